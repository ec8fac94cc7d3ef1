// Host-side state of the library: the per-device sticky error word, the launch
// counter, SM counts and the tile-shape choice of each operator.
#include <atomic>
#include <mutex>
#include <unordered_map>

#include "common.cuh"
#include "tiles.h"

namespace crys {
namespace {

// Sticky error bits set by kernels (CRYS_DEV_*).  One copy per device that loads the
// library; kernels receive its address as an argument.
__device__ int32_t g_device_error = 0;

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
int32_t* g_error_ptr[kMaxDevices] = {};
int g_sms[kMaxDevices] = {};
std::atomic<int64_t> g_launches{0};
std::atomic<int> g_variant[CRYS_NUM_OPS] = {};
// pending crys_debug_stall request (op, first tile, wait bound), taken by the next call
std::mutex g_stall_mutex;
int g_stall_op = -1;
uint32_t g_stall_first = 0;
uint64_t g_stall_ns = 0;

int current_device() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return 0;
  return dev;
}

}  // namespace

int32_t* device_error_word() {
  const int dev = current_device();
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_error_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_device_error) != cudaSuccess) return nullptr;
    g_error_ptr[dev] = static_cast<int32_t*>(p);
  }
  return g_error_ptr[dev];
}

void note_launch(int kernels) { g_launches.fetch_add(kernels, std::memory_order_relaxed); }

int sm_count() {
  const int dev = current_device();
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_sms[dev]) {
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    g_sms[dev] = v > 0 ? v : 1;
  }
  return g_sms[dev];
}

bool set_dynamic_smem(const void* kernel, size_t bytes) {
  static std::mutex m;
  static std::unordered_map<const void*, size_t> done[kMaxDevices];
  const int dev = current_device();
  std::lock_guard<std::mutex> lock(m);
  auto it = done[dev].find(kernel);
  if (it != done[dev].end() && it->second >= bytes) return true;
  if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           static_cast<int>(bytes)) != cudaSuccess)
    return false;
  done[dev][kernel] = bytes;
  return true;
}

int blocks_per_sm(const void* kernel, int threads, size_t smem) {
  struct Key {
    const void* kernel;
    int threads;
    size_t smem;
    bool operator==(const Key& o) const { return kernel == o.kernel && threads == o.threads && smem == o.smem; }
  };
  struct KeyHash {
    size_t operator()(const Key& k) const {
      return std::hash<const void*>()(k.kernel) ^ (static_cast<size_t>(k.threads) << 1) ^ (k.smem << 12);
    }
  };
  static std::mutex m;
  static std::unordered_map<Key, int, KeyHash> known[kMaxDevices];
  const int dev = current_device();
  const Key key{kernel, threads, smem};
  {
    std::lock_guard<std::mutex> lock(m);
    auto it = known[dev].find(key);
    if (it != known[dev].end()) return it->second;
  }
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem) != cudaSuccess || per_sm < 1)
    per_sm = 1;
  std::lock_guard<std::mutex> lock(m);
  known[dev][key] = per_sm;
  return per_sm;
}

bool take_stall(int op, uint32_t* first_tile, uint64_t* wait_ns) {
  std::lock_guard<std::mutex> lock(g_stall_mutex);
  *first_tile = 0;
  *wait_ns = kWaitBoundNs;
  if (g_stall_op != op) return false;
  *first_tile = g_stall_first;
  *wait_ns = g_stall_ns;
  g_stall_op = -1;
  return true;
}

int tile_variant(int op) {
  if (op < 0 || op >= CRYS_NUM_OPS) return 0;
  return g_variant[op].load(std::memory_order_relaxed);
}

}  // namespace crys

extern "C" {

const char* crys_strerror(int status) {
  switch (status) {
    case CRYS_OK: return "ok";
    case CRYS_EINVAL: return "invalid argument (null, misaligned or out-of-range value, bad plan)";
    case CRYS_ENOMEM: return "scratch buffer smaller than required";
    case CRYS_EFULL: return "hash table capacity too small";
    case CRYS_ETIMEOUT: return "wait exceeded its bound";
    case CRYS_ECUDA: return "CUDA runtime error";
    default: return "unknown status";
  }
}

int crys_device_errors(int32_t* flags, int clear, crys_stream s) {
  if (!flags) return CRYS_EINVAL;
  int32_t* word = crys::device_error_word();
  if (!word) return CRYS_ECUDA;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(s);
  int32_t host = 0;
  if (cudaMemcpyAsync(&host, word, sizeof(int32_t), cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return CRYS_ECUDA;
  if (clear && cudaMemsetAsync(word, 0, sizeof(int32_t), st) != cudaSuccess) return CRYS_ECUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return CRYS_ECUDA;
  *flags = host;
  return CRYS_OK;
}

int64_t crys_launch_count(void) { return crys::g_launches.load(); }

int crys_debug_stall(int op, int32_t first_tile, int64_t wait_limit_ns) {
  if ((op != CRYS_OP_SELECT && op != CRYS_OP_SORT) || first_tile < 0 || wait_limit_ns < 1000 ||
      wait_limit_ns > static_cast<int64_t>(crys::kWaitBoundNs))
    return CRYS_EINVAL;
  std::lock_guard<std::mutex> lock(crys::g_stall_mutex);
  crys::g_stall_op = op;
  crys::g_stall_first = static_cast<uint32_t>(first_tile);
  crys::g_stall_ns = static_cast<uint64_t>(wait_limit_ns);
  return CRYS_OK;
}

int crys_tile_variants(int op, int32_t* threads, int32_t* items, int32_t max) {
  if (op < 0 || op >= CRYS_NUM_OPS) return CRYS_EINVAL;
  const int n = crys::kNumVariants[op];
  for (int i = 0; i < n && i < max; ++i) {
    if (threads) threads[i] = crys::kTiles[op][i].threads;
    if (items) items[i] = crys::kTiles[op][i].items;
  }
  return n;
}

int crys_set_tile(int op, int32_t variant) {
  if (op < 0 || op >= CRYS_NUM_OPS || variant < 0 || variant >= crys::kNumVariants[op])
    return CRYS_EINVAL;
  crys::g_variant[op].store(variant);
  return CRYS_OK;
}

int crys_get_tile(int op) {
  if (op < 0 || op >= CRYS_NUM_OPS) return CRYS_EINVAL;
  return crys::g_variant[op].load();
}

}  // extern "C"
