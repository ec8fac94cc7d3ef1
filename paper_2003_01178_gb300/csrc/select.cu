// Selection (Section 3.2 query Q0, Section 4.2 query Q3) as one persistent kernel.
//
// Per tile: BlockLoad (bulk copy into a shared-memory stage) -> BlockPred (range
// predicate into a per-thread bitmap in registers) -> BlockScan (a warp scan of packed
// per-thread counts, then one warp scans the warps' totals) -> one output reservation
// per tile -> BlockShuffle (each warp compacts its rows into its own shared-memory
// run) -> BlockStore (coalesced stores of each warp's run).
//
// Each warp owns a contiguous run of ITEMS*32 rows of the tile (lane l reads the
// 4-value groups j*128 + 4l, j < ITEMS/4) and compacts its selected values in input
// order into its own shared-memory run.  A first block barrier publishes the warp totals
// (the stage goes back to the copy engine right after it); warp 0 turns them into
// offsets and makes the tile's single output reservation; after a second barrier every
// warp stores its run with coalesced writes.  In the unordered mode a tile without
// matches stops after the first barrier.  Full tiles read the stage without tail checks.
//
// Output reservation: mode 0 adds the tile's count to the global cursor with one
// atomic (the paper's scheme); mode 1 chains tiles with a decoupled look-back (tile
// ids handed out in order by an atomic counter, so a tile only waits on tiles that
// running blocks already hold) and the result is in input order.
#include <mutex>
#include <type_traits>

#include "common.cuh"
#include "pipeline.cuh"
#include "tiles.h"

namespace crys {
namespace {

constexpr uint64_t kFlagAggregate = 1ull << 62;
constexpr uint64_t kFlagInclusive = 2ull << 62;
constexpr uint64_t kValueMask = (1ull << 62) - 1;

struct SelectArgs {
  const int32_t* x;
  int64_t n;
  int32_t lo, hi;
  uint32_t span;  // hi - lo; only used when lo <= hi
  int32_t* out;
  unsigned long long* count;  // cursor (mode 0) / final count (mode 1)
  uint64_t* tile_state;       // mode 1: one status word per tile
  unsigned int* tile_counter; // mode 1: next tile id (scratch header, word 0)
  unsigned int* abort_word;   // mode 1: set by the first block of this call that gives up
  uint32_t tile_base;         // mode 1: first tile id handed out (0 unless a test stalls)
  uint64_t wait_ns;           // mode 1: bound of a look-back wait
  int32_t* err;
  int32_t stages;
};

// Decoupled look-back over tiles 0..t-1 (thread 0 only).  Returns the number of
// selected rows in all earlier tiles, or -1 if a predecessor never published within
// the wait bound, or another block of the same call already gave up (its abort word,
// in this call's scratch: a failure of an earlier call does not reach this one).
__device__ int64_t lookback_exclusive(uint64_t* state, int64_t t, uint64_t total, const SelectArgs& a) {
  if (t == 0) {
    st_relaxed_u64(&state[0], kFlagInclusive | total);
    return 0;
  }
  st_relaxed_u64(&state[t], kFlagAggregate | total);
  uint64_t excl = 0;
  int64_t p = t - 1;
  uint64_t t0 = 0;
  bool timing = false;
  while (p >= 0) {
    const uint64_t w = ld_relaxed_u64(&state[p]);
    const uint64_t flag = w >> 62;
    if (flag == 0) {
      if (!timing) {
        t0 = global_timer_ns();
        timing = true;
      } else if (global_timer_ns() - t0 > a.wait_ns) {
        set_error(a.err, CRYS_DEV_TIMEOUT);
        st_relaxed_u32(a.abort_word, 1u);
        return -1;
      }
      if (ld_relaxed_u32(a.abort_word)) return -1;
      continue;
    }
    timing = false;
    excl += w & kValueMask;
    if (flag == 2) break;
    --p;
  }
  st_relaxed_u64(&state[t], kFlagInclusive | (excl + total));
  return static_cast<int64_t>(excl);
}

template <int THREADS, int ITEMS, bool ORDERED>
__global__ void __launch_bounds__(THREADS) select_kernel(SelectArgs a) {
  constexpr int TILE = THREADS * ITEMS;
  constexpr int VEC = ITEMS / 4;
  constexpr int WARPS = THREADS / kWarp;
  constexpr int WROWS = ITEMS * kWarp;  // rows of a tile owned by one warp, contiguous
  static_assert(ITEMS % 4 == 0 && VEC <= 4, "4..16 items per thread");
  static_assert(WARPS <= kWarp, "one warp scans the warp totals");

  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int S = a.stages;
  int32_t* stages = reinterpret_cast<int32_t*>(smem_raw);    // S x TILE
  int32_t* wbuf_all = stages + S * TILE;                     // per-warp compaction runs
  __shared__ StageRing ring;
  __shared__ int32_t wtot[WARPS];
  __shared__ int32_t woff[WARPS];
  __shared__ long long out_base;

  const int tid = threadIdx.x, lane = tid % kWarp, warp = tid / kWarp;
  int32_t* wbuf = wbuf_all + warp * WROWS;
  const int64_t ntiles = (a.n + TILE - 1) / TILE;
  const uint64_t pol = policy_evict_first();
  int64_t issued = 0;  // thread 0 only

  auto issue = [&](int s) {
    int64_t t = ORDERED ? static_cast<int64_t>(a.tile_base) + static_cast<int64_t>(atomicAdd(a.tile_counter, 1u))
                        : static_cast<int64_t>(blockIdx.x) + issued * gridDim.x;
    ++issued;
    if (t >= ntiles) {
      ring.tile[s] = -1;
      return;
    }
    ring.tile[s] = t;
    const int64_t row = t * TILE;
    const int64_t valid = (a.n - row) < TILE ? (a.n - row) : TILE;
    ring_issue(&ring.full[s], stages + s * TILE, TILE, &a.x, 1, row, valid, pol);
  };

  ring_init(ring, S);
  if (tid == 0)
    for (int s = 0; s < S; ++s) issue(s);
  __syncthreads();

  for (int64_t k = 0;; ++k) {
    const int s = static_cast<int>(k % S);
    const int64_t t = ring.tile[s];
    if (t < 0) break;
    if (!ring_wait(ring, k, S, a.err)) {
      if (tid == 0) ring_drain(ring, k, S, a.err);
      return;
    }
    const int32_t* st = stages + s * TILE;
    const int64_t row0 = t * TILE;
    const int valid = static_cast<int>((a.n - row0) < TILE ? (a.n - row0) : TILE);
    const int bulk = valid & ~3;

    // BlockLoad + BlockPred: this warp's rows warp*WROWS + j*128 + lane*4 + e, values and
    // bitmap in registers.
    int32_t v[ITEMS];
    uint32_t bits = 0;
    // a full tile (all but possibly the last) reads the stage without tail checks
    auto load_pred = [&](auto full_tag) {
      constexpr bool FULL = decltype(full_tag)::value;
#pragma unroll
      for (int j = 0; j < VEC; ++j) {
        const int p = warp * WROWS + j * 128 + lane * 4;
        const int4 q = FULL ? *reinterpret_cast<const int4*>(st + p) : stage_read4(st, a.x + row0, p, bulk, valid);
        v[4 * j + 0] = q.x;
        v[4 * j + 1] = q.y;
        v[4 * j + 2] = q.z;
        v[4 * j + 3] = q.w;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          // lo <= v <= hi as one unsigned comparison (span = hi - lo, lo <= hi)
          const bool hit = (FULL || p + e < valid) &&
                           static_cast<uint32_t>(v[4 * j + e]) - static_cast<uint32_t>(a.lo) <= a.span;
          bits |= static_cast<uint32_t>(hit) << (4 * j + e);
        }
      }
    };
    if (valid == TILE)
      load_pred(std::true_type{});
    else
      load_pred(std::false_type{});
    // BlockScan inside the warp: one scan of the per-lane counts of all VEC groups at
    // once (group j's count in byte j; a group's warp total is at most 128).
    uint32_t packed = 0;
#pragma unroll
    for (int j = 0; j < VEC; ++j) packed |= static_cast<uint32_t>(__popc((bits >> (4 * j)) & 0xFu)) << (8 * j);
    const uint32_t incl = static_cast<uint32_t>(warp_inclusive_scan(static_cast<int32_t>(packed), lane));
    const uint32_t excl = incl - packed;
    const uint32_t totals = __shfl_sync(0xFFFFFFFFu, incl, kWarp - 1);
    // BlockShuffle inside the warp: its selected values, in input order, to its own run.
    int run = 0;
#pragma unroll
    for (int j = 0; j < VEC; ++j) {
      int pos = run + static_cast<int>((excl >> (8 * j)) & 0xFFu);
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        if (bits & (1u << (4 * j + e))) wbuf[pos++] = v[4 * j + e];
      }
      run += static_cast<int>((totals >> (8 * j)) & 0xFFu);
    }
    if (lane == 0) wtot[warp] = run;
    __syncthreads();  // every warp has read the stage and published its count
    if (!ORDERED) {
      // A tile without matches needs no reservation and no store: every thread sees the
      // same warp totals, so the whole block skips the second barrier together.  (The
      // totals are next written after the next iteration's stage barrier.)
      int tile_total = 0;
#pragma unroll
      for (int w = 0; w < WARPS; ++w) tile_total += wtot[w];
      if (tile_total == 0) {
        if (tid == 0) {
          fence_proxy_async_smem();
          issue(s);
        }
        continue;
      }
    }
    if (warp == 0) {
      if (lane == 0) {  // the stage is free: refill it now, while the tile is written
        fence_proxy_async_smem();
        issue(s);
      }
      const int32_t x = lane < WARPS ? wtot[lane] : 0;
      const int32_t inc = warp_inclusive_scan(x, lane);
      if (lane < WARPS) woff[lane] = inc - x;
      const int32_t total = __shfl_sync(0xFFFFFFFFu, inc, kWarp - 1);
      if (lane == 0) {
        long long base;
        if (ORDERED) {
          base = lookback_exclusive(a.tile_state, t, static_cast<uint64_t>(total), a);
          if (base >= 0 && t == ntiles - 1) *a.count = static_cast<unsigned long long>(base + total);
        } else {
          base = total ? static_cast<long long>(atomicAdd(a.count, static_cast<unsigned long long>(total))) : 0;
        }
        if (base >= 0 && base + total > a.n) {
          set_error(a.err, CRYS_DEV_BOUNDS);
          base = -1;
        }
        out_base = base;
      }
    }
    __syncthreads();
    const long long base = out_base;
    if (base < 0) {  // look-back gave up (or bounds): abandon uniformly
      if (tid == 0) ring_drain(ring, k + 1, S, a.err);
      return;
    }
    // BlockStore: each warp writes its run with coalesced stores.
    int32_t* dst = a.out + base + woff[warp];
    for (int i = lane; i < run; i += kWarp) dst[i] = wbuf[i];
  }
}

template <int THREADS, int ITEMS>
int launch(SelectArgs a, bool ordered, cudaStream_t s) {
  constexpr int TILE = THREADS * ITEMS;
  const size_t tile_bytes = static_cast<size_t>(TILE) * sizeof(int32_t);
  // The select body is issue-bound: keep about 32 warps per SM resident and give each
  // block the stages that still fit.
  a.stages = stages_for(tile_bytes, tile_bytes + 1024, (32 * kWarp) / THREADS);
  const size_t smem = static_cast<size_t>(a.stages + 1) * tile_bytes;
  const int64_t ntiles = (a.n + TILE - 1) / TILE;
  if (ordered) {
    auto k = select_kernel<THREADS, ITEMS, true>;
    if (!allow_smem(k, smem)) return CRYS_ECUDA;
    k<<<persistent_grid(k, THREADS, smem, ntiles), THREADS, smem, s>>>(a);
  } else {
    auto k = select_kernel<THREADS, ITEMS, false>;
    if (!allow_smem(k, smem)) return CRYS_ECUDA;
    k<<<persistent_grid(k, THREADS, smem, ntiles), THREADS, smem, s>>>(a);
  }
  note_launch();
  return check_launch();
}

constexpr int kOp = CRYS_OP_SELECT;

int64_t min_tile() {
  int64_t m = INT64_MAX;
  for (int i = 0; i < kNumVariants[kOp]; ++i) {
    const int64_t t = static_cast<int64_t>(kTiles[kOp][i].threads) * kTiles[kOp][i].items;
    if (t < m) m = t;
  }
  return m;
}

}  // namespace
}  // namespace crys

extern "C" int crys_select(const int32_t* x, int64_t n, int32_t lo, int32_t hi, int32_t* out,
                           int64_t* d_count, int order_preserving, void* d_temp,
                           size_t* temp_bytes, crys_stream stream) {
  using namespace crys;
  if (n < 0 || (order_preserving != 0 && order_preserving != 1)) return CRYS_EINVAL;
  const int64_t max_tiles = (n + min_tile() - 1) / min_tile();
  const size_t need = order_preserving ? (static_cast<size_t>(max_tiles) * 8 + 256) : 0;
  if (!d_temp && temp_bytes) {
    *temp_bytes = need;
    return CRYS_OK;
  }
  if (need && (!d_temp || !temp_bytes)) return CRYS_EINVAL;
  if (need && *temp_bytes < need) return CRYS_ENOMEM;
  if (!d_count || (n > 0 && (!x || !out))) return CRYS_EINVAL;
  if (n > 0 && !aligned16(x)) return CRYS_EINVAL;
  if (need && (reinterpret_cast<uintptr_t>(d_temp) & 255u)) return CRYS_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (cudaMemsetAsync(d_count, 0, sizeof(int64_t), s) != cudaSuccess) return CRYS_ECUDA;
  if (n == 0) return CRYS_OK;
  if (lo > hi) {  // empty range: nothing selected (d_count already zeroed)
    if (order_preserving && cudaMemsetAsync(d_temp, 0, need, s) != cudaSuccess) return CRYS_ECUDA;
    return CRYS_OK;
  }
  SelectArgs a;
  a.x = x;
  a.n = n;
  a.lo = lo;
  a.hi = hi;
  a.span = static_cast<uint32_t>(hi) - static_cast<uint32_t>(lo);
  a.out = out;
  a.count = reinterpret_cast<unsigned long long*>(d_count);
  a.tile_counter = nullptr;
  a.abort_word = nullptr;
  a.tile_state = nullptr;
  a.tile_base = 0;
  a.wait_ns = kWaitBoundNs;
  a.err = device_error_word();
  if (!a.err) return CRYS_ECUDA;
  if (order_preserving) {
    a.tile_counter = static_cast<unsigned int*>(d_temp);
    a.abort_word = static_cast<unsigned int*>(d_temp) + 1;
    a.tile_state = reinterpret_cast<uint64_t*>(static_cast<char*>(d_temp) + 256);
    take_stall(CRYS_OP_SELECT, &a.tile_base, &a.wait_ns);
    if (cudaMemsetAsync(d_temp, 0, need, s) != cudaSuccess) return CRYS_ECUDA;
  }
  const bool ord = order_preserving != 0;
  switch (tile_variant(CRYS_OP_SELECT)) {
    case 1: return launch<kTiles[kOp][1].threads, kTiles[kOp][1].items>(a, ord, s);
    case 2: return launch<kTiles[kOp][2].threads, kTiles[kOp][2].items>(a, ord, s);
    case 3: return launch<kTiles[kOp][3].threads, kTiles[kOp][3].items>(a, ord, s);
    default: return launch<kTiles[kOp][0].threads, kTiles[kOp][0].items>(a, ord, s);
  }
}

// ---------------------------------------------------------------------------
// Allocation-free order-preserving selection: the look-back scratch is a static device
// array of this file instead of caller-supplied memory.

namespace crys {
namespace {

static_assert(CRYS_SELECT_STATIC_SCRATCH_BYTES >= 256 + (CRYS_SELECT_STATIC_MAX_ROWS / 512) * 8,
              "static scratch covers the smallest tile shape");

static __device__ __align__(256) unsigned char g_select_scratch[CRYS_SELECT_STATIC_SCRATCH_BYTES];

constexpr int kMaxStaticDevices = 64;
std::mutex g_static_mutex;
void* g_static_ptr[kMaxStaticDevices] = {};

// Device address of g_select_scratch on the current device (looked up once per device
// with that device current; the host-side name is only a stand-in for the symbol).
void* static_scratch() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxStaticDevices) return nullptr;
  std::lock_guard<std::mutex> lock(g_static_mutex);
  if (!g_static_ptr[dev]) {
    void* ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_select_scratch) != cudaSuccess) return nullptr;
    g_static_ptr[dev] = ptr;
  }
  return g_static_ptr[dev];
}

}  // namespace
}  // namespace crys

extern "C" int crys_select_static(const int32_t* x, int64_t n, int32_t lo, int32_t hi,
                                  int32_t* out, int64_t* d_count, crys_stream stream) {
  using namespace crys;
  if (n < 0 || n > CRYS_SELECT_STATIC_MAX_ROWS) return CRYS_EINVAL;
  size_t need = 0;
  if (crys_select(nullptr, n, lo, hi, nullptr, nullptr, 1, nullptr, &need, stream) != CRYS_OK)
    return CRYS_EINVAL;
  if (need > CRYS_SELECT_STATIC_SCRATCH_BYTES) return CRYS_EINVAL;
  void* scratch = static_scratch();
  if (!scratch) return CRYS_ECUDA;
  size_t have = CRYS_SELECT_STATIC_SCRATCH_BYTES;
  // crys_select clears the `need` bytes it uses on `stream` before its kernel runs.
  return crys_select(x, n, lo, hi, out, d_count, 1, scratch, &have, stream);
}
