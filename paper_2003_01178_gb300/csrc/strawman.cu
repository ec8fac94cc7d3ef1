// The "independent threads" selection the paper uses as its point of comparison for the
// tile-based model (Section 3.2, Figure "tile"): every thread owns a contiguous chunk of
// the input, as a CPU thread would, and the selection takes three kernels:
//   K1  each thread counts the rows of its chunk that satisfy the predicate;
//   K2  an exclusive prefix sum of the per-thread counts gives each thread its offset;
//   K3  each thread reads its chunk again and writes its matches from its offset.
// Neighbouring threads read addresses a chunk apart (no coalescing) and the input is read
// twice; the output is in input order.  Kept as an ablation beside select_kernel.
#include "common.cuh"

namespace crys {
namespace {

constexpr int kStrawThreads = 256;
constexpr int kScanThreads = 1024;

__global__ void __launch_bounds__(kStrawThreads)
    straw_count_kernel(const int32_t* __restrict__ x, int64_t n, int32_t lo, uint32_t span, int64_t chunk,
                       int64_t* __restrict__ counts) {
  const int64_t t = static_cast<int64_t>(blockIdx.x) * kStrawThreads + threadIdx.x;
  const int64_t b = t * chunk;
  const int64_t e = b + chunk < n ? b + chunk : n;
  int64_t c = 0;
  for (int64_t i = b; i < e; ++i) c += static_cast<uint32_t>(x[i]) - static_cast<uint32_t>(lo) <= span;
  counts[t] = c;
}

// Exclusive scan of m counts in place by one block: each thread sums a contiguous run,
// the block scans the run totals, then each thread writes its run's offsets.
__global__ void __launch_bounds__(kScanThreads) straw_scan_kernel(int64_t* __restrict__ counts, int64_t m,
                                                                  unsigned long long* __restrict__ total) {
  __shared__ int64_t part[kScanThreads];
  const int tid = threadIdx.x;
  const int64_t per = (m + kScanThreads - 1) / kScanThreads;
  const int64_t b = tid * per;
  const int64_t e = b + per < m ? b + per : m;
  int64_t s = 0;
  for (int64_t i = b; i < e; ++i) s += counts[i];
  part[tid] = s;
  __syncthreads();
  for (int d = 1; d < kScanThreads; d <<= 1) {  // Hillis-Steele inclusive scan of the totals
    const int64_t v = tid >= d ? part[tid - d] : 0;
    __syncthreads();
    part[tid] += v;
    __syncthreads();
  }
  int64_t run = part[tid] - s;
  for (int64_t i = b; i < e; ++i) {
    const int64_t c = counts[i];
    counts[i] = run;
    run += c;
  }
  if (tid == kScanThreads - 1) *total = static_cast<unsigned long long>(part[tid]);
}

__global__ void __launch_bounds__(kStrawThreads)
    straw_write_kernel(const int32_t* __restrict__ x, int64_t n, int32_t lo, uint32_t span, int64_t chunk,
                       const int64_t* __restrict__ offsets, int32_t* __restrict__ out) {
  const int64_t t = static_cast<int64_t>(blockIdx.x) * kStrawThreads + threadIdx.x;
  const int64_t b = t * chunk;
  const int64_t e = b + chunk < n ? b + chunk : n;
  int64_t o = offsets[t];
  for (int64_t i = b; i < e; ++i) {
    const int32_t v = x[i];
    if (static_cast<uint32_t>(v) - static_cast<uint32_t>(lo) <= span) out[o++] = v;
  }
}

// Threads of the independent-threads launch: every SM fully occupied, 8 blocks of 256.
int64_t straw_threads() { return static_cast<int64_t>(sm_count()) * 8 * kStrawThreads; }

}  // namespace
}  // namespace crys

extern "C" int crys_select_strawman(const int32_t* x, int64_t n, int32_t lo, int32_t hi, int32_t* out,
                                    int64_t* d_count, void* d_temp, size_t* temp_bytes, crys_stream stream) {
  using namespace crys;
  if (n < 0) return CRYS_EINVAL;
  const int64_t threads = straw_threads();
  const size_t need = static_cast<size_t>(threads) * sizeof(int64_t);
  if (!d_temp && temp_bytes) {
    *temp_bytes = need;
    return CRYS_OK;
  }
  if (!d_temp || !temp_bytes || *temp_bytes < need) return CRYS_EINVAL;
  if (!d_count || (n > 0 && (!x || !out))) return CRYS_EINVAL;
  if (reinterpret_cast<uintptr_t>(d_temp) & 7u) return CRYS_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (cudaMemsetAsync(d_count, 0, sizeof(int64_t), s) != cudaSuccess) return CRYS_ECUDA;
  if (n == 0 || lo > hi) return CRYS_OK;
  const uint32_t span = static_cast<uint32_t>(hi) - static_cast<uint32_t>(lo);
  const int64_t chunk = (n + threads - 1) / threads;
  int64_t* counts = static_cast<int64_t*>(d_temp);
  const unsigned blocks = static_cast<unsigned>(threads / kStrawThreads);
  straw_count_kernel<<<blocks, kStrawThreads, 0, s>>>(x, n, lo, span, chunk, counts);
  note_launch();
  straw_scan_kernel<<<1, kScanThreads, 0, s>>>(counts, threads, reinterpret_cast<unsigned long long*>(d_count));
  note_launch();
  straw_write_kernel<<<blocks, kStrawThreads, 0, s>>>(x, n, lo, span, chunk, counts, out);
  note_launch();
  return check_launch();
}
