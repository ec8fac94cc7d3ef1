// Device-side twin of datagen/__init__.py: fills int32/float32 columns in HBM with the
// same counter-based values (SplitMix64 words, Lemire range reduction, Feistel
// permutation with cycle walking).  Input generation only; no query operator lives here.
// Built into libcrysgen.so, separate from the operator library.
#include <cuda_runtime.h>
#include <stdint.h>

namespace {

constexpr uint64_t kGamma = 0x9E3779B97F4A7C15ull;

__host__ __device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__host__ __device__ __forceinline__ uint64_t stream_base(uint64_t seed, uint64_t stream) {
  return mix64(seed ^ mix64(stream));
}

__device__ __forceinline__ uint64_t word_at(uint64_t base, uint64_t i) {
  return mix64(base + (i + 1ull) * kGamma);
}

template <int KIND>
__global__ void fill_kernel(uint64_t base, int64_t start, int64_t n, int32_t lo, uint64_t span,
                            void* out) {
  int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    uint64_t w = word_at(base, (uint64_t)(start + i));
    if (KIND == 0) {  // uniform int32 in [lo, lo + span)
      uint64_t off = ((w >> 32) * span) >> 32;
      ((int32_t*)out)[i] = (int32_t)((int64_t)lo + (int64_t)off);
    } else if (KIND == 1) {  // uniform float32 in [0, 1)
      ((float*)out)[i] = (float)((double)(w >> 40) * (1.0 / 16777216.0));
    } else {  // raw 32-bit pattern
      ((uint32_t*)out)[i] = (uint32_t)(w >> 32);
    }
  }
}

__device__ __forceinline__ uint64_t feistel(uint64_t x, const uint64_t* keys, int half) {
  uint64_t mask = (1ull << half) - 1ull;
  uint64_t l = x >> half, r = x & mask;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    uint64_t f = mix64(r + keys[k]) & mask;
    uint64_t nl = r;
    r = l ^ f;
    l = nl;
  }
  return (l << half) | r;
}

struct FeistelKeys { uint64_t k[4]; };

__global__ void perm_kernel(FeistelKeys keys, int half, int64_t n_domain, int64_t start, int64_t count,
                            int32_t* out) {
  int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride) {
    uint64_t y = feistel((uint64_t)(start + i), keys.k, half);
    // Cycle walking ends: the walk from an in-range start returns to the domain
    // [0, n) within at most 2^k - n steps because the Feistel network is a
    // permutation; the cap is only a guard and is never reached.
    for (int step = 0; y >= (uint64_t)n_domain && step < (1 << 30); ++step)
      y = feistel(y, keys.k, half);
    out[i] = y < (uint64_t)n_domain ? (int32_t)y : -1;
  }
}

int grid_for(int64_t n) {
  int64_t blocks = (n + 255) / 256;
  if (blocks > 152 * 32) blocks = 152 * 32;
  if (blocks < 1) blocks = 1;
  return (int)blocks;
}

}  // namespace

extern "C" {

// Fill out[0..n) with element start+i of uniform int32 in [lo, hi] of (seed, stream).
int dg_uniform_i32(uint64_t seed, uint64_t stream, int64_t start, int64_t n, int32_t lo,
                   int32_t hi, int32_t* out, cudaStream_t s) {
  if (n < 0 || hi < lo) return -1;
  if (n == 0) return 0;
  uint64_t span = (uint64_t)((int64_t)hi - (int64_t)lo + 1);
  fill_kernel<0><<<grid_for(n), 256, 0, s>>>(stream_base(seed, stream), start, n, lo, span, out);
  return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

int dg_uniform_f32(uint64_t seed, uint64_t stream, int64_t start, int64_t n, float* out,
                   cudaStream_t s) {
  if (n < 0) return -1;
  if (n == 0) return 0;
  fill_kernel<1><<<grid_for(n), 256, 0, s>>>(stream_base(seed, stream), start, n, 0, 0, out);
  return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

int dg_bits_i32(uint64_t seed, uint64_t stream, int64_t start, int64_t n, int32_t* out,
                cudaStream_t s) {
  if (n < 0) return -1;
  if (n == 0) return 0;
  fill_kernel<2><<<grid_for(n), 256, 0, s>>>(stream_base(seed, stream), start, n, 0, 0, out);
  return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

// Elements start..start+count of the seeded permutation of [0, n_domain).
int dg_perm_i32(uint64_t seed, uint64_t stream, int64_t n_domain, int64_t start, int64_t count,
                int32_t* out, cudaStream_t s) {
  if (count < 0 || n_domain < 0 || n_domain > (1ll << 31) || start < 0 ||
      start + count > n_domain)
    return -1;
  if (count == 0) return 0;
  int k = 2;
  if (n_domain > 1) {
    uint64_t v = (uint64_t)(n_domain - 1);
    int bl = 0;
    while (v) { ++bl; v >>= 1; }
    k = bl < 2 ? 2 : bl;
  }
  k += (k & 1);
  FeistelKeys keys;
  uint64_t base = stream_base(seed, stream);
  for (int r = 0; r < 4; ++r) keys.k[r] = mix64(base + (uint64_t)(r + 1) * kGamma);
  perm_kernel<<<grid_for(count), 256, 0, s>>>(keys, k / 2, n_domain, start, count, out);
  return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

}  // extern "C"
