// Projection (Section 4.1, queries Q1 and Q2) as one persistent kernel: two BlockLoads
// (bulk copies of the x1 and x2 tiles into one shared-memory stage), the arithmetic in
// registers, and a BlockStore of 16-byte vectors straight from registers (the output
// of a tile is contiguous and 16-byte aligned, so no shared-memory staging is needed).
#include "common.cuh"
#include "pipeline.cuh"
#include "tiles.h"

namespace crys {
namespace {


struct ProjectArgs {
  const float* x1;
  const float* x2;
  int64_t n;
  float a, b;
  float* y;
  int32_t* err;
  int32_t stages;
};

template <int OP>
__device__ __forceinline__ float project_one(float a, float b, float x1, float x2) {
  // one rounding per product and per sum, as written: a*x1 + b*x2
  const float lin = __fadd_rn(__fmul_rn(a, x1), __fmul_rn(b, x2));
  if (OP == CRYS_PROJ_SIGMOID) return 1.0f / (1.0f + expf(-lin));
  return lin;
}

__device__ __forceinline__ void st_stream_v4(float* p, float4 v) {
  asm volatile("st.global.cs.v4.f32 [%0], {%1,%2,%3,%4};" ::"l"(p), "f"(v.x), "f"(v.y), "f"(v.z),
               "f"(v.w)
               : "memory");
}

template <int THREADS, int ITEMS, int OP>
__global__ void __launch_bounds__(THREADS) project_kernel(ProjectArgs a) {
  constexpr int TILE = THREADS * ITEMS;
  constexpr int VEC = ITEMS / 4;
  static_assert(ITEMS % 4 == 0, "items per thread must be a multiple of 4");
  extern __shared__ __align__(128) unsigned char smem_raw[];
  int32_t* stages = reinterpret_cast<int32_t*>(smem_raw);  // per stage: x1 tile, x2 tile
  __shared__ StageRing ring;
  const int S = a.stages;

  const int tid = threadIdx.x;
  const int64_t ntiles = (a.n + TILE - 1) / TILE;
  const uint64_t pol = policy_evict_first();
  const int32_t* cols[2] = {reinterpret_cast<const int32_t*>(a.x1),
                            reinterpret_cast<const int32_t*>(a.x2)};
  int64_t issued = 0;

  auto issue = [&](int s) {
    const int64_t t = static_cast<int64_t>(blockIdx.x) + issued * gridDim.x;
    ++issued;
    if (t >= ntiles) {
      ring.tile[s] = -1;
      return;
    }
    ring.tile[s] = t;
    const int64_t row = t * TILE;
    const int64_t valid = (a.n - row) < TILE ? (a.n - row) : TILE;
    ring_issue(&ring.full[s], stages + s * 2 * TILE, TILE, cols, 2, row, valid, pol);
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
    const int32_t* st1 = stages + s * 2 * TILE;
    const int32_t* st2 = st1 + TILE;
    const int64_t row0 = t * TILE;
    const int valid = static_cast<int>((a.n - row0) < TILE ? (a.n - row0) : TILE);
    const int bulk = valid & ~3;
#pragma unroll
    for (int j = 0; j < VEC; ++j) {
      const int p = (j * THREADS + tid) * 4;
      if (p >= valid) break;
      const int4 q1 = stage_read4(st1, cols[0] + row0, p, bulk, valid);
      const int4 q2 = stage_read4(st2, cols[1] + row0, p, bulk, valid);
      float4 r;
      r.x = project_one<OP>(a.a, a.b, __int_as_float(q1.x), __int_as_float(q2.x));
      r.y = project_one<OP>(a.a, a.b, __int_as_float(q1.y), __int_as_float(q2.y));
      r.z = project_one<OP>(a.a, a.b, __int_as_float(q1.z), __int_as_float(q2.z));
      r.w = project_one<OP>(a.a, a.b, __int_as_float(q1.w), __int_as_float(q2.w));
      float* dst = a.y + row0 + p;
      if (p + 4 <= valid) {
        st_stream_v4(dst, r);
      } else {
        const float rr[4] = {r.x, r.y, r.z, r.w};
        for (int e = 0; p + e < valid; ++e) dst[e] = rr[e];
      }
    }
    __syncthreads();
    if (tid == 0) {
      fence_proxy_async_smem();
      issue(s);
    }
  }
}

template <int THREADS, int ITEMS>
int launch(ProjectArgs a, int op, cudaStream_t s) {
  constexpr int TILE = THREADS * ITEMS;
  const size_t stage_bytes = static_cast<size_t>(2) * TILE * sizeof(int32_t);
  a.stages = stages_for(stage_bytes, 1024, THREADS >= 512 ? 1 : 2);
  const size_t smem = static_cast<size_t>(a.stages) * stage_bytes;
  const int64_t ntiles = (a.n + TILE - 1) / TILE;
  if (op == CRYS_PROJ_SIGMOID) {
    auto k = project_kernel<THREADS, ITEMS, CRYS_PROJ_SIGMOID>;
    if (!allow_smem(k, smem)) return CRYS_ECUDA;
    k<<<persistent_grid(k, THREADS, smem, ntiles), THREADS, smem, s>>>(a);
  } else {
    auto k = project_kernel<THREADS, ITEMS, CRYS_PROJ_LINEAR>;
    if (!allow_smem(k, smem)) return CRYS_ECUDA;
    k<<<persistent_grid(k, THREADS, smem, ntiles), THREADS, smem, s>>>(a);
  }
  note_launch();
  return check_launch();
}

constexpr int kOp = CRYS_OP_PROJECT;

}  // namespace
}  // namespace crys

extern "C" int crys_project(const float* x1, const float* x2, int64_t n, float a, float b, int op,
                            float* y, crys_stream stream) {
  using namespace crys;
  if (n < 0 || (op != CRYS_PROJ_LINEAR && op != CRYS_PROJ_SIGMOID)) return CRYS_EINVAL;
  if (n == 0) return CRYS_OK;
  if (!x1 || !x2 || !y || !aligned16(x1) || !aligned16(x2) || !aligned16(y)) return CRYS_EINVAL;
  ProjectArgs args;
  args.x1 = x1;
  args.x2 = x2;
  args.n = n;
  args.a = a;
  args.b = b;
  args.y = y;
  args.err = device_error_word();
  if (!args.err) return CRYS_ECUDA;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  switch (tile_variant(kOp)) {
    case 1: return launch<kTiles[kOp][1].threads, kTiles[kOp][1].items>(args, op, s);
    case 2: return launch<kTiles[kOp][2].threads, kTiles[kOp][2].items>(args, op, s);
    case 3: return launch<kTiles[kOp][3].threads, kTiles[kOp][3].items>(args, op, s);
    default: return launch<kTiles[kOp][0].threads, kTiles[kOp][0].items>(args, op, s);
  }
}
