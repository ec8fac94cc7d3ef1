// Staged tile loading for the streaming kernels: each persistent thread block owns a
// ring of S shared-memory stages; thread 0 fills a stage with one bulk asynchronous
// copy (TMA) per column and the block consumes it after the stage's mbarrier phase
// completes.  This is the paper's BlockLoad (Section 3.3) with the copy engine doing
// the loads, so a block keeps S tiles in flight without spending registers on them.
//
// Stage reuse is ordered by __syncthreads: a stage is refilled only after every thread
// of the block has finished with it, so no "empty" barrier is needed.  Every wait is
// bounded; a block whose wait runs out abandons its work (uniformly, via
// __syncthreads_or) after draining the copies it still has in flight.
#pragma once

#include "common.cuh"

namespace crys {

constexpr int kMaxStages = 8;

// The number of stages S (2..kMaxStages) is chosen per launch by the host so that a
// block's stages fill its share of shared memory.
struct StageRing {
  uint64_t full[kMaxStages];  // completion barrier of each stage (1 arrival + tx bytes)
  int64_t tile[kMaxStages];   // tile held by each stage, -1 when none was issued
};

__device__ __forceinline__ void ring_init(StageRing& r, int S) {
  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&r.full[s], 1);
      r.tile[s] = -1;
    }
    fence_barrier_init();
  }
  __syncthreads();
}

// Thread 0: arms stage `bar` for `ncols` column slices of `valid` rows starting at
// `row` and issues the bulk copies.  Only whole 16-byte groups are copied; the last
// (valid % 4) rows of a ragged final tile are read by the consumers from global memory.
__device__ __forceinline__ void ring_issue(uint64_t* bar, int32_t* stage, int col_stride,
                                           const int32_t* const* cols, int ncols, int64_t row,
                                           int64_t valid, uint64_t policy) {
  const uint32_t bytes = static_cast<uint32_t>(valid / 4) * 16u;
  mbar_arrive_expect_tx(bar, bytes * static_cast<uint32_t>(ncols));
  if (bytes) {
    for (int c = 0; c < ncols; ++c)
      bulk_load(stage + c * col_stride, cols[c] + row, bytes, bar, policy);
  }
}

// All threads: waits for the stage of local iteration k.  Returns false in every thread
// when any thread's wait ran out.
__device__ __forceinline__ bool ring_wait(StageRing& r, int64_t k, int S, int32_t* err) {
  const bool ok = mbar_wait_bounded(&r.full[k % S], static_cast<uint32_t>((k / S) & 1), err);
  return !__syncthreads_or(!ok);
}

// Thread 0 after an abandoned iteration k: waits (bounded) for the copies of the
// iterations k .. k+S-1 that were issued, so no copy lands after the block exits.
__device__ __forceinline__ void ring_drain(StageRing& r, int64_t k, int S, int32_t* err) {
  for (int j = 0; j < S; ++j) {
    const int64_t kk = k + j;
    const int s = static_cast<int>(kk % S);
    if (r.tile[s] >= 0) mbar_wait_bounded(&r.full[s], static_cast<uint32_t>((kk / S) & 1), err);
  }
}

// Reads 4 consecutive values of a staged column slice at element p of a tile with
// `valid` rows of which the first `bulk` (valid rounded down to 4) were copied; rows
// past `bulk` come from global memory and rows past `valid` read as 0.
__device__ __forceinline__ int4 stage_read4(const int32_t* st, const int32_t* gcol, int p,
                                            int bulk, int valid) {
  if (p + 4 <= bulk) return *reinterpret_cast<const int4*>(st + p);
  int v[4];
#pragma unroll
  for (int e = 0; e < 4; ++e) v[e] = (p + e < bulk) ? st[p + e] : (p + e < valid ? gcol[p + e] : 0);
  return make_int4(v[0], v[1], v[2], v[3]);
}

}  // namespace crys
