// Host-side internals shared by the operator translation units (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "crystal.h"

namespace crys {

// Device pointer of the calling device's sticky error word (see crys_device_errors).
int32_t* device_error_word();

// Counts one kernel launch of this library.
void note_launch(int kernels = 1);

// Number of SMs of the current device.
int sm_count();

// Current tile variant of an operator (index into its variant table).
int tile_variant(int op);

// The stall requested by crys_debug_stall for the next call of `op`, consumed by this
// call: tile ids start at *first_tile and look-back waits give up after *wait_ns.
// Without a request: 0 and the default bound.  Returns whether a request was taken.
bool take_stall(int op, uint32_t* first_tile, uint64_t* wait_ns);

inline bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

inline int check_launch() { return cudaGetLastError() == cudaSuccess ? CRYS_OK : CRYS_ECUDA; }

inline uint32_t log2_pow2(uint64_t v) {
  uint32_t r = 0;
  while ((1ull << r) < v) ++r;
  return r;
}

inline bool is_pow2(int64_t v) { return v > 0 && (v & (v - 1)) == 0; }

// Number of shared-memory stages for a streaming kernel: as many as fit in a block's
// share of the SM's shared memory when `blocks_per_sm` blocks are resident, between 2
// and 8 (the more tiles in flight per SM, the closer a scan gets to HBM bandwidth).
inline int stages_for(size_t stage_bytes, size_t extra_bytes, int blocks_per_sm) {
  const size_t per_block = (220u * 1024u) / static_cast<size_t>(blocks_per_sm > 0 ? blocks_per_sm : 1);
  const size_t room = per_block > extra_bytes ? per_block - extra_bytes : 0;
  size_t s = room / (stage_bytes > 0 ? stage_bytes : 1);
  if (s < 2) s = 2;
  if (s > 8) s = 8;
  return static_cast<int>(s);
}

// Resident blocks per SM of a kernel launched with `threads` threads and `smem` bytes of
// dynamic shared memory (the occupancy calculator), at least 1; remembered per device,
// kernel and launch shape, since a short launch cannot afford the query every time.
int blocks_per_sm(const void* kernel, int threads, size_t smem);

// Persistent grid: resident blocks per SM x SMs, capped by the number of tiles.
template <typename K>
int persistent_grid(K kernel, int threads, size_t smem, int64_t tiles) {
  const int per_sm = blocks_per_sm(reinterpret_cast<const void*>(kernel), threads, smem);
  int64_t g = static_cast<int64_t>(per_sm) * sm_count();
  if (tiles < g) g = tiles;
  return g < 1 ? 1 : static_cast<int>(g);
}

// Opts a kernel into `bytes` of dynamic shared memory.  Without the opt-in, static
// plus dynamic shared memory of a block is limited to 48 KB, so every kernel that
// takes dynamic shared memory sets the attribute (once per kernel and size).
bool set_dynamic_smem(const void* kernel, size_t bytes);

template <typename K>
bool allow_smem(K kernel, size_t bytes) {
  if (bytes == 0) return true;
  return set_dynamic_smem(reinterpret_cast<const void*>(kernel), bytes);
}

}  // namespace crys
