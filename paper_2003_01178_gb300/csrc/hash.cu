// No-partitioning hash join (Section 4.3): build into a linear-probing table of 8-byte
// slots, and probe fused with SUM aggregation (query Q4).
//
// Probe kernel per tile: BlockLoad of the key and payload tiles (bulk copies into a
// shared-memory stage), BlockLookup with the first slot of every item loaded before any
// is resolved (ITEMS independent random reads in flight per thread), continuations past
// the home slots issued a probing step at a time for all items together, per-thread int64
// sums, and BlockAggregate once per persistent block (one atomic per block).  A table of
// at most 32 KB is first copied into each block's shared memory and probed there.
#include "common.cuh"
#include "pipeline.cuh"
#include "tiles.h"

namespace crys {
namespace {

constexpr int kMaxBuildFilters = 4;

__global__ void fill_empty_kernel(uint64_t* slots, int64_t n) {
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += stride)
    slots[i] = kEmptySlot;
}

struct BuildArgs {
  const int32_t* keys;
  const int32_t* vals;
  int64_t n;
  int32_t n_filters;
  crys_pred filters[kMaxBuildFilters];
  uint64_t* slots;
  HashFn hash;
  int32_t* err;
};

__global__ void __launch_bounds__(256) build_kernel(const __grid_constant__ BuildArgs a) {
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < a.n; i += stride) {
    bool keep = true;
    for (int f = 0; f < a.n_filters; ++f) {
      const int32_t v = a.filters[f].col[i];
      keep = keep && v >= a.filters[f].lo && v <= a.filters[f].hi;
    }
    if (!keep) continue;
    const int32_t key = a.keys[i];
    const int32_t val = a.vals ? a.vals[i] : 0;
    if (key == -1 || !hash_may_hold(key, a.hash)) {  // reserved, or outside a direct table
      set_error(a.err, CRYS_DEV_BAD_KEY);
      continue;
    }
    const uint64_t packed = static_cast<uint64_t>(static_cast<uint32_t>(key)) |
                            (static_cast<uint64_t>(static_cast<uint32_t>(val)) << 32);
    uint32_t h = hash_slot(key, a.hash);
    bool placed = false;
    for (uint32_t probe = 0; probe <= a.hash.steps; ++probe) {
      uint64_t cur = a.slots[h];
      if (cur == kEmptySlot) {
        cur = atomicCAS(reinterpret_cast<unsigned long long*>(a.slots + h), kEmptySlot, packed);
        if (cur == kEmptySlot) {
          placed = true;
          break;
        }
      }
      if (static_cast<uint32_t>(cur) == static_cast<uint32_t>(key)) {
        set_error(a.err, CRYS_DEV_DUP_KEY);
        placed = true;
        break;
      }
      h = (h + 1) & a.hash.mask;
    }
    if (!placed) set_error(a.err, CRYS_DEV_TABLE_FULL);
  }
}

struct ProbeArgs {
  const int32_t* fk;
  const int32_t* pay;
  int64_t n;
  const uint64_t* slots;
  HashFn hash;
  unsigned long long* sum;
  unsigned long long* matches;
  int32_t* err;
  int32_t stages;
  int32_t table_slots;  // SMEM_TABLE: the whole table, copied into shared memory
};

// A table of at most this many bytes is copied into every block's shared memory: random
// slot reads then cost shared-memory wavefronts instead of L1 tag lookups.
constexpr int64_t kSmemTableBytes = 32 * 1024;
static_assert(kSmemTableBytes / 8 <= kSmallHashSlots, "a table in shared memory hashes with one multiply");

template <int THREADS, int ITEMS, bool SMEM_TABLE>
__global__ void __launch_bounds__(THREADS) probe_kernel(ProbeArgs a) {
  constexpr int TILE = THREADS * ITEMS;
  constexpr int VEC = ITEMS / 4;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  int32_t* stages = reinterpret_cast<int32_t*>(smem_raw);  // per stage: fk tile, payload tile
  __shared__ StageRing ring;
  __shared__ uint64_t red[THREADS / kWarp];
  const int S = a.stages;

  const int tid = threadIdx.x;
  const int64_t ntiles = (a.n + TILE - 1) / TILE;
  const uint64_t pol = policy_evict_first();
  const uint64_t pol_table = policy_evict_last();
  const int32_t* cols[2] = {a.fk, a.pay};
  int64_t issued = 0;
  uint64_t sum = 0, matches = 0;

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
  uint64_t* tbl = reinterpret_cast<uint64_t*>(stages + S * 2 * TILE);
  if (SMEM_TABLE)
    for (int i = tid; i < a.table_slots; i += THREADS) tbl[i] = ld_slot(a.slots + i, pol_table);
  __syncthreads();
  // Linear probing continued in the shared-memory copy of the table.
  auto resolve_smem = [&](uint32_t h, uint64_t sl, int32_t key, int32_t* value) -> bool {
    for (uint32_t probe = 0;; ++probe) {
      if (sl == kEmptySlot) return false;
      if (static_cast<uint32_t>(sl) == static_cast<uint32_t>(key)) {
        *value = static_cast<int32_t>(sl >> 32);
        return true;
      }
      if (probe >= a.hash.steps) return false;
      h = (h + 1) & a.hash.mask;
      sl = tbl[h];
    }
  };

  bool aborted = false;
  for (int64_t k = 0;; ++k) {
    const int s = static_cast<int>(k % S);
    const int64_t t = ring.tile[s];
    if (t < 0) break;
    if (!ring_wait(ring, k, S, a.err)) {
      if (tid == 0) ring_drain(ring, k, S, a.err);
      aborted = true;
      break;
    }
    const int32_t* stk = stages + s * 2 * TILE;
    const int32_t* stp = stk + TILE;
    const int64_t row0 = t * TILE;
    const int valid = static_cast<int>((a.n - row0) < TILE ? (a.n - row0) : TILE);
    const int bulk = valid & ~3;
    int32_t key[ITEMS], pay[ITEMS];
    uint32_t live = 0;
    if (valid == TILE) {  // a full tile: the stage holds every row
#pragma unroll
      for (int j = 0; j < VEC; ++j) {
        const int p = (j * THREADS + tid) * 4;
        const int4 qk = *reinterpret_cast<const int4*>(stk + p);
        const int4 qp = *reinterpret_cast<const int4*>(stp + p);
        key[4 * j + 0] = qk.x; key[4 * j + 1] = qk.y; key[4 * j + 2] = qk.z; key[4 * j + 3] = qk.w;
        pay[4 * j + 0] = qp.x; pay[4 * j + 1] = qp.y; pay[4 * j + 2] = qp.z; pay[4 * j + 3] = qp.w;
      }
      live = ITEMS == 32 ? 0xFFFFFFFFu : ((1u << ITEMS) - 1u);
    } else {
#pragma unroll
      for (int j = 0; j < VEC; ++j) {
        const int p = (j * THREADS + tid) * 4;
        const int4 qk = stage_read4(stk, cols[0] + row0, p, bulk, valid);
        const int4 qp = stage_read4(stp, cols[1] + row0, p, bulk, valid);
        key[4 * j + 0] = qk.x; key[4 * j + 1] = qk.y; key[4 * j + 2] = qk.z; key[4 * j + 3] = qk.w;
        pay[4 * j + 0] = qp.x; pay[4 * j + 1] = qp.y; pay[4 * j + 2] = qp.z; pay[4 * j + 3] = qp.w;
#pragma unroll
        for (int e = 0; e < 4; ++e) live |= static_cast<uint32_t>(p + e < valid) << (4 * j + e);
      }
    }
    // BlockLookup: all first-slot reads issued before any is examined.
    uint32_t h[ITEMS];
    uint64_t slot[ITEMS];
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
      h[i] = SMEM_TABLE ? hash_slot_small(key[i], a.hash) : hash_slot(key[i], a.hash);
      const bool look = ((live >> i) & 1u) && hash_may_hold(key[i], a.hash);
      if (SMEM_TABLE)
        slot[i] = look ? tbl[h[i]] : kEmptySlot;
      else
        slot[i] = look ? ld_slot(a.slots + h[i], pol_table) : kEmptySlot;
    }
    if (SMEM_TABLE) {
#pragma unroll
      for (int i = 0; i < ITEMS; ++i) {
        int32_t value;
        if (((live >> i) & 1u) && resolve_smem(h[i], slot[i], key[i], &value)) {
          sum += static_cast<uint64_t>(static_cast<int64_t>(pay[i]) * static_cast<int64_t>(value));
          matches += 1;
        }
      }
    } else {
      // continuations past the home slot: one round trip per probing step for all items
      int32_t value[ITEMS];
      const uint32_t found = hash_resolve_all<ITEMS>(a.slots, a.hash, h, slot, key, live, value, pol_table);
#pragma unroll
      for (int i = 0; i < ITEMS; ++i)
        if ((found >> i) & 1u) {
          sum += static_cast<uint64_t>(static_cast<int64_t>(pay[i]) * static_cast<int64_t>(value[i]));
          matches += 1;
        }
    }
    __syncthreads();
    if (tid == 0) {
      fence_proxy_async_smem();
      issue(s);
    }
  }
  // BlockAggregate: one atomic per block for the sum and one for the match count.  A block
  // whose stage wait ran out (CRYS_DEV_TIMEOUT is set) still adds the rows it did finish,
  // so the partial result and the error flag arrive together.
  (void)aborted;
  const uint64_t bsum = block_sum_u64<THREADS>(sum, red);
  const uint64_t bmatch = block_sum_u64<THREADS>(matches, red);
  if (tid == 0) {
    if (bsum) atomicAdd(a.sum, static_cast<unsigned long long>(bsum));
    if (a.matches && bmatch) atomicAdd(a.matches, static_cast<unsigned long long>(bmatch));
  }
}

template <int THREADS, int ITEMS>
int launch_probe(ProbeArgs a, cudaStream_t s) {
  constexpr int TILE = THREADS * ITEMS;
  // Probes need warps more than deep staging, and a small table wants L1 left over:
  // two stages per block.
  a.stages = 2;
  const size_t stage_bytes = static_cast<size_t>(a.stages) * 2 * TILE * sizeof(int32_t);
  const int64_t ntiles = (a.n + TILE - 1) / TILE;
  if (a.table_slots > 0) {
    const size_t smem = stage_bytes + static_cast<size_t>(a.table_slots) * 8;
    auto k = probe_kernel<THREADS, ITEMS, true>;
    if (!allow_smem(k, smem)) return CRYS_ECUDA;
    k<<<persistent_grid(k, THREADS, smem, ntiles), THREADS, smem, s>>>(a);
  } else {
    auto k = probe_kernel<THREADS, ITEMS, false>;
    if (!allow_smem(k, stage_bytes)) return CRYS_ECUDA;
    k<<<persistent_grid(k, THREADS, stage_bytes, ntiles), THREADS, stage_bytes, s>>>(a);
  }
  note_launch();
  return check_launch();
}

bool valid_table(const crys_hash* ht) {
  if (!ht || !ht->slots || (reinterpret_cast<uintptr_t>(ht->slots) & 7u) != 0 || ht->capacity > (1ll << 31))
    return false;
  if (ht->kind == CRYS_HASH_DIRECT) return ht->capacity >= 1;
  return (ht->kind == CRYS_HASH_MULT || ht->kind == CRYS_HASH_IDENT) && is_pow2(ht->capacity) &&
         ht->capacity >= 2;
}

int grid_for(int64_t n, int threads) {
  const int64_t cap = static_cast<int64_t>(sm_count()) * 16;
  int64_t g = (n + threads - 1) / threads;
  if (g > cap) g = cap;
  return g < 1 ? 1 : static_cast<int>(g);
}

constexpr int kOp = CRYS_OP_PROBE;

}  // namespace
}  // namespace crys

extern "C" {

int crys_hash_init(const crys_hash* ht, crys_stream stream) {
  using namespace crys;
  if (!valid_table(ht)) return CRYS_EINVAL;
  fill_empty_kernel<<<grid_for(ht->capacity, 256), 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
      ht->slots, ht->capacity);
  note_launch();
  return check_launch();
}

int crys_hash_build(const int32_t* keys, const int32_t* vals, int64_t n, const crys_pred* filters,
                    int32_t n_filters, const crys_hash* ht, crys_stream stream) {
  using namespace crys;
  if (n < 0 || !valid_table(ht) || n_filters < 0 || n_filters > kMaxBuildFilters) return CRYS_EINVAL;
  if (n_filters > 0 && !filters) return CRYS_EINVAL;
  if (n == 0) return CRYS_OK;
  if (!keys) return CRYS_EINVAL;
  if (n_filters == 0 && ht->capacity < n) return CRYS_EFULL;
  BuildArgs a;
  a.keys = keys;
  a.vals = vals;
  a.n = n;
  a.n_filters = n_filters;
  for (int f = 0; f < n_filters; ++f) {
    if (!filters[f].col) return CRYS_EINVAL;
    a.filters[f] = filters[f];
  }
  a.slots = ht->slots;
  a.hash = make_hash(ht->kind, ht->capacity);
  a.err = device_error_word();
  if (!a.err) return CRYS_ECUDA;
  build_kernel<<<grid_for(n, 256), 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(a);
  note_launch();
  return check_launch();
}

int crys_probe_aggregate(const int32_t* fk, const int32_t* payload, int64_t n, const crys_hash* ht,
                         int64_t* d_sum, int64_t* d_matches, crys_stream stream) {
  using namespace crys;
  if (n < 0 || !valid_table(ht) || !d_sum) return CRYS_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (cudaMemsetAsync(d_sum, 0, sizeof(int64_t), s) != cudaSuccess) return CRYS_ECUDA;
  if (d_matches && cudaMemsetAsync(d_matches, 0, sizeof(int64_t), s) != cudaSuccess) return CRYS_ECUDA;
  if (n == 0) return CRYS_OK;
  if (!fk || !payload || !aligned16(fk) || !aligned16(payload)) return CRYS_EINVAL;
  ProbeArgs a;
  a.fk = fk;
  a.pay = payload;
  a.n = n;
  a.slots = ht->slots;
  a.hash = make_hash(ht->kind, ht->capacity);
  a.sum = reinterpret_cast<unsigned long long*>(d_sum);
  a.matches = reinterpret_cast<unsigned long long*>(d_matches);
  a.err = device_error_word();
  if (!a.err) return CRYS_ECUDA;
  a.table_slots = ht->capacity * 8 <= kSmemTableBytes ? static_cast<int32_t>(ht->capacity) : 0;
  switch (tile_variant(kOp)) {
    case 1: return launch_probe<kTiles[kOp][1].threads, kTiles[kOp][1].items>(a, s);
    case 2: return launch_probe<kTiles[kOp][2].threads, kTiles[kOp][2].items>(a, s);
    case 3: return launch_probe<kTiles[kOp][3].threads, kTiles[kOp][3].items>(a, s);
    default: return launch_probe<kTiles[kOp][0].threads, kTiles[kOp][0].items>(a, s);
  }
}

}  // extern "C"
