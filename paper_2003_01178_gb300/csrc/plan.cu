// Fused select-join-aggregate pipelines (Section 5.3; Figure "tile-extension"): after
// the dimension tables are built, ONE kernel streams the fact table in tiles and, per
// tile, applies the fact predicates (BlockPred), probes the dimension tables
// (BlockLookup), checks the dimension predicates on bit fields of the joined values,
// forms the group id and accumulates SUM(expr) and COUNT per group (BlockAggregate into
// per-block partials, flushed with one atomic per non-empty group and block).
//
// Kernels:
//  * plan_kernel        one query.  The copy engine prefetches each tile's columns into
//                       L2 a few tiles ahead (bulk prefetch), and the evaluation is
//                       branch-light: every column the query reads is loaded for every
//                       row and predicates only clear bits of a row bitmap.
//                       With few tiles per block, all of a tile's loads are issued
//                       before any value is used.
//  * shared_scan_kernel up to 32 queries over the same fact table: each tile of the
//                       union of their columns crosses HBM once, and each (foreign
//                       key, table) pair that several queries join through is probed
//                       once per row for all of them.  Serves batches with joins on
//                       tables that are not direct.
//  * annotate_kernel, tagged_scan_kernel (and the graph-replayable prepare_kernel,
//                       tagged_scan_kernel_dev) the shared scan over direct dimension
//                       tables with per-batch query bitmaps (see below).
#include "common.cuh"
#include "pipeline.cuh"
#include "tiles.h"

namespace crys {
namespace {

enum AccMode : int32_t { kAccSingle = 0, kAccShared = 1, kAccGlobal = 2 };
constexpr int kMaxProbes = 8;  // distinct (fk column, table) pairs probed once per batch

struct DevJoin {
  const uint64_t* slots;
  HashFn hash;
  int32_t fk_col;
  int32_t card;    // 0: not grouped
  int32_t stride;  // mixed-radix weight of this join's group code
  uint32_t gshift, gmask;
  int32_t n_fp;
  uint32_t fp_shift[CRYS_MAX_FIELD_PREDS], fp_mask[CRYS_MAX_FIELD_PREDS];
  int32_t fp_lo[CRYS_MAX_FIELD_PREDS], fp_hi[CRYS_MAX_FIELD_PREDS];
  uint32_t fp_span[CRYS_MAX_FIELD_PREDS];  // hi - lo (an empty range has mask 0, lo 1, span 0)
  int32_t probe;    // index of the batch-wide probe that serves this join, -1: probe here
  int32_t fk_slot;  // staged slice of fk_col (shared scan)
};

struct DevQuery {
  int32_t n_preds;
  int32_t pred_col[CRYS_MAX_PREDS];
  int32_t pred_lo[CRYS_MAX_PREDS];
  int32_t pred_hi[CRYS_MAX_PREDS];
  uint32_t pred_span[CRYS_MAX_PREDS];  // hi - lo
  int32_t pred_slot[CRYS_MAX_PREDS];   // staged slice of pred_col (shared scan)
  int32_t never;                       // an empty range: no row can qualify
  int32_t n_joins;
  DevJoin joins[CRYS_MAX_JOINS];
  int32_t agg_op, agg_a, agg_b;
  int32_t agg_a_slot, agg_b_slot;      // staged slices (shared scan)
  int32_t first_join;                  // shared scan: join tested on every row (-1: none)
  int32_t first_pred;                  // shared scan: fact predicate tested on every row (-1)
  int32_t acc_mode;
  int32_t acc_off;  // first shared-memory accumulator of this query
  int64_t groups;
  unsigned long long* sums;
  unsigned long long* counts;
};

// Bit field of a joined value: the whole value when the mask is all ones.
__device__ __forceinline__ int32_t field_of(int32_t v, uint32_t shift, uint32_t mask) {
  return static_cast<int32_t>((static_cast<uint32_t>(v) >> shift) & mask);
}

// Column access from global memory (plan_kernel).  Tiles start at multiples of 4 rows
// from a 4-row-aligned segment start, so full groups are 16-byte vector loads.
struct GlobalCols {
  const int32_t* const* cols;
  int64_t row0;
  int valid;
  uint64_t pol;
  __device__ __forceinline__ int4 load4(int c, int p) const {
    const int32_t* src = cols[c] + row0 + p;
    if (p + 4 <= valid) return ld_stream_v4(src, pol);
    int v[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) v[e] = p + e < valid ? ld_stream(src + e, pol) : 0;
    return make_int4(v[0], v[1], v[2], v[3]);
  }
};

// Column access for a tile known to be full: every 16-byte group exists.
struct FullTileCols {
  const int32_t* const* cols;
  int64_t row0;
  uint64_t pol;
  __device__ __forceinline__ int4 load4(int c, int p) const { return ld_stream_v4(cols[c] + row0 + p, pol); }
};

// Column loads that stay in L1: the columns a shared scan's queries read for predicates
// and aggregates are read by several queries of the batch in a row.  In L2 they are the
// first lines to go: the tile is not read again once its queries are done with it.
__device__ __forceinline__ int4 ld_cached_v4(const int32_t* p) {
  int4 v;
  asm volatile("ld.global.nc.L2::cache_hint.v4.s32 {%0,%1,%2,%3}, [%4], %5;"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "l"(p), "l"(policy_evict_first()));
  return v;
}
__device__ __forceinline__ int32_t ld_cached(const int32_t* p) {
  int32_t v;
  asm volatile("ld.global.nc.L2::cache_hint.s32 %0, [%1], %2;" : "=r"(v) : "l"(p), "l"(policy_evict_first()));
  return v;
}

struct CachedCols {
  const int32_t* const* cols;
  int64_t row0;
  int valid;
  __device__ __forceinline__ int4 load4(int c, int p) const {
    const int32_t* src = cols[c] + row0 + p;
    if (p + 4 <= valid) return ld_cached_v4(src);
    int v[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) v[e] = p + e < valid ? ld_cached(src + e) : 0;
    return make_int4(v[0], v[1], v[2], v[3]);
  }
};

__device__ __forceinline__ void unpack4(int4 q, int32_t* dst) {
  dst[0] = q.x;
  dst[1] = q.y;
  dst[2] = q.z;
  dst[3] = q.w;
}

// Probes one table for this thread's ITEMS rows: all first-slot reads are issued before
// any is resolved.  (Continuations go item by item here: resolving them together, as the
// probe kernel does, costs this kernel 20 more registers and half its resident blocks.)  Returns the bitmap of rows whose key was found; values in `value`.
template <int ITEMS>
__device__ __forceinline__ uint32_t probe_items(const uint64_t* slots, const HashFn& hf,
                                                const int32_t (&key)[ITEMS], uint32_t live,
                                                int32_t (&value)[ITEMS], uint64_t pol) {
  uint32_t h[ITEMS];
  uint64_t slot[ITEMS];
  if (hf.steps == 0u && hf.mult_hi == 1u && hf.mult_lo == 0u && hf.shift == 0u && hf.mask == 0xFFFFFFFFu) {
    // direct table (uniform branch): a key below the capacity is in slot `key` or
    // absent, one read per row
    uint32_t found = 0;
#pragma unroll
    for (int i = 0; i < ITEMS; ++i)
      slot[i] = ((live >> i) & 1u) && static_cast<uint32_t>(key[i]) < hf.limit ? ld_slot(slots + key[i], pol) : kEmptySlot;
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
      const bool hit = slot[i] != kEmptySlot && static_cast<uint32_t>(slot[i]) == static_cast<uint32_t>(key[i]);
      value[i] = hit ? static_cast<int32_t>(slot[i] >> 32) : 0;
      found |= static_cast<uint32_t>(hit) << i;
    }
    return found;
  }
#pragma unroll
  for (int i = 0; i < ITEMS; ++i) {
    h[i] = hash_slot(key[i], hf);
    slot[i] = ((live >> i) & 1u) && hash_may_hold(key[i], hf) ? ld_slot(slots + h[i], pol) : kEmptySlot;
  }
  uint32_t found = 0;
#pragma unroll
  for (int i = 0; i < ITEMS; ++i) {
    value[i] = 0;
    if (((live >> i) & 1u) && hash_resolve(slots, hf, h[i], slot[i], key[i], &value[i], pol))
      found |= 1u << i;
  }
  return found;
}

// Range test lo <= v <= hi as one unsigned comparison (span = hi - lo).
__device__ __forceinline__ bool in_span(int32_t v, int32_t lo, uint32_t span) {
  return static_cast<uint32_t>(v) - static_cast<uint32_t>(lo) <= span;
}

// Evaluation of one query of a shared scan on this thread's rows, cheapest tests first:
// (1) dimension predicates on values probed once for the batch (found bits, then bit
// fields of the 16-byte vectors of probed values; the join chosen on the host as most
// selective first), (2) fact predicates, (3) joins this query alone uses (probed now, for
// surviving rows only), (4) group codes and the aggregate, only while a row survives.
// Probed values for probe d, vector j of thread t at pv[(d * VEC + j) * THREADS + t];
// found bits at pf[d * THREADS + t].
template <int THREADS, int ITEMS>
__device__ __forceinline__ uint32_t eval_shared(const DevQuery& q, const CachedCols& cols, uint32_t alive,
                                                const int4* pv, const uint32_t* pf,
                                                int32_t (&gid)[ITEMS], int64_t (&val)[ITEMS],
                                                int32_t* err, uint64_t pol_table) {
  constexpr int VEC = ITEMS / 4;
  const int tid = threadIdx.x;
  if (q.never) return 0;
  // (1)
  for (int k = -1; k < q.n_joins && alive; ++k) {
    const int jn = k < 0 ? q.first_join : k;
    if (jn < 0 || (k >= 0 && jn == q.first_join)) continue;
    const DevJoin& J = q.joins[jn];
    if (J.probe < 0) continue;
    alive &= pf[J.probe * THREADS + tid];
    for (int f = 0; f < J.n_fp && alive; ++f) {
      const uint32_t sh = J.fp_shift[f], mk = J.fp_mask[f], span = J.fp_span[f];
      const int32_t lo = J.fp_lo[f];
#pragma unroll
      for (int j = 0; j < VEC; ++j) {
        const int4 v4 = pv[(J.probe * VEC + j) * THREADS + tid];
        const int32_t v[4] = {v4.x, v4.y, v4.z, v4.w};
#pragma unroll
        for (int e = 0; e < 4; ++e)
          if (!in_span(field_of(v[e], sh, mk), lo, span)) alive &= ~(1u << (4 * j + e));
      }
    }
  }
  // (2)
  for (int f = 0; f < q.n_preds && alive; ++f) {
    const int c = q.pred_col[f];
    const int32_t lo = q.pred_lo[f];
    const uint32_t span = q.pred_span[f];
#pragma unroll
    for (int j = 0; j < VEC; ++j) {
      if (!((alive >> (4 * j)) & 0xFu)) continue;
      int32_t v[4];
      unpack4(cols.load4(c, (j * THREADS + tid) * 4), v);
#pragma unroll
      for (int e = 0; e < 4; ++e)
        if (!in_span(v[e], lo, span)) alive &= ~(1u << (4 * j + e));
    }
  }
  if (!alive) return 0;
#pragma unroll
  for (int i = 0; i < ITEMS; ++i) gid[i] = 0;
  // (3) joins served by no batch-wide probe
  for (int jn = 0; jn < q.n_joins && alive; ++jn) {
    const DevJoin& J = q.joins[jn];
    if (J.probe >= 0) continue;
    int32_t key[ITEMS], value[ITEMS];
#pragma unroll
    for (int j = 0; j < VEC; ++j) {
      if ((alive >> (4 * j)) & 0xFu)
        unpack4(cols.load4(J.fk_col, (j * THREADS + tid) * 4), key + 4 * j);
      else
        key[4 * j] = key[4 * j + 1] = key[4 * j + 2] = key[4 * j + 3] = 0;
    }
    alive &= probe_items<ITEMS>(J.slots, J.hash, key, alive, value, pol_table);
    for (int f = 0; f < J.n_fp; ++f) {
#pragma unroll
      for (int i = 0; i < ITEMS; ++i)
        if (!in_span(field_of(value[i], J.fp_shift[f], J.fp_mask[f]), J.fp_lo[f], J.fp_span[f]))
          alive &= ~(1u << i);
    }
    if (J.card > 0) {
#pragma unroll
      for (int i = 0; i < ITEMS; ++i) {
        const uint32_t code = static_cast<uint32_t>(field_of(value[i], J.gshift, J.gmask));
        if (((alive >> i) & 1u) && code >= static_cast<uint32_t>(J.card)) {
          set_error(err, CRYS_DEV_BAD_GROUP);
          alive &= ~(1u << i);
        }
        gid[i] += static_cast<int32_t>(code) * J.stride;
      }
    }
  }
  if (!alive) return 0;
  // (4)
  for (int jn = 0; jn < q.n_joins; ++jn) {
    const DevJoin& J = q.joins[jn];
    if (J.probe < 0 || J.card <= 0) continue;
    const uint32_t card = static_cast<uint32_t>(J.card);
#pragma unroll
    for (int j = 0; j < VEC; ++j) {
      const int4 v4 = pv[(J.probe * VEC + j) * THREADS + tid];
      const int32_t v[4] = {v4.x, v4.y, v4.z, v4.w};
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int i = 4 * j + e;
        const uint32_t code = static_cast<uint32_t>(field_of(v[e], J.gshift, J.gmask));
        if (((alive >> i) & 1u) && code >= card) {
          set_error(err, CRYS_DEV_BAD_GROUP);
          alive &= ~(1u << i);
        }
        gid[i] += static_cast<int32_t>(code) * J.stride;
      }
    }
  }
#pragma unroll
  for (int j = 0; j < VEC; ++j) {
    if (!((alive >> (4 * j)) & 0xFu)) continue;
    const int p = (j * THREADS + tid) * 4;
    int32_t va[4], vb[4] = {0, 0, 0, 0};
    unpack4(cols.load4(q.agg_a, p), va);
    if (q.agg_op != CRYS_AGG_A) unpack4(cols.load4(q.agg_b, p), vb);
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int64_t x = va[e], y = vb[e];
      int64_t r;
      switch (q.agg_op) {
        case CRYS_AGG_A_MUL_B: r = x * y; break;
        case CRYS_AGG_A_SUB_B: r = x - y; break;
        case CRYS_AGG_A_ADD_B: r = x + y; break;
        default: r = x; break;
      }
      val[4 * j + e] = r;
    }
  }
  return alive;
}

// Branch-light evaluation of one query on this thread's rows for plan_kernel.  The
// tile's columns are already on their way to L2 (bulk prefetch), so every column the
// query reads is loaded for all rows (no selective loads and no per-group branches);
// predicates only clear bits of the row bitmap and dead rows contribute 0.
template <int THREADS, int ITEMS, bool SEL = false>
__device__ __forceinline__ uint32_t eval_eager_loop(const DevQuery& q, const GlobalCols& cols, uint32_t alive,
                                               int32_t (&gid)[ITEMS], int64_t (&val)[ITEMS],
                                               int32_t* err, uint64_t pol_table) {
  constexpr int VEC = ITEMS / 4;
  const int tid = threadIdx.x;
  for (int f = 0; f < q.n_preds; ++f) {
    const int c = q.pred_col[f];
    const int32_t lo = q.pred_lo[f];
    const uint32_t span = q.pred_span[f];
#pragma unroll
    for (int j = 0; j < VEC; ++j) {
      int32_t v[4];
      unpack4(cols.load4(c, (j * THREADS + tid) * 4), v);
#pragma unroll
      for (int e = 0; e < 4; ++e) alive &= ~(static_cast<uint32_t>(!in_span(v[e], lo, span)) << (4 * j + e));
    }
  }
#pragma unroll
  for (int i = 0; i < ITEMS; ++i) gid[i] = 0;
  for (int jn = 0; jn < q.n_joins; ++jn) {
    const DevJoin& J = q.joins[jn];
    int32_t key[ITEMS], value[ITEMS];
#pragma unroll
    for (int j = 0; j < VEC; ++j) unpack4(cols.load4(J.fk_col, (j * THREADS + tid) * 4), key + 4 * j);
    alive &= probe_items<ITEMS>(J.slots, J.hash, key, alive, value, pol_table);
    for (int f = 0; f < J.n_fp; ++f) {
      const uint32_t sh = J.fp_shift[f], mk = J.fp_mask[f], span = J.fp_span[f];
      const int32_t lo = J.fp_lo[f];
#pragma unroll
      for (int i = 0; i < ITEMS; ++i)
        alive &= ~(static_cast<uint32_t>(!in_span(field_of(value[i], sh, mk), lo, span)) << i);
    }
    if (J.card > 0) {
      const uint32_t card = static_cast<uint32_t>(J.card);
      uint32_t bad = 0;
#pragma unroll
      for (int i = 0; i < ITEMS; ++i) {
        const uint32_t code = static_cast<uint32_t>(field_of(value[i], J.gshift, J.gmask));
        bad |= static_cast<uint32_t>(code >= card) << i;
        gid[i] += static_cast<int32_t>(code) * J.stride;
      }
      bad &= alive;
      if (bad) {
        set_error(err, CRYS_DEV_BAD_GROUP);
        alive &= ~bad;
      }
    }
  }
  // the aggregate operands; with SEL a 16-byte group with no live row is not read
  // (selective load: the Section 5.3 model's later-column term, one line per surviving
  // row at most), otherwise every group is read and the loads can go out early
#pragma unroll
  for (int j = 0; j < VEC; ++j) {
    const int p = (j * THREADS + tid) * 4;
    int32_t va[4] = {0, 0, 0, 0}, vb[4] = {0, 0, 0, 0};
    if (!SEL || ((alive >> (4 * j)) & 0xFu)) {
      unpack4(cols.load4(q.agg_a, p), va);
      if (q.agg_op != CRYS_AGG_A) unpack4(cols.load4(q.agg_b, p), vb);
    }
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int64_t x = va[e], y = vb[e];
      int64_t r;
      switch (q.agg_op) {
        case CRYS_AGG_A_MUL_B: r = x * y; break;
        case CRYS_AGG_A_SUB_B: r = x - y; break;
        case CRYS_AGG_A_ADD_B: r = x + y; break;
        default: r = x; break;
      }
      val[4 * j + e] = ((alive >> (4 * j + e)) & 1u) ? r : 0;
    }
  }
  return alive;
}

// The column vectors of one tile that go out before any is used: up to two fact
// predicates, up to two joins' foreign keys and the aggregate operands.
template <int ITEMS>
struct TileVectors {
  static constexpr int VEC = ITEMS / 4;
  static constexpr int KP = 2;  // fact predicates whose columns go out up front
  static constexpr int KJ = 2;  // joins whose keys go out up front
  int4 pv[KP][VEC], kv[KJ][VEC], av[VEC], bv[VEC];
};

template <int THREADS, int ITEMS, typename Cols>
__device__ __forceinline__ void load_tile_vectors(const DevQuery& q, const Cols& cols, TileVectors<ITEMS>& r) {
  using R = TileVectors<ITEMS>;
  const int tid = static_cast<int>(threadIdx.x);
#pragma unroll
  for (int j = 0; j < R::VEC; ++j) {
    const int p = (j * THREADS + tid) * 4;
#pragma unroll
    for (int f = 0; f < R::KP; ++f) r.pv[f][j] = f < q.n_preds ? cols.load4(q.pred_col[f], p) : make_int4(0, 0, 0, 0);
#pragma unroll
    for (int jn = 0; jn < R::KJ; ++jn)
      r.kv[jn][j] = jn < q.n_joins ? cols.load4(q.joins[jn].fk_col, p) : make_int4(0, 0, 0, 0);
    r.av[j] = cols.load4(q.agg_a, p);
    r.bv[j] = q.agg_op != CRYS_AGG_A ? cols.load4(q.agg_b, p) : make_int4(0, 0, 0, 0);
  }
}

// Evaluation of a tile whose leading column vectors are already in registers.
template <int THREADS, int ITEMS, typename Cols>
__device__ __forceinline__ uint32_t eval_tile_vectors(const DevQuery& q, const Cols& cols,
                                                      const TileVectors<ITEMS>& tv, uint32_t alive,
                                                      int32_t (&gid)[ITEMS], int64_t (&val)[ITEMS],
                                                      int32_t* err, uint64_t pol_table) {
  static_assert(ITEMS == 4 || ITEMS == 8, "one or two 16-byte vectors per column and thread");
  constexpr int VEC = ITEMS / 4;
  constexpr int KP = TileVectors<ITEMS>::KP;
  constexpr int KJ = TileVectors<ITEMS>::KJ;
  const int tid = static_cast<int>(threadIdx.x);
  const auto& pv = tv.pv;
  const auto& kv = tv.kv;
  const auto& av = tv.av;
  const auto& bv = tv.bv;
  auto pred = [&](const int32_t (&v)[ITEMS], int32_t lo, uint32_t span) {
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) alive &= ~(static_cast<uint32_t>(!in_span(v[i], lo, span)) << i);
  };
#pragma unroll
  for (int f = 0; f < KP; ++f) {
    if (f >= q.n_preds) break;
    int32_t v[ITEMS];
#pragma unroll
    for (int j = 0; j < VEC; ++j) unpack4(pv[f][j], v + 4 * j);
    pred(v, q.pred_lo[f], q.pred_span[f]);
  }
  for (int f = KP; f < q.n_preds; ++f) {
    int32_t v[ITEMS];
#pragma unroll
    for (int j = 0; j < VEC; ++j) unpack4(cols.load4(q.pred_col[f], (j * THREADS + tid) * 4), v + 4 * j);
    pred(v, q.pred_lo[f], q.pred_span[f]);
  }
#pragma unroll
  for (int i = 0; i < ITEMS; ++i) gid[i] = 0;
#pragma unroll
  for (int jn = 0; jn < CRYS_MAX_JOINS; ++jn) {
    if (jn >= q.n_joins) break;
    const DevJoin& J = q.joins[jn];
    int32_t key[ITEMS], value[ITEMS];
#pragma unroll
    for (int j = 0; j < VEC; ++j) {
      if (jn < KJ) unpack4(kv[jn < KJ ? jn : 0][j], key + 4 * j);
      else unpack4(cols.load4(J.fk_col, (j * THREADS + tid) * 4), key + 4 * j);
    }
    alive &= probe_items<ITEMS>(J.slots, J.hash, key, alive, value, pol_table);
    for (int f = 0; f < J.n_fp; ++f) {
      const uint32_t sh = J.fp_shift[f], mk = J.fp_mask[f], span = J.fp_span[f];
      const int32_t lo = J.fp_lo[f];
#pragma unroll
      for (int i = 0; i < ITEMS; ++i)
        alive &= ~(static_cast<uint32_t>(!in_span(field_of(value[i], sh, mk), lo, span)) << i);
    }
    if (J.card > 0) {
      const uint32_t card = static_cast<uint32_t>(J.card);
      uint32_t bad = 0;
#pragma unroll
      for (int i = 0; i < ITEMS; ++i) {
        const uint32_t code = static_cast<uint32_t>(field_of(value[i], J.gshift, J.gmask));
        bad |= static_cast<uint32_t>(code >= card) << i;
        gid[i] += static_cast<int32_t>(code) * J.stride;
      }
      bad &= alive;
      if (bad) {
        set_error(err, CRYS_DEV_BAD_GROUP);
        alive &= ~bad;
      }
    }
  }
#pragma unroll
  for (int j = 0; j < VEC; ++j) {
    int32_t va[4], vb[4];
    unpack4(av[j], va);
    unpack4(bv[j], vb);
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int64_t x = va[e], y = vb[e];
      int64_t r;
      switch (q.agg_op) {
        case CRYS_AGG_A_MUL_B: r = x * y; break;
        case CRYS_AGG_A_SUB_B: r = x - y; break;
        case CRYS_AGG_A_ADD_B: r = x + y; break;
        default: r = x; break;
      }
      val[4 * j + e] = ((alive >> (4 * j + e)) & 1u) ? r : 0;
    }
  }
  return alive;
}

// The same evaluation with every leading column load of the tile issued before any value
// is used, so that one L2 round trip serves the tile instead of one per step; for tiles
// of 4 or 8 rows per thread, where the loaded vectors fit in registers.
template <int THREADS, int ITEMS>
__device__ __forceinline__ uint32_t eval_eager_preload(const DevQuery& q, const GlobalCols& cols, uint32_t alive,
                                                       int32_t (&gid)[ITEMS], int64_t (&val)[ITEMS],
                                                       int32_t* err, uint64_t pol_table) {
  TileVectors<ITEMS> r;
  load_tile_vectors<THREADS, ITEMS>(q, cols, r);
  return eval_tile_vectors<THREADS, ITEMS>(q, cols, r, alive, gid, val, err, pol_table);
}

template <int THREADS, int ITEMS, bool PRELOAD>
__device__ __forceinline__ uint32_t eval_eager(const DevQuery& q, const GlobalCols& cols, uint32_t alive,
                                               int32_t (&gid)[ITEMS], int64_t (&val)[ITEMS],
                                               int32_t* err, uint64_t pol_table) {
  if constexpr (PRELOAD && (ITEMS == 4 || ITEMS == 8)) {
    return eval_eager_preload<THREADS, ITEMS>(q, cols, alive, gid, val, err, pol_table);
  } else {
    return eval_eager_loop<THREADS, ITEMS>(q, cols, alive, gid, val, err, pol_table);
  }
}

// Rows of this thread that exist in a tile with `valid` rows.
template <int THREADS, int ITEMS>
__device__ __forceinline__ uint32_t rows_present(int valid) {
  constexpr int VEC = ITEMS / 4;
  uint32_t live = 0;
#pragma unroll
  for (int j = 0; j < VEC; ++j) {
    const int p = (j * THREADS + static_cast<int>(threadIdx.x)) * 4;
#pragma unroll
    for (int e = 0; e < 4; ++e) live |= static_cast<uint32_t>(p + e < valid) << (4 * j + e);
  }
  return live;
}

// Accumulator shared memory of a block: sums (8 B) then counts (4 B) per group.
struct SharedAcc {
  unsigned long long* sums;
  unsigned int* counts;
};

// 64-bit add to a shared-memory accumulator made of 32-bit atomics (the low word comes
// first: the GPU is little-endian).  The add to the low word returns its previous value,
// which tells whether it carried; the high word then receives the value's high half plus
// that carry (skipped when both are zero).  Every carry is counted by the add that made
// it, so the two words hold the exact sum modulo 2^64 once all adds are done.  On sm_103a
// this measured faster than the 64-bit shared-memory atomic.
__device__ __forceinline__ void shared_add_u64(unsigned long long* p, unsigned long long v) {
  const uint32_t lo = static_cast<uint32_t>(v), hi = static_cast<uint32_t>(v >> 32);
  uint32_t* w = reinterpret_cast<uint32_t*>(p);
  const uint32_t old = atomicAdd(w, lo);
  const uint32_t up = hi + (old + lo < old ? 1u : 0u);
  if (up) atomicAdd(w + 1, up);
}

__device__ __forceinline__ SharedAcc shared_acc(unsigned char* base, int groups) {
  SharedAcc s;
  s.sums = reinterpret_cast<unsigned long long*>(base);
  s.counts = reinterpret_cast<unsigned int*>(base + static_cast<size_t>(groups) * 8);
  return s;
}

template <int THREADS>
__device__ __forceinline__ void flush_shared(const SharedAcc& acc, int first, int64_t groups,
                                             unsigned long long* sums, unsigned long long* counts) {
  for (int64_t g = threadIdx.x; g < groups; g += THREADS) {
    const unsigned int c = acc.counts[first + g];
    if (c) {
      atomicAdd(sums + g, acc.sums[first + g]);
      if (counts) atomicAdd(counts + g, static_cast<unsigned long long>(c));
    }
  }
}

// ------------------------------------------------------------------ one query

// Programmatic dependent launch: the query kernel is launched while the kernel that
// clears its outputs still runs, and waits for that kernel (its completion and its
// stores) only where it first touches the outputs; without a programmatic launch the
// wait returns at once.
__device__ __forceinline__ void wait_for_prerequisite_grid() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Clears a query's sums and counts; lets the dependent query kernel start right away.
__global__ void __launch_bounds__(256) zero_outputs_kernel(unsigned long long* sums, unsigned long long* counts,
                                                           int64_t groups) {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t g = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; g < groups; g += stride) {
    sums[g] = 0;
    if (counts) counts[g] = 0;
  }
}

struct PlanArgs {
  const int32_t* cols[CRYS_MAX_COLS];
  int64_t row_begin, row_end;
  DevQuery q;
  int32_t* err;
  uint32_t col_mask;   // fact columns the query reads
  uint32_t late_mask;  // columns read only by the aggregate (selective loads, see plan_kernel)
};

// Thread 0 asks the copy engine to bring tile `t` of every column in `mask` into L2
// (one bulk prefetch per column slice), so that the dependent loads of a later
// iteration (predicate -> key -> probe -> aggregate) each wait for L2 instead of HBM.
__device__ __forceinline__ void prefetch_tile(const int32_t* const* cols, uint32_t mask, int64_t row_begin,
                                              int64_t t, int64_t tile, int64_t nrows) {
  const int64_t row0 = row_begin + t * tile;
  const int64_t valid = (nrows - t * tile) < tile ? (nrows - t * tile) : tile;
  const uint32_t bytes = static_cast<uint32_t>(valid / 4) * 16u;
  if (!bytes) return;
  for (uint32_t m = mask; m; m &= m - 1) bulk_prefetch_l2(cols[__ffs(m) - 1] + row0, bytes);
}

constexpr int kPrefetchTiles = 2;  // tiles of a block prefetched ahead of the one in work
constexpr int kTagPrefetchTiles = 1;  // the same for the tagged scan, whose tiles stay in work longer

template <int THREADS, int ITEMS, bool PRELOAD>
__global__ void __launch_bounds__(THREADS) plan_kernel(const __grid_constant__ PlanArgs a) {
  constexpr int TILE = THREADS * ITEMS;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ uint64_t red[THREADS / kWarp];
  const DevQuery& q = a.q;
  const int groups_sh = q.acc_mode == kAccShared ? static_cast<int>(q.groups) : 0;
  const SharedAcc acc = shared_acc(smem_raw, groups_sh);
  for (int g = threadIdx.x; g < groups_sh; g += THREADS) {
    acc.sums[g] = 0;
    acc.counts[g] = 0;
  }
  __syncthreads();

  const int64_t nrows = a.row_end - a.row_begin;
  const int64_t ntiles = (nrows + TILE - 1) / TILE;
  uint64_t my_sum = 0, my_count = 0;
  if (q.acc_mode == kAccGlobal) wait_for_prerequisite_grid();  // adds go to the outputs from the first tile on
  const uint64_t pol = policy_evict_first();
  const uint64_t pol_table = policy_evict_last();
  if (threadIdx.x == 0)
    for (int d = 0; d < kPrefetchTiles; ++d) {
      const int64_t tt = blockIdx.x + static_cast<int64_t>(d) * gridDim.x;
      if (tt < ntiles) prefetch_tile(a.cols, a.col_mask, a.row_begin, tt, TILE, nrows);
    }
  // Selective loads of the late columns (read by the aggregate only): every warp counts
  // the 128-byte lines of those columns its live rows needed (an L2 miss fills a whole
  // line, so a line is saved only when all its 32 rows failed).  Once fewer than a third
  // were needed, the warp reads them for live 16-byte groups only, and thread 0 stops
  // prefetching them into L2 (by warp 0's counts), so their dead lines stay in DRAM.
  auto tile_cols = [&](int64_t t) {
    GlobalCols c;
    c.pol = pol;
    c.cols = a.cols;
    c.row0 = a.row_begin + t * TILE;
    c.valid = static_cast<int>((nrows - t * TILE) < TILE ? (nrows - t * TILE) : TILE);
    return c;
  };
  // BlockAggregate of one tile's rows into this thread's sums or the accumulators
  auto accumulate = [&](uint32_t alive, const int32_t (&gid)[ITEMS], const int64_t (&val)[ITEMS]) {
    if (q.acc_mode == kAccSingle) {
#pragma unroll
      for (int i = 0; i < ITEMS; ++i) my_sum += static_cast<uint64_t>(val[i]);
      my_count += __popc(alive);
      return;
    }
    if (!alive) return;
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
      if (!((alive >> i) & 1u)) continue;
      if (q.acc_mode == kAccShared) {
        shared_add_u64(acc.sums + gid[i], static_cast<unsigned long long>(val[i]));
        atomicAdd(acc.counts + gid[i], 1u);
      } else {
        red_add_global(q.sums + gid[i], static_cast<unsigned long long>(val[i]), pol_table);
        if (q.counts) red_add_global(q.counts + gid[i], 1ull, pol_table);
      }
    }
  };
  if constexpr (PRELOAD && ITEMS == 4) {
    // A software pipeline: the next tile's leading column vectors are loaded into
    // registers before this tile is evaluated, so that their latency overlaps the
    // evaluation instead of every warp of the SM waiting on its loads and then computing
    // in step with the others.
    // Full tiles (all but possibly the last) load without per-group bounds tests.
    auto full_cols = [&](const GlobalCols& c) { return FullTileCols{c.cols, c.row0, c.pol}; };
    auto load = [&](int64_t tt, TileVectors<ITEMS>& r) {
      const GlobalCols c = tile_cols(tt);
      if (c.valid == TILE)
        load_tile_vectors<THREADS, ITEMS>(q, full_cols(c), r);
      else
        load_tile_vectors<THREADS, ITEMS>(q, c, r);
    };
    TileVectors<ITEMS> cur, nxt;
    int64_t t = blockIdx.x;
    if (t < ntiles && !q.never) load(t, cur);
    for (; t < ntiles; t += gridDim.x) {
      const int64_t ahead = t + static_cast<int64_t>(kPrefetchTiles) * gridDim.x;
      if (threadIdx.x == 0 && ahead < ntiles) prefetch_tile(a.cols, a.col_mask, a.row_begin, ahead, TILE, nrows);
      const GlobalCols cols = tile_cols(t);
      const int64_t tn = t + gridDim.x;
      if (tn < ntiles && !q.never) load(tn, nxt);
      int32_t gid[ITEMS];
      int64_t val[ITEMS];
#pragma unroll
      for (int i = 0; i < ITEMS; ++i) {
        gid[i] = 0;
        val[i] = 0;
      }
      uint32_t alive = 0;
      if (!q.never) {
        if (cols.valid == TILE)
          alive = eval_tile_vectors<THREADS, ITEMS>(q, full_cols(cols), cur, (1u << ITEMS) - 1u, gid, val, a.err,
                                                    pol_table);
        else
          alive = eval_tile_vectors<THREADS, ITEMS>(q, cols, cur, rows_present<THREADS, ITEMS>(cols.valid), gid, val,
                                                    a.err, pol_table);
      }
      accumulate(alive, gid, val);
      cur = nxt;
    }
  } else {
    uint32_t need_lines = 0, seen_lines = 0;
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
      const bool sparse = a.late_mask && seen_lines >= 64u && 3u * need_lines < seen_lines;
      const int64_t ahead = t + static_cast<int64_t>(kPrefetchTiles) * gridDim.x;
      if (threadIdx.x == 0 && ahead < ntiles)
        prefetch_tile(a.cols, sparse ? (a.col_mask & ~a.late_mask) : a.col_mask, a.row_begin, ahead, TILE, nrows);
      const GlobalCols cols = tile_cols(t);
      int32_t gid[ITEMS];
      int64_t val[ITEMS];
      uint32_t alive = 0;
      if (!q.never) {
        const uint32_t present = rows_present<THREADS, ITEMS>(cols.valid);
        if (PRELOAD || !sparse)
          alive = eval_eager<THREADS, ITEMS, PRELOAD>(q, cols, present, gid, val, a.err, pol_table);
        else
          alive = eval_eager_loop<THREADS, ITEMS, true>(q, cols, present, gid, val, a.err, pol_table);
      }
      if (!PRELOAD && a.late_mask) {
#pragma unroll
        for (int j = 0; j < ITEMS / 4; ++j) {
          // lanes 8m .. 8m+7 read the 16-byte groups of 128-byte line m of the warp's 512 bytes
          const uint32_t b = __ballot_sync(0xFFFFFFFFu, ((alive >> (4 * j)) & 0xFu) != 0u);
          need_lines += static_cast<uint32_t>((b & 0xFFu) != 0) + ((b & 0xFF00u) != 0) + ((b & 0xFF0000u) != 0) +
                        ((b & 0xFF000000u) != 0);
          seen_lines += 4u;
        }
      }
      accumulate(alive, gid, val);
    }
  }
  if (q.acc_mode == kAccSingle) {
    const uint64_t s = block_sum_u64<THREADS>(my_sum, red);
    const uint64_t c = block_sum_u64<THREADS>(my_count, red);
    if (threadIdx.x == 0 && c) {
      wait_for_prerequisite_grid();
      atomicAdd(q.sums, static_cast<unsigned long long>(s));
      if (q.counts) atomicAdd(q.counts, static_cast<unsigned long long>(c));
    }
  } else if (q.acc_mode == kAccShared) {
    __syncthreads();
    wait_for_prerequisite_grid();
    flush_shared<THREADS>(acc, 0, q.groups, q.sums, q.counts);
  }
}

// ------------------------------------------------------------------ one query, fixed shape
//
// Plans of the Q1 family (Section 5.3's query 1.x: one or two fact predicates, one join on
// a direct dimension table with its field predicates, one output group, SUM(a * b) or
// SUM(a)) compiled for their shape: no loops over plan fields, no switch on the aggregate,
// full tiles without bounds tests, and the next tile's column vectors in flight while the
// current one is evaluated.
//
// Selective loads (Section 3.3's BlockLoadSel): every warp counts the 128-byte lines of the
// aggregate-only ("late") columns that its live rows needed (an L2 miss fills a whole
// line, so a line is saved only when all of its 32 rows failed).  Once fewer than a third
// were needed, the warp stops loading those columns ahead and reads them after the
// predicates and the probe, for the 16-byte groups with a live row only; thread 0 stops
// prefetching them into L2 (by warp 0's counts), so their dead lines stay in DRAM.  Only
// the 4-row shapes carry this: with 8-row items its registers cost the dense case 5% (Q1
// at 2^28 rows), so the tile-shape tuner picks between a selective 4-row and a plain 8-row
// kernel per workload.
template <int THREADS, int ITEMS, int NP, int AGG>
__global__ void __launch_bounds__(THREADS) plan_fixed_kernel(const __grid_constant__ PlanArgs a) {
  static_assert(ITEMS == 4 || ITEMS == 8, "one or two 16-byte vectors per column and thread");
  static_assert(NP >= 1 && NP <= 2, "one or two fact predicates");
  constexpr int TILE = THREADS * ITEMS;
  constexpr int VEC = ITEMS / 4;
  constexpr bool TWO = AGG != CRYS_AGG_A;  // the aggregate reads a second column
  __shared__ uint64_t red[THREADS / kWarp];
  const DevQuery& q = a.q;
  const DevJoin& J = q.joins[0];
  const int tid = static_cast<int>(threadIdx.x);
  const int64_t nrows = a.row_end - a.row_begin;
  const int64_t ntiles = (nrows + TILE - 1) / TILE;
  const uint64_t pol = policy_evict_first();
  const uint64_t pol_table = policy_evict_last();
  const int32_t* pcol[NP];
#pragma unroll
  for (int f = 0; f < NP; ++f) pcol[f] = a.cols[q.pred_col[f]] + a.row_begin;
  const int32_t* kcol = a.cols[J.fk_col] + a.row_begin;
  const int32_t* xcol = a.cols[q.agg_a] + a.row_begin;
  const int32_t* ycol = a.cols[TWO ? q.agg_b : q.agg_a] + a.row_begin;
  constexpr bool SELECTIVE = ITEMS == 4;
  const uint32_t late_mask = SELECTIVE ? a.late_mask : 0u;
  const bool x_late = (late_mask >> q.agg_a) & 1u;
  const bool y_late = TWO && ((late_mask >> q.agg_b) & 1u);
  struct Vecs {
    int4 p[NP][VEC], k[VEC], x[VEC], y[VEC];
    bool sel;  // the late columns were not loaded ahead
  };
  auto load4 = [&](const int32_t* col, int64_t row0, int p, int valid) -> int4 {
    if (p + 4 <= valid) return ld_stream_v4(col + row0 + p, pol);
    int v[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) v[e] = p + e < valid ? ld_stream(col + row0 + p + e, pol) : 0;
    return make_int4(v[0], v[1], v[2], v[3]);
  };
  auto load = [&](int64_t t, Vecs& V, bool sparse) {
    const int64_t row0 = t * TILE;
    const int valid = static_cast<int>((nrows - row0) < TILE ? (nrows - row0) : TILE);
    V.sel = sparse;
    const bool lx = !(sparse && x_late), ly = TWO && !(sparse && y_late);
#pragma unroll
    for (int j = 0; j < VEC; ++j) {
      const int p = (j * THREADS + tid) * 4;
      V.x[j] = make_int4(0, 0, 0, 0);
      V.y[j] = make_int4(0, 0, 0, 0);
      if (valid == TILE) {
#pragma unroll
        for (int f = 0; f < NP; ++f) V.p[f][j] = ld_stream_v4(pcol[f] + row0 + p, pol);
        V.k[j] = ld_stream_v4(kcol + row0 + p, pol);
        if (lx) V.x[j] = ld_stream_v4(xcol + row0 + p, pol);
        if (ly) V.y[j] = ld_stream_v4(ycol + row0 + p, pol);
      } else {
#pragma unroll
        for (int f = 0; f < NP; ++f) V.p[f][j] = load4(pcol[f], row0, p, valid);
        V.k[j] = load4(kcol, row0, p, valid);
        if (lx) V.x[j] = load4(xcol, row0, p, valid);
        if (ly) V.y[j] = load4(ycol, row0, p, valid);
      }
    }
  };
  uint64_t my_sum = 0, my_count = 0;
  uint32_t need_lines = 0, seen_lines = 0;
  if (threadIdx.x == 0)
    for (int d = 0; d < kPrefetchTiles; ++d) {
      const int64_t tt = blockIdx.x + static_cast<int64_t>(d) * gridDim.x;
      if (tt < ntiles) prefetch_tile(a.cols, a.col_mask, a.row_begin, tt, TILE, nrows);
    }
  Vecs cur, nxt;
  int64_t t = blockIdx.x;
  if (t < ntiles && !q.never) load(t, cur, false);
  for (; t < ntiles && !q.never; t += gridDim.x) {
    const bool sparse = late_mask && seen_lines >= 64u && 3u * need_lines < seen_lines;
    const int64_t ahead = t + static_cast<int64_t>(kPrefetchTiles) * gridDim.x;
    if (threadIdx.x == 0 && ahead < ntiles)
      prefetch_tile(a.cols, sparse ? (a.col_mask & ~late_mask) : a.col_mask, a.row_begin, ahead, TILE, nrows);
    const int64_t tn = t + gridDim.x;
    if (tn < ntiles) load(tn, nxt, sparse);
    const int64_t row0 = t * TILE;
    const int valid = static_cast<int>((nrows - row0) < TILE ? (nrows - row0) : TILE);
#pragma unroll
    for (int j = 0; j < VEC; ++j) {
      const int p = (j * THREADS + tid) * 4;
      int32_t pv[NP][4], key[4];
#pragma unroll
      for (int f = 0; f < NP; ++f) unpack4(cur.p[f][j], pv[f]);
      unpack4(cur.k[j], key);
      // BlockPred, then the probe of the surviving rows, all four slot reads in flight
      bool ok[4];
      uint64_t slot[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        ok[e] = p + e < valid;
#pragma unroll
        for (int f = 0; f < NP; ++f) ok[e] = ok[e] && in_span(pv[f][e], q.pred_lo[f], q.pred_span[f]);
        slot[e] = ok[e] && static_cast<uint32_t>(key[e]) < J.hash.limit ? ld_slot(J.slots + key[e], pol_table)
                                                                        : kEmptySlot;
      }
      bool hit[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        hit[e] = ok[e] && slot[e] != kEmptySlot && static_cast<uint32_t>(slot[e]) == static_cast<uint32_t>(key[e]);
        const int32_t v = static_cast<int32_t>(slot[e] >> 32);
        for (int f = 0; f < J.n_fp; ++f)
          hit[e] = hit[e] && in_span(field_of(v, J.fp_shift[f], J.fp_mask[f]), J.fp_lo[f], J.fp_span[f]);
      }
      const bool live = hit[0] || hit[1] || hit[2] || hit[3];
      if constexpr (SELECTIVE) {
        // lanes 8m .. 8m+7 hold the 16-byte groups of 128-byte line m of the warp's 512 bytes
        const uint32_t b = __ballot_sync(0xFFFFFFFFu, live);
        need_lines += static_cast<uint32_t>((b & 0xFFu) != 0) + ((b & 0xFF00u) != 0) + ((b & 0xFF0000u) != 0) +
                      ((b & 0xFF000000u) != 0);
        seen_lines += 4u;
      }
      int4 x4 = cur.x[j], y4 = TWO ? cur.y[j] : make_int4(0, 0, 0, 0);
      if (SELECTIVE && cur.sel && live) {  // the late columns of this group, read only now that a row is live
        if (x_late) x4 = load4(xcol, row0, p, valid);
        if (y_late) y4 = load4(ycol, row0, p, valid);
      }
      int32_t xv[4], yv[4];
      unpack4(x4, xv);
      unpack4(y4, yv);
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        int64_t r;
        if (AGG == CRYS_AGG_A_MUL_B) r = static_cast<int64_t>(xv[e]) * yv[e];
        else if (AGG == CRYS_AGG_A_SUB_B) r = static_cast<int64_t>(xv[e]) - yv[e];
        else if (AGG == CRYS_AGG_A_ADD_B) r = static_cast<int64_t>(xv[e]) + yv[e];
        else r = xv[e];
        my_sum += hit[e] ? static_cast<uint64_t>(r) : 0ull;
        my_count += hit[e] ? 1u : 0u;
      }
    }
    cur = nxt;
  }
  const uint64_t s = block_sum_u64<THREADS>(my_sum, red);
  const uint64_t c = block_sum_u64<THREADS>(my_count, red);
  if (threadIdx.x == 0 && c) {
    wait_for_prerequisite_grid();
    atomicAdd(q.sums, static_cast<unsigned long long>(s));
    if (q.counts) atomicAdd(q.counts, static_cast<unsigned long long>(c));
  }
}

// ------------------------------------------------------------------ shared scan

struct ProbeSpec {
  const uint64_t* slots;
  HashFn hash;
  int32_t fk_col;
  int32_t fk_slot;  // staged slice of fk_col
};

struct ScanArgs {
  const int32_t* cols[CRYS_MAX_COLS];
  int32_t slot_of[CRYS_MAX_COLS];     // table column -> staged slice, -1 if unused
  int32_t union_cols[CRYS_MAX_COLS];  // staged slice -> table column
  int32_t n_union;
  int32_t stages;
  int64_t row_begin, row_end;
  int32_t n_queries;
  int32_t n_probes;       // batch-wide probes (0: every join probes for its own query)
  int32_t shared_groups;  // accumulators held in shared memory, all queries
  int32_t* err;
  ProbeSpec probes[kMaxProbes];
  DevQuery q[CRYS_MAX_PLANS];
};

// The shared scan keeps no staging ring: each thread loads its own rows' foreign keys
// (16-byte vectors, read once per tile for the whole batch) and probes every shared
// dimension table once; predicate and aggregate columns are read with L1-cached loads,
// so the second and later queries of the batch that read a column find the tile in L1.
// Shared memory holds only each thread's probe results and the group accumulators,
// which keeps several blocks per SM resident to hide the probes' latency; no barrier is
// needed inside the tile loop.
template <int THREADS, int ITEMS>
__global__ void __launch_bounds__(THREADS, (24 * kWarp) / THREADS > 0 ? (24 * kWarp) / THREADS : 1)
    shared_scan_kernel(const __grid_constant__ ScanArgs a) {
  constexpr int TILE = THREADS * ITEMS;
  constexpr int VEC = ITEMS / 4;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int tid = threadIdx.x, lane = tid % kWarp;
  int4* pv = reinterpret_cast<int4*>(smem_raw);                                   // probes x TILE
  uint32_t* pf = reinterpret_cast<uint32_t*>(pv + static_cast<size_t>(a.n_probes) * VEC * THREADS);
  const SharedAcc acc = shared_acc(reinterpret_cast<unsigned char*>(pf + a.n_probes * THREADS),
                                   a.shared_groups);
  for (int g = tid; g < a.shared_groups; g += THREADS) {
    acc.sums[g] = 0;
    acc.counts[g] = 0;
  }
  __syncthreads();

  const int64_t nrows = a.row_end - a.row_begin;
  const int64_t ntiles = (nrows + TILE - 1) / TILE;
  const uint64_t pol = policy_evict_first();
  const uint64_t pol_table = policy_evict_last();
  uint32_t union_mask = 0;
  for (int u = 0; u < a.n_union; ++u) union_mask |= 1u << a.union_cols[u];
  if (tid == 0)
    for (int d = 0; d < kPrefetchTiles; ++d) {
      const int64_t tt = blockIdx.x + static_cast<int64_t>(d) * gridDim.x;
      if (tt < ntiles) prefetch_tile(a.cols, union_mask, a.row_begin, tt, TILE, nrows);
    }
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int64_t ahead = t + static_cast<int64_t>(kPrefetchTiles) * gridDim.x;
    if (tid == 0 && ahead < ntiles) prefetch_tile(a.cols, union_mask, a.row_begin, ahead, TILE, nrows);
    const int64_t row0 = a.row_begin + t * TILE;
    const int valid = static_cast<int>((nrows - t * TILE) < TILE ? (nrows - t * TILE) : TILE);
    const uint32_t live = rows_present<THREADS, ITEMS>(valid);
    GlobalCols fk_cols;
    fk_cols.cols = a.cols;
    fk_cols.row0 = row0;
    fk_cols.valid = valid;
    fk_cols.pol = pol;
    // Batch-wide BlockLookup: each shared (fk column, table) pair once per row; up to PW
    // probes at a time with all their first-slot reads in flight together.
    constexpr int PW = ITEMS <= 4 ? 2 : 1;
    for (int d0 = 0; d0 < a.n_probes; d0 += PW) {
      int32_t key[PW][ITEMS];
      uint32_t h[PW][ITEMS];
      uint64_t slot[PW][ITEMS];
#pragma unroll
      for (int dd = 0; dd < PW; ++dd) {
        if (d0 + dd >= a.n_probes) break;
        const ProbeSpec& P = a.probes[d0 + dd];
#pragma unroll
        for (int j = 0; j < VEC; ++j) unpack4(fk_cols.load4(P.fk_col, (j * THREADS + tid) * 4), key[dd] + 4 * j);
#pragma unroll
        for (int i = 0; i < ITEMS; ++i) {
          h[dd][i] = hash_slot(key[dd][i], P.hash);
          slot[dd][i] = ((live >> i) & 1u) && hash_may_hold(key[dd][i], P.hash)
                            ? ld_slot(P.slots + h[dd][i], pol_table)
                            : kEmptySlot;
        }
      }
#pragma unroll
      for (int dd = 0; dd < PW; ++dd) {
        const int d = d0 + dd;
        if (d >= a.n_probes) break;
        const ProbeSpec& P = a.probes[d];
        int32_t value[ITEMS];
        uint32_t found = 0;
#pragma unroll
        for (int i = 0; i < ITEMS; ++i) {
          value[i] = 0;
          if (((live >> i) & 1u) &&
              hash_resolve(P.slots, P.hash, h[dd][i], slot[dd][i], key[dd][i], &value[i], pol_table))
            found |= 1u << i;
        }
        pf[d * THREADS + tid] = found;
#pragma unroll
        for (int j = 0; j < VEC; ++j)
          pv[(d * VEC + j) * THREADS + tid] = make_int4(value[4 * j], value[4 * j + 1], value[4 * j + 2], value[4 * j + 3]);
      }
    }
    CachedCols cols;
    cols.cols = a.cols;
    cols.row0 = row0;
    cols.valid = valid;
    for (int qi = 0; qi < a.n_queries; ++qi) {
      const DevQuery& q = a.q[qi];
      int32_t gid[ITEMS];
      int64_t val[ITEMS];
      const uint32_t alive = eval_shared<THREADS, ITEMS>(q, cols, live, pv, pf, gid, val, a.err, pol_table);
      if (q.acc_mode == kAccSingle) {
        if (!__any_sync(0xFFFFFFFFu, alive != 0)) continue;
        uint64_t s_sum = 0, s_cnt = 0;
#pragma unroll
        for (int i = 0; i < ITEMS; ++i) {
          if ((alive >> i) & 1u) {
            s_sum += static_cast<uint64_t>(val[i]);
            s_cnt += 1;
          }
        }
        s_sum = warp_sum_u64(s_sum);
        s_cnt = warp_sum_u64(s_cnt);
        if (lane == 0 && s_cnt) {
          shared_add_u64(acc.sums + q.acc_off, static_cast<unsigned long long>(s_sum));
          atomicAdd(acc.counts + q.acc_off, static_cast<unsigned int>(s_cnt));
        }
      } else if (alive) {
#pragma unroll
        for (int i = 0; i < ITEMS; ++i) {
          if (!((alive >> i) & 1u)) continue;
          if (q.acc_mode == kAccShared) {
            shared_add_u64(acc.sums + q.acc_off + gid[i], static_cast<unsigned long long>(val[i]));
            atomicAdd(acc.counts + q.acc_off + gid[i], 1u);
          } else {
            red_add_global(q.sums + gid[i], static_cast<unsigned long long>(val[i]), pol_table);
            if (q.counts) red_add_global(q.counts + gid[i], 1ull, pol_table);
          }
        }
      }
    }
  }
  __syncthreads();
  for (int qi = 0; qi < a.n_queries; ++qi) {
    const DevQuery& q = a.q[qi];
    if (q.acc_mode != kAccGlobal) flush_shared<THREADS>(acc, q.acc_off, q.groups, q.sums, q.counts);
  }
}

// ------------------------------------------------------------------ tagged shared scan
//
// Query bitmaps over direct dimension tables (the shared join of CJOIN, Candea et al.,
// VLDB 2009, applied to one batch of a shared scan).  For every distinct (fact column,
// table) pair of the batch, annotate_kernel writes one 8-byte entry per table slot:
// the slot's value in the high word and, in the low word, the bitmap of the batch's
// queries the dimension row satisfies (bit q set when query q does not join through the
// pair, or joins it and the row passes all of q's bit-field predicates on it).  The
// fact scan then needs one lookup per pair and row to know every query's dimension
// verdict at once: the AND of the entries' bitmaps.  Only the (row, query) pairs left
// set are expanded, compacted per warp and finished one pair per lane (fact predicates,
// group code, aggregate), so a query costs in proportion to the rows it keeps.
//
// Finishing reads, per pair, the pairs' values of its row and the fact columns of its
// query's predicates and aggregate.  Both are put in shared memory by the warp that owns
// the rows, during the lookups: one region of values per pair and one per fact column the
// batch finishes with ("staged" columns), all with the same item-major layout (value of
// item i of thread t at i * (THREADS + 16) + t).  The lanes of a round finish rows of
// different threads of the warp, so distinct rows fall in distinct banks; regions are
// padded by 8 words so that one row's values in different regions do too.
//
// Fact predicates on columns of small range are folded into the row's bitmap the same
// way: when every fact predicate of the batch lies on at most kMaxPredTags columns, each
// within kPredTagLen consecutive values, a table per column maps a value to the bitmap
// of the queries whose predicates on that column it passes.  Finishing then tests no
// predicate, and rows that fail them never become pairs.

constexpr int kMaxTagPairs = 8;
constexpr int kMaxPredTags = 2;
constexpr int kPredTagLen = 256;
// Tagged-scan blocks resident per SM: two blocks of 512 threads (32 warps) measured
// faster than three of 256, with the same shared memory left to each block's group
// accumulators.  A block of 1024 threads has the SM to itself: its shared memory also
// holds the entries of the batch's smallest table (see kTagSmemBytes), which two blocks
// could only hold twice.
__host__ __device__ constexpr int tag_blocks_per_sm(int threads) { return threads >= 1024 ? 1 : 2; }
constexpr int kMaxTagEntries = CRYS_MAX_PLANS * CRYS_MAX_JOINS;
// A query's descriptor: kDescWords 32-bit fields (a column field holds the index of the
// column's value region), stored field-major in shared memory: field f of query q at
// f * CRYS_MAX_PLANS + q.  The lanes of a finishing round read the same field of the
// queries they finish, so distinct queries fall in distinct banks and equal ones share a
// broadcast: one wavefront per field read.  Unused predicates and groups hold entries
// that always pass, so every lane runs the same instructions whatever query it finishes.
// What every pair reads is also packed into few words (kDPack, kDGroupW): shared-memory
// wavefronts, not instructions, bound finishing.
constexpr int kDescWords = 56;
enum DescField : int {
  kDAggA = 0, kDAggB = 1,                     // aggregate operands (value regions)
  kDAccMode = 2, kDAccOff = 3,                // shared-memory accumulators (offset) or global
  kDP0Col = 4, kDP0Lo = 5, kDP0Span = 6,      // fact predicate 0: region, lo, span
  kDP1Col = 7, kDP1Lo = 8, kDP1Span = 9,      // fact predicate 1
  kDPreds = 10, kDGroups = 11,                // fact predicates, grouped joins
  kDMulAB = 12, kDCoefA = 13, kDCoefB = 14,   // val = a*b, or ca*a + cb*b
  // region of a | region of b << 5 | operator << 10 (0 a, 1 a*b, 2 a-b, 3 a+b) |
  // grouped joins << 12 | global accumulators << 15
  kDPack = 15,
  kDGroup0 = 16,      // 4 grouped joins of 4 words: pair << 8 | shift, mask, card, stride
  kDSums = 32,        // output pointers: sums (2 words), then counts (2 words)
  kDCounts = 34,
  kDMorePreds = 36,   // fact predicates 2..7: region, lo, span
  kDGroupW = 54,      // grouped joins 0, 1: pair | shift << 4 | mask bits << 9
};
static_assert(kDMorePreds + 3 * (CRYS_MAX_PREDS - 2) <= kDGroupW && kDGroupW + 2 <= kDescWords, "descriptor fields");
static_assert(kMaxTagPairs + CRYS_MAX_COLS <= 32, "a value region index fits 5 bits");

// Field access to one query's descriptor in the field-major layout.
template <typename T>
struct DescView {
  T* base;  // field 0 of the query
  __host__ __device__ __forceinline__ T& operator[](int f) const { return base[f * CRYS_MAX_PLANS]; }
};

struct TagPair {
  const uint64_t* slots;  // the direct table
  uint64_t* ann;          // per-batch entries, one per slot
  uint32_t limit;         // capacity
  int32_t fk_col;
  uint32_t nonjoin;       // queries that do not join through the pair
  uint32_t join;          // queries that do
  int32_t first_entry, n_entries;
};

struct TagEntry {  // one join of one query through a pair
  int32_t q;
  int32_t n_fp;
  uint32_t fp_shift[CRYS_MAX_FIELD_PREDS], fp_mask[CRYS_MAX_FIELD_PREDS], fp_span[CRYS_MAX_FIELD_PREDS];
  int32_t fp_lo[CRYS_MAX_FIELD_PREDS];
};

struct AnnotateArgs {
  int32_t n_pairs;
  TagPair pairs[kMaxTagPairs];
  TagEntry entries[kMaxTagEntries];
};

__device__ __forceinline__ void annotate_pair(const AnnotateArgs& a, int pair) {
  const TagPair& P = a.pairs[pair];
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < P.limit; i += stride) {
    const uint64_t s = P.slots[i];
    const int32_t v = static_cast<int32_t>(s >> 32);
    uint32_t bits = P.nonjoin;
    if (s != kEmptySlot) {
      uint32_t fail = 0;
      for (int e = P.first_entry; e < P.first_entry + P.n_entries; ++e) {
        const TagEntry& E = a.entries[e];
        bool ok = true;
        for (int f = 0; f < E.n_fp; ++f)
          ok = ok && in_span(field_of(v, E.fp_shift[f], E.fp_mask[f]), E.fp_lo[f], E.fp_span[f]);
        if (!ok) fail |= 1u << E.q;
      }
      bits |= P.join & ~fail;
    }
    P.ann[i] = (static_cast<uint64_t>(static_cast<uint32_t>(v)) << 32) | bits;
  }
}

__global__ void __launch_bounds__(256) annotate_kernel(const __grid_constant__ AnnotateArgs a) {
  annotate_pair(a, blockIdx.y);
}

struct TagScanPair {
  const uint64_t* ann;
  uint32_t limit;
  int32_t fk_col;
  uint32_t nonjoin;
  int32_t in_l1;  // entries small enough to stay in L1 (read with L1 allocation)
};

// Entries of a table up to this size are read through L1, where every tile's lookups
// find them; the others bypass L1 so that they do not evict the small ones.
constexpr int64_t kTagL1Bytes = 24 * 1024;
// In a block that has its SM to itself, the entries of one table up to this size are
// copied into shared memory once and looked up there: a warp's 32 random lookups then
// cost a few bank-conflict wavefronts instead of one L1 request per distinct line.
constexpr int64_t kTagSmemBytes = 24 * 1024;

__device__ __forceinline__ uint64_t ld_tag_l1(const uint64_t* p, uint64_t pol) {
  uint64_t v;
  asm volatile("ld.global.nc.L1::evict_last.L2::cache_hint.u64 %0, [%1], %2;" : "=l"(v) : "l"(p), "l"(pol));
  return v;
}
__device__ __forceinline__ uint64_t ld_tag_bypass(const uint64_t* p, uint64_t pol) {
  uint64_t v;
  asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.u64 %0, [%1], %2;" : "=l"(v) : "l"(p), "l"(pol));
  return v;
}

// Everything a tagged scan launch needs except the query descriptors (TagHead), and the
// descriptors after it (TagArgs).
struct TagHead {
  const int32_t* cols[CRYS_MAX_COLS];
  uint32_t col_mask;  // fact columns the batch reads
  int64_t row_begin, row_end;
  int32_t n_pairs;
  int32_t n_queries;
  uint32_t all_mask;     // queries that can qualify at all
  uint32_t global_mask;  // queries whose groups are added in global memory
  int32_t shared_groups;
  int32_t tile_shape;  // THREADS << 16 | ITEMS of the shape the arguments were prepared for
  int32_t smem_bytes;  // dynamic shared memory the launch provides
  int32_t* err;
  TagScanPair pairs[kMaxTagPairs];
  int32_t n_stage;                    // fact columns staged for finishing
  int32_t stage_col[CRYS_MAX_COLS];   // staged column s -> fact column (region n_pairs + s)
  int32_t smem_pair;                  // pair whose entries are looked up in shared memory, or -1
  int32_t smem_slots;                 // its entries (its table's capacity)
  int32_t preds_in_bitmap;            // every fact predicate is folded into the bitmaps
  int32_t n_ptags;                    // fact columns whose predicates are table lookups
  int32_t ptag_col[kMaxPredTags];
  int32_t ptag_base[kMaxPredTags];    // the value of entry 0
  uint32_t ptag_len[kMaxPredTags];    // entries
  uint32_t ptag_out[kMaxPredTags];    // the bitmap of a value outside the entries
  uint32_t ptag[kMaxPredTags][kPredTagLen];  // bitmap of the queries value base + k passes
};

struct TagArgs : TagHead {
  int32_t desc[CRYS_MAX_PLANS * kDescWords];
};

// Finishes one (row, query) pair whose dimension verdicts all passed: fact predicates
// (unless PREDS is false: the bitmaps held them), group code from the pairs' values,
// aggregate, accumulation.  `vals` holds the value regions (pairs, then staged columns;
// PVS words apart) and `t` is the row's item-major index in them.
template <int PVS, bool PREDS>
__device__ __forceinline__ void finish_pair(const DescView<const int32_t> D, const int32_t* vals, int t,
                                            const SharedAcc& acc, int32_t* err) {
  const int32_t* row = vals + t;
  const uint32_t pk = static_cast<uint32_t>(D[kDPack]);
  const int32_t xa = row[(pk & 31u) * PVS];
  const int32_t xb = row[((pk >> 5) & 31u) * PVS];
  if (PREDS) {
    const int32_t x0 = row[D[kDP0Col] * PVS];
    const int32_t x1 = row[D[kDP1Col] * PVS];
    bool ok = in_span(x0, D[kDP0Lo], static_cast<uint32_t>(D[kDP0Span])) &
              in_span(x1, D[kDP1Lo], static_cast<uint32_t>(D[kDP1Span]));
    const int n_preds = D[kDPreds];
    for (int f = 2; f < n_preds; ++f) {
      const int b = kDMorePreds + 3 * (f - 2);
      ok = ok && in_span(row[D[b] * PVS], D[b + 1], static_cast<uint32_t>(D[b + 2]));
    }
    if (!ok) return;
  }
  int32_t gid = 0;
  uint32_t bad = 0;
  auto group = [&](int g) {
    const int32_t gx = D[kDGroup0 + 4 * g];
    const uint32_t code = (static_cast<uint32_t>(row[(gx >> 8) * PVS]) >> (gx & 31)) &
                          static_cast<uint32_t>(D[kDGroup0 + 4 * g + 1]);
    bad |= static_cast<uint32_t>(code >= static_cast<uint32_t>(D[kDGroup0 + 4 * g + 2]));
    gid += static_cast<int32_t>(code) * D[kDGroup0 + 4 * g + 3];
  };
  auto group_packed = [&](int g) {  // grouped joins 0 and 1 from their packed words
    const uint32_t w = static_cast<uint32_t>(D[kDGroupW + g]);
    const uint32_t mb = (w >> 9) & 63u;
    const uint32_t mask = mb >= 32u ? 0xFFFFFFFFu : ((1u << mb) - 1u);
    const uint32_t code = (static_cast<uint32_t>(row[(w & 15u) * PVS]) >> ((w >> 4) & 31u)) & mask;
    bad |= static_cast<uint32_t>(code >= static_cast<uint32_t>(D[kDGroup0 + 4 * g + 2]));
    gid += static_cast<int32_t>(code) * D[kDGroup0 + 4 * g + 3];
  };
  group_packed(0);
  group_packed(1);
  const int n_groups = static_cast<int>((pk >> 12) & 7u);
  for (int g = 2; g < n_groups; ++g) group(g);
  if (bad) {
    set_error(err, CRYS_DEV_BAD_GROUP);
    return;
  }
  const uint32_t op = (pk >> 10) & 3u;
  const int64_t a64 = xa, b64 = xb;
  const int64_t val = op == 1u ? a64 * b64 : a64 + (op == 2u ? -b64 : (op == 3u ? b64 : int64_t{0}));
  if (!((pk >> 15) & 1u)) {
    const int slot = D[kDAccOff] + gid;
    shared_add_u64(acc.sums + slot, static_cast<unsigned long long>(val));
    atomicAdd(acc.counts + slot, 1u);
  } else {
    unsigned long long* sums = reinterpret_cast<unsigned long long*>(
        (static_cast<uint64_t>(static_cast<uint32_t>(D[kDSums + 1])) << 32) | static_cast<uint32_t>(D[kDSums]));
    unsigned long long* counts = reinterpret_cast<unsigned long long*>(
        (static_cast<uint64_t>(static_cast<uint32_t>(D[kDCounts + 1])) << 32) | static_cast<uint32_t>(D[kDCounts]));
    const uint64_t keep = policy_evict_last();
    red_add_global(sums + gid, static_cast<unsigned long long>(val), keep);
    if (counts) red_add_global(counts + gid, 1ull, keep);
  }
}

// Shared memory of a block: query descriptors, the value regions of the tile's rows
// (n_vals = pairs + staged columns, PVS words each), one (row, query) list per warp, the
// entries of the pair looked up in shared memory (tag_slots of them, possibly none), then
// the group accumulators.
template <int THREADS, int ITEMS>
struct TagSmem {
  static constexpr int TILE = THREADS * ITEMS;
  // item slot i of thread t at i * IST + t: a lane's rows of consecutive item slots,
  // which one finishing list holds, fall 16 banks apart
  static constexpr int IST = THREADS + 16;
  static constexpr int PVS = ITEMS * IST + 8;  // region stride in words
  static constexpr int LIST = 256;      // list window of a warp (a round averages a few per lane)
  static constexpr size_t desc_bytes = CRYS_MAX_PLANS * kDescWords * 4;
  static constexpr size_t vals_off = (desc_bytes + 15) / 16 * 16;
  __host__ __device__ static size_t list_off(int n_vals) { return vals_off + static_cast<size_t>(n_vals) * PVS * 4; }
  __host__ __device__ static size_t tags_off(int n_vals) {
    return (list_off(n_vals) + static_cast<size_t>(THREADS / kWarp) * LIST * 2 + 15) / 16 * 16;
  }
  __host__ __device__ static size_t acc_off(int n_vals, int tag_slots) {
    return tags_off(n_vals) + static_cast<size_t>(tag_slots) * 8;
  }
};

template <int THREADS, int ITEMS>
__device__ __forceinline__ void tagged_scan_body(const TagHead& a, const int32_t* desc_src) {
  using L = TagSmem<THREADS, ITEMS>;
  constexpr int TILE = L::TILE;
  constexpr int VEC = ITEMS / 4;
  static_assert(ITEMS <= 8, "a list entry holds a 3-bit item slot and a lane");
  constexpr int PVS = L::PVS;
  constexpr int IST = L::IST;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int tid = threadIdx.x, lane = tid % kWarp, warp = tid / kWarp;
  const int n_vals = a.n_pairs + a.n_stage;
  int32_t* desc = reinterpret_cast<int32_t*>(smem_raw);
  int32_t* vals = reinterpret_cast<int32_t*>(smem_raw + L::vals_off);
  uint16_t* list = reinterpret_cast<uint16_t*>(smem_raw + L::list_off(n_vals)) + warp * L::LIST;
  uint64_t* stag = reinterpret_cast<uint64_t*>(smem_raw + L::tags_off(n_vals));
  const int tag_slots = a.smem_pair >= 0 ? a.smem_slots : 0;
  // arguments prepared for another tile shape, or accumulators past the shared memory
  // this launch has: refuse the work (uniformly in every block) instead of overrunning
  uint32_t dyn_smem;
  asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dyn_smem));
  bool ptags_ok = a.n_ptags >= 0 && a.n_ptags <= kMaxPredTags;
  for (int c = 0; c < kMaxPredTags && ptags_ok; ++c)
    ptags_ok = c >= a.n_ptags || (a.ptag_len[c] <= static_cast<uint32_t>(kPredTagLen) && a.ptag_col[c] >= 0 &&
                                  a.ptag_col[c] < CRYS_MAX_COLS);
  if (a.tile_shape != ((THREADS << 16) | ITEMS) || a.n_stage < 1 || a.n_stage > CRYS_MAX_COLS || !ptags_ok ||
      a.smem_pair >= a.n_pairs || tag_slots < 0 ||
      (a.smem_pair >= 0 && static_cast<uint32_t>(tag_slots) != a.pairs[a.smem_pair].limit) ||
      L::acc_off(n_vals, tag_slots) + static_cast<size_t>(a.shared_groups) * 12 > dyn_smem) {
    if (tid == 0) set_error(a.err, CRYS_DEV_BOUNDS);
    return;
  }
  const SharedAcc acc = shared_acc(smem_raw + L::acc_off(n_vals, tag_slots), a.shared_groups);
  for (int w = tid; w < CRYS_MAX_PLANS * kDescWords; w += THREADS) desc[w] = desc_src[w];
  if (a.smem_pair >= 0) {
    const uint64_t* src = a.pairs[a.smem_pair].ann;
    for (int w = tid; w < tag_slots; w += THREADS) stag[w] = src[w];
  }
  for (int g = tid; g < a.shared_groups; g += THREADS) {
    acc.sums[g] = 0;
    acc.counts[g] = 0;
  }
  __syncthreads();

  const int64_t nrows = a.row_end - a.row_begin;
  const int64_t ntiles = (nrows + TILE - 1) / TILE;
  const uint64_t pol = policy_evict_first();
  const uint64_t pol_table = policy_evict_last();
  if (tid == 0)
    for (int d = 0; d < kTagPrefetchTiles; ++d) {
      const int64_t tt = blockIdx.x + static_cast<int64_t>(d) * gridDim.x;
      if (tt < ntiles) prefetch_tile(a.cols, a.col_mask, a.row_begin, tt, TILE, nrows);
    }
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int64_t ahead = t + static_cast<int64_t>(kTagPrefetchTiles) * gridDim.x;
    if (tid == 0 && ahead < ntiles) prefetch_tile(a.cols, a.col_mask, a.row_begin, ahead, TILE, nrows);
    const int64_t row0 = a.row_begin + t * TILE;
    const int valid = static_cast<int>((nrows - t * TILE) < TILE ? (nrows - t * TILE) : TILE);
    const uint32_t live = rows_present<THREADS, ITEMS>(valid);
    GlobalCols fk_cols;
    fk_cols.cols = a.cols;
    fk_cols.row0 = row0;
    fk_cols.valid = valid;
    fk_cols.pol = pol;
    uint32_t rm[ITEMS];
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) rm[i] = ((live >> i) & 1u) ? a.all_mask : 0u;
    // fact predicates folded into the bitmaps: one table lookup per column and row
    for (int c = 0; c < a.n_ptags; ++c) {
      int32_t x[ITEMS];
#pragma unroll
      for (int j = 0; j < VEC; ++j) unpack4(fk_cols.load4(a.ptag_col[c], (j * THREADS + tid) * 4), x + 4 * j);
#pragma unroll
      for (int i = 0; i < ITEMS; ++i) {
        const uint32_t k = static_cast<uint32_t>(x[i]) - static_cast<uint32_t>(a.ptag_base[c]);
        rm[i] &= k < a.ptag_len[c] ? a.ptag[c][k] : a.ptag_out[c];
      }
    }
    __syncwarp();  // the warp is done with the previous tile's values
    // one lookup per pair and row: AND of the dimension verdicts, values kept for groups.
    // Two pairs at a time: the second pair's lookups go out before the first pair's
    // verdicts are in (gated only on what the row had before both), so a warp waits for
    // one L2 round trip per two pairs.
    auto lookup = [&](const TagScanPair& P, bool in_smem, const int32_t (&key)[ITEMS], uint64_t (&e)[ITEMS]) {
      if (in_smem) {
#pragma unroll
        for (int i = 0; i < ITEMS; ++i)
          e[i] = (rm[i] && static_cast<uint32_t>(key[i]) < P.limit) ? stag[key[i]] : static_cast<uint64_t>(P.nonjoin);
      } else if (P.in_l1) {
#pragma unroll
        for (int i = 0; i < ITEMS; ++i)
          e[i] = (rm[i] && static_cast<uint32_t>(key[i]) < P.limit) ? ld_tag_l1(P.ann + key[i], pol_table)
                                                                    : static_cast<uint64_t>(P.nonjoin);
      } else {
#pragma unroll
        for (int i = 0; i < ITEMS; ++i)
          e[i] = (rm[i] && static_cast<uint32_t>(key[i]) < P.limit) ? ld_tag_bypass(P.ann + key[i], pol_table)
                                                                    : static_cast<uint64_t>(P.nonjoin);
      }
    };
    for (int p = 0; p < a.n_pairs; p += 2) {
      const bool two = p + 1 < a.n_pairs;
      int32_t key0[ITEMS], key1[ITEMS];
      uint64_t e0[ITEMS], e1[ITEMS];
#pragma unroll
      for (int j = 0; j < VEC; ++j) unpack4(fk_cols.load4(a.pairs[p].fk_col, (j * THREADS + tid) * 4), key0 + 4 * j);
      if (two) {
#pragma unroll
        for (int j = 0; j < VEC; ++j)
          unpack4(fk_cols.load4(a.pairs[p + 1].fk_col, (j * THREADS + tid) * 4), key1 + 4 * j);
      }
      lookup(a.pairs[p], p == a.smem_pair, key0, e0);
      if (two) lookup(a.pairs[p + 1], p + 1 == a.smem_pair, key1, e1);
#pragma unroll
      for (int i = 0; i < ITEMS; ++i) {
        rm[i] &= static_cast<uint32_t>(e0[i]);
        vals[p * PVS + i * IST + tid] = static_cast<int32_t>(e0[i] >> 32);
      }
      if (two) {
#pragma unroll
        for (int i = 0; i < ITEMS; ++i) {
          rm[i] &= static_cast<uint32_t>(e1[i]);
          vals[(p + 1) * PVS + i * IST + tid] = static_cast<int32_t>(e1[i] >> 32);
        }
      }
    }
    uint32_t any = 0;
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) any |= rm[i];
    if (!__any_sync(0xFFFFFFFFu, any != 0)) continue;  // no pair of the warp's rows survives
    // the fact columns the batch finishes with, beside the pairs' values
    for (int c = 0; c < a.n_stage; ++c) {
      int32_t x[ITEMS];
#pragma unroll
      for (int j = 0; j < VEC; ++j) unpack4(fk_cols.load4(a.stage_col[c], (j * THREADS + tid) * 4), x + 4 * j);
#pragma unroll
      for (int i = 0; i < ITEMS; ++i) vals[(a.n_pairs + c) * PVS + i * IST + tid] = x[i];
    }
    __syncwarp();  // values of the warp's rows visible to all its lanes
    // Item slots SLOTS at a time: expand each lane's (row, query) pairs of those slots into
    // the warp's list, then finish them 32 at a time (one pair per lane).  Two slots per
    // list leave fewer partly filled rounds than one.  Pairs of queries with shared-memory
    // accumulators come first in the list and those with global ones after, so that all
    // but one round take a single accumulation path.
    constexpr int SLOTS = ITEMS % 2 == 0 ? 2 : 1;
    auto finish_window = [&](int wn) {
      for (int base = 0; base < wn; base += kWarp) {
        if (base + lane < wn) {
          const uint32_t ent = list[base + lane];
          // item-major index of the entry's row: item slot, then the warp's lane
          const int row = static_cast<int>((ent >> 5) & 7u) * IST + warp * kWarp + static_cast<int>(ent & 31u);
          const DescView<const int32_t> D{desc + (ent >> 8)};
          if (a.preds_in_bitmap)
            finish_pair<PVS, false>(D, vals, row, acc, a.err);
          else
            finish_pair<PVS, true>(D, vals, row, acc, a.err);
        }
      }
    };
#pragma unroll
    for (int i = 0; i < ITEMS; i += SLOTS) {
      // bit 32 s + q: query q on the lane's row of item slot i + s
      uint64_t ms = 0, mg = 0;
#pragma unroll
      for (int s = 0; s < SLOTS; ++s) {
        ms |= static_cast<uint64_t>(rm[i + s] & ~a.global_mask) << (32 * s);
        mg |= static_cast<uint64_t>(rm[i + s] & a.global_mask) << (32 * s);
      }
      const int ns = __popcll(ms), ng = __popcll(mg);
      const int incl_s = warp_inclusive_scan(ns, lane), incl_g = warp_inclusive_scan(ng, lane);
      const int total_s = __shfl_sync(0xFFFFFFFFu, incl_s, kWarp - 1);
      const int total = total_s + __shfl_sync(0xFFFFFFFFu, incl_g, kWarp - 1);
      if (total == 0) continue;
      // list entry: query << 8 | item slot << 5 | lane
      auto entry = [&](uint64_t m) {
        const int b = __ffsll(static_cast<long long>(m)) - 1;
        return static_cast<uint16_t>(((b & 31) << 8) | ((i + (b >> 5)) << 5) | lane);
      };
      if (total <= L::LIST) {  // the usual case: one window
        int k = incl_s - ns;
        for (uint64_t m = ms; m; m &= m - 1, ++k) list[k] = entry(m);
        k = total_s + incl_g - ng;
        for (uint64_t m = mg; m; m &= m - 1, ++k) list[k] = entry(m);
        __syncwarp();
        finish_window(total);
        __syncwarp();  // the list is reused by the next slots
        continue;
      }
      // more pairs than the list holds: windows of L::LIST entries
      for (int w0 = 0; w0 < total; w0 += L::LIST) {
        int k = incl_s - ns;
        for (uint64_t m = ms; m; m &= m - 1, ++k)
          if (k >= w0 && k < w0 + L::LIST) list[k - w0] = entry(m);
        k = total_s + incl_g - ng;
        for (uint64_t m = mg; m; m &= m - 1, ++k)
          if (k >= w0 && k < w0 + L::LIST) list[k - w0] = entry(m);
        __syncwarp();
        finish_window((total - w0) < L::LIST ? (total - w0) : L::LIST);
        __syncwarp();  // the list is reused by the next window or slots
      }
    }
  }
  __syncthreads();
  for (int qi = 0; qi < a.n_queries; ++qi) {
    const DescView<const int32_t> D{desc + qi};
    if (D[kDAccMode] == kAccGlobal) continue;
    unsigned long long* sums = reinterpret_cast<unsigned long long*>(
        (static_cast<uint64_t>(static_cast<uint32_t>(D[kDSums + 1])) << 32) | static_cast<uint32_t>(D[kDSums]));
    unsigned long long* counts = reinterpret_cast<unsigned long long*>(
        (static_cast<uint64_t>(static_cast<uint32_t>(D[kDCounts + 1])) << 32) | static_cast<uint32_t>(D[kDCounts]));
    int64_t groups = 1;
    for (int g = 0; g < D[kDGroups]; ++g) groups *= D[kDGroup0 + 4 * g + 2];
    flush_shared<THREADS>(acc, D[kDAccOff], groups, sums, counts);
  }
}

template <int THREADS, int ITEMS>
__global__ void __launch_bounds__(THREADS, tag_blocks_per_sm(THREADS))
    tagged_scan_kernel(const __grid_constant__ TagArgs a) {
  // the head is read on every tile: a shared-memory copy is cheaper than the parameter
  // bank, whose cache does not hold a 9 KB argument block
  __shared__ __align__(16) TagHead head;
  static_assert(sizeof(TagHead) % 4 == 0, "copied as 32-bit words");
  for (int w = threadIdx.x; w < static_cast<int>(sizeof(TagHead) / 4); w += THREADS)
    reinterpret_cast<uint32_t*>(&head)[w] = reinterpret_cast<const uint32_t*>(&a)[w];
  __syncthreads();
  tagged_scan_body<THREADS, ITEMS>(head, a.desc);
}

// ------------------------------------------------------------------ graph-replayable launch
//
// A serving loop launches the tagged scan once per row segment with a batch that changes
// at segment boundaries.  Its arguments then live in a device block (TagLaunch) that the
// host refills, through a pinned copy, before every launch; the launch itself (shape and
// shared memory fixed per tile shape) never changes, so one CUDA graph of
// {copy, prepare_kernel, tagged_scan_kernel_dev} can be captured once and replayed.

struct TagLaunch {
  TagArgs scan;
  AnnotateArgs ann;
  int32_t annotate;  // the batch changed since the previous launch: re-tag its pairs
  int32_t variant;   // tile shape the block was prepared for
  int32_t n_zero;    // outputs that start at zero in this launch
  unsigned long long* zero_ptr[2 * CRYS_MAX_PLANS];
  int64_t zero_words[2 * CRYS_MAX_PLANS];
};

// blockIdx.y < kMaxTagPairs: annotation of pair y (when asked for); the last row of
// blocks zeroes the outputs of the queries that join the batch in this launch.
__global__ void __launch_bounds__(256) prepare_kernel(const TagLaunch* __restrict__ L) {
  if (blockIdx.y < kMaxTagPairs) {
    if (L->annotate && static_cast<int>(blockIdx.y) < L->ann.n_pairs) annotate_pair(L->ann, blockIdx.y);
    return;
  }
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int z = 0; z < L->n_zero; ++z) {
    unsigned long long* p = L->zero_ptr[z];
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < L->zero_words[z]; i += stride)
      p[i] = 0ull;
  }
}

template <int THREADS, int ITEMS>
__global__ void __launch_bounds__(THREADS, tag_blocks_per_sm(THREADS))
    tagged_scan_kernel_dev(const TagArgs* __restrict__ a) {
  // the head is read on every tile: one shared-memory copy per block
  __shared__ __align__(16) TagHead head;
  static_assert(sizeof(TagHead) % 4 == 0, "copied as 32-bit words");
  for (int w = threadIdx.x; w < static_cast<int>(sizeof(TagHead) / 4); w += THREADS)
    reinterpret_cast<uint32_t*>(&head)[w] = reinterpret_cast<const uint32_t*>(a)[w];
  __syncthreads();
  tagged_scan_body<THREADS, ITEMS>(head, a->desc);
}

// ------------------------------------------------------------------ packing

struct PackArgs {
  const int32_t* cols[8];
  uint32_t shift[8], mask[8];
  int32_t n_fields;
  int64_t n;
  int32_t* out;
};

__global__ void __launch_bounds__(256) pack_kernel(const __grid_constant__ PackArgs a) {
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < a.n; i += stride) {
    uint32_t v = 0;
    for (int k = 0; k < a.n_fields; ++k)
      v |= (static_cast<uint32_t>(a.cols[k][i]) & a.mask[k]) << a.shift[k];
    a.out[i] = static_cast<int32_t>(v);
  }
}

// ------------------------------------------------------------------ host side

constexpr int64_t kMaxGroups = 1ll << 28;
constexpr size_t kSharedBudget = 200 * 1024;  // dynamic shared memory a block may use
constexpr int kScanBlocksPerSM = 3;           // shared-scan blocks resident per SM (target)

uint32_t field_mask(int32_t bits) {
  return (bits <= 0 || bits >= 32) ? 0xFFFFFFFFu : ((1u << bits) - 1u);
}

bool field_ok(int32_t shift, int32_t bits) {
  if (bits < 0 || bits > 32 || shift < 0 || shift > 31) return false;
  if (bits == 0 || bits == 32) return shift == 0;
  return shift + bits <= 32;
}

int groups_of(const crys_plan& p, int64_t* groups) {
  if (p.n_joins < 0 || p.n_joins > CRYS_MAX_JOINS) return CRYS_EINVAL;
  int64_t g = 1;
  for (int j = 0; j < p.n_joins; ++j) {
    const int32_t c = p.joins[j].group_card;
    if (c < 0) return CRYS_EINVAL;
    if (c > 0) {
      g *= c;
      if (g > kMaxGroups) return CRYS_EINVAL;
    }
  }
  *groups = g;
  return CRYS_OK;
}

bool table_ok(const crys_hash& h) {
  if (!h.slots || (reinterpret_cast<uintptr_t>(h.slots) & 7u) != 0 || h.capacity > (1ll << 31)) return false;
  if (h.kind == CRYS_HASH_DIRECT) return h.capacity >= 1;
  return (h.kind == CRYS_HASH_MULT || h.kind == CRYS_HASH_IDENT) && is_pow2(h.capacity) && h.capacity >= 2;
}

int to_device(const crys_table& t, const crys_plan& p, DevQuery* d, uint32_t* col_mask) {
  int64_t groups = 0;
  if (groups_of(p, &groups) != CRYS_OK) return CRYS_EINVAL;
  if (p.n_preds < 0 || p.n_preds > CRYS_MAX_PREDS) return CRYS_EINVAL;
  if (p.agg_op < CRYS_AGG_A || p.agg_op > CRYS_AGG_A_ADD_B) return CRYS_EINVAL;
  if (!p.d_sums) return CRYS_EINVAL;
  auto col_ok = [&](int32_t c) { return c >= 0 && c < t.n_cols; };
  uint32_t mask = 0;
  d->n_preds = p.n_preds;
  for (int f = 0; f < p.n_preds; ++f) {
    if (!col_ok(p.preds[f].col)) return CRYS_EINVAL;
    d->pred_col[f] = p.preds[f].col;
    d->pred_lo[f] = p.preds[f].lo;
    d->pred_hi[f] = p.preds[f].hi;
    d->pred_span[f] = static_cast<uint32_t>(p.preds[f].hi) - static_cast<uint32_t>(p.preds[f].lo);
    mask |= 1u << p.preds[f].col;
  }
  d->never = 0;
  for (int f = 0; f < p.n_preds; ++f)
    if (p.preds[f].lo > p.preds[f].hi) d->never = 1;
  d->n_joins = p.n_joins;
  // mixed-radix weights: first grouped join most significant
  int64_t weight = groups;
  for (int j = 0; j < p.n_joins; ++j) {
    const crys_join& J = p.joins[j];
    DevJoin& D = d->joins[j];
    if (!col_ok(J.fk_col) || !table_ok(J.ht)) return CRYS_EINVAL;
    if (!field_ok(J.group_shift, J.group_bits) || J.n_preds < 0 || J.n_preds > CRYS_MAX_FIELD_PREDS)
      return CRYS_EINVAL;
    D.slots = J.ht.slots;
    D.hash = make_hash(J.ht.kind, J.ht.capacity);
    D.fk_col = J.fk_col;
    D.card = J.group_card;
    D.stride = 0;
    if (J.group_card > 0) {
      weight /= J.group_card;
      D.stride = static_cast<int32_t>(weight);
    }
    D.gshift = static_cast<uint32_t>(J.group_shift);
    D.gmask = field_mask(J.group_bits);
    D.n_fp = J.n_preds;
    for (int f = 0; f < J.n_preds; ++f) {
      if (!field_ok(J.preds[f].shift, J.preds[f].bits)) return CRYS_EINVAL;
      D.fp_shift[f] = static_cast<uint32_t>(J.preds[f].shift);
      D.fp_mask[f] = field_mask(J.preds[f].bits);
      D.fp_lo[f] = J.preds[f].lo;
      D.fp_hi[f] = J.preds[f].hi;
      D.fp_span[f] = static_cast<uint32_t>(J.preds[f].hi) - static_cast<uint32_t>(J.preds[f].lo);
      if (J.preds[f].lo > J.preds[f].hi) {  // never true: compare the constant 0 with [1, 1]
        D.fp_mask[f] = 0;
        D.fp_lo[f] = 1;
        D.fp_span[f] = 0;
      }
    }
    D.probe = -1;
    mask |= 1u << J.fk_col;
  }
  if (!col_ok(p.agg_a)) return CRYS_EINVAL;
  mask |= 1u << p.agg_a;
  if (p.agg_op != CRYS_AGG_A) {
    if (!col_ok(p.agg_b)) return CRYS_EINVAL;
    mask |= 1u << p.agg_b;
  }
  d->agg_op = p.agg_op;
  d->agg_a = p.agg_a;
  d->agg_b = p.agg_op != CRYS_AGG_A ? p.agg_b : p.agg_a;
  d->groups = groups;
  d->sums = reinterpret_cast<unsigned long long*>(p.d_sums);
  d->counts = reinterpret_cast<unsigned long long*>(p.d_counts);
  d->acc_mode = kAccGlobal;
  d->acc_off = 0;
  *col_mask = mask;
  return CRYS_OK;
}

int check_table(const crys_table* t) {
  if (!t || t->n_cols < 1 || t->n_cols > CRYS_MAX_COLS || t->n_rows < 0) return CRYS_EINVAL;
  for (int c = 0; c < t->n_cols; ++c)
    if (t->n_rows > 0 && (!t->cols[c] || !aligned16(t->cols[c]))) return CRYS_EINVAL;
  return CRYS_OK;
}

int zero_outputs(const DevQuery& q, cudaStream_t s) {
  if (cudaMemsetAsync(q.sums, 0, static_cast<size_t>(q.groups) * 8, s) != cudaSuccess) return CRYS_ECUDA;
  if (q.counts && cudaMemsetAsync(q.counts, 0, static_cast<size_t>(q.groups) * 8, s) != cudaSuccess)
    return CRYS_ECUDA;
  return CRYS_OK;
}

// Clears a query's outputs on the stream: the kernel the query kernel is launched behind
// (programmatic dependent launch).
int launch_zero_outputs(const DevQuery& q, cudaStream_t s) {
  const int64_t zb = q.groups > 256 ? (q.groups + 255) / 256 : 1;
  const int64_t zcap = static_cast<int64_t>(sm_count()) * 4;
  zero_outputs_kernel<<<static_cast<unsigned>(zb < zcap ? zb : zcap), 256, 0, s>>>(q.sums, q.counts, q.groups);
  note_launch();
  return check_launch();
}

// Per-block accumulators are 32-bit counts: a block must see fewer than 2^32 rows.
bool counts_fit(int64_t rows, int grid) { return (rows / (grid > 0 ? grid : 1)) + (1 << 16) < (1ll << 32); }

template <int THREADS, int ITEMS>
int launch_plan(PlanArgs& a, cudaStream_t s) {
  constexpr int TILE = THREADS * ITEMS;
  size_t smem = 0;
  if (a.q.groups == 1) {
    a.q.acc_mode = kAccSingle;
  } else if (static_cast<size_t>(a.q.groups) * 12 <= kSharedBudget) {
    a.q.acc_mode = kAccShared;
    smem = static_cast<size_t>(a.q.groups) * 12;
  } else {
    a.q.acc_mode = kAccGlobal;
  }
  // All of a tile's leading column loads go out together (4- and 8-row items), and with
  // 4-row items the next tile's loads are in flight while a tile is evaluated: measured
  // faster than the step-by-step evaluation at every size (Q1 at 2^28 rows, hashed date
  // table: 0.665 against 0.818 ms).  The step-by-step evaluation, with selective loads of
  // the late columns, remains for other tile shapes.
  const int64_t ntiles = (a.row_end - a.row_begin + TILE - 1) / TILE;
  auto kl = plan_kernel<THREADS, ITEMS, false>;
  if (!allow_smem(kl, smem)) return CRYS_ECUDA;
  int grid = persistent_grid(kl, THREADS, smem, ntiles);
  const bool preload = ITEMS == 4 || ITEMS == 8;
  auto k = preload ? plan_kernel<THREADS, ITEMS, true> : kl;
  if (preload) {
    if (!allow_smem(k, smem)) return CRYS_ECUDA;
    grid = persistent_grid(k, THREADS, smem, ntiles);
  }
  // a plan of the Q1 family: the kernel compiled for its shape
  const DevJoin& J0 = a.q.joins[0];
  const bool fixed = preload && a.q.acc_mode == kAccSingle && a.q.n_joins == 1 &&
                     (a.q.n_preds == 1 || a.q.n_preds == 2) && J0.card <= 0 && J0.hash.steps == 0u &&
                     J0.hash.mult_hi == 1u && J0.hash.mult_lo == 0u && J0.hash.shift == 0u && J0.hash.mask == 0xFFFFFFFFu &&
                     (a.q.agg_op == CRYS_AGG_A_MUL_B || a.q.agg_op == CRYS_AGG_A);
  if (fixed) {
    const bool mul = a.q.agg_op == CRYS_AGG_A_MUL_B;
    if (a.q.n_preds == 2)
      k = mul ? plan_fixed_kernel<THREADS, ITEMS, 2, CRYS_AGG_A_MUL_B> : plan_fixed_kernel<THREADS, ITEMS, 2, CRYS_AGG_A>;
    else
      k = mul ? plan_fixed_kernel<THREADS, ITEMS, 1, CRYS_AGG_A_MUL_B> : plan_fixed_kernel<THREADS, ITEMS, 1, CRYS_AGG_A>;
    grid = persistent_grid(k, THREADS, 0, ntiles);
  }
  if (!counts_fit(a.row_end - a.row_begin, grid)) return CRYS_EINVAL;
  // every host check passed: clear the outputs, then launch the query kernel while the
  // clearing kernel still runs
  if (launch_zero_outputs(a.q, s) != CRYS_OK) return CRYS_ECUDA;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(static_cast<unsigned>(grid));
  cfg.blockDim = dim3(THREADS);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (cudaLaunchKernelEx(&cfg, k, a) != cudaSuccess) return CRYS_ECUDA;
  note_launch();
  return check_launch();
}

template <int THREADS, int ITEMS>
int launch_scan(ScanArgs& a, cudaStream_t s) {
  constexpr int TILE = THREADS * ITEMS;
  const size_t probe_bytes = static_cast<size_t>(a.n_probes) * (TILE + THREADS) * sizeof(int32_t);
  // Shared memory per block: probe results plus accumulators for as many queries as
  // fit (smallest group counts first: they have the most rows per group, where global
  // atomics would contend most) within a share that keeps kScanBlocksPerSM blocks
  // resident; the rest accumulate with global atomics.
  const size_t share = (220u * 1024u) / kScanBlocksPerSM;
  const size_t budget = share > probe_bytes ? share - probe_bytes : 0;
  int order[CRYS_MAX_PLANS];
  for (int qi = 0; qi < a.n_queries; ++qi) order[qi] = qi;
  for (int i = 1; i < a.n_queries; ++i)
    for (int j = i; j > 0 && a.q[order[j]].groups < a.q[order[j - 1]].groups; --j) {
      const int t = order[j];
      order[j] = order[j - 1];
      order[j - 1] = t;
    }
  int64_t used = 0;
  for (int oi = 0; oi < a.n_queries; ++oi) {
    DevQuery& q = a.q[order[oi]];
    if (static_cast<size_t>(used + q.groups) * 12 <= budget) {
      q.acc_mode = q.groups == 1 ? kAccSingle : kAccShared;
      q.acc_off = static_cast<int32_t>(used);
      used += q.groups;
    } else {
      q.acc_mode = kAccGlobal;
    }
  }
  a.shared_groups = static_cast<int32_t>(used);
  const size_t smem = probe_bytes + static_cast<size_t>(used) * 12;
  auto k = shared_scan_kernel<THREADS, ITEMS>;
  if (!allow_smem(k, smem)) return CRYS_ECUDA;
  const int64_t ntiles = (a.row_end - a.row_begin + TILE - 1) / TILE;
  const int grid = persistent_grid(k, THREADS, smem, ntiles);
  if (!counts_fit(a.row_end - a.row_begin, grid)) return CRYS_EINVAL;
  k<<<grid, THREADS, smem, s>>>(a);
  note_launch();
  return check_launch();
}

// Assigns batch-wide probes: a (fk column, table) pair joined by two or more queries of
// the batch is probed once per row for all of them (up to kMaxProbes pairs, most used
// first); a pair only one query joins is probed by that query itself, after its own
// predicates have removed rows.
void assign_probes(ScanArgs& a) {
  struct Pair {
    ProbeSpec spec;
    int uses;
  };
  Pair pairs[CRYS_MAX_PLANS * CRYS_MAX_JOINS];
  int n = 0;
  auto same = [](const ProbeSpec& p, const DevJoin& J) {
    return p.slots == J.slots && p.fk_col == J.fk_col && p.hash.mask == J.hash.mask && p.hash.limit == J.hash.limit &&
           p.hash.mult_hi == J.hash.mult_hi && p.hash.mult_lo == J.hash.mult_lo;
  };
  for (int qi = 0; qi < a.n_queries; ++qi) {
    for (int j = 0; j < a.q[qi].n_joins; ++j) {
      const DevJoin& J = a.q[qi].joins[j];
      int found = -1;
      for (int d = 0; d < n && found < 0; ++d)
        if (same(pairs[d].spec, J)) found = d;
      if (found < 0) {
        pairs[n].spec = {J.slots, J.hash, J.fk_col, 0};
        pairs[n].uses = 0;
        found = n++;
      }
      pairs[found].uses += 1;
    }
  }
  // most used first (stable insertion sort; n <= 128)
  for (int i = 1; i < n; ++i)
    for (int j = i; j > 0 && pairs[j].uses > pairs[j - 1].uses; --j) {
      const Pair t = pairs[j];
      pairs[j] = pairs[j - 1];
      pairs[j - 1] = t;
    }
  int m = 0;
  while (m < n && m < kMaxProbes && pairs[m].uses >= 2) {
    a.probes[m] = pairs[m].spec;
    ++m;
  }
  for (int qi = 0; qi < a.n_queries; ++qi)
    for (int j = 0; j < a.q[qi].n_joins; ++j)
      for (int d = 0; d < m; ++d)
        if (same(a.probes[d], a.q[qi].joins[j])) a.q[qi].joins[j].probe = d;
  a.n_probes = m;
}

// Tagging a batch: the distinct (fact column, direct table) pairs, their annotation
// entries, the scratch layout and the per-query descriptors.  Returns false when the
// batch cannot be tagged (a join on a table that is not direct, or too many pairs).
struct TagBatch {
  AnnotateArgs ann;
  TagArgs scan;
  int64_t bytes;   // scratch the annotations need
  int64_t max_slots;
};

bool tag_batch(const crys_plan* plans, const DevQuery* q, int n, TagBatch* tb) {
  AnnotateArgs& A = tb->ann;
  TagArgs& S = tb->scan;
  A.n_pairs = 0;
  int pair_of[CRYS_MAX_PLANS][CRYS_MAX_JOINS];
  for (int qi = 0; qi < n; ++qi) {
    for (int j = 0; j < plans[qi].n_joins; ++j) {
      const crys_join& J = plans[qi].joins[j];
      if (J.ht.kind != CRYS_HASH_DIRECT) return false;
      int found = -1;
      for (int p = 0; p < A.n_pairs && found < 0; ++p)
        if (A.pairs[p].slots == J.ht.slots && A.pairs[p].fk_col == J.fk_col &&
            A.pairs[p].limit == static_cast<uint32_t>(J.ht.capacity))
          found = p;
      if (found < 0) {
        if (A.n_pairs == kMaxTagPairs) return false;
        found = A.n_pairs++;
        TagPair& P = A.pairs[found];
        P.slots = J.ht.slots;
        P.ann = nullptr;
        P.limit = static_cast<uint32_t>(J.ht.capacity);
        P.fk_col = J.fk_col;
        P.join = 0;
        P.n_entries = 0;
      }
      pair_of[qi][j] = found;
      A.pairs[found].join |= 1u << qi;
      A.pairs[found].n_entries += 1;
    }
  }
  // entries grouped by pair
  int next[kMaxTagPairs];
  int first = 0;
  for (int p = 0; p < A.n_pairs; ++p) {
    A.pairs[p].first_entry = first;
    next[p] = first;
    first += A.pairs[p].n_entries;
  }
  const uint32_t everyone = n == 32 ? 0xFFFFFFFFu : ((1u << n) - 1u);
  for (int qi = 0; qi < n; ++qi)
    for (int j = 0; j < q[qi].n_joins; ++j) {
      const DevJoin& J = q[qi].joins[j];
      TagEntry& E = A.entries[next[pair_of[qi][j]]++];
      E.q = qi;
      E.n_fp = J.n_fp;
      for (int f = 0; f < CRYS_MAX_FIELD_PREDS; ++f) {
        E.fp_shift[f] = f < J.n_fp ? J.fp_shift[f] : 0;
        E.fp_mask[f] = f < J.n_fp ? J.fp_mask[f] : 0;
        E.fp_lo[f] = f < J.n_fp ? J.fp_lo[f] : 0;
        E.fp_span[f] = f < J.n_fp ? J.fp_span[f] : 0;
      }
    }
  tb->bytes = 0;
  tb->max_slots = 0;
  S.n_pairs = A.n_pairs;
  for (int p = 0; p < A.n_pairs; ++p) {
    TagPair& P = A.pairs[p];
    P.nonjoin = everyone & ~P.join;
    S.pairs[p].limit = P.limit;
    S.pairs[p].fk_col = P.fk_col;
    S.pairs[p].nonjoin = P.nonjoin;
    S.pairs[p].in_l1 = static_cast<int64_t>(P.limit) * 8 <= kTagL1Bytes ? 1 : 0;
    tb->bytes += (static_cast<int64_t>(P.limit) * 8 + 15) / 16 * 16;
    if (P.limit > tb->max_slots) tb->max_slots = P.limit;
  }
  // fact columns the batch finishes with: staged in value regions after the pairs'
  int region_of[CRYS_MAX_COLS];
  for (int c = 0; c < CRYS_MAX_COLS; ++c) {
    region_of[c] = -1;
    S.stage_col[c] = 0;
  }
  S.n_stage = 0;
  S.smem_pair = -1;
  S.smem_slots = 0;
  auto region = [&](int32_t c) {
    if (region_of[c] < 0) {
      region_of[c] = A.n_pairs + S.n_stage;
      S.stage_col[S.n_stage++] = c;
    }
    return region_of[c];
  };
  // fact predicates folded into the bitmaps, when each column's predicates in the batch
  // span at most kPredTagLen values and at most kMaxPredTags columns have any
  // (queries that no row can satisfy are left out: their bit is never set)
  S.preds_in_bitmap = 1;
  S.n_ptags = 0;
  int64_t plo[CRYS_MAX_COLS], phi[CRYS_MAX_COLS];
  uint32_t pq[CRYS_MAX_COLS];
  for (int c = 0; c < CRYS_MAX_COLS; ++c) {
    plo[c] = INT64_MAX;
    phi[c] = INT64_MIN;
    pq[c] = 0;
  }
  for (int qi = 0; qi < n; ++qi) {
    if (q[qi].never) continue;
    for (int f = 0; f < q[qi].n_preds; ++f) {
      const int c = q[qi].pred_col[f];
      plo[c] = q[qi].pred_lo[f] < plo[c] ? q[qi].pred_lo[f] : plo[c];
      phi[c] = q[qi].pred_hi[f] > phi[c] ? q[qi].pred_hi[f] : phi[c];
      pq[c] |= 1u << qi;
    }
  }
  for (int c = 0; c < CRYS_MAX_COLS && S.preds_in_bitmap; ++c) {
    if (!pq[c]) continue;
    if (S.n_ptags == kMaxPredTags || phi[c] - plo[c] + 1 > kPredTagLen) {
      S.preds_in_bitmap = 0;
      break;
    }
    const int t = S.n_ptags++;
    S.ptag_col[t] = c;
    S.ptag_base[t] = static_cast<int32_t>(plo[c]);
    S.ptag_len[t] = static_cast<uint32_t>(phi[c] - plo[c] + 1);
    S.ptag_out[t] = everyone & ~pq[c];
    for (int k = 0; k < kPredTagLen; ++k) {
      uint32_t bits = S.ptag_out[t];
      const int64_t v = plo[c] + k;
      if (k < static_cast<int>(S.ptag_len[t]))
        for (int qi = 0; qi < n; ++qi) {
          if (!((pq[c] >> qi) & 1u)) continue;
          bool ok = true;
          for (int f = 0; f < q[qi].n_preds; ++f)
            if (q[qi].pred_col[f] == c) ok = ok && q[qi].pred_lo[f] <= v && v <= q[qi].pred_hi[f];
          if (ok) bits |= 1u << qi;
        }
      S.ptag[t][k] = k < static_cast<int>(S.ptag_len[t]) ? bits : 0u;
    }
  }
  if (!S.preds_in_bitmap) S.n_ptags = 0;
  // descriptors
  S.n_queries = n;
  S.all_mask = 0;
  for (int w = 0; w < CRYS_MAX_PLANS * kDescWords; ++w) S.desc[w] = 0;
  for (int qi = 0; qi < n; ++qi) {
    const DevQuery& Q = q[qi];
    const DescView<int32_t> D{S.desc + qi};
    if (!Q.never) S.all_mask |= 1u << qi;
    // fact predicates: the first two in fixed fields (an unused one always passes: any
    // value of the aggregate column lies in [0, 0 + 2^32 - 1]), the rest in a list
    // (none when the bitmaps hold them: finishing then reads no predicate field)
    const int np = S.preds_in_bitmap ? 0 : Q.n_preds;
    D[kDPreds] = np;
    const int32_t pc[2] = {np > 0 ? Q.pred_col[0] : Q.agg_a, np > 1 ? Q.pred_col[1] : Q.agg_a};
    const int32_t pl[2] = {np > 0 ? Q.pred_lo[0] : 0, np > 1 ? Q.pred_lo[1] : 0};
    const uint32_t ps[2] = {np > 0 ? Q.pred_span[0] : 0xFFFFFFFFu, np > 1 ? Q.pred_span[1] : 0xFFFFFFFFu};
    D[kDP0Col] = region(pc[0]);
    D[kDP0Lo] = pl[0];
    D[kDP0Span] = static_cast<int32_t>(ps[0]);
    D[kDP1Col] = region(pc[1]);
    D[kDP1Lo] = pl[1];
    D[kDP1Span] = static_cast<int32_t>(ps[1]);
    for (int f = 2; f < np; ++f) {
      D[kDMorePreds + 3 * (f - 2)] = region(Q.pred_col[f]);
      D[kDMorePreds + 3 * (f - 2) + 1] = Q.pred_lo[f];
      D[kDMorePreds + 3 * (f - 2) + 2] = static_cast<int32_t>(Q.pred_span[f]);
    }
    // grouped joins; unused entries give code 0 of cardinality 1
    int ng = 0;
    for (int g = 0; g < 4; ++g) {
      D[kDGroup0 + 4 * g] = 0;
      D[kDGroup0 + 4 * g + 1] = 0;
      D[kDGroup0 + 4 * g + 2] = 1;
      D[kDGroup0 + 4 * g + 3] = 0;
    }
    for (int j = 0; j < Q.n_joins; ++j) {
      const DevJoin& J = Q.joins[j];
      if (J.card <= 0) continue;
      D[kDGroup0 + 4 * ng] = (pair_of[qi][j] << 8) | static_cast<int32_t>(J.gshift);
      if (ng < 2)
        D[kDGroupW + ng] = pair_of[qi][j] | static_cast<int32_t>(J.gshift << 4) |
                           (__builtin_popcount(J.gmask) << 9);
      D[kDGroup0 + 4 * ng + 1] = static_cast<int32_t>(J.gmask);
      D[kDGroup0 + 4 * ng + 2] = J.card;
      D[kDGroup0 + 4 * ng + 3] = J.stride;
      ++ng;
    }
    D[kDGroups] = ng;
    // aggregate: a*b, or ca*a + cb*b (a: ca 1 cb 0 with b = a; a-b: 1, -1; a+b: 1, 1)
    D[kDAggA] = region(Q.agg_a);
    D[kDAggB] = region(Q.agg_op == CRYS_AGG_A ? Q.agg_a : Q.agg_b);
    D[kDMulAB] = Q.agg_op == CRYS_AGG_A_MUL_B ? 1 : 0;
    D[kDCoefA] = Q.agg_op == CRYS_AGG_A_MUL_B ? 0 : 1;
    D[kDCoefB] = Q.agg_op == CRYS_AGG_A_SUB_B ? -1 : (Q.agg_op == CRYS_AGG_A_ADD_B ? 1 : 0);
    const int32_t op = Q.agg_op == CRYS_AGG_A_MUL_B ? 1 : (Q.agg_op == CRYS_AGG_A_SUB_B ? 2 : (Q.agg_op == CRYS_AGG_A_ADD_B ? 3 : 0));
    D[kDPack] = D[kDAggA] | (D[kDAggB] << 5) | (op << 10) | (ng << 12);  // accumulators: assign_accumulators
    const uint64_t sp = reinterpret_cast<uint64_t>(Q.sums), cp = reinterpret_cast<uint64_t>(Q.counts);
    D[kDSums] = static_cast<int32_t>(static_cast<uint32_t>(sp));
    D[kDSums + 1] = static_cast<int32_t>(static_cast<uint32_t>(sp >> 32));
    D[kDCounts] = static_cast<int32_t>(static_cast<uint32_t>(cp));
    D[kDCounts + 1] = static_cast<int32_t>(static_cast<uint32_t>(cp >> 32));
  }
  return true;
}

// Places the annotations in scratch and launches the annotation and the scan.
// Points each pair's annotations into scratch.
void place_annotations(TagBatch& tb, unsigned char* scratch) {
  int64_t off = 0;
  for (int p = 0; p < tb.ann.n_pairs; ++p) {
    tb.ann.pairs[p].ann = reinterpret_cast<uint64_t*>(scratch + off);
    tb.scan.pairs[p].ann = tb.ann.pairs[p].ann;
    off += (static_cast<int64_t>(tb.ann.pairs[p].limit) * 8 + 15) / 16 * 16;
  }
}

// Expected fraction of fact rows a query keeps, from its dimension predicates on bit
// fields, taking field values as uniform (1 where it cannot tell, 0 when no row can
// qualify).  Only orders queries for the shared accumulators; no result depends on it.
double kept_fraction(const DevQuery& Q) {
  if (Q.never) return 0.0;
  double f = 1.0;
  for (int j = 0; j < Q.n_joins; ++j)
    for (int k = 0; k < Q.joins[j].n_fp; ++k) {
      const uint32_t mask = Q.joins[j].fp_mask[k];
      if (mask == 0xFFFFFFFFu) continue;
      const int64_t lo = Q.joins[j].fp_lo[k] < 0 ? 0 : Q.joins[j].fp_lo[k];
      const int64_t hi = Q.joins[j].fp_hi[k] > static_cast<int64_t>(mask) ? mask : Q.joins[j].fp_hi[k];
      f *= hi < lo ? 0.0 : static_cast<double>(hi - lo + 1) / (static_cast<double>(mask) + 1.0);
    }
  return f;
}

// Group accumulators in shared memory for as many queries as fit in `budget` bytes, the
// queries with the most expected rows per group first (their global atomics would be the
// most frequent and contend most); the rest accumulate with global atomics.  Returns the
// groups held.
int64_t assign_accumulators(TagArgs& S, const DevQuery* q, size_t budget) {
  int order[CRYS_MAX_PLANS];
  double density[CRYS_MAX_PLANS];
  for (int qi = 0; qi < S.n_queries; ++qi) {
    order[qi] = qi;
    density[qi] = kept_fraction(q[qi]) / static_cast<double>(q[qi].groups < 1 ? 1 : q[qi].groups);
  }
  auto before = [&](int x, int y) {  // x goes first
    return density[x] != density[y] ? density[x] > density[y] : q[x].groups < q[y].groups;
  };
  for (int i = 1; i < S.n_queries; ++i)
    for (int j = i; j > 0 && before(order[j], order[j - 1]); --j) {
      const int t = order[j];
      order[j] = order[j - 1];
      order[j - 1] = t;
    }
  int64_t used = 0;
  for (int oi = 0; oi < S.n_queries; ++oi) {
    const int qi = order[oi];
    const DescView<int32_t> D{S.desc + qi};
    if (static_cast<size_t>(used + q[qi].groups) * 12 <= budget) {
      D[kDAccMode] = kAccShared;
      D[kDAccOff] = static_cast<int32_t>(used);
      used += q[qi].groups;
    } else {
      D[kDAccMode] = kAccGlobal;
      D[kDAccOff] = 0;
    }
  }
  S.shared_groups = static_cast<int32_t>(used);
  S.global_mask = 0;
  for (int qi = 0; qi < S.n_queries; ++qi) {
    const DescView<int32_t> D{S.desc + qi};
    const bool global = D[kDAccMode] == kAccGlobal;
    if (global) S.global_mask |= 1u << qi;
    D[kDPack] = (D[kDPack] & ~(1 << 15)) | (global ? 1 << 15 : 0);
  }
  return used;
}

// Shared memory of one tagged-scan block: a block alone on its SM takes all but its
// static head of the 227 KB a block may have; two blocks take 110 KB each.
constexpr size_t tag_share(int threads) { return tag_blocks_per_sm(threads) == 1 ? 224u * 1024u : 110u * 1024u; }
static_assert(224u * 1024u + sizeof(TagHead) <= 227u * 1024u, "one block's shared memory");
static_assert(2 * (110u * 1024u + sizeof(TagHead) + 1024u) <= 228u * 1024u, "two blocks' shared memory");

// The pair whose entries a block of this shape looks up in shared memory: the smallest
// table of at most kTagSmemBytes, in blocks that have their SM to itself (-1: none).
template <int THREADS>
void choose_smem_pair(TagArgs& S) {
  S.smem_pair = -1;
  S.smem_slots = 0;
  if constexpr (tag_blocks_per_sm(THREADS) == 1) {
    for (int p = 0; p < S.n_pairs; ++p) {
      const int64_t bytes = static_cast<int64_t>(S.pairs[p].limit) * 8;
      if (bytes <= kTagSmemBytes && (S.smem_pair < 0 || S.pairs[p].limit < S.pairs[S.smem_pair].limit)) {
        S.smem_pair = p;
        S.smem_slots = static_cast<int32_t>(S.pairs[p].limit);
      }
    }
  }
}

template <int THREADS, int ITEMS>
int launch_tagged(TagBatch& tb, const DevQuery* q, unsigned char* scratch, cudaStream_t s) {
  using L = TagSmem<THREADS, ITEMS>;
  constexpr int TILE = L::TILE;
  constexpr size_t kTagShare = tag_share(THREADS);
  AnnotateArgs& A = tb.ann;
  TagArgs& S = tb.scan;
  place_annotations(tb, scratch);
  choose_smem_pair<THREADS>(S);
  if (A.n_pairs > 0) {
    int64_t gx = (tb.max_slots + 255) / 256;
    const int64_t cap = static_cast<int64_t>(sm_count()) * 8;
    if (gx > cap) gx = cap;
    annotate_kernel<<<dim3(static_cast<unsigned>(gx < 1 ? 1 : gx), static_cast<unsigned>(A.n_pairs)), 256, 0, s>>>(A);
    note_launch();
    const int rc = check_launch();
    if (rc != CRYS_OK) return rc;
  }
  size_t fixed = L::acc_off(S.n_pairs + S.n_stage, S.smem_slots);
  if (fixed > kTagShare && S.smem_pair >= 0) {  // no room for the entries: read them through L1
    S.smem_pair = -1;
    S.smem_slots = 0;
    fixed = L::acc_off(S.n_pairs + S.n_stage, 0);
  }
  const int64_t used = assign_accumulators(S, q, kTagShare > fixed ? kTagShare - fixed : 0);
  S.tile_shape = (THREADS << 16) | ITEMS;
  S.smem_bytes = static_cast<int32_t>(fixed + static_cast<size_t>(used) * 12);
  auto k = tagged_scan_kernel<THREADS, ITEMS>;
  if (!allow_smem(k, S.smem_bytes)) return CRYS_ECUDA;
  const int64_t ntiles = (S.row_end - S.row_begin + TILE - 1) / TILE;
  const int grid = persistent_grid(k, THREADS, S.smem_bytes, ntiles);
  if (!counts_fit(S.row_end - S.row_begin, grid)) return CRYS_EINVAL;
  k<<<grid, THREADS, S.smem_bytes, s>>>(S);
  note_launch();
  return check_launch();
}

// The fixed launch of a TagLaunch block for tile shape (THREADS, ITEMS): grid and shared
// memory depend only on the shape, so the launch can be captured once and replayed.
template <int THREADS, int ITEMS>
int fixed_scan_grid(int* grid) {
  constexpr size_t kTagShare = tag_share(THREADS);
  auto k = tagged_scan_kernel_dev<THREADS, ITEMS>;
  if (!allow_smem(k, kTagShare)) return CRYS_ECUDA;
  *grid = persistent_grid(k, THREADS, kTagShare, int64_t{1} << 40);
  return *grid > 0 ? CRYS_OK : CRYS_ECUDA;
}

template <int THREADS, int ITEMS>
int prepare_block(TagBatch& tb, const DevQuery* q, unsigned char* scratch, TagLaunch* out) {
  using L = TagSmem<THREADS, ITEMS>;
  constexpr size_t kTagShare = tag_share(THREADS);
  place_annotations(tb, scratch);
  TagArgs& S = tb.scan;
  choose_smem_pair<THREADS>(S);
  size_t fixed = L::acc_off(S.n_pairs + S.n_stage, S.smem_slots);
  if (fixed > kTagShare && S.smem_pair >= 0) {  // no room for the entries: read them through L1
    S.smem_pair = -1;
    S.smem_slots = 0;
    fixed = L::acc_off(S.n_pairs + S.n_stage, 0);
  }
  if (fixed > kTagShare) return CRYS_EINVAL;
  assign_accumulators(S, q, kTagShare - fixed);
  S.tile_shape = (THREADS << 16) | ITEMS;
  S.smem_bytes = static_cast<int32_t>(kTagShare);
  int grid = 0;
  const int rc = fixed_scan_grid<THREADS, ITEMS>(&grid);
  if (rc != CRYS_OK) return rc;
  if (!counts_fit(S.row_end - S.row_begin, grid)) return CRYS_EINVAL;
  out->scan = S;
  out->ann = tb.ann;
  return CRYS_OK;
}

template <int THREADS, int ITEMS>
int launch_block(const TagLaunch* dev, cudaStream_t s) {
  int grid = 0;
  int rc = fixed_scan_grid<THREADS, ITEMS>(&grid);
  if (rc != CRYS_OK) return rc;
  prepare_kernel<<<dim3(static_cast<unsigned>(sm_count() * 4), kMaxTagPairs + 1), 256, 0, s>>>(dev);
  note_launch();
  rc = check_launch();
  if (rc != CRYS_OK) return rc;
  tagged_scan_kernel_dev<THREADS, ITEMS><<<grid, THREADS, tag_share(THREADS), s>>>(&dev->scan);
  note_launch();
  return check_launch();
}

}  // namespace
}  // namespace crys

extern "C" {

int crys_plan_groups(const crys_plan* plan, int64_t* groups) {
  if (!plan || !groups) return CRYS_EINVAL;
  return crys::groups_of(*plan, groups);
}

int crys_pack_fields(const int32_t* const* cols, const int32_t* shifts, const int32_t* bits,
                     int32_t n_fields, int64_t n, int32_t* out, crys_stream stream) {
  using namespace crys;
  if (n < 0 || n_fields < 1 || n_fields > 8 || !cols || !shifts || !bits) return CRYS_EINVAL;
  PackArgs a;
  uint64_t used = 0;
  for (int k = 0; k < n_fields; ++k) {
    if (bits[k] < 1 || bits[k] > 31 || shifts[k] < 0 || shifts[k] + bits[k] > 31) return CRYS_EINVAL;
    const uint64_t m = ((1ull << bits[k]) - 1) << shifts[k];
    if (used & m) return CRYS_EINVAL;
    used |= m;
    if (n > 0 && !cols[k]) return CRYS_EINVAL;
    a.cols[k] = cols[k];
    a.shift[k] = static_cast<uint32_t>(shifts[k]);
    a.mask[k] = (1u << bits[k]) - 1u;
  }
  if (n == 0) return CRYS_OK;
  if (!out) return CRYS_EINVAL;
  a.n_fields = n_fields;
  a.n = n;
  a.out = out;
  int64_t g = (n + 255) / 256;
  const int64_t cap = static_cast<int64_t>(sm_count()) * 16;
  if (g > cap) g = cap;
  pack_kernel<<<static_cast<unsigned int>(g), 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(a);
  note_launch();
  return check_launch();
}

int crys_run_plan(const crys_table* fact, const crys_plan* plan, crys_stream stream) {
  using namespace crys;
  if (check_table(fact) != CRYS_OK || !plan) return CRYS_EINVAL;
  static PlanArgs zero_args;  // zero-initialised template
  PlanArgs a = zero_args;
  uint32_t mask = 0;
  if (to_device(*fact, *plan, &a.q, &mask) != CRYS_OK) return CRYS_EINVAL;
  for (int c = 0; c < fact->n_cols; ++c) a.cols[c] = fact->cols[c];
  a.col_mask = mask;
  // columns only the aggregate reads, when a filter runs before it (a fact predicate or a
  // join): candidates for selective loads
  a.late_mask = 0;
  if (a.q.n_preds > 0 || a.q.n_joins > 0) {
    uint32_t early = 0;
    for (int f = 0; f < a.q.n_preds; ++f) early |= 1u << a.q.pred_col[f];
    for (int j = 0; j < a.q.n_joins; ++j) early |= 1u << a.q.joins[j].fk_col;
    a.late_mask = ((1u << a.q.agg_a) | (1u << a.q.agg_b)) & ~early;
  }
  a.row_begin = 0;
  a.row_end = fact->n_rows;
  a.err = device_error_word();
  if (!a.err) return CRYS_ECUDA;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (fact->n_rows == 0) return launch_zero_outputs(a.q, s) == CRYS_OK ? CRYS_OK : CRYS_ECUDA;
  constexpr int kOp = CRYS_OP_PLAN;
  switch (tile_variant(kOp)) {
    case 1: return launch_plan<kTiles[kOp][1].threads, kTiles[kOp][1].items>(a, s);
    case 2: return launch_plan<kTiles[kOp][2].threads, kTiles[kOp][2].items>(a, s);
    case 3: return launch_plan<kTiles[kOp][3].threads, kTiles[kOp][3].items>(a, s);
    default: return launch_plan<kTiles[kOp][0].threads, kTiles[kOp][0].items>(a, s);
  }
}

int crys_run_plans(const crys_table* fact, const crys_plan* plans, int32_t n_plans,
                   int64_t row_begin, int64_t row_end, int flags, crys_stream stream) {
  using namespace crys;
  if (check_table(fact) != CRYS_OK || n_plans < 0 || n_plans > CRYS_MAX_PLANS) return CRYS_EINVAL;
  if (n_plans > 0 && !plans) return CRYS_EINVAL;
  if (row_begin < 0 || row_end < row_begin || row_end > fact->n_rows || (row_begin & 3)) return CRYS_EINVAL;
  if (flags & ~CRYS_ACCUMULATE) return CRYS_EINVAL;
  static ScanArgs zero_args;
  ScanArgs* a = new ScanArgs(zero_args);
  uint32_t mask = 0;
  for (int qi = 0; qi < n_plans; ++qi) {
    uint32_t m = 0;
    if (to_device(*fact, plans[qi], &a->q[qi], &m) != CRYS_OK) {
      delete a;
      return CRYS_EINVAL;
    }
    mask |= m;
  }
  a->n_queries = n_plans;
  a->n_union = 0;
  for (int c = 0; c < CRYS_MAX_COLS; ++c) {
    a->cols[c] = c < fact->n_cols ? fact->cols[c] : nullptr;
    a->slot_of[c] = -1;
    if (mask & (1u << c)) {
      a->slot_of[c] = a->n_union;
      a->union_cols[a->n_union++] = c;
    }
  }
  assign_probes(*a);
  // staged slices of every column a query or probe reads
  for (int qi = 0; qi < n_plans; ++qi) {
    DevQuery& q = a->q[qi];
    for (int f = 0; f < q.n_preds; ++f) q.pred_slot[f] = a->slot_of[q.pred_col[f]];
    q.agg_a_slot = a->slot_of[q.agg_a];
    q.agg_b_slot = a->slot_of[q.agg_b];
    for (int j = 0; j < q.n_joins; ++j) q.joins[j].fk_slot = a->slot_of[q.joins[j].fk_col];
  }
  for (int d = 0; d < a->n_probes; ++d) a->probes[d].fk_slot = a->slot_of[a->probes[d].fk_col];
  // The filter each query tests on every row of a tile: the batch-probed join whose
  // predicates keep the smallest share of their fields' value range (codes assumed
  // spread over the field), else the first fact predicate, else none.
  for (int qi = 0; qi < n_plans; ++qi) {
    DevQuery& q = a->q[qi];
    q.first_join = -1;
    q.first_pred = -1;
    double best = 2.0;
    for (int j = 0; j < q.n_joins; ++j) {
      const DevJoin& J = q.joins[j];
      if (J.probe < 0 || J.n_fp == 0) continue;
      double est = 1.0;
      for (int f = 0; f < J.n_fp; ++f) {
        const double top = static_cast<double>(J.fp_mask[f]);
        const double lo = J.fp_lo[f] < 0 ? 0.0 : static_cast<double>(J.fp_lo[f]);
        const double hi = static_cast<double>(J.fp_hi[f]) > top ? top : static_cast<double>(J.fp_hi[f]);
        est *= hi >= lo ? (hi - lo + 1.0) / (top + 1.0) : 0.0;
      }
      if (est < best) {
        best = est;
        q.first_join = j;
      }
    }
    if (q.first_join < 0 && q.n_preds > 0) q.first_pred = 0;
  }
  a->row_begin = row_begin;
  a->row_end = row_end;
  a->err = device_error_word();
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  int rc = a->err ? CRYS_OK : CRYS_ECUDA;
  if (rc == CRYS_OK && !(flags & CRYS_ACCUMULATE)) {
    for (int qi = 0; qi < n_plans && rc == CRYS_OK; ++qi) rc = zero_outputs(a->q[qi], s);
  }
  if (rc == CRYS_OK && n_plans > 0 && row_end > row_begin) {
    constexpr int kOp = CRYS_OP_SHARED_SCAN;
    switch (tile_variant(kOp)) {
      case 1: rc = launch_scan<kTiles[kOp][1].threads, kTiles[kOp][1].items>(*a, s); break;
      case 2: rc = launch_scan<kTiles[kOp][2].threads, kTiles[kOp][2].items>(*a, s); break;
      case 3: rc = launch_scan<kTiles[kOp][3].threads, kTiles[kOp][3].items>(*a, s); break;
      default: rc = launch_scan<kTiles[kOp][0].threads, kTiles[kOp][0].items>(*a, s); break;
    }
  }
  delete a;
  return rc;
}

int crys_run_plans_tagged_bytes(const crys_table* fact, const crys_plan* plans, int32_t n_plans,
                                int64_t* bytes) {
  using namespace crys;
  if (!bytes || check_table(fact) != CRYS_OK || n_plans < 0 || n_plans > CRYS_MAX_PLANS) return CRYS_EINVAL;
  if (n_plans > 0 && !plans) return CRYS_EINVAL;
  *bytes = 0;
  DevQuery* q = new DevQuery[CRYS_MAX_PLANS]();
  TagBatch* tb = new TagBatch();
  int rc = CRYS_OK;
  for (int qi = 0; qi < n_plans && rc == CRYS_OK; ++qi) {
    uint32_t m = 0;
    rc = to_device(*fact, plans[qi], &q[qi], &m);
  }
  if (rc == CRYS_OK && tag_batch(plans, q, n_plans, tb)) *bytes = tb->bytes;
  delete tb;
  delete[] q;
  return rc;
}

int crys_run_plans_tagged(const crys_table* fact, const crys_plan* plans, int32_t n_plans,
                          int64_t row_begin, int64_t row_end, int flags, void* scratch,
                          int64_t scratch_bytes, crys_stream stream) {
  using namespace crys;
  if (check_table(fact) != CRYS_OK || n_plans < 0 || n_plans > CRYS_MAX_PLANS) return CRYS_EINVAL;
  if (n_plans > 0 && !plans) return CRYS_EINVAL;
  if (row_begin < 0 || row_end < row_begin || row_end > fact->n_rows || (row_begin & 3)) return CRYS_EINVAL;
  if (flags & ~CRYS_ACCUMULATE) return CRYS_EINVAL;
  if (scratch_bytes < 0 || (scratch && !aligned16(scratch))) return CRYS_EINVAL;
  DevQuery* q = new DevQuery[CRYS_MAX_PLANS]();
  TagBatch* tb = new TagBatch();
  uint32_t mask = 0;
  int rc = CRYS_OK;
  for (int qi = 0; qi < n_plans && rc == CRYS_OK; ++qi) {
    uint32_t m = 0;
    rc = to_device(*fact, plans[qi], &q[qi], &m);
    mask |= m;
  }
  const bool tagged = rc == CRYS_OK && tag_batch(plans, q, n_plans, tb) && scratch && tb->bytes <= scratch_bytes;
  if (rc == CRYS_OK && !tagged) {
    delete tb;
    delete[] q;
    return crys_run_plans(fact, plans, n_plans, row_begin, row_end, flags, stream);
  }
  TagArgs& S = tb->scan;
  for (int c = 0; c < CRYS_MAX_COLS; ++c) S.cols[c] = c < fact->n_cols ? fact->cols[c] : nullptr;
  S.col_mask = mask;
  S.row_begin = row_begin;
  S.row_end = row_end;
  S.err = device_error_word();
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (rc == CRYS_OK && !S.err) rc = CRYS_ECUDA;
  if (rc == CRYS_OK && !(flags & CRYS_ACCUMULATE))
    for (int qi = 0; qi < n_plans && rc == CRYS_OK; ++qi) rc = zero_outputs(q[qi], s);
  if (rc == CRYS_OK && n_plans > 0 && row_end > row_begin) {
    unsigned char* base = static_cast<unsigned char*>(scratch);
    constexpr int kOp = CRYS_OP_TAGGED_SCAN;
    switch (tile_variant(kOp)) {
      case 1: rc = launch_tagged<kTiles[kOp][1].threads, kTiles[kOp][1].items>(*tb, q, base, s); break;
      case 2: rc = launch_tagged<kTiles[kOp][2].threads, kTiles[kOp][2].items>(*tb, q, base, s); break;
      case 3: rc = launch_tagged<kTiles[kOp][3].threads, kTiles[kOp][3].items>(*tb, q, base, s); break;
      default: rc = launch_tagged<kTiles[kOp][0].threads, kTiles[kOp][0].items>(*tb, q, base, s); break;
    }
  }
  delete tb;
  delete[] q;
  return rc;
}

int crys_tagged_block_bytes(int64_t* bytes) {
  if (!bytes) return CRYS_EINVAL;
  *bytes = (static_cast<int64_t>(sizeof(crys::TagLaunch)) + 255) / 256 * 256;
  return CRYS_OK;
}

int crys_tagged_prepare(const crys_table* fact, const crys_plan* plans, int32_t n_plans, int64_t row_begin,
                        int64_t row_end, int flags, const int32_t* zero_plans, int32_t n_zero, void* scratch,
                        int64_t scratch_bytes, void* host_block) {
  using namespace crys;
  if (!host_block || check_table(fact) != CRYS_OK || n_plans < 1 || n_plans > CRYS_MAX_PLANS || !plans)
    return CRYS_EINVAL;
  if (row_begin < 0 || row_end < row_begin || row_end > fact->n_rows || (row_begin & 3)) return CRYS_EINVAL;
  if ((flags & ~CRYS_TAG_ANNOTATE) || n_zero < 0 || n_zero > n_plans || (n_zero > 0 && !zero_plans))
    return CRYS_EINVAL;
  if (!scratch || !aligned16(scratch) || scratch_bytes < 0) return CRYS_EINVAL;
  DevQuery* q = new DevQuery[CRYS_MAX_PLANS]();
  TagBatch* tb = new TagBatch();
  TagLaunch* out = static_cast<TagLaunch*>(host_block);
  uint32_t mask = 0;
  int rc = CRYS_OK;
  for (int qi = 0; qi < n_plans && rc == CRYS_OK; ++qi) {
    uint32_t m = 0;
    rc = to_device(*fact, plans[qi], &q[qi], &m);
    mask |= m;
  }
  if (rc == CRYS_OK && (!tag_batch(plans, q, n_plans, tb) || tb->bytes > scratch_bytes)) rc = CRYS_EINVAL;
  if (rc == CRYS_OK) {
    TagArgs& S = tb->scan;
    for (int c = 0; c < CRYS_MAX_COLS; ++c) S.cols[c] = c < fact->n_cols ? fact->cols[c] : nullptr;
    S.col_mask = mask;
    S.row_begin = row_begin;
    S.row_end = row_end;
    S.err = device_error_word();
    if (!S.err) rc = CRYS_ECUDA;
  }
  if (rc == CRYS_OK) {
    unsigned char* base = static_cast<unsigned char*>(scratch);
    constexpr int kOp = CRYS_OP_TAGGED_SCAN;
    const int v = tile_variant(kOp);
    switch (v) {
      case 1: rc = prepare_block<kTiles[kOp][1].threads, kTiles[kOp][1].items>(*tb, q, base, out); break;
      case 2: rc = prepare_block<kTiles[kOp][2].threads, kTiles[kOp][2].items>(*tb, q, base, out); break;
      case 3: rc = prepare_block<kTiles[kOp][3].threads, kTiles[kOp][3].items>(*tb, q, base, out); break;
      default: rc = prepare_block<kTiles[kOp][0].threads, kTiles[kOp][0].items>(*tb, q, base, out); break;
    }
    out->variant = v;
  }
  if (rc == CRYS_OK) {
    out->annotate = (flags & CRYS_TAG_ANNOTATE) ? 1 : 0;
    out->n_zero = 0;
    for (int z = 0; z < n_zero && rc == CRYS_OK; ++z) {
      const int qi = zero_plans[z];
      if (qi < 0 || qi >= n_plans) {
        rc = CRYS_EINVAL;
        break;
      }
      out->zero_ptr[out->n_zero] = q[qi].sums;
      out->zero_words[out->n_zero++] = q[qi].groups;
      if (q[qi].counts) {
        out->zero_ptr[out->n_zero] = q[qi].counts;
        out->zero_words[out->n_zero++] = q[qi].groups;
      }
    }
  }
  delete tb;
  delete[] q;
  return rc;
}

int crys_tagged_launch(const void* dev_block, crys_stream stream) {
  using namespace crys;
  if (!dev_block || !aligned16(dev_block)) return CRYS_EINVAL;
  const TagLaunch* L = static_cast<const TagLaunch*>(dev_block);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  constexpr int kOp = CRYS_OP_TAGGED_SCAN;
  switch (tile_variant(kOp)) {
    case 1: return launch_block<kTiles[kOp][1].threads, kTiles[kOp][1].items>(L, s);
    case 2: return launch_block<kTiles[kOp][2].threads, kTiles[kOp][2].items>(L, s);
    case 3: return launch_block<kTiles[kOp][3].threads, kTiles[kOp][3].items>(L, s);
    default: return launch_block<kTiles[kOp][0].threads, kTiles[kOp][0].items>(L, s);
  }
}

}  // extern "C"
