/* crystal.h — C ABI of the GB300 (sm_103a) tile-based query operators.
 *
 * The operators follow the statements of the problems in "A Study of the Fundamental
 * Performance Characteristics of GPUs and CPUs for Database Analytics" (Shanbhag,
 * Madden, Yu; SIGMOD 2020), Section 3 (tile-based execution model), Section 4
 * (project, select, hash join, sort) and Section 5.3 (fused select-join-aggregate
 * query kernels).
 *
 * Conventions shared by every call
 *  - All column pointers are caller-owned DEVICE memory on the current device; the
 *    library never frees them.  Column pointers must be 16-byte aligned (the kernels
 *    move whole 16-byte vectors); a misaligned pointer returns CRYS_EINVAL.
 *  - Every call is asynchronous on the given stream (NULL = legacy default stream).
 *    Outputs in device memory are valid once that stream is synchronised.
 *  - Return value: CRYS_OK or a negative CRYS_E* status detected on the host before
 *    anything was launched (nothing was enqueued in that case).
 *  - Conditions only the GPU can see (a wait that exceeded its time bound, a full
 *    hash table, a reserved or duplicate key, a group code out of range) set sticky
 *    bits in a per-device error word read with crys_device_errors(); the kernels
 *    never trap, and a kernel that detects one of these stops its own work early.
 *  - n == 0 is legal everywhere and produces empty / zero results.
 *  - Scratch: calls that need scratch take (void* d_temp, size_t* temp_bytes).  With
 *    d_temp == NULL the call only stores the required size in *temp_bytes and returns
 *    CRYS_OK; otherwise *temp_bytes must be at least that size (else CRYS_ENOMEM).
 *    Scratch is caller-owned device memory, 256-byte aligned, used only while the call's
 *    work runs on its stream.
 */
#ifndef CRYSTAL_H
#define CRYSTAL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* crys_stream; /* the same type as cudaStream_t */

/* ------------------------------------------------------------------ status */
#define CRYS_OK 0
#define CRYS_EINVAL (-1)   /* bad argument: null/misaligned pointer, bad size, bad plan */
#define CRYS_ENOMEM (-2)   /* scratch smaller than required */
#define CRYS_EFULL (-3)    /* hash table capacity too small for the rows to insert */
#define CRYS_ETIMEOUT (-4) /* reserved for host waits that exceeded their bound */
#define CRYS_ECUDA (-5)    /* a CUDA runtime call failed (launch or memset) */

/* Bits of the per-device error word (crys_device_errors). */
#define CRYS_DEV_TIMEOUT 0x1    /* a bounded spin-wait (mbarrier, look-back) gave up */
#define CRYS_DEV_TABLE_FULL 0x2 /* an insert probed the whole table without a free slot */
#define CRYS_DEV_BAD_KEY 0x4    /* key -1 (0xFFFFFFFF, the empty-slot marker) on build */
#define CRYS_DEV_DUP_KEY 0x8    /* a build key was inserted twice */
#define CRYS_DEV_BAD_GROUP 0x10 /* a joined group code was outside [0, group_card) */
#define CRYS_DEV_BOUNDS 0x20    /* an output position fell outside its buffer (skipped) */

/* Human-readable text for a status code. */
const char* crys_strerror(int status);

/* Copies the calling device's error word into *flags after synchronising `s`; when
 * `clear` is non-zero the word is reset to 0 (also ordered on `s`). */
int crys_device_errors(int32_t* flags, int clear, crys_stream s);

/* Total number of kernels this library has launched in this process (all devices). */
int64_t crys_launch_count(void);

/* Test hook for the bounded waits (failure detection; the paper has no counterpart).
 * The NEXT call of `op` in this process - an order-preserving crys_select (also through
 * crys_select_static) or a crys_sort - hands out tile ids starting at `first_tile`
 * instead of 0 and bounds its look-back waits by `wait_limit_ns` (1 us .. 2 s) instead
 * of 2 s.  With first_tile > 0 the tiles before it never publish their counts, so the
 * tile after them waits for a flag that nothing sets: the call's blocks give up once
 * the bound has passed, CRYS_DEV_TIMEOUT is set in the device error word and the call's
 * outputs are incomplete; nothing hangs and nothing traps.  A call that gives up marks
 * only its own scratch (the per-call abort word), so later calls run normally whether or
 * not the error word was cleared.  One-shot: the request is consumed by that call.
 * CRYS_EINVAL for another op, a negative tile or a bound outside the range. */
int crys_debug_stall(int op, int32_t first_tile, int64_t wait_limit_ns);

/* ------------------------------------------------------------------ selection
 * Section 3.2 (query Q0, Figure "tile-example") and Section 4.2 (query Q3):
 * SELECT x FROM R WHERE lo <= x <= hi, as one kernel: each thread block loads a tile,
 * evaluates the predicate, computes per-thread offsets with a block-wide scan, reserves
 * its output range once per tile and writes the compacted tile with coalesced stores.
 * The inclusive range expresses "<", "<=", "==", ">" and BETWEEN on int32.
 *   x          n int32 values (device)
 *   out        capacity for n int32 values (device); receives the selected values
 *   d_count    one int64 (device); receives the number of selected values
 *   order_preserving
 *              0: the paper's scheme, one atomic reservation per tile — tiles land in
 *                 completion order, values inside a tile keep input order.  No scratch.
 *              1: tiles are chained by a decoupled look-back scan so that `out` is in
 *                 input order.  Needs scratch (see conventions).
 */
int crys_select(const int32_t* x, int64_t n, int32_t lo, int32_t hi, int32_t* out,
                int64_t* d_count, int order_preserving, void* d_temp, size_t* temp_bytes,
                crys_stream s);

/* Allocation-free variant of the order-preserving selection (no counterpart in the
 * paper; it exists for callers that cannot allocate device memory on the call path:
 * query executors and plugins that run inside a host process owning a fixed,
 * pre-reserved device memory pool, or real-time pipelines that forbid allocation after
 * start-up).  Same result as crys_select(..., order_preserving = 1, ...), but the
 * look-back scratch lives in a file-scope static device array of the library
 * (CRYS_SELECT_STATIC_SCRATCH_BYTES bytes, held by every device that loads the
 * library until the process exits).  The caller still passes x, out and d_count.
 *   n > CRYS_SELECT_STATIC_MAX_ROWS returns CRYS_EINVAL (nothing enqueued).
 *   The first call on a device looks up the array's device address with that device
 *   current; make that first call before any stream capture.
 *   All calls share the one array: the call clears the part it uses on its stream, and
 *   calls whose work overlaps on the GPU (other streams, other threads) race on it.
 *   No cudaMalloc, cudaFree or allocating library routine is called. */
#define CRYS_SELECT_STATIC_MAX_ROWS (1ll << 25)
#define CRYS_SELECT_STATIC_SCRATCH_BYTES (256 + (CRYS_SELECT_STATIC_MAX_ROWS / 512) * 8)
int crys_select_static(const int32_t* x, int64_t n, int32_t lo, int32_t hi, int32_t* out,
                       int64_t* d_count, crys_stream s);

/* The "independent threads" selection the paper compares the tile model against
 * (Section 3.2, Figure "tile"): each thread of a fixed launch owns a contiguous chunk of
 * x; one kernel counts each thread's matches, one scans the counts, one re-reads the
 * chunks and writes the matches.  Same result as crys_select with order_preserving = 1
 * (input order); kept as an ablation.  Scratch: one int64 per launched thread, two-call
 * size query as in crys_select (d_temp NULL: *temp_bytes receives the size). */
int crys_select_strawman(const int32_t* x, int64_t n, int32_t lo, int32_t hi, int32_t* out,
                         int64_t* d_count, void* d_temp, size_t* temp_bytes, crys_stream s);

/* ------------------------------------------------------------------ projection
 * Section 4.1, queries Q1 and Q2: y = a*x1 + b*x2 (CRYS_PROJ_LINEAR) or the sigmoid
 * 1/(1 + exp(-(a*x1 + b*x2))) (CRYS_PROJ_SIGMOID), float32 in and out, one rounding per
 * multiply and per add (no fused multiply-add), IEEE division and expf.
 *   x1, x2, y  n float32 values each (device); y may alias x1 or x2. */
#define CRYS_PROJ_LINEAR 0
#define CRYS_PROJ_SIGMOID 1
int crys_project(const float* x1, const float* x2, int64_t n, float a, float b, int op, float* y,
                 crys_stream s);

/* ------------------------------------------------------------------ hash join
 * Section 4.3: no-partitioning hash join over a linear-probing table that is a plain
 * array of 8-byte slots (no pointers).  Slot = key in the low 32 bits, value in the high
 * 32 bits; an empty slot is all ones, so key -1 cannot be stored.  The paper's tables run
 * at 50% fill, i.e. capacity = 2 * rows.  Home slot of key k:
 *   CRYS_HASH_MULT   (0, default) multiplicative (Fibonacci) hashing, the top
 *                    log2(capacity) bits of the 64-bit product
 *                    (uint64)(uint32)k * 0x9E3779B97F4A7C15; for a capacity of at most
 *                    4096 slots, (uint32)(k * 2654435769) >> (32 - log2(capacity));
 *   CRYS_HASH_IDENT  (1) k mod capacity: perfect hashing when the keys are dense
 *                    (0..n-1 with capacity >= n, as for star-schema dimension keys; the
 *                    paper's Section 5.3 cost model assumes perfect hashing), so a table
 *                    needs only capacity >= n and every probe reads one slot;
 * then linear probing with wrap-around (capacity a power of two, >= 2); or
 *   CRYS_HASH_DIRECT (2) slot k holds key k: every key must lie in [0, capacity) (the
 *                    build flags CRYS_DEV_BAD_KEY otherwise), capacity is any value >= 1
 *                    (no power of two needed: n dense keys need exactly n slots), and a
 *                    lookup reads one slot, or none for a key outside [0, capacity).
 *                    Direct tables also let a shared scan tag dimension rows with query
 *                    bitmaps (crys_run_plans_tagged). */
#define CRYS_HASH_MULT 0
#define CRYS_HASH_IDENT 1
#define CRYS_HASH_DIRECT 2
typedef struct {
  uint64_t* slots;  /* capacity slots (device), caller-owned, 8-byte aligned */
  int64_t capacity; /* <= 2^31; a power of two >= 2 unless CRYS_HASH_DIRECT */
  int32_t kind;     /* CRYS_HASH_MULT, CRYS_HASH_IDENT or CRYS_HASH_DIRECT */
} crys_hash;

/* Conjunctive range predicate on a device column: lo <= col[row] <= hi. */
typedef struct {
  const int32_t* col;
  int32_t lo, hi;
} crys_pred;

/* Marks every slot empty.  Must precede the first build into a table. */
int crys_hash_init(const crys_hash* ht, crys_stream s);

/* Build phase: inserts (keys[i], vals[i]) for every row i passing all `n_filters`
 * predicates (the dimension filter of a select-join query is applied at build time,
 * Section 5.3).  vals may be NULL (value 0, membership only).  Keys must be unique and
 * != -1.  Without filters the capacity must be at least n (CRYS_EFULL otherwise); a
 * completely full table still answers probes (bounded by the capacity). */
int crys_hash_build(const int32_t* keys, const int32_t* vals, int64_t n,
                    const crys_pred* filters, int32_t n_filters, const crys_hash* ht,
                    crys_stream s);

/* Probe phase fused with aggregation (Section 4.3, query Q4 with SUM(payload * value)):
 * for each probe row whose key is in the table, sum += (int64)payload[i] * value.
 * Per-thread sums are reduced per thread block and added to *d_sum with one atomic per
 * block.  Sums wrap modulo 2^64.
 *   d_sum      one int64 (device), overwritten
 *   d_matches  one int64 (device) counting matching probe rows, or NULL */
int crys_probe_aggregate(const int32_t* fk, const int32_t* payload, int64_t n,
                         const crys_hash* ht, int64_t* d_sum, int64_t* d_matches,
                         crys_stream s);

/* ------------------------------------------------------------------ sort
 * Section 4.4: least-significant-digit radix sort of (key, value) pairs by signed int32
 * key, 8-bit digits, 4 passes, stable.  One up-front pass histograms all four digits;
 * each digit pass ranks a tile stably inside the thread block and finds the tile's
 * output offsets with a chained (decoupled look-back) scan.  n <= 2^30 - 1.
 * keys_out/vals_out must not overlap the inputs; the inputs are not modified. */
int crys_sort(const int32_t* keys_in, const int32_t* vals_in, int32_t* keys_out,
              int32_t* vals_out, int64_t n, void* d_temp, size_t* temp_bytes, crys_stream s);

/* Most-significant-digit radix sort (Section 4.4: the GPU sort behind the paper's sort
 * figure is an MSB radix sort, not stable).  Two 8-bit partition passes on the top two
 * digits (signed order: the sign bit is flipped), each a histogram, a scan and a scatter
 * whose tiles rank their keys with shared-memory atomics and reserve each digit's run with
 * one global atomic; then every bucket of the top 16 bits is sorted inside one thread
 * block by the low 16 bits (4 stable passes of 4 bits in shared memory) and stored.
 * Keys come out in ascending signed order; rows with EQUAL keys may come out in any order
 * (unstable), so (key, value) pairs are a permutation of the input pairs.  A bucket of
 * more than 8192 rows (heavily repeated top bits) is sorted by one block through global
 * memory: correct for every input, slow only for such skew.  n <= 2^31 - 1; keys_out /
 * vals_out must not overlap the inputs.  Scratch (two-call size query): n keys + n values
 * plus about 1.3 MB of bucket arrays. */
int crys_sort_msb(const int32_t* keys_in, const int32_t* vals_in, int32_t* keys_out,
                  int32_t* vals_out, int64_t n, void* d_temp, size_t* temp_bytes, crys_stream s);

/* Radix-partitioned hash join with aggregation (Section 4.3 names partitioned joins as the
 * alternative to the no-partitioning join when the build side is far beyond the caches).
 * Build side (bkeys[i], bvals[i]), nb rows, unique keys; probe side (fk[j], payload[j]), np
 * rows.  Both sides are partitioned in up to two passes by the top bits of the
 * multiplicative hash key * 2654435769 (bits chosen so that a build partition averages at
 * most 2048 rows), then each probe tile builds its partition's table in shared memory and
 * probes it.  A build partition too large for shared memory (heavily skewed keys) gets its
 * table in scratch.  Same result as crys_hash_build + crys_probe_aggregate:
 *   d_sum      one int64: SUM(payload * value) over matching probe rows (wraps mod 2^64)
 *   d_matches  one int64 counting matching probe rows, or NULL
 * Keys must be unique (a repeated build key sets CRYS_DEV_DUP_KEY).  nb <= 2^30,
 * np <= 2^31 - 1.  Scratch (two-call size query): two copies of each side plus 32 bytes per
 * build row for the oversized-partition tables. */
int crys_join_partitioned(const int32_t* bkeys, const int32_t* bvals, int64_t nb,
                          const int32_t* fk, const int32_t* payload, int64_t np, int64_t* d_sum,
                          int64_t* d_matches, void* d_temp, size_t* temp_bytes, crys_stream s);

/* ------------------------------------------------------------------ query plans
 * Section 5.3: a select-join-aggregate query runs as build kernels for its dimension
 * tables and ONE probe kernel over the fact table that, per tile, applies the fact
 * predicates, probes the dimension tables (rows that miss are dropped), checks the
 * dimension predicates, forms the group id from the joined values, and accumulates
 * SUM(expr) and COUNT per group.
 *
 * A dimension table maps key -> a 32-bit value.  Two ways to use it:
 *  - the paper's plan: build the table with the dimension filter applied at build time
 *    (crys_hash_build filters) and the group attribute as the value; the join then has
 *    no predicates and takes the whole value as its group code;
 *  - resident tables: build ONE table per dimension whose value packs several
 *    attribute codes into bit fields (crys_pack_fields); each query then states its
 *    dimension predicates and its group attribute as bit fields of the value, and all
 *    queries share the table (no per-query build).
 * Field (shift, bits) of a value v is (v >> shift) & (2^bits - 1) for 0 < bits < 32 and
 * the whole int32 v for bits == 0 or 32.  The group id g is the mixed-radix number of
 * the grouped joins' codes in plan order (first grouped join most significant); the
 * number of groups G is the product of their group_card (1 when nothing is grouped). */
#define CRYS_MAX_COLS 16
#define CRYS_MAX_PREDS 8
#define CRYS_MAX_JOINS 4
#define CRYS_MAX_FIELD_PREDS 2
#define CRYS_MAX_PLANS 32

#define CRYS_AGG_A 0       /* SUM(a) */
#define CRYS_AGG_A_MUL_B 1 /* SUM(a * b) */
#define CRYS_AGG_A_SUB_B 2 /* SUM(a - b) */
#define CRYS_AGG_A_ADD_B 3 /* SUM(a + b) */

typedef struct {
  const int32_t* cols[CRYS_MAX_COLS]; /* device columns, n_rows values each */
  int32_t n_cols;
  int64_t n_rows;
} crys_table;

typedef struct {
  int32_t col; /* fact column index */
  int32_t lo, hi;
} crys_col_pred;

typedef struct {
  int32_t shift, bits; /* bit field of the joined value (see above) */
  int32_t lo, hi;      /* lo <= field <= hi */
} crys_field_pred;

typedef struct {
  int32_t fk_col;                 /* fact column holding the foreign key */
  crys_hash ht;                   /* dimension table: key -> value */
  int32_t group_card;             /* 0: not grouped; else group code in [0, group_card) */
  int32_t group_shift, group_bits; /* bit field of the value holding the group code */
  int32_t n_preds;                /* dimension predicates on bit fields of the value */
  crys_field_pred preds[CRYS_MAX_FIELD_PREDS];
} crys_join;

typedef struct {
  int32_t n_preds;
  crys_col_pred preds[CRYS_MAX_PREDS];
  int32_t n_joins;
  crys_join joins[CRYS_MAX_JOINS];
  int32_t agg_op, agg_a, agg_b; /* CRYS_AGG_*, fact column indices */
  int64_t* d_sums;              /* G int64 (device) */
  int64_t* d_counts;            /* G int64 (device) or NULL */
} crys_plan;

/* Number of groups G of a plan (product of group_card over grouped joins). */
int crys_plan_groups(const crys_plan* plan, int64_t* groups);

/* out[i] = OR over k of (cols[k][i] & (2^bits[k] - 1)) << shifts[k], for the dimension
 * value of a resident table (done once when a dimension is loaded; the paper likewise
 * dictionary-encodes attributes before loading, Section 5.2).  cols is a HOST array of
 * n_fields (1..8) device column pointers; fields must not overlap or pass bit 31. */
int crys_pack_fields(const int32_t* const* cols, const int32_t* shifts, const int32_t* bits,
                     int32_t n_fields, int64_t n, int32_t* out, crys_stream s);

/* One query over all fact rows; overwrites the plan's outputs. */
int crys_run_plan(const crys_table* fact, const crys_plan* plan, crys_stream s);

/* Shared scan: up to CRYS_MAX_PLANS queries over rows [row_begin, row_end) of the same
 * fact table in ONE kernel: each tile of the union of the queries' columns is read from
 * HBM once (bulk-prefetched into L2 a few tiles ahead, then read through L1) and every
 * query is evaluated on it.  A (fact column, table) pair that two or more of the queries
 * join on is probed once per row for the whole batch (the 8 most used such pairs) and
 * those queries read the probed value; any other join is probed by its own query.  With
 * CRYS_ACCUMULATE the outputs are added to instead of overwritten, so a query can be
 * carried across several row segments (a circular scan that queries join and leave at
 * segment boundaries).  row_begin must be a multiple of 4. */
#define CRYS_ACCUMULATE 0x1
int crys_run_plans(const crys_table* fact, const crys_plan* plans, int32_t n_plans,
                   int64_t row_begin, int64_t row_end, int flags, crys_stream s);

/* Shared scan with query bitmaps: the shared join of CJOIN (Candea, Polyzotis and
 * Vingralek, VLDB 2009) applied to one batch.  When every join of every plan is on a
 * CRYS_HASH_DIRECT table (at most 8 distinct (fact column, table) pairs), each pair gets
 * a per-batch array of `capacity` 8-byte entries: the slot's value in the high word and,
 * in the low word, the bitmap of the batch's plans that the dimension row satisfies (bit
 * q set when plan q does not join through the pair, or joins it and the row passes all
 * of q's bit-field predicates on it).  The fact scan ANDs one entry per pair into each
 * row's bitmap and finishes only the (row, plan) pairs still set: fact predicates, group
 * code, aggregate.  When the batch's fact predicates lie on at most two columns, each
 * within 256 consecutive values, they too become bitmaps (a per-batch table per column,
 * looked up once per row) and finishing tests none.  Results are those of
 * crys_run_plans, and so is every argument rule.
 *   crys_run_plans_tagged_bytes  scratch bytes the bitmaps of this batch need; 0 when the
 *                                batch cannot be tagged.
 *   scratch       device memory, 16-byte aligned, rebuilt by every call.  With scratch
 *                 NULL or smaller than needed, or a batch that cannot be tagged, the call
 *                 runs crys_run_plans instead (same results, no bitmaps). */
int crys_run_plans_tagged_bytes(const crys_table* fact, const crys_plan* plans, int32_t n_plans,
                                int64_t* bytes);
int crys_run_plans_tagged(const crys_table* fact, const crys_plan* plans, int32_t n_plans,
                          int64_t row_begin, int64_t row_end, int flags, void* scratch,
                          int64_t scratch_bytes, crys_stream s);

/* The tagged scan as a fixed, graph-replayable launch for serving loops (no counterpart in
 * the paper, which runs one query per kernel).  Everything a launch needs - the batch's
 * query descriptors, pairs, row range, annotation flag and the outputs to clear - lives in
 * one argument block in device memory:
 *   crys_tagged_block_bytes  size of the block (host and device copies).
 *   crys_tagged_prepare      fills a HOST block (plain or pinned memory, not read by the
 *                            device) for `plans` over rows [row_begin, row_end): outputs are
 *                            always added to; the n_zero plans listed in zero_plans (indexes
 *                            into plans) have their sums and counts cleared first; with
 *                            CRYS_TAG_ANNOTATE the batch's query bitmaps are rebuilt in
 *                            scratch (needed whenever the batch differs from the one of the
 *                            previous launch on the same scratch).  CRYS_EINVAL when the batch
 *                            cannot be tagged or scratch is smaller than
 *                            crys_run_plans_tagged_bytes(); the caller then uses
 *                            crys_run_plans_tagged.
 *   crys_tagged_launch       launches the work of a DEVICE copy of a block: a prepare kernel
 *                            (clearing, annotation) and the scan.  Its grid and shared memory
 *                            depend only on the tile shape, so a stream capture of
 *                            {copy of the block from pinned memory, crys_tagged_launch} can be
 *                            replayed for every launch of a serving loop.  The tile shape must
 *                            be the one the block was prepared with; a block prepared for
 *                            another shape does no work and raises CRYS_DEV_BOUNDS. */
#define CRYS_TAG_ANNOTATE 0x2
int crys_tagged_block_bytes(int64_t* bytes);
int crys_tagged_prepare(const crys_table* fact, const crys_plan* plans, int32_t n_plans,
                        int64_t row_begin, int64_t row_end, int flags, const int32_t* zero_plans,
                        int32_t n_zero, void* scratch, int64_t scratch_bytes, void* host_block);
int crys_tagged_launch(const void* dev_block, crys_stream s);

/* ------------------------------------------------------------------ tile shapes
 * Each operator is compiled for several tile shapes (threads per block x items per
 * thread, Section 3.3).  crys_tile_variants lists them; crys_set_tile picks the one
 * used by later calls in this process (an autotuner sweeps and persists the choice).
 * CRYS_OP_SHARED_SCAN is crys_run_plans (also when crys_run_plans_tagged falls back to
 * it); CRYS_OP_TAGGED_SCAN is the tagged scan of crys_run_plans_tagged and of the
 * replayable launch (a block must be launched under the shape it was prepared for). */
#define CRYS_OP_SELECT 0
#define CRYS_OP_PROJECT 1
#define CRYS_OP_PROBE 2
#define CRYS_OP_PLAN 3
#define CRYS_OP_SHARED_SCAN 4
#define CRYS_OP_SORT 5
#define CRYS_OP_TAGGED_SCAN 6
#define CRYS_NUM_OPS 7
/* Writes up to `max` (threads, items) pairs; returns the number of variants (or <0). */
int crys_tile_variants(int op, int32_t* threads, int32_t* items, int32_t max);
int crys_set_tile(int op, int32_t variant);
int crys_get_tile(int op);

#ifdef __cplusplus
}
#endif
#endif /* CRYSTAL_H */
