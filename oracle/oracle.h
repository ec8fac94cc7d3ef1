/* Oracle for the Crystal operators: TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, row-at-a-time CPU statement of what each GPU operator computes,
 * written from the paper's definitions ("A Study of the Fundamental Performance
 * Characteristics of GPUs and CPUs for Database Analytics", Shanbhag, Madden, Yu,
 * SIGMOD 2020).  Only the tests, __graft_entry__.smoke() and bench.py's cpu_baseline /
 * reference arm may load it.  It shares no code, header, table or constant with the
 * CUDA library; the only thing both sides share is the seeded input generator.
 *
 * Every function is an exact definition (integer work, or float64 arithmetic rounded
 * once to float32 for projection), so no result here depends on evaluation order,
 * tile shape or hashing.
 */
#ifndef CRYSTAL_ORACLE_H
#define CRYSTAL_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Selection Q0/Q3 (Section 3.2, Section 4.2): every x[i] with lo <= x[i] <= hi is
 * appended to out in input order; returns the number appended.  out holds n slots. */
int64_t orc_select(const int32_t* x, int64_t n, int32_t lo, int32_t hi, int32_t* out);
/* Same rows, input range split evenly over nthreads threads; output identical. */
int64_t orc_select_mt(const int32_t* x, int64_t n, int32_t lo, int32_t hi, int32_t* out,
                      int nthreads);

/* Tile-model scan of Section 3.2 (Figure "tile-example"): a tile of threads*items
 * flags where thread t owns items t, t+threads, t+2*threads, ...  Per-thread match
 * counts, their exclusive prefix sums, the total, and the compacted order (thread t
 * writes its matched item indices, in its own item order, starting at offsets[t]). */
void orc_tile_scan(const uint8_t* flags, int32_t threads, int32_t items, int32_t* counts,
                   int32_t* offsets, int32_t* total, int32_t* order);

/* Projection Q1/Q2 (Section 4.1): y = a*x1 + b*x2 (op 0) or 1/(1+exp(-(a*x1+b*x2)))
 * (op 1), evaluated in float64 and rounded once to float32. */
void orc_project(const float* x1, const float* x2, int64_t n, float a, float b, int op,
                 float* y);
void orc_project_mt(const float* x1, const float* x2, int64_t n, float a, float b, int op,
                    float* y, int nthreads);

/* Equi-join with aggregation (Section 4.3, Q4 with the payload product as the
 * aggregate): for every probe row whose key appears among the build keys,
 * sum += payload[i] * value_of(fk[i]).  Build keys must be unique.  Sums wrap mod 2^64.
 * *matches receives the number of probe rows that found their key.  Returns the sum.
 * The build side is indexed by sorting (key, row) pairs and binary search; no hash
 * table is involved.  Returns INT64_MIN and sets *matches = -1 on duplicate keys. */
int64_t orc_join_sum(const int32_t* bkeys, const int32_t* bvals, int64_t nb,
                     const int32_t* fk, const int32_t* payload, int64_t np, int64_t* matches);
int64_t orc_join_sum_mt(const int32_t* bkeys, const int32_t* bvals, int64_t nb,
                        const int32_t* fk, const int32_t* payload, int64_t np,
                        int64_t* matches, int nthreads);

/* Sort (Section 4.4): (key, value) pairs ordered by signed int32 key, stable (equal
 * keys keep their input order).  Plain top-down merge sort. */
void orc_sort(const int32_t* keys, const int32_t* vals, int64_t n, int32_t* keys_out,
              int32_t* vals_out);

/* Select-join-group-by pipeline (Section 5.3; Figure "query11", Figure "q21-query").
 * For each fact row: all fact predicates hold; for each join the row's foreign key
 * names a dimension row (by unique key) that passes all that join's dimension
 * predicates; then group id g = mixed-radix number of the joined group attributes
 * (first grouped join most significant) and sums[g] += expr(row), counts[g] += 1.
 * expr: op 0 A, 1 A*B, 2 A-B, 3 A+B over fact columns, each in int64. */
#define ORC_MAX_COLS 16
#define ORC_MAX_PREDS 8
#define ORC_MAX_JOINS 4
#define ORC_MAX_DIM_PREDS 4

typedef struct {
  const int32_t* col; /* dimension column */
  int32_t lo, hi;     /* lo <= col[d] <= hi */
} orc_dim_pred;

typedef struct {
  int32_t fk_col;           /* fact column holding the foreign key */
  const int32_t* dim_keys;  /* unique dimension keys */
  int64_t dim_rows;
  int32_t n_preds;
  orc_dim_pred preds[ORC_MAX_DIM_PREDS];
  const int32_t* group_attr; /* group code per dimension row, or NULL */
  int32_t group_card;        /* codes lie in [0, group_card); 1 when not grouped */
} orc_join;

typedef struct {
  int32_t col, lo, hi; /* lo <= fact[col][r] <= hi */
} orc_fact_pred;

typedef struct {
  const int32_t* cols[ORC_MAX_COLS];
  int32_t n_cols;
  int64_t n_rows;
  int32_t n_preds;
  orc_fact_pred preds[ORC_MAX_PREDS];
  int32_t n_joins;
  orc_join joins[ORC_MAX_JOINS];
  int32_t agg_op, agg_a, agg_b;
} orc_plan;

/* Returns 0, or -1 for an invalid plan (bad column index, group code out of range,
 * duplicate dimension key).  sums/counts hold prod(group_card) entries. */
int orc_run_plan(const orc_plan* p, int64_t* sums, int64_t* counts);
int orc_run_plan_mt(const orc_plan* p, int64_t* sums, int64_t* counts, int nthreads);

int orc_hardware_threads(void);

#ifdef __cplusplus
}
#endif
#endif
