/* Oracle for the Crystal operators: TEST INFRASTRUCTURE ONLY (see oracle.h).
 * Plain row-at-a-time loops; the _mt variants run the very same loops on disjoint row
 * ranges in pthreads and merge the results, for the CPU baseline timing. */
#include "oracle.h"

#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

int orc_hardware_threads(void) {
  long n = sysconf(_SC_NPROCESSORS_ONLN);
  return n > 0 ? (int)n : 1;
}

/* ---------------------------------------------------------------- selection */

/* Section 4.2, query Q3 / Section 3.2, query Q0: keep the entries that satisfy the
 * predicate, in input order (the branching form of Figure "selscan-example"). */
int64_t orc_select(const int32_t* x, int64_t n, int32_t lo, int32_t hi, int32_t* out) {
  int64_t count = 0;
  for (int64_t i = 0; i < n; ++i) {
    if (x[i] >= lo && x[i] <= hi) {
      out[count] = x[i];
      count += 1;
    }
  }
  return count;
}

typedef struct {
  const int32_t* x;
  int64_t begin, end;
  int32_t lo, hi;
  int32_t* out; /* this range's own region, written from out[begin] */
  int64_t count;
} sel_task;

static void* sel_worker(void* arg) {
  sel_task* t = (sel_task*)arg;
  t->count = orc_select(t->x + t->begin, t->end - t->begin, t->lo, t->hi, t->out + t->begin);
  return NULL;
}

int64_t orc_select_mt(const int32_t* x, int64_t n, int32_t lo, int32_t hi, int32_t* out,
                      int nthreads) {
  if (nthreads < 1) nthreads = 1;
  sel_task* tasks = (sel_task*)calloc((size_t)nthreads, sizeof(sel_task));
  pthread_t* th = (pthread_t*)calloc((size_t)nthreads, sizeof(pthread_t));
  for (int t = 0; t < nthreads; ++t) {
    tasks[t].x = x;
    tasks[t].begin = n * t / nthreads;
    tasks[t].end = n * (t + 1) / nthreads;
    tasks[t].lo = lo;
    tasks[t].hi = hi;
    tasks[t].out = out;
    pthread_create(&th[t], NULL, sel_worker, &tasks[t]);
  }
  int64_t total = 0;
  for (int t = 0; t < nthreads; ++t) {
    pthread_join(th[t], NULL);
    /* ranges are in order and each range's output starts at or after `total` */
    memmove(out + total, out + tasks[t].begin, (size_t)tasks[t].count * sizeof(int32_t));
    total += tasks[t].count;
  }
  free(tasks);
  free(th);
  return total;
}

/* Section 3.2, Figure "tile-example": thread t evaluates items t, t+T, t+2T, ...;
 * counts its matches; the block's exclusive prefix sum of the counts gives each
 * thread's write offset; the sum of all counts is the tile's total. */
void orc_tile_scan(const uint8_t* flags, int32_t threads, int32_t items, int32_t* counts,
                   int32_t* offsets, int32_t* total, int32_t* order) {
  for (int32_t t = 0; t < threads; ++t) {
    int32_t c = 0;
    for (int32_t k = 0; k < items; ++k) c += flags[t + k * threads] ? 1 : 0;
    counts[t] = c;
  }
  int32_t running = 0;
  for (int32_t t = 0; t < threads; ++t) {
    offsets[t] = running;
    running += counts[t];
  }
  *total = running;
  for (int32_t t = 0; t < threads; ++t) {
    int32_t pos = offsets[t];
    for (int32_t k = 0; k < items; ++k) {
      int32_t item = t + k * threads;
      if (flags[item]) order[pos++] = item;
    }
  }
}

/* ---------------------------------------------------------------- projection */

/* Section 4.1, Q1 and Q2: a*x1 + b*x2 and its sigmoid 1/(1+e^-y), in float64,
 * rounded once to the 4-byte output. */
void orc_project(const float* x1, const float* x2, int64_t n, float a, float b, int op,
                 float* y) {
  for (int64_t i = 0; i < n; ++i) {
    double lin = (double)a * (double)x1[i] + (double)b * (double)x2[i];
    double r = op == 1 ? 1.0 / (1.0 + exp(-lin)) : lin;
    y[i] = (float)r;
  }
}

typedef struct {
  const float *x1, *x2;
  int64_t begin, end;
  float a, b;
  int op;
  float* y;
} proj_task;

static void* proj_worker(void* arg) {
  proj_task* t = (proj_task*)arg;
  orc_project(t->x1 + t->begin, t->x2 + t->begin, t->end - t->begin, t->a, t->b, t->op,
              t->y + t->begin);
  return NULL;
}

void orc_project_mt(const float* x1, const float* x2, int64_t n, float a, float b, int op,
                    float* y, int nthreads) {
  if (nthreads < 1) nthreads = 1;
  proj_task* tasks = (proj_task*)calloc((size_t)nthreads, sizeof(proj_task));
  pthread_t* th = (pthread_t*)calloc((size_t)nthreads, sizeof(pthread_t));
  for (int t = 0; t < nthreads; ++t) {
    proj_task v = {x1, x2, n * t / nthreads, n * (t + 1) / nthreads, a, b, op, y};
    tasks[t] = v;
    pthread_create(&th[t], NULL, proj_worker, &tasks[t]);
  }
  for (int t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);
  free(tasks);
  free(th);
}

/* ---------------------------------------------------------------- sorting */

typedef struct {
  int32_t key;
  int32_t val;
} kv;

/* Top-down merge sort of a[lo, hi) using tmp; ties take the left run first, which
 * keeps equal keys in input order. */
static void merge_sort_rec(kv* a, kv* tmp, int64_t lo, int64_t hi) {
  if (hi - lo < 2) return;
  int64_t mid = lo + (hi - lo) / 2;
  merge_sort_rec(a, tmp, lo, mid);
  merge_sort_rec(a, tmp, mid, hi);
  int64_t i = lo, j = mid, k = lo;
  while (i < mid && j < hi) {
    if (a[j].key < a[i].key)
      tmp[k++] = a[j++];
    else
      tmp[k++] = a[i++];
  }
  while (i < mid) tmp[k++] = a[i++];
  while (j < hi) tmp[k++] = a[j++];
  memcpy(a + lo, tmp + lo, (size_t)(hi - lo) * sizeof(kv));
}

static void stable_sort_kv(kv* a, int64_t n) {
  if (n < 2) return;
  kv* tmp = (kv*)malloc((size_t)n * sizeof(kv));
  merge_sort_rec(a, tmp, 0, n);
  free(tmp);
}

/* Section 4.4: the result radix sort produces, stated as a stable sort by key. */
void orc_sort(const int32_t* keys, const int32_t* vals, int64_t n, int32_t* keys_out,
              int32_t* vals_out) {
  kv* a = (kv*)malloc((size_t)(n > 0 ? n : 1) * sizeof(kv));
  for (int64_t i = 0; i < n; ++i) {
    a[i].key = keys[i];
    a[i].val = vals[i];
  }
  stable_sort_kv(a, n);
  for (int64_t i = 0; i < n; ++i) {
    keys_out[i] = a[i].key;
    vals_out[i] = a[i].val;
  }
  free(a);
}

/* ---------------------------------------------------------------- joins */

/* Index of a build side: (key, row) pairs sorted by key. */
typedef struct {
  kv* pairs; /* key, row index */
  int64_t n;
  int duplicate;
} key_index;

static key_index index_build(const int32_t* keys, int64_t n) {
  key_index ix;
  ix.n = n;
  ix.duplicate = 0;
  ix.pairs = (kv*)malloc((size_t)(n > 0 ? n : 1) * sizeof(kv));
  for (int64_t i = 0; i < n; ++i) {
    ix.pairs[i].key = keys[i];
    ix.pairs[i].val = (int32_t)i;
  }
  stable_sort_kv(ix.pairs, n);
  for (int64_t i = 1; i < n; ++i)
    if (ix.pairs[i].key == ix.pairs[i - 1].key) ix.duplicate = 1;
  return ix;
}

/* Row of the build side holding `key`, or -1. */
static int64_t index_find(const key_index* ix, int32_t key) {
  int64_t lo = 0, hi = ix->n;
  while (lo < hi) {
    int64_t mid = lo + (hi - lo) / 2;
    if (ix->pairs[mid].key < key)
      lo = mid + 1;
    else
      hi = mid;
  }
  if (lo < ix->n && ix->pairs[lo].key == key) return ix->pairs[lo].val;
  return -1;
}

typedef struct {
  const key_index* ix;
  const int32_t* bvals;
  const int32_t *fk, *payload;
  int64_t begin, end;
  uint64_t sum;
  int64_t matches;
} join_task;

static void* join_worker(void* arg) {
  join_task* t = (join_task*)arg;
  uint64_t sum = 0;
  int64_t matches = 0;
  for (int64_t i = t->begin; i < t->end; ++i) {
    int64_t row = index_find(t->ix, t->fk[i]);
    if (row >= 0) {
      sum += (uint64_t)((int64_t)t->payload[i] * (int64_t)t->bvals[row]);
      matches += 1;
    }
  }
  t->sum = sum;
  t->matches = matches;
  return NULL;
}

/* Section 4.3, query Q4: equi-join of probe rows with build rows on the key, summing
 * the product of the probe payload and the build value over matching pairs. */
int64_t orc_join_sum_mt(const int32_t* bkeys, const int32_t* bvals, int64_t nb,
                        const int32_t* fk, const int32_t* payload, int64_t np,
                        int64_t* matches, int nthreads) {
  if (nthreads < 1) nthreads = 1;
  key_index ix = index_build(bkeys, nb);
  if (ix.duplicate) {
    free(ix.pairs);
    if (matches) *matches = -1;
    return INT64_MIN;
  }
  join_task* tasks = (join_task*)calloc((size_t)nthreads, sizeof(join_task));
  pthread_t* th = (pthread_t*)calloc((size_t)nthreads, sizeof(pthread_t));
  for (int t = 0; t < nthreads; ++t) {
    join_task v = {&ix, bvals, fk, payload, np * t / nthreads, np * (t + 1) / nthreads, 0, 0};
    tasks[t] = v;
    pthread_create(&th[t], NULL, join_worker, &tasks[t]);
  }
  uint64_t sum = 0;
  int64_t m = 0;
  for (int t = 0; t < nthreads; ++t) {
    pthread_join(th[t], NULL);
    sum += tasks[t].sum;
    m += tasks[t].matches;
  }
  if (matches) *matches = m;
  free(tasks);
  free(th);
  free(ix.pairs);
  return (int64_t)sum;
}

int64_t orc_join_sum(const int32_t* bkeys, const int32_t* bvals, int64_t nb,
                     const int32_t* fk, const int32_t* payload, int64_t np, int64_t* matches) {
  return orc_join_sum_mt(bkeys, bvals, nb, fk, payload, np, matches, 1);
}

/* ---------------------------------------------------------------- query plans */

typedef struct {
  const orc_plan* p;
  const key_index* ix; /* one per join */
  int64_t begin, end;
  int64_t groups;
  uint64_t* sums;
  int64_t* counts;
  int bad;
} plan_task;

static int64_t agg_value(const orc_plan* p, int64_t r) {
  int64_t a = p->cols[p->agg_a][r];
  int64_t b = p->agg_op == 0 ? 0 : p->cols[p->agg_b][r];
  switch (p->agg_op) {
    case 1: return a * b;
    case 2: return a - b;
    case 3: return a + b;
    default: return a;
  }
}

static void* plan_worker(void* arg) {
  plan_task* t = (plan_task*)arg;
  const orc_plan* p = t->p;
  for (int64_t r = t->begin; r < t->end; ++r) {
    int keep = 1;
    for (int32_t k = 0; k < p->n_preds && keep; ++k) {
      int32_t v = p->cols[p->preds[k].col][r];
      keep = v >= p->preds[k].lo && v <= p->preds[k].hi;
    }
    int64_t g = 0;
    for (int32_t j = 0; j < p->n_joins && keep; ++j) {
      const orc_join* jn = &p->joins[j];
      int64_t d = index_find(&t->ix[j], p->cols[jn->fk_col][r]);
      if (d < 0) {
        keep = 0;
        break;
      }
      for (int32_t k = 0; k < jn->n_preds && keep; ++k) {
        int32_t v = jn->preds[k].col[d];
        keep = v >= jn->preds[k].lo && v <= jn->preds[k].hi;
      }
      if (!keep) break;
      if (jn->group_attr) {
        int32_t code = jn->group_attr[d];
        if (code < 0 || code >= jn->group_card) {
          t->bad = 1;
          keep = 0;
          break;
        }
        g = g * jn->group_card + code;
      }
    }
    if (!keep) continue;
    t->sums[g] += (uint64_t)agg_value(p, r);
    t->counts[g] += 1;
  }
  return NULL;
}

static int plan_valid(const orc_plan* p, int64_t* groups) {
  if (p->n_cols < 0 || p->n_cols > ORC_MAX_COLS || p->n_preds < 0 ||
      p->n_preds > ORC_MAX_PREDS || p->n_joins < 0 || p->n_joins > ORC_MAX_JOINS)
    return 0;
  for (int32_t k = 0; k < p->n_preds; ++k)
    if (p->preds[k].col < 0 || p->preds[k].col >= p->n_cols) return 0;
  if (p->agg_op < 0 || p->agg_op > 3) return 0;
  if (p->agg_a < 0 || p->agg_a >= p->n_cols) return 0;
  if (p->agg_op != 0 && (p->agg_b < 0 || p->agg_b >= p->n_cols)) return 0;
  int64_t g = 1;
  for (int32_t j = 0; j < p->n_joins; ++j) {
    const orc_join* jn = &p->joins[j];
    if (jn->fk_col < 0 || jn->fk_col >= p->n_cols) return 0;
    if (jn->n_preds < 0 || jn->n_preds > ORC_MAX_DIM_PREDS) return 0;
    if (jn->group_attr) {
      if (jn->group_card < 1) return 0;
      g *= jn->group_card;
    }
  }
  *groups = g;
  return 1;
}

int orc_run_plan_mt(const orc_plan* p, int64_t* sums, int64_t* counts, int nthreads) {
  int64_t groups = 0;
  if (!plan_valid(p, &groups)) return -1;
  if (nthreads < 1) nthreads = 1;
  key_index ix[ORC_MAX_JOINS];
  int dup = 0;
  for (int32_t j = 0; j < p->n_joins; ++j) {
    ix[j] = index_build(p->joins[j].dim_keys, p->joins[j].dim_rows);
    dup |= ix[j].duplicate;
  }
  int rc = 0;
  if (dup) {
    rc = -1;
  } else {
    plan_task* tasks = (plan_task*)calloc((size_t)nthreads, sizeof(plan_task));
    pthread_t* th = (pthread_t*)calloc((size_t)nthreads, sizeof(pthread_t));
    for (int t = 0; t < nthreads; ++t) {
      tasks[t].p = p;
      tasks[t].ix = ix;
      tasks[t].begin = p->n_rows * t / nthreads;
      tasks[t].end = p->n_rows * (t + 1) / nthreads;
      tasks[t].groups = groups;
      tasks[t].sums = (uint64_t*)calloc((size_t)groups, sizeof(uint64_t));
      tasks[t].counts = (int64_t*)calloc((size_t)groups, sizeof(int64_t));
      pthread_create(&th[t], NULL, plan_worker, &tasks[t]);
    }
    for (int64_t g = 0; g < groups; ++g) {
      sums[g] = 0;
      if (counts) counts[g] = 0;
    }
    for (int t = 0; t < nthreads; ++t) {
      pthread_join(th[t], NULL);
      if (tasks[t].bad) rc = -1;
      for (int64_t g = 0; g < groups; ++g) {
        sums[g] = (int64_t)((uint64_t)sums[g] + tasks[t].sums[g]);
        if (counts) counts[g] += tasks[t].counts[g];
      }
      free(tasks[t].sums);
      free(tasks[t].counts);
    }
    free(tasks);
    free(th);
  }
  for (int32_t j = 0; j < p->n_joins; ++j) free(ix[j].pairs);
  return rc;
}

int orc_run_plan(const orc_plan* p, int64_t* sums, int64_t* counts) {
  return orc_run_plan_mt(p, sums, counts, 1);
}
