/*
 * Oracle — plain CPU definitions of every result the GPU library computes.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is compiled into oracle/liboracle.so and
 * is loaded by tests/, by __graft_entry__.smoke() and by the CPU-baseline leg of
 * bench.py — never by the library itself.  It shares no code, header, table or
 * helper with the CUDA path (paper_2502_09541_gb300/csrc); the two only read the
 * same host buffers written by datagen/.
 *
 * Everything here is integer except the MLP CDF model (fp64).  Integer results
 * are exact definitions: two's-complement wrapping int64 sums (computed in
 * uint64), ascending row ids, stable orders.  Dimension and build-side lookups
 * use qsort + bsearch over (key, row) pairs — library primitives — so a reader
 * can check each function against the paper by eye.
 *
 * Multi-threaded variants split rows into contiguous ranges and add the
 * per-range partial results; wrapping addition is associative and commutative,
 * so the result does not depend on the thread count.
 */
#define _GNU_SOURCE /* qsort_r */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "oracle.h"

#define OR_EXPORT __attribute__((visibility("default")))

/* ------------------------------------------------------------------ */
/* predicates: op codes match the row predicate vocabulary of Section 6.3
 * (selection predicates sigma_a, sigma_b); all compare int32 values. */
static int pred_holds(int32_t v, int32_t op, int32_t lo, int32_t hi) {
  switch (op) {
    case OR_BETWEEN: return lo <= v && v <= hi;
    case OR_EQ: return v == lo;
    case OR_NE: return v != lo;
    case OR_LT: return v < lo;
    case OR_LE: return v <= lo;
    case OR_GT: return v > lo;
    case OR_GE: return v >= lo;
    default: return 0;
  }
}

/* ------------------------------------------------------------------ */
/* sorted (key,row) index of a dimension, for bsearch lookups */
typedef struct { int32_t key; uint32_t row; } kr32;

static int cmp_kr32(const void *a, const void *b) {
  const kr32 *x = (const kr32 *)a, *y = (const kr32 *)b;
  if (x->key != y->key) return x->key < y->key ? -1 : 1;
  return x->row < y->row ? -1 : (x->row > y->row);
}
static int cmp_key32(const void *k, const void *e) {
  int32_t a = *(const int32_t *)k, b = ((const kr32 *)e)->key;
  return a < b ? -1 : (a > b);
}

/* builds the index; returns 0, or OR_E_DUPKEY if a key repeats */
static int build_index(const int32_t *key, uint64_t rows, kr32 **out) {
  kr32 *ix = (kr32 *)malloc(sizeof(kr32) * (rows ? rows : 1));
  for (uint64_t i = 0; i < rows; ++i) { ix[i].key = key[i]; ix[i].row = (uint32_t)i; }
  qsort(ix, rows, sizeof(kr32), cmp_kr32);
  for (uint64_t i = 1; i < rows; ++i)
    if (ix[i].key == ix[i - 1].key) { free(ix); return OR_E_DUPKEY; }
  *out = ix;
  return 0;
}

static int64_t lookup(const kr32 *ix, uint64_t rows, int32_t k) {
  const kr32 *e = (const kr32 *)bsearch(&k, ix, rows, sizeof(kr32), cmp_key32);
  return e ? (int64_t)e->row : -1;
}

/* ------------------------------------------------------------------ */
/* O1: single-dimension query (Section 7.1 star-join shape): join fact rows to
 * the date dimension, keep year == year_eq AND disc_lo <= discount <= disc_hi
 * AND quantity < qty_lt, return SUM(price * discount) in wrapping int64. */
OR_EXPORT int or_q1(const int32_t *date_fk, const int32_t *quantity, const int32_t *discount,
                    const int32_t *price, uint64_t n, const int32_t *dim_key, const int32_t *dim_year,
                    uint64_t dim_rows, int32_t year_eq, int32_t disc_lo, int32_t disc_hi,
                    int32_t qty_lt, int64_t *sum, uint64_t *count) {
  kr32 *ix;
  int st = build_index(dim_key, dim_rows, &ix);
  if (st) return st;
  uint64_t s = 0, c = 0;
  for (uint64_t i = 0; i < n; ++i) {
    int64_t r = lookup(ix, dim_rows, date_fk[i]);
    if (r < 0) continue;
    if (dim_year[r] != year_eq) continue;
    if (discount[i] < disc_lo || discount[i] > disc_hi) continue;
    if (quantity[i] >= qty_lt) continue;
    s += (uint64_t)((int64_t)price[i] * (int64_t)discount[i]);
    c += 1;
  }
  free(ix);
  *sum = (int64_t)s;
  *count = c;
  return 0;
}

/* ------------------------------------------------------------------ */
/* O2: star query.  Per dimension: the fact foreign key column is looked up in
 * the dimension (inner join — a missing key drops the row), the dimension
 * predicates are applied to the matched dimension row (Section 7.1: filter the
 * dimension tables, then probe), the fact predicates are applied to the fact
 * row, the group id is the mixed-radix number of the group-key codes (first
 * key most significant), and sum[g] += agg(a, b), cnt[g] += 1 in wrapping
 * int64. */
typedef struct {
  const or_star_query *q;
  kr32 **ix;
  uint64_t begin, end;
  uint64_t *sums, *cnts;
  int status;
} star_job;

static void star_range(star_job *j) {
  const or_star_query *q = j->q;
  for (uint64_t i = j->begin; i < j->end; ++i) {
    int keep = 1;
    for (int p = 0; p < q->n_fact_preds && keep; ++p) {
      const or_pred *fp = &q->fact_preds[p];
      keep = pred_holds(fp->col[i], fp->op, fp->lo, fp->hi);
    }
    if (!keep) continue;
    int64_t drow[OR_MAX_DIMS];
    for (int d = 0; d < q->n_dims && keep; ++d) {
      const or_dim *dm = &q->dims[d];
      drow[d] = lookup(j->ix[d], dm->rows, dm->fact_fk[i]);
      if (drow[d] < 0) { keep = 0; break; }
      for (int p = 0; p < dm->n_preds && keep; ++p)
        keep = pred_holds(dm->attr[dm->pred_attr[p]][drow[d]], dm->pred_op[p], dm->pred_lo[p],
                          dm->pred_hi[p]);
    }
    if (!keep) continue;
    uint64_t g = 0;
    for (int k = 0; k < q->n_group_keys; ++k) {
      const or_gkey *gk = &q->group_keys[k];
      int32_t code = gk->dim < 0 ? gk->fact_col[i] : q->dims[gk->dim].attr[gk->attr][drow[gk->dim]];
      if (code < 0 || code >= gk->card) { j->status = OR_E_RANGE; return; }
      g = g * (uint64_t)gk->card + (uint64_t)code;
    }
    int64_t a = q->agg_a ? q->agg_a[i] : 0, b = q->agg_b ? q->agg_b[i] : 0, v;
    switch (q->agg_op) {
      case OR_AGG_SUM: v = a; break;
      case OR_AGG_MUL: v = a * b; break;
      case OR_AGG_SUB: v = a - b; break;
      default: v = 0; break; /* COUNT only */
    }
    j->sums[g] += (uint64_t)v;
    j->cnts[g] += 1;
  }
}

static void *star_thread(void *p) { star_range((star_job *)p); return NULL; }

OR_EXPORT uint64_t or_star_groups(const or_star_query *q) {
  uint64_t g = 1;
  for (int k = 0; k < q->n_group_keys; ++k) g *= (uint64_t)q->group_keys[k].card;
  return g;
}

OR_EXPORT int or_star(const or_star_query *q, int64_t *sums, uint64_t *counts, int nthreads) {
  if (q->n_dims > OR_MAX_DIMS) return OR_E_RANGE;
  kr32 *ix[OR_MAX_DIMS] = {0};
  int st = 0;
  for (int d = 0; d < q->n_dims && !st; ++d) st = build_index(q->dims[d].key, q->dims[d].rows, &ix[d]);
  uint64_t G = or_star_groups(q);
  memset(sums, 0, G * sizeof(int64_t));
  memset(counts, 0, G * sizeof(uint64_t));
  if (nthreads < 1) nthreads = 1;
  if (nthreads > 256) nthreads = 256;
  star_job jobs[256];
  pthread_t th[256];
  for (int t = 0; t < nthreads && !st; ++t) {
    jobs[t].q = q; jobs[t].ix = ix; jobs[t].status = 0;
    jobs[t].begin = q->n * (uint64_t)t / (uint64_t)nthreads;
    jobs[t].end = q->n * (uint64_t)(t + 1) / (uint64_t)nthreads;
    jobs[t].sums = (uint64_t *)calloc(G, 8);
    jobs[t].cnts = (uint64_t *)calloc(G, 8);
    if (nthreads == 1) star_range(&jobs[t]);
    else pthread_create(&th[t], NULL, star_thread, &jobs[t]);
  }
  if (!st) {
    for (int t = 0; t < nthreads; ++t) {
      if (nthreads > 1) pthread_join(th[t], NULL);
      if (jobs[t].status) st = jobs[t].status;
      for (uint64_t g = 0; g < G; ++g) {
        sums[g] = (int64_t)((uint64_t)sums[g] + jobs[t].sums[g]);
        counts[g] += jobs[t].cnts[g];
      }
      free(jobs[t].sums);
      free(jobs[t].cnts);
    }
  }
  for (int d = 0; d < q->n_dims; ++d) free(ix[d]);
  return st;
}

/* ------------------------------------------------------------------ */
/* Filter with stream compaction (Section 6.3 selection): the ascending row ids
 * (row0 + i) of rows satisfying every predicate.  Writes at most cap ids,
 * always returns the full count. */
OR_EXPORT int or_filter(uint64_t n, uint64_t row0, int n_preds, const or_pred *preds, uint64_t *out_rows,
                        uint64_t cap, uint64_t *out_count) {
  uint64_t c = 0;
  for (uint64_t i = 0; i < n; ++i) {
    int keep = 1;
    for (int p = 0; p < n_preds && keep; ++p) keep = pred_holds(preds[p].col[i], preds[p].op, preds[p].lo, preds[p].hi);
    if (!keep) continue;
    if (out_rows && c < cap) out_rows[c] = row0 + i;
    c += 1;
  }
  *out_count = c;
  return 0;
}

/* ------------------------------------------------------------------ */
/* O3: sort of (uint64 key, uint32 row id) pairs, stable by key (Section 6.1
 * sorts 64-bit integers; equal keys keep input order).  Implemented as qsort
 * on the unique composite (key, input index). */
static int cmp_ki(const void *a, const void *b, void *ctx) {
  const uint64_t *keys = (const uint64_t *)ctx;
  uint64_t x = *(const uint64_t *)a, y = *(const uint64_t *)b;
  if (keys[x] != keys[y]) return keys[x] < keys[y] ? -1 : 1;
  return x < y ? -1 : (x > y);
}

OR_EXPORT int or_sort_pairs(const uint64_t *keys, const uint32_t *rowids, uint64_t n, uint64_t *out_keys,
                            uint32_t *out_rowids) {
  uint64_t *idx = (uint64_t *)malloc(sizeof(uint64_t) * (n ? n : 1));
  if (!idx) return OR_E_NOMEM;
  for (uint64_t i = 0; i < n; ++i) idx[i] = i;
  qsort_r(idx, n, sizeof(uint64_t), cmp_ki, (void *)keys);
  for (uint64_t i = 0; i < n; ++i) {
    out_keys[i] = keys[idx[i]];
    out_rowids[i] = rowids[idx[i]];
  }
  free(idx);
  return 0;
}

/* Exact cut of sorted runs (Section 6.1, MergeExKernel data mapping: regroup
 * sorted chunks into partitions with max(P_i) <= min(P_i+1)).  The runs are
 * consecutive pieces [run_off[r], run_off[r+1]) of keys.  Definition: order
 * all n keys stably (by key, then by position), take the first k of that
 * order, and count how many of them lie in each run.  k >= n takes every
 * element. */
OR_EXPORT int or_exact_cut(const uint64_t *keys, const uint64_t *run_off, uint32_t n_runs, uint64_t k,
                           uint64_t *out) {
  const uint64_t n = run_off[n_runs];
  uint64_t *idx = (uint64_t *)malloc(sizeof(uint64_t) * (n ? n : 1));
  if (!idx) return OR_E_NOMEM;
  for (uint64_t i = 0; i < n; ++i) idx[i] = i;
  qsort_r(idx, n, sizeof(uint64_t), cmp_ki, (void *)keys);
  for (uint32_t r = 0; r < n_runs; ++r) out[r] = 0;
  for (uint64_t i = 0; i < k && i < n; ++i) {
    uint32_t r = 0;
    while (idx[i] >= run_off[r + 1]) ++r;
    out[r] += 1;
  }
  free(idx);
  return 0;
}

/* ------------------------------------------------------------------ */
/* SplitMix64 output finalizer (Steele, Lea & Flood 2014): the mixing function
 * of the join pair fingerprint. */
static uint64_t fmix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
static uint64_t rotl64(uint64_t x, int r) { return (x << r) | (x >> (64 - r)); }

OR_EXPORT uint64_t or_pair_fp(uint64_t probe_row, uint64_t payload) { return fmix(probe_row ^ rotl64(payload, 17)); }

/* O4: equi-join A.key == B.key (Section 6.2; build keys unique).  For every
 * probe row j whose key matches build row r: count += 1, psum += payload[r],
 * fp += fmix(j ^ rotl(payload[r], 17)), all wrapping. */
typedef struct { int64_t key; uint64_t row; } kr64;
static int cmp_kr64(const void *a, const void *b) {
  const kr64 *x = (const kr64 *)a, *y = (const kr64 *)b;
  if (x->key != y->key) return x->key < y->key ? -1 : 1;
  return x->row < y->row ? -1 : (x->row > y->row);
}
static int cmp_key64(const void *k, const void *e) {
  int64_t a = *(const int64_t *)k, b = ((const kr64 *)e)->key;
  return a < b ? -1 : (a > b);
}

typedef struct {
  const kr64 *ix; const int64_t *bpay; uint64_t nb;
  const int64_t *pkeys; uint64_t row0, begin, end;
  uint64_t count, psum, fp;
} join_job;

static void *join_thread(void *p) {
  join_job *j = (join_job *)p;
  uint64_t c = 0, s = 0, f = 0;
  for (uint64_t i = j->begin; i < j->end; ++i) {
    const kr64 *e = (const kr64 *)bsearch(&j->pkeys[i], j->ix, j->nb, sizeof(kr64), cmp_key64);
    if (!e) continue;
    uint64_t pay = (uint64_t)j->bpay[e->row];
    c += 1;
    s += pay;
    f += or_pair_fp(j->row0 + i, pay);
  }
  j->count = c; j->psum = s; j->fp = f;
  return NULL;
}

OR_EXPORT int or_join(const int64_t *bkeys, const int64_t *bpay, uint64_t nb, const int64_t *pkeys, uint64_t np,
                      uint64_t probe_row0, uint64_t *count, uint64_t *psum, uint64_t *fp, int nthreads) {
  kr64 *ix = (kr64 *)malloc(sizeof(kr64) * (nb ? nb : 1));
  if (!ix) return OR_E_NOMEM;
  for (uint64_t i = 0; i < nb; ++i) { ix[i].key = bkeys[i]; ix[i].row = i; }
  qsort(ix, nb, sizeof(kr64), cmp_kr64);
  for (uint64_t i = 1; i < nb; ++i)
    if (ix[i].key == ix[i - 1].key) { free(ix); return OR_E_DUPKEY; }
  if (nthreads < 1) nthreads = 1;
  if (nthreads > 256) nthreads = 256;
  join_job jobs[256];
  pthread_t th[256];
  for (int t = 0; t < nthreads; ++t) {
    join_job jj = {ix, bpay, nb, pkeys, probe_row0, np * (uint64_t)t / (uint64_t)nthreads,
                   np * (uint64_t)(t + 1) / (uint64_t)nthreads, 0, 0, 0};
    jobs[t] = jj;
    if (nthreads == 1) join_thread(&jobs[t]);
    else pthread_create(&th[t], NULL, join_thread, &jobs[t]);
  }
  uint64_t c = 0, s = 0, f = 0;
  for (int t = 0; t < nthreads; ++t) {
    if (nthreads > 1) pthread_join(th[t], NULL);
    c += jobs[t].count; s += jobs[t].psum; f += jobs[t].fp;
  }
  free(ix);
  *count = c; *psum = s; *fp = f;
  return 0;
}

/* ------------------------------------------------------------------ */
/* find_boundary (Section 6.2.1, Fig. 9): input hashes already clustered
 * (non-decreasing); boundary has N+1 entries.  (1) every entry starts as a
 * placeholder; (2) position i whose hash differs from the previous position's
 * (or i == 0) records i at entry hash[i]; the last entry is n; (3) every
 * remaining placeholder is replaced by the next valid boundary to its right. */
OR_EXPORT void or_find_boundary(const uint32_t *hash, uint64_t n, uint32_t N, uint64_t *boundary) {
  const uint64_t NA = UINT64_MAX;
  for (uint32_t g = 0; g <= N; ++g) boundary[g] = NA;
  for (uint64_t i = 0; i < n; ++i)
    if (i == 0 || hash[i] != hash[i - 1]) boundary[hash[i]] = i;
  boundary[N] = n;
  for (int64_t g = (int64_t)N - 1; g >= 0; --g)
    if (boundary[g] == NA) boundary[g] = boundary[g + 1];
}

/* ------------------------------------------------------------------ */
/* Range partition (Section 6.2.1 clustering, with a monotone range function in
 * place of low key bits): pid(key) = number of splitters <= key, so partition
 * p holds [s_{p-1}, s_p).  Output is a stable scatter (input order kept inside
 * each partition) and the P+1 boundary array of partition starts. */
OR_EXPORT uint32_t or_pid(uint64_t key, const uint64_t *splitters, uint32_t P) {
  uint32_t c = 0;
  for (uint32_t j = 0; j + 1 < P; ++j) c += splitters[j] <= key;
  return c;
}

OR_EXPORT void or_range_partition(const uint64_t *keys, const uint32_t *rowids, uint64_t n,
                                  const uint64_t *splitters, uint32_t P, uint64_t *out_keys,
                                  uint32_t *out_rowids, uint64_t *boundary) {
  uint64_t *cnt = (uint64_t *)calloc(P + 1, 8);
  for (uint64_t i = 0; i < n; ++i) cnt[or_pid(keys[i], splitters, P)] += 1;
  boundary[0] = 0;
  for (uint32_t p = 0; p < P; ++p) boundary[p + 1] = boundary[p] + cnt[p];
  uint64_t *cur = (uint64_t *)malloc(8 * (P + 1));
  memcpy(cur, boundary, 8 * (P + 1));
  for (uint64_t i = 0; i < n; ++i) {
    uint32_t p = or_pid(keys[i], splitters, P);
    out_keys[cur[p]] = keys[i];
    out_rowids[cur[p]] = rowids[i];
    cur[p] += 1;
  }
  free(cur);
  free(cnt);
}

/* ------------------------------------------------------------------ */
/* Splitters.  Sample splitters: with the sample sorted, s_p = sample[p*m/P]
 * (p = 1..P-1).  Piecewise-linear CDF model (1024 segments): knot j is the
 * sample order statistic at index j*(m-1)/S, the model's CDF is j/S at knot j
 * and linear between knots; the splitter of partition boundary p is the model's
 * inverse at p/P, evaluated in exact integer arithmetic. */
static int cmp_u64(const void *a, const void *b) {
  uint64_t x = *(const uint64_t *)a, y = *(const uint64_t *)b;
  return x < y ? -1 : (x > y);
}

OR_EXPORT void or_sort_u64(uint64_t *a, uint64_t n) { qsort(a, n, 8, cmp_u64); }

OR_EXPORT void or_sample_splitters(const uint64_t *sorted_sample, uint64_t m, uint32_t P, uint64_t *splitters) {
  for (uint32_t p = 1; p < P; ++p) splitters[p - 1] = sorted_sample[(uint64_t)p * m / P];
}

OR_EXPORT void or_pl_knots(const uint64_t *sorted_sample, uint64_t m, uint32_t S, uint64_t *knots) {
  for (uint32_t j = 0; j <= S; ++j) knots[j] = sorted_sample[(uint64_t)j * (m - 1) / S];
}

OR_EXPORT void or_pl_splitters(const uint64_t *knots, uint32_t S, uint32_t P, uint64_t *splitters) {
  for (uint32_t p = 1; p < P; ++p) {
    uint64_t num = (uint64_t)p * S; /* position p*S/P on the knot axis */
    uint64_t j = num / P, rem = num % P;
    if (j >= S) { splitters[p - 1] = knots[S]; continue; }
    uint64_t gap = knots[j + 1] - knots[j];
    splitters[p - 1] = knots[j] + (uint64_t)(((unsigned __int128)gap * rem) / P);
  }
}

/* ------------------------------------------------------------------ */
/* Monotone CDF MLP, 1 -> H -> 1 (fp64):
 *   y(x) = gamma + sum_j softplus(alpha_j) * sigmoid(softplus(omega_j) * x + beta_j)
 * Both weight layers pass through softplus, so y is non-decreasing in x.
 * Loss L = (1/m) sum_i (y(x_i) - t_i)^2.  Parameter layout:
 *   theta = [omega(H), beta(H), alpha(H), gamma]. */
static double softplus(double v) { return v > 30 ? v : log1p(exp(v)); }
static double sigm(double v) { return 1.0 / (1.0 + exp(-v)); }

OR_EXPORT double or_mlp_forward(const double *theta, int H, double x) {
  const double *om = theta, *be = theta + H, *al = theta + 2 * H;
  double y = theta[3 * H];
  for (int j = 0; j < H; ++j) y += softplus(al[j]) * sigm(softplus(om[j]) * x + be[j]);
  return y;
}

/* Returns L and writes dL/dtheta (3H+1 entries). */
OR_EXPORT double or_mlp_loss_grad(const double *theta, int H, const double *x, const double *t, uint64_t m,
                                  double *grad) {
  const double *om = theta, *be = theta + H, *al = theta + 2 * H;
  for (int k = 0; k < 3 * H + 1; ++k) grad[k] = 0;
  double L = 0;
  for (uint64_t i = 0; i < m; ++i) {
    double y = or_mlp_forward(theta, H, x[i]);
    double r = y - t[i];
    L += r * r;
    double dy = 2.0 * r / (double)m;
    grad[3 * H] += dy;
    for (int j = 0; j < H; ++j) {
      double w = softplus(om[j]);
      double z = w * x[i] + be[j];
      double s = sigm(z);
      double a = softplus(al[j]);
      double ds = s * (1.0 - s);
      grad[2 * H + j] += dy * sigm(al[j]) * s;           /* d softplus(al) = sigmoid(al) */
      grad[H + j] += dy * a * ds;                         /* d/d beta */
      grad[j] += dy * a * ds * x[i] * sigm(om[j]);        /* d/d omega via softplus */
    }
  }
  return L / (double)m;
}

/* One Adam step (Kingma & Ba 2015), fp64, step number t >= 1. */
OR_EXPORT void or_adam_step(double *theta, const double *grad, double *m1, double *m2, int n, int t, double lr,
                            double b1, double b2, double eps) {
  double c1 = 1.0 - pow(b1, t), c2 = 1.0 - pow(b2, t);
  for (int k = 0; k < n; ++k) {
    m1[k] = b1 * m1[k] + (1 - b1) * grad[k];
    m2[k] = b2 * m2[k] + (1 - b2) * grad[k] * grad[k];
    theta[k] -= lr * (m1[k] / c1) / (sqrt(m2[k] / c2) + eps);
  }
}

/* ------------------------------------------------------------------ */
/* Zero-copy threshold (Section 6.3): TH = E / (C_l2 * N_exchange), generalised
 * to one host link as TH = (E / G) * (B_zc / B_ce) where G is the bytes that
 * cross the link per sparse element gather, B_zc the zero-copy streaming
 * bandwidth and B_ce the aggregate copy-engine bandwidth.  With G = C_l2 and
 * B_ce = N_exchange * B_zc (copies spread over N_exchange equal links while a
 * zero-copy gather uses one) it is the paper's formula. */
OR_EXPORT double or_zero_copy_threshold(double elem_bytes, double gather_bytes, double bw_zero_copy, double bw_copy) {
  return (elem_bytes / gather_bytes) * (bw_zero_copy / bw_copy);
}

/* Heavy-key isolation of splitters (P requested partitions, sorted sample of
 * m keys).  Walking the splitters left to right: a splitter not above the last
 * one kept becomes that one + 1 (one at UINT64_MAX is dropped); then, if the
 * kept value v occurs at least m / (2P) times in the sample (half a
 * partition's share), v + 1 is added as the next boundary so that [v, v + 1)
 * holds v alone.  Returns the number of splitters written (at most 2(P-1)). */
OR_EXPORT uint32_t or_isolate_splitters(const uint64_t *spl, uint32_t n_spl, const uint64_t *sample, uint64_t m,
                                        uint32_t P, uint64_t *out) {
  uint32_t k = 0;
  for (uint32_t j = 0; j < n_spl; ++j) {
    uint64_t v = spl[j];
    if (k > 0 && v <= out[k - 1]) {
      if (out[k - 1] == UINT64_MAX) continue;
      v = out[k - 1] + 1;
    }
    out[k++] = v;
    uint64_t c = 0;
    for (uint64_t i = 0; i < m; ++i) c += sample[i] == v;
    if (c * 2 * (uint64_t)P >= m && v != UINT64_MAX) out[k++] = v + 1;
  }
  return k;
}
