/*
 * vxgen — seeded, counter-based synthetic column generators.
 *
 * This module is the single producer of input data for both the CPU oracle and
 * the GPU library; it holds no query arithmetic (no predicates, joins, sums,
 * partitioning or sorting of the method).  Every value is a pure function of
 * (seed, column salt, global row index), so a column can be filled in any
 * order, by any number of threads, or in row ranges, with identical bytes.
 *
 * Random source: the SplitMix64 output finalizer (Steele, Lea & Flood,
 * "Fast splittable pseudorandom number generators", OOPSLA 2014), applied to a
 * per-column base plus the row index.  Bounded integers use Lemire's
 * multiply-shift range reduction ("Fast random integer generation in an
 * interval", ACM TOMACS 2019).  Zipf ranks use rejection-inversion
 * (Hörmann & Derflinger, "Rejection-inversion to generate variates from
 * monotone discrete distributions", ACM TOMACS 1996).
 *
 * Portable C11 + pthreads; no architecture intrinsics (runs on x86-64 and
 * aarch64 with identical output).
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define VXG_EXPORT __attribute__((visibility("default")))

static const uint64_t PHI = 0x9E3779B97F4A7C15ull;
static const uint64_t PSI = 0xD1B54A32D192ED03ull;

VXG_EXPORT uint64_t vxg_mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

/* Base of the counter stream of one column: unrelated bases for different
 * (seed, salt) pairs. */
VXG_EXPORT uint64_t vxg_base(uint64_t seed, uint64_t salt) {
  return vxg_mix64(vxg_mix64(seed * PHI + 1) ^ (salt * PSI));
}

/* The row-th 64-bit uniform of a column. */
VXG_EXPORT uint64_t vxg_u64(uint64_t base, uint64_t row) { return vxg_mix64(base + row * PHI); }

static inline uint64_t bounded(uint64_t u, uint64_t range) {
  return (uint64_t)(((unsigned __int128)u * range) >> 64);
}

/* ---- thread fan-out -------------------------------------------------- */

typedef struct job job;
typedef void (*fill_fn)(const job *, uint64_t, uint64_t);
struct job {
  fill_fn fn;
  void *out;
  uint64_t row0, base;
  int64_t lo, hi;
  uint64_t n_items, aux;
  double s;
  uint64_t begin, end; /* per-thread slice */
};

static void *run_job(void *p) {
  job *j = (job *)p;
  j->fn(j, j->begin, j->end);
  return NULL;
}

static void fan_out(job proto, uint64_t n, int nthreads) {
  if (nthreads < 1) nthreads = 1;
  if (nthreads > 256) nthreads = 256;
  if ((uint64_t)nthreads > n / 65536 + 1) nthreads = (int)(n / 65536 + 1);
  if (nthreads == 1) {
    proto.fn(&proto, 0, n);
    return;
  }
  pthread_t th[256];
  job jobs[256];
  for (int t = 0; t < nthreads; ++t) {
    jobs[t] = proto;
    jobs[t].begin = n * (uint64_t)t / (uint64_t)nthreads;
    jobs[t].end = n * (uint64_t)(t + 1) / (uint64_t)nthreads;
    pthread_create(&th[t], NULL, run_job, &jobs[t]);
  }
  for (int t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);
}

/* ---- int32 uniform in [lo, hi] (inclusive) ---------------------------- */

static void f_i32_uniform(const job *j, uint64_t b, uint64_t e) {
  int32_t *o = (int32_t *)j->out;
  uint64_t range = (uint64_t)(j->hi - j->lo + 1);
  for (uint64_t i = b; i < e; ++i)
    o[i] = (int32_t)(j->lo + (int64_t)bounded(vxg_u64(j->base, j->row0 + i), range));
}

VXG_EXPORT void vxg_fill_i32_uniform(int32_t *out, uint64_t n, uint64_t row0, uint64_t seed,
                                     uint64_t salt, int32_t lo, int32_t hi, int nthreads) {
  job p = {0};
  p.fn = f_i32_uniform; p.out = out; p.row0 = row0; p.base = vxg_base(seed, salt);
  p.lo = lo; p.hi = hi;
  fan_out(p, n, nthreads);
}

/* ---- uint64 uniform over the full range ------------------------------- */

static void f_u64_uniform(const job *j, uint64_t b, uint64_t e) {
  uint64_t *o = (uint64_t *)j->out;
  for (uint64_t i = b; i < e; ++i) o[i] = vxg_u64(j->base, j->row0 + i);
}

VXG_EXPORT void vxg_fill_u64_uniform(uint64_t *out, uint64_t n, uint64_t row0, uint64_t seed,
                                     uint64_t salt, int nthreads) {
  job p = {0};
  p.fn = f_u64_uniform; p.out = out; p.row0 = row0; p.base = vxg_base(seed, salt);
  fan_out(p, n, nthreads);
}

/* ---- row ids: (row0 + i) mod 2^32 ------------------------------------- */

static void f_rowid(const job *j, uint64_t b, uint64_t e) {
  uint32_t *o = (uint32_t *)j->out;
  for (uint64_t i = b; i < e; ++i) o[i] = (uint32_t)(j->row0 + i);
}

VXG_EXPORT void vxg_fill_rowid_u32(uint32_t *out, uint64_t n, uint64_t row0, int nthreads) {
  job p = {0};
  p.fn = f_rowid; p.out = out; p.row0 = row0;
  fan_out(p, n, nthreads);
}

/* ---- Zipf(s) ranks in [1, N] by rejection-inversion -------------------
 * h(x) = x^-s is the (unnormalised) density of the continuous hat; H is its
 * antiderivative and Hinv the inverse.  Written in the numerically stable
 * form with helper functions log1p/expm1 so that s = 1 is continuous. */

static double helper1(double x) { /* log1p(x)/x, -> 1 as x -> 0 */
  return fabs(x) > 1e-8 ? log1p(x) / x : 1.0 - x * (0.5 - x * (1.0 / 3.0 - 0.25 * x));
}
static double helper2(double x) { /* expm1(x)/x, -> 1 as x -> 0 */
  return fabs(x) > 1e-8 ? expm1(x) / x : 1.0 + x * 0.5 * (1.0 + x * (1.0 / 3.0) * (1.0 + 0.25 * x));
}
static double zH(double x, double s) { /* integral of t^-s: (x^(1-s) - 1)/(1-s) */
  double lx = log(x);
  return helper2((1.0 - s) * lx) * lx;
}
static double zHinv(double y, double s) {
  double t = y * (1.0 - s);
  if (t < -1.0) t = -1.0;
  return exp(helper1(t) * y);
}
static double zh(double x, double s) { return exp(-s * log(x)); }

typedef struct {
  double s, hx1, hN, shift;
  uint64_t N;
} zipf_t;

static zipf_t zipf_init(uint64_t N, double s) {
  zipf_t z;
  z.s = s; z.N = N;
  z.hx1 = zH(1.5, s) - 1.0;
  z.hN = zH((double)N + 0.5, s);
  z.shift = 2.0 - zHinv(zH(2.5, s) - zh(2.0, s), s);
  return z;
}

/* One rank drawn from the per-row substream (base, row): attempt k uses the
 * uniform vxg_mix64(rowbase + k*PSI). */
static uint64_t zipf_draw(const zipf_t *z, uint64_t rowbase) {
  for (uint64_t k = 0;; ++k) {
    uint64_t u64 = vxg_mix64(rowbase + k * PSI);
    double u01 = (double)(u64 >> 11) * (1.0 / 9007199254740992.0); /* [0,1) */
    double u = z->hN + u01 * (z->hx1 - z->hN);
    double x = zHinv(u, z->s);
    double kf = floor(x + 0.5);
    if (kf < 1.0) kf = 1.0;
    if (kf > (double)z->N) kf = (double)z->N;
    if (kf - x <= z->shift || u >= zH(kf + 0.5, z->s) - zh(kf, z->s)) return (uint64_t)kf;
  }
}

/* map: 0 -> key = mix64(rank); 1 -> key = rank */
static void f_zipf(const job *j, uint64_t b, uint64_t e) {
  uint64_t *o = (uint64_t *)j->out;
  zipf_t z = zipf_init(j->n_items, j->s);
  for (uint64_t i = b; i < e; ++i) {
    uint64_t r = zipf_draw(&z, vxg_u64(j->base, j->row0 + i));
    o[i] = j->aux == 0 ? vxg_mix64(r) : r;
  }
}

VXG_EXPORT void vxg_fill_u64_zipf(uint64_t *out, uint64_t n, uint64_t row0, uint64_t seed,
                                  uint64_t salt, uint64_t N, double s, int map, int nthreads) {
  job p = {0};
  p.fn = f_zipf; p.out = out; p.row0 = row0; p.base = vxg_base(seed, salt);
  p.n_items = N; p.s = s; p.aux = (uint64_t)map;
  fan_out(p, n, nthreads);
}

/* Single Zipf rank for a row (tests check the sampler's frequencies). */
VXG_EXPORT uint64_t vxg_zipf_rank(uint64_t seed, uint64_t salt, uint64_t row, uint64_t N, double s) {
  zipf_t z = zipf_init(N, s);
  return zipf_draw(&z, vxg_u64(vxg_base(seed, salt), row));
}

/* ---- presorted runs ----------------------------------------------------
 * total rows split into n_runs equal runs (the last takes the remainder);
 * inside a run of length L the key at position q is q*stride + (u mod stride)
 * with stride = floor(2^64 / L): a stratified uniform sample, non-decreasing
 * inside the run. */
static void f_runs(const job *j, uint64_t b, uint64_t e) {
  uint64_t *o = (uint64_t *)j->out;
  uint64_t total = j->n_items, runs = j->aux;
  uint64_t L = total / runs;
  for (uint64_t i = b; i < e; ++i) {
    uint64_t g = j->row0 + i;
    uint64_t r = g / L;
    if (r >= runs) r = runs - 1;
    uint64_t start = r * L;
    uint64_t len = (r == runs - 1) ? total - start : L;
    uint64_t q = g - start;
    uint64_t stride = len ? (uint64_t)((((unsigned __int128)1) << 64) / len) : 0;
    if (stride == 0) stride = 1;
    o[i] = q * stride + vxg_u64(j->base, g) % stride;
  }
}

VXG_EXPORT void vxg_fill_u64_presorted_runs(uint64_t *out, uint64_t n, uint64_t row0, uint64_t total,
                                            uint64_t n_runs, uint64_t seed, uint64_t salt, int nthreads) {
  job p = {0};
  p.fn = f_runs; p.out = out; p.row0 = row0; p.base = vxg_base(seed, salt);
  p.n_items = total; p.aux = n_runs ? n_runs : 1;
  fan_out(p, n, nthreads);
}

/* ---- join inputs --------------------------------------------------------
 * build row i: key = mix64(i), payload = mix64(i ^ PAYLOAD_SALT).
 * probe row t: with probability match (Bernoulli from the counter stream) a
 * build index b (uniform, or Zipf(s) rank r mapped by (a*r + c) mod n_build),
 * key = mix64(b); otherwise key = mix64(n_build + t), which no build key
 * equals because mix64 is a bijection. */
#define PAYLOAD_SALT 0x5DEECE66DA3B1C27ull

static void f_build_keys(const job *j, uint64_t b, uint64_t e) {
  int64_t *o = (int64_t *)j->out;
  for (uint64_t i = b; i < e; ++i) o[i] = (int64_t)vxg_mix64(j->row0 + i);
}
static void f_build_payload(const job *j, uint64_t b, uint64_t e) {
  int64_t *o = (int64_t *)j->out;
  for (uint64_t i = b; i < e; ++i) o[i] = (int64_t)vxg_mix64((j->row0 + i) ^ PAYLOAD_SALT);
}
VXG_EXPORT void vxg_fill_build_keys(int64_t *out, uint64_t n, uint64_t row0, int nthreads) {
  job p = {0};
  p.fn = f_build_keys; p.out = out; p.row0 = row0;
  fan_out(p, n, nthreads);
}
VXG_EXPORT void vxg_fill_build_payload(int64_t *out, uint64_t n, uint64_t row0, int nthreads) {
  job p = {0};
  p.fn = f_build_payload; p.out = out; p.row0 = row0;
  fan_out(p, n, nthreads);
}

static const uint64_t ZMAP_A = 2654435761ull; /* odd, not divisible by 5 */

static void f_probe(const job *j, uint64_t b, uint64_t e) {
  int64_t *o = (int64_t *)j->out;
  uint64_t nb = j->n_items;
  double match = (double)j->lo / 1e6; /* match rate in millionths */
  uint64_t thr = match >= 1.0 ? UINT64_MAX : (uint64_t)(match * 18446744073709551616.0);
  zipf_t z;
  if (j->s > 0) z = zipf_init(nb, j->s);
  for (uint64_t i = b; i < e; ++i) {
    uint64_t t = j->row0 + i;
    uint64_t u0 = vxg_u64(j->base, 3 * t);
    int hit = match >= 1.0 ? 1 : (u0 < thr);
    if (!hit) {
      o[i] = (int64_t)vxg_mix64(nb + t);
      continue;
    }
    uint64_t bi;
    if (j->s > 0) {
      uint64_t r = zipf_draw(&z, vxg_u64(j->base, 3 * t + 1));
      bi = (uint64_t)(((unsigned __int128)ZMAP_A * r + 12345u) % nb);
    } else {
      bi = bounded(vxg_u64(j->base, 3 * t + 2), nb);
    }
    o[i] = (int64_t)vxg_mix64(bi);
  }
}

/* zipf_s <= 0 selects uniform; match_ppm = match rate in parts per million. */
VXG_EXPORT void vxg_fill_probe_keys(int64_t *out, uint64_t n, uint64_t row0, uint64_t n_build,
                                    int64_t match_ppm, double zipf_s, uint64_t seed, uint64_t salt,
                                    int nthreads) {
  job p = {0};
  p.fn = f_probe; p.out = out; p.row0 = row0; p.base = vxg_base(seed, salt);
  p.n_items = n_build; p.lo = match_ppm; p.s = zipf_s;
  fan_out(p, n, nthreads);
}

/* Generator-side ground truth of the join: the number of probe rows that were
 * drawn as matches and the wrapping sum of the payloads they reference,
 * recomputed from the draw itself (no table lookup). */
VXG_EXPORT void vxg_probe_truth(uint64_t n, uint64_t row0, uint64_t n_build, int64_t match_ppm,
                                double zipf_s, uint64_t seed, uint64_t salt, uint64_t *count,
                                uint64_t *payload_sum) {
  uint64_t base = vxg_base(seed, salt);
  double match = (double)match_ppm / 1e6;
  uint64_t thr = match >= 1.0 ? UINT64_MAX : (uint64_t)(match * 18446744073709551616.0);
  zipf_t z;
  if (zipf_s > 0) z = zipf_init(n_build, zipf_s);
  uint64_t c = 0, s = 0;
  for (uint64_t i = 0; i < n; ++i) {
    uint64_t t = row0 + i;
    uint64_t u0 = vxg_u64(base, 3 * t);
    int hit = match >= 1.0 ? 1 : (u0 < thr);
    if (!hit) continue;
    uint64_t bi;
    if (zipf_s > 0) {
      uint64_t r = zipf_draw(&z, vxg_u64(base, 3 * t + 1));
      bi = (uint64_t)(((unsigned __int128)ZMAP_A * r + 12345u) % n_build);
    } else {
      bi = bounded(vxg_u64(base, 3 * t + 2), n_build);
    }
    c += 1;
    s += vxg_mix64(bi ^ PAYLOAD_SALT);
  }
  *count = c;
  *payload_sum = s;
}

/* ---- dimension tables ---------------------------------------------------
 * Keys: a seeded Fisher-Yates shuffle of 0..n-1 (stored order is shuffled so
 * that a join is a real lookup). */
VXG_EXPORT void vxg_permutation_i32(int32_t *out, uint64_t n, uint64_t seed, uint64_t salt) {
  uint64_t base = vxg_base(seed, salt);
  for (uint64_t i = 0; i < n; ++i) out[i] = (int32_t)i;
  for (uint64_t i = n; i > 1; --i) {
    uint64_t k = bounded(vxg_u64(base, i), i); /* k in [0, i) */
    int32_t t = out[i - 1];
    out[i - 1] = out[k];
    out[k] = t;
  }
}

/* Calendar of the date dimension: key d is day 1992-01-01 + d of the
 * proleptic Gregorian calendar.  Writes year (e.g. 1993) and month (1..12). */
static int is_leap(int y) { return (y % 4 == 0 && y % 100 != 0) || y % 400 == 0; }
VXG_EXPORT void vxg_date_of_key(int32_t key, int32_t *year, int32_t *month) {
  static const int mdays[12] = {31, 28, 31, 30, 31, 30, 31, 31, 30, 31, 30, 31};
  int y = 1992, d = key;
  while (d >= (is_leap(y) ? 366 : 365)) {
    d -= is_leap(y) ? 366 : 365;
    ++y;
  }
  int m = 0;
  for (;;) {
    int md = mdays[m] + (m == 1 && is_leap(y));
    if (d < md) break;
    d -= md;
    ++m;
  }
  *year = y;
  *month = m + 1;
}

/* Hierarchical attribute: code = parent * fanout + u(fanout); parent may be
 * NULL (then code = u(card)). */
VXG_EXPORT void vxg_fill_child_code(int32_t *out, const int32_t *parent, uint64_t n, int32_t fanout,
                                    int32_t card, uint64_t seed, uint64_t salt) {
  uint64_t base = vxg_base(seed, salt);
  for (uint64_t i = 0; i < n; ++i) {
    uint64_t u = vxg_u64(base, i);
    out[i] = parent ? parent[i] * fanout + (int32_t)bounded(u, (uint64_t)fanout)
                    : (int32_t)bounded(u, (uint64_t)card);
  }
}

/* Clustered column: row g of a total-row table gets floor(g * card / total), a
 * non-decreasing ramp (a fact table appended in key order). */
static void f_ramp(const job *j, uint64_t b, uint64_t e) {
  int32_t *o = (int32_t *)j->out;
  for (uint64_t i = b; i < e; ++i)
    o[i] = (int32_t)(((unsigned __int128)(j->row0 + i) * (uint64_t)j->hi) / j->n_items);
}

VXG_EXPORT void vxg_fill_i32_ramp(int32_t *out, uint64_t n, uint64_t row0, uint64_t total, int32_t card,
                                  int nthreads) {
  job p = {0};
  p.fn = f_ramp; p.out = out; p.row0 = row0; p.n_items = total ? total : 1; p.hi = card;
  fan_out(p, n, nthreads);
}

/* Sample positions: m positions drawn uniformly with replacement from [0, n). */
VXG_EXPORT void vxg_sample_positions(uint64_t *out, uint64_t m, uint64_t n, uint64_t seed, uint64_t salt) {
  uint64_t base = vxg_base(seed, salt);
  for (uint64_t i = 0; i < m; ++i) out[i] = bounded(vxg_u64(base, i), n);
}
