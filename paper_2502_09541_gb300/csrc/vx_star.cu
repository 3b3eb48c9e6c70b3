// Star-join pipeline: dimension hash tables (build), fused chunk kernel (filter
// -> chained probes -> group-by aggregate with zero-copy late
// materialization), filter with ordered stream compaction, and the
// vx_run_plan / vx_groupby / vx_filter entry points.
//
// Section 7.1: dimension tables are filtered and hashed on the device and kept
// there; fact chunks stream through one fused kernel per chunk.  Section 6.3:
// aggregate columns whose estimated selectivity is below TH are not staged;
// the kernel reads them from mapped host memory for qualifying rows only.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdio>

#include "vx_bulk.cuh"
#include "vx_internal.h"
#include "vx_probe.cuh"
#include "vx_star.cuh"

namespace vx {

// ================================================================== device code

// Inserts every dimension row: value = group-code contribution of the row if
// it passes the dimension predicates, HT_FILTERED otherwise (so duplicate keys
// are detected over the whole dimension, not only its qualifying rows).
__global__ void ht_build_kernel(const DimBuildParams p) {
  const uint32_t mask = (1u << p.log2cap) - 1u;
  unsigned long long passed = 0;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < p.rows;
       i += (uint64_t)gridDim.x * blockDim.x) {
    const int32_t key = p.key[i];
    bool ok = true;
    for (int q = 0; q < p.n_preds && ok; ++q) ok = pred_ok(p.attr[p.pred_attr[q]][i], p.pred_op[q], p.pred_lo[q], p.pred_hi[q]);
    uint32_t val = HT_FILTERED;
    if (ok) {
      uint64_t g = 0;
      for (int a = 0; a < p.n_attr; ++a) {
        if (p.stride[a] == 0) continue;
        int32_t code = p.attr[a][i];
        if (code < 0 || code >= p.card[a]) {
          atomicOr(p.err, ERR_RANGE);
          code = 0;
        }
        g += (uint64_t)code * p.stride[a];
      }
      val = (uint32_t)g;
      ++passed;
    }
    if (p.dmap) {  // dense keys: one value per key
      const uint32_t idx = (uint32_t)(key - p.kmin);
      if (idx >= p.span) {
        atomicOr(p.err, ERR_HT_FULL);
        continue;
      }
      if (atomicCAS(&p.dmap[idx], HT_EMPTY_VAL, val) != HT_EMPTY_VAL) atomicOr(p.err, ERR_DUPKEY);
      continue;
    }
    const unsigned long long packed = ((unsigned long long)val << 32) | (uint32_t)key;
    uint32_t h = ht_hash32(key, p.log2cap);
    bool done = false;
    for (uint32_t n = 0; n <= mask; ++n) {
      unsigned long long old = atomicCAS((unsigned long long *)&p.slots[h], HT_EMPTY, packed);
      if (old == HT_EMPTY) { done = true; break; }
      if ((int32_t)(uint32_t)old == key) { atomicOr(p.err, ERR_DUPKEY); done = true; break; }
      h = (h + 1u) & mask;
    }
    if (!done) atomicOr(p.err, ERR_HT_FULL);
  }
  // passed-row count (planner's dimension selectivity)
  for (int off = 16; off > 0; off >>= 1) passed += __shfl_down_sync(0xffffffffu, passed, off);
  if ((threadIdx.x & 31) == 0 && passed) atomicAdd(p.passed, passed);
}

__global__ void fill_u64_kernel(uint64_t *p, uint64_t n, uint64_t v) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
    p[i] = v;
}

// Fused chunk kernel: per row (kRows rows per thread, strided by blockDim for
// coalescing) — fact predicates, chained probes into the dimension tables,
// mixed-radix group id, aggregate.  Accumulators live in shared memory when
// the groups fit (kSmem), else in global memory.
// survivors of one block tile, collected in shared memory (split mode)
template <uint32_t kCap>
struct SurvTileT {
  unsigned int n, base;
  uint2 e[kCap];  // (chunk row, group id)
};
using SurvTile = SurvTileT<kStarTileRows>;

// rows base + j * blockDim.x (j < kRows) of one chunk.  kSplit: surviving
// rows are appended to the block's survivor list instead of being aggregated
// (their late payload columns are read by star_gather_kernel).
template <bool kSmem, int kRows, bool kSplit = false>
__device__ __forceinline__ void star_rows(const ChunkParams &p, uint64_t base, unsigned long long *ssum,
                                          unsigned long long *scnt, unsigned long long &surv,
                                          SurvTile *st = nullptr) {
  {
    uint64_t row[kRows];
    bool alive[kRows];
    uint32_t g[kRows];
#pragma unroll
    for (int j = 0; j < kRows; ++j) {
      row[j] = base + (uint64_t)j * blockDim.x;
      alive[j] = row[j] < p.n;
      g[j] = 0;
    }
    for (int q = 0; q < p.n_fact_preds; ++q) {
      int32_t v[kRows];
#pragma unroll
      for (int j = 0; j < kRows; ++j) v[j] = alive[j] ? load_role(p, p.fp_role[q], row[j]) : 0;
      const PredRange r = pred_range(p.fp_op[q], p.fp_lo[q], p.fp_hi[q]);
#pragma unroll
      for (int j = 0; j < kRows; ++j) alive[j] = alive[j] && pred_in(r, v[j]);
    }
    for (int d = 0; d < p.n_dims; ++d) {
      const uint64_t *__restrict__ slots = p.ht[d];
      const uint32_t l2c = p.ht_log2[d];
      const uint32_t mask = (1u << l2c) - 1u;
      int32_t key[kRows];
      uint32_t h[kRows];
      uint64_t sl[kRows];
#pragma unroll
      for (int j = 0; j < kRows; ++j) key[j] = alive[j] ? load_role(p, p.dim_role[d], row[j]) : 0;
      if (p.dspan[d]) {  // direct map: one load per row, no probing
        const int32_t kmin = p.dmin[d];
        const uint32_t span = p.dspan[d], vb = p.dvb[d];
        uint32_t v[kRows];
#pragma unroll
        for (int j = 0; j < kRows; ++j) {
          const uint32_t idx = (uint32_t)(key[j] - kmin);
          v[j] = (alive[j] && idx < span) ? dmap_get(slots, vb, idx) : HT_EMPTY_VAL;
        }
#pragma unroll
        for (int j = 0; j < kRows; ++j) {
          const bool hit = alive[j] && v[j] < HT_FILTERED;
          g[j] += hit ? v[j] : 0u;
          alive[j] = hit;
        }
        continue;
      }
      // first probe of every row issued before any is resolved (memory-level
      // parallelism); linear probing continues only on collisions
#pragma unroll
      for (int j = 0; j < kRows; ++j) {
        h[j] = ht_hash32(key[j], l2c);
        sl[j] = alive[j] ? __ldg(&slots[h[j]]) : HT_EMPTY;
      }
#pragma unroll
      for (int j = 0; j < kRows; ++j) {
        if (!alive[j]) continue;
        uint64_t s = sl[j];
        uint32_t hh = h[j];
        bool hit = false;
        for (uint32_t n = 0; n <= mask; ++n) {
          const uint32_t v = (uint32_t)(s >> 32);
          if (v == HT_EMPTY_VAL) break;
          if ((int32_t)(uint32_t)s == key[j]) {
            hit = v != HT_FILTERED;
            g[j] += v;
            break;
          }
          hh = (hh + 1u) & mask;
          s = __ldg(&slots[hh]);
        }
        alive[j] = hit;
      }
    }
    for (int k = 0; k < p.n_fgk; ++k) {
#pragma unroll
      for (int j = 0; j < kRows; ++j) {
        if (!alive[j]) continue;
        int32_t code = load_role(p, p.fgk_role[k], row[j]);
        if (code < 0 || code >= p.fgk_card[k]) {
          atomicOr(p.err, ERR_RANGE);
          alive[j] = false;
          continue;
        }
        g[j] += (uint32_t)code * p.fgk_stride[k];
      }
    }
    if (p.chunk_surv) {
#pragma unroll
      for (int j = 0; j < kRows; ++j) surv += alive[j];
    }
    if constexpr (kSplit) {
#pragma unroll
      for (int j = 0; j < kRows; ++j) {
        if (!alive[j]) continue;
        const unsigned int k = atomicAdd(&st->n, 1u);
        st->e[k] = make_uint2((uint32_t)row[j], g[j]);
      }
    } else {
      int32_t av[kRows], bv[kRows];
#pragma unroll
      for (int j = 0; j < kRows; ++j) {  // aggregate inputs of all rows in flight together
        av[j] = (alive[j] && p.agg_a_role >= 0) ? load_role(p, p.agg_a_role, row[j]) : 0;
        bv[j] = (alive[j] && p.agg_b_role >= 0) ? load_role(p, p.agg_b_role, row[j]) : 0;
      }
#pragma unroll
      for (int j = 0; j < kRows; ++j) {
        if (!alive[j]) continue;
        const int64_t a = av[j], b = bv[j];
        int64_t v = p.agg_op == VX_AGG_SUM ? a : p.agg_op == VX_AGG_MUL ? a * b : p.agg_op == VX_AGG_SUB ? a - b : 0;
        if (kSmem) {
          atomicAdd(&ssum[g[j]], (unsigned long long)v);
          atomicAdd(&scnt[g[j]], 1ull);
        } else {
          atomicAdd(&p.g_sum[g[j]], (unsigned long long)v);
          atomicAdd(&p.g_cnt[g[j]], 1ull);
        }
      }
    }
  }
}

constexpr uint32_t kVecTileRows = 1024;  // one group of 4 rows per thread of 256

// row j of a vector-path thread whose first row is r0 (group j / 4, lane j % 4)
__device__ __forceinline__ uint64_t row_of(uint64_t r0, int j) {
  return r0 + (uint64_t)(j >> 2) * kVecTileRows + (uint64_t)(j & 3);
}

__device__ __forceinline__ int32_t lane4(const int4 &v, int j) { return j == 0 ? v.x : j == 1 ? v.y : j == 2 ? v.z : v.w; }

// value of row j from the row-logic slot `slot` (compile-time select over the
// kR loaded vectors, so the values stay in registers)
template <int kR>
__device__ __forceinline__ int32_t slot_val(const int4 (&vals)[kR], int slot, int j) {
  int32_t x = 0;
#pragma unroll
  for (int k = 0; k < kR; ++k)
    if (k == slot) x = lane4(vals[k], j);
  return x;
}

// where the vector path reads row j's value of a row-logic slot: the loaded
// vectors in registers, or the thread's own 16-byte slots in shared memory
// (slot k of thread t at sv[k * 256 + t])
template <int kR, int kV>
struct RegVals {
  const int4 (&v)[kV][kR];
  __device__ __forceinline__ int32_t operator()(int slot, int j) const { return slot_val(v[j >> 2], slot, j & 3); }
};

// Vector path: kV groups of 4 consecutive rows, r0 + v * kVecTileRows + 0..3
// (r0 a multiple of 4, staged columns 16-byte aligned).  Every row-logic
// column is loaded with one 16-byte load per group before any row is
// evaluated, so the rows' memory latency overlaps;
// then predicates, probes (direct map or hash, all 4 rows' lookups in flight)
// and the group id are computed from registers.  Survivors are aggregated
// (kSplit = false) or appended to the block's survivor list.
template <int kR, int kV>
__device__ __forceinline__ void star_load4(const ChunkParams &p, uint64_t r0, int4 (&vals)[kV][kR]) {
#pragma unroll
  for (int v = 0; v < kV; ++v) {
    const uint64_t rv = r0 + (uint64_t)v * kVecTileRows;
    const bool full = rv + 3 < p.n;
#pragma unroll
    for (int k = 0; k < kR; ++k) {
      const int32_t *col = p.staged[k < p.n_rowroles ? p.rowrole[k] : p.rowrole[0]];
      if (full) {
        vals[v][k] = __ldg(reinterpret_cast<const int4 *>(col + rv));
      } else {
        vals[v][k].x = rv < p.n ? __ldg(col + rv) : 0;
        vals[v][k].y = rv + 1 < p.n ? __ldg(col + rv + 1) : 0;
        vals[v][k].z = rv + 2 < p.n ? __ldg(col + rv + 2) : 0;
        vals[v][k].w = 0;
      }
    }
  }
}

// the fact predicates of kN rows (alive[j] &= row j passes them)
template <int kN, class Vals>
__device__ __forceinline__ void star_fact_preds(const ChunkParams &p, const Vals &vals, bool (&alive)[kN]) {
  for (int q = 0; q < p.n_fact_preds; ++q) {
    const int s = p.fp_slot[q];
    const PredRange r = pred_range(p.fp_op[q], p.fp_lo[q], p.fp_hi[q]);
#pragma unroll
    for (int j = 0; j < kN; ++j) alive[j] = alive[j] && pred_in(r, vals(s, j));
  }
}

// the probes (dimension predicates and group-code contributions) and fact
// group keys of kN rows: alive[j] &= row j finds a qualifying row in every
// dimension, g[j] += its group code
template <int kN, class Vals>
__device__ __forceinline__ void star_probe_dims(const ChunkParams &p, const Vals &vals, bool (&alive)[kN],
                                                uint32_t (&g)[kN]) {
  for (int d = 0; d < p.n_dims; ++d) {
    const int s = p.dim_slot[d];
    int32_t key[kN];
#pragma unroll
    for (int j = 0; j < kN; ++j) key[j] = vals(s, j);
    if (p.dspan[d]) {
      const uint32_t vb = p.dvb[d];
      uint32_t v[kN];
#pragma unroll
      for (int j = 0; j < kN; ++j) {
        const uint32_t idx = (uint32_t)(key[j] - p.dmin[d]);
        v[j] = (alive[j] && idx < p.dspan[d]) ? dmap_get(p.ht[d], vb, idx) : HT_EMPTY_VAL;
      }
#pragma unroll
      for (int j = 0; j < kN; ++j) {
        const bool hit = alive[j] && v[j] < HT_FILTERED;
        g[j] += hit ? v[j] : 0u;
        alive[j] = hit;
      }
    } else {
      const uint64_t *__restrict__ slots = p.ht[d];
      const uint32_t l2c = p.ht_log2[d], mask = (1u << l2c) - 1u;
      uint32_t h[kN];
      uint64_t sl[kN];
#pragma unroll
      for (int j = 0; j < kN; ++j) {
        h[j] = ht_hash32(key[j], l2c);
        sl[j] = alive[j] ? __ldg(&slots[h[j]]) : HT_EMPTY;
      }
#pragma unroll
      for (int j = 0; j < kN; ++j) {
        if (!alive[j]) continue;
        uint64_t sv = sl[j];
        uint32_t hh = h[j];
        bool hit = false;
        for (uint32_t n = 0; n <= mask; ++n) {
          const uint32_t v = (uint32_t)(sv >> 32);
          if (v == HT_EMPTY_VAL) break;
          if ((int32_t)(uint32_t)sv == key[j]) {
            hit = v != HT_FILTERED;
            g[j] += v;
            break;
          }
          hh = (hh + 1u) & mask;
          sv = __ldg(&slots[hh]);
        }
        alive[j] = hit;
      }
    }
  }
  for (int k = 0; k < p.n_fgk; ++k) {
    const int s = p.fgk_slot[k];
#pragma unroll
    for (int j = 0; j < kN; ++j) {
      if (!alive[j]) continue;
      const int32_t code = vals(s, j);
      if (code < 0 || code >= p.fgk_card[k]) {
        atomicOr(p.err, ERR_RANGE);
        alive[j] = false;
        continue;
      }
      g[j] += (uint32_t)code * p.fgk_stride[k];
    }
  }
}

// predicates, probes and fact group keys of a thread's 4 x kV rows: alive[j]
// = row j qualifies, g[j] = its group id
template <int kV, class Vals>
__device__ __forceinline__ void star_eval4(const ChunkParams &p, uint64_t r0, const Vals &vals, bool (&alive)[4 * kV],
                                           uint32_t (&g)[4 * kV]) {
  constexpr int kN = 4 * kV;
#pragma unroll
  for (int j = 0; j < kN; ++j) {
    alive[j] = row_of(r0, j) >= p.row_lo && row_of(r0, j) < p.n;
    g[j] = 0;
  }
  star_fact_preds<kN>(p, vals, alive);
  star_probe_dims<kN>(p, vals, alive, g);
}

template <bool kSmem, bool kSplit, int kV, class Vals, class Tile>
__device__ __forceinline__ void star_rows4(const ChunkParams &p, uint64_t r0, const Vals &vals,
                                           unsigned long long *ssum, unsigned long long *scnt,
                                           unsigned long long &surv, Tile *st) {
  constexpr int kN = 4 * kV;  // rows of this thread
  bool alive[kN];
  uint32_t g[kN];
  star_eval4<kV>(p, r0, vals, alive, g);
  if (p.chunk_surv) {
#pragma unroll
    for (int j = 0; j < kN; ++j) surv += alive[j];
  }
  if constexpr (kSplit) {
#pragma unroll
    for (int j = 0; j < kN; ++j)
      if (alive[j]) st->e[atomicAdd(&st->n, 1u)] = make_uint2((uint32_t)row_of(r0, j), g[j]);
  } else {
#pragma unroll
    for (int j = 0; j < kN; ++j) {
      if (!alive[j]) continue;
      const int64_t a = p.agg_a_role < 0    ? 0
                        : p.agg_slot[0] >= 0 ? vals(p.agg_slot[0], j)
                                             : load_role(p, p.agg_a_role, row_of(r0, j));
      const int64_t b = p.agg_b_role < 0    ? 0
                        : p.agg_slot[1] >= 0 ? vals(p.agg_slot[1], j)
                                             : load_role(p, p.agg_b_role, row_of(r0, j));
      const int64_t v = p.agg_op == VX_AGG_SUM ? a : p.agg_op == VX_AGG_MUL ? a * b : p.agg_op == VX_AGG_SUB ? a - b : 0;
      if (kSmem) {
        atomicAdd(&ssum[g[j]], (unsigned long long)v);
        atomicAdd(&scnt[g[j]], 1ull);
      } else {
        atomicAdd(&p.g_sum[g[j]], (unsigned long long)v);
        atomicAdd(&p.g_cnt[g[j]], 1ull);
      }
    }
  }
}


// column values of the vector path: in registers, or staged by each thread into
// its own shared-memory slots with cp.async and read back per access (no
// column vectors in registers: 32-40 instead of 48-116 registers).  Measured
// per 2.8M-row chunk, shared-memory slots won in split mode (28.0 vs 30.1 µs
// with 4 columns, 31.4 vs 35.0 with 6) and with 8 columns (37.7 vs 48.0), and
// lost with 6 columns and shared-memory group accumulators (47.2 vs 40.5).
constexpr bool vec_cols(bool split, int kr) { return split || kr >= 8; }

// groups of 4 rows per thread (a block tile is groups x kVecTileRows rows):
// one.  Two raised registers to 62-128 with register-held columns, and with
// shared-memory slots of 4 columns (48 registers, 4 resident blocks) measured
// 29.5 / 34.3 µs against 29.0 / 29.2 µs per chunk for T2 at 0.1 / 1 %.
constexpr int kVecGroups = 1;
constexpr int vec_groups(bool split, int kr) { return (void)split, (void)kr, kVecGroups; }
static_assert(2 * kVecTileRows <= kStarTileRows, "a block tile's survivors must fit its list");
// dynamic shared memory of the column slots, after the group accumulators
constexpr size_t vec_col_bytes(bool split, int kr) {
  return vec_cols(split, kr) ? (size_t)kr * vec_groups(split, kr) * 256 * sizeof(int4) : 0;
}

struct StageVals {  // row-logic slot k of the thread's 4 rows at base[k * stride]
  const int4 *base;
  uint32_t stride;
  __device__ __forceinline__ int32_t operator()(int slot, int j) const { return lane4(base[slot * stride], j & 3); }
};

// thread t's rows r0 + v * kVecTileRows + 0..3 of every row-logic column into
// scol[(k * kV + v) * 256 + t]
template <int kR, int kV>
__device__ __forceinline__ void star_stage4(const ChunkParams &p, uint64_t r0, int4 *scol) {
#pragma unroll
  for (int v = 0; v < kV; ++v) {
    const uint64_t rv = r0 + (uint64_t)v * kVecTileRows;
    const bool full = rv + 3 < p.n;
#pragma unroll
    for (int k = 0; k < kR; ++k) {
      const int32_t *col = p.staged[k < p.n_rowroles ? p.rowrole[k] : p.rowrole[0]];
      int4 *dst = &scol[(k * kV + v) * 256 + threadIdx.x];
      if (full) {  // 16-byte aligned: staged columns are, and rv is a multiple of 4
        const unsigned sa = (unsigned)__cvta_generic_to_shared(dst);
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(col + rv) : "memory");
      } else {
        *dst = make_int4(rv < p.n ? __ldg(col + rv) : 0, rv + 1 < p.n ? __ldg(col + rv + 1) : 0,
                         rv + 2 < p.n ? __ldg(col + rv + 2) : 0, 0);
      }
    }
  }
  asm volatile("cp.async.commit_group;\n" ::: "memory");
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");  // the thread reads only its own slots
}

// Vector path kernel over whole block tiles of kVecGroups x kVecTileRows rows,
// one block per tile (the hardware keeps as many resident as registers and
// shared memory allow).
template <bool kSmem, bool kSplit, int kR>
__global__ void __launch_bounds__(256) star_vec_kernel(const ChunkParams p) {
  constexpr bool kCols = vec_cols(kSplit, kR);
  constexpr int kG = vec_groups(kSplit, kR);
  static_assert(kG == 1, "thread slots hold one group of 4 rows");
  extern __shared__ __align__(16) unsigned long long sacc[];  // [2 * n_groups] when kSmem, then column slots
  __shared__ SurvTileT<kG * kVecTileRows> st;
  int4 *scol = reinterpret_cast<int4 *>(sacc + (kSmem ? 2 * p.n_groups : 0));  // 16-byte aligned: even count
  unsigned long long *ssum = sacc, *scnt = sacc + p.n_groups;
  if (kSmem) {
    for (uint32_t g = threadIdx.x; g < 2 * p.n_groups; g += blockDim.x) sacc[g] = 0;
  }
  if (threadIdx.x == 0) st.n = 0;
  __syncthreads();
  unsigned long long surv = 0;
  constexpr uint64_t kTile = (uint64_t)kG * kVecTileRows;
  for (uint64_t t0 = (uint64_t)blockIdx.x * kTile; t0 < p.n; t0 += (uint64_t)gridDim.x * kTile) {
    const uint64_t r0 = t0 + 4ull * threadIdx.x;
    if (kCols) {
      star_stage4<kR, kG>(p, r0, scol);
      star_rows4<kSmem, kSplit, kG>(p, r0, StageVals{scol + threadIdx.x, 256}, ssum, scnt, surv, &st);
    } else {
      int4 cur[kVecGroups][kR];
      star_load4<kR, kVecGroups>(p, r0, cur);
      star_rows4<kSmem, kSplit, kVecGroups>(p, r0, RegVals<kR, kVecGroups>{cur}, ssum, scnt, surv, &st);
    }
    if (kSplit) {
      __syncthreads();
      const unsigned int n = st.n;
      if (n) {
        if (threadIdx.x == 0) st.base = atomicAdd(p.surv_cnt, n);
        __syncthreads();
        for (unsigned int k = threadIdx.x; k < n; k += blockDim.x)
          if (st.base + k < p.surv_cap) p.surv_list[st.base + k] = st.e[k];
        __syncthreads();
        if (threadIdx.x == 0) st.n = 0;
        __syncthreads();
      }
    }
  }
  if (kSmem) {
    __syncthreads();
    for (uint32_t q = threadIdx.x; q < p.n_groups; q += blockDim.x) {
      if (scnt[q]) {
        atomicAdd(&p.g_sum[q], ssum[q]);
        atomicAdd(&p.g_cnt[q], scnt[q]);
      }
    }
  }
  if (p.chunk_surv) {
    for (int off = 16; off > 0; off >>= 1) surv += __shfl_down_sync(0xffffffffu, surv, off);
    if ((threadIdx.x & 31) == 0 && surv) atomicAdd(&p.chunk_surv[p.chunk_idx], surv);
  }
}

// Bulk-copy pipeline of the fused chunk kernel (the automatic vector path).
// Persistent blocks of 256 threads walk their 1024-row tiles of the chunk.
// Thread 0 copies each tile's row-logic columns into one stage of a ring of
// shared-memory stages with cp.async.bulk, counted on the stage's mbarrier by
// bytes, n_stages tiles ahead of the block; every thread waits on the stage's
// barrier, evaluates its four rows from shared memory, and after the block's
// barrier (every read of the stage done) thread 0 refills the stage with the
// tile n_stages further on.  The copies of the next tiles stream from HBM
// while the current tile's dimension lookups run.  Survivors (split mode) are
// placed by warp ballots and one global atomic per tile that has any.  Waits
// are bounded: a wait that gives up sets ERR_WAIT, the block stops after the
// tile's barrier (the same decision in every thread), and thread 0 waits,
// bounded again, for the copies it issued to land before the block exits.
constexpr uint32_t kBulkTile = kVecTileRows;  // 4 rows per thread of 256
constexpr uint32_t kBulkColBytes = kBulkTile * 4;
constexpr int kBulkMaxStages = 8;

// tile k of the block (global tile blockIdx.x + k gridDim.x) into stage s
__device__ __forceinline__ void bulk_issue(const ChunkParams &p, uint32_t nr, uint32_t tile, int4 *stage,
                                           uint64_t *bar) {
  const uint32_t row0 = tile * kBulkTile;
  const uint32_t rows = (uint32_t)p.n - row0 < kBulkTile ? (uint32_t)p.n - row0 : kBulkTile;
  const uint32_t bytes = (rows & ~3u) * 4u;  // the partial last group of rows is read by its thread
  if (bytes) {
    mbar_arrive_expect_tx(bar, nr * bytes);
    for (uint32_t k = 0; k < nr; ++k)
      bulk_g2s(reinterpret_cast<char *>(stage) + k * kBulkColBytes, p.staged[p.rowrole[k]] + row0, bytes, bar);
  } else {
    mbar_arrive(bar);
  }
}

template <bool kSmem, bool kSplit>
__global__ void __launch_bounds__(256, 6) star_bulk_kernel(const ChunkParams p, uint32_t n_stages) {
  extern __shared__ __align__(128) unsigned long long sacc[];  // [2 * n_groups] when kSmem, then the stages
  __shared__ __align__(8) uint64_t full[kBulkMaxStages];
  __shared__ uint32_t s_wcnt[2][8], s_base[2], s_abort[2];
  __shared__ int4 s_tail[8];  // the chunk's partial last group of rows (one thread in the grid)
  const uint32_t nr = (uint32_t)p.n_rowroles;
  const uint32_t stage_i4 = nr * (kBulkTile / 4);  // int4 per stage
  int4 *stages = reinterpret_cast<int4 *>(sacc + (kSmem ? 2 * p.n_groups : 0));  // 16-byte aligned
  unsigned long long *ssum = sacc, *scnt = sacc + p.n_groups;
  const uint32_t tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t n = (uint32_t)p.n;  // chunk rows (< 2^31 on this path)
  const uint32_t n_tiles = (n + kBulkTile - 1) / kBulkTile;
  const uint32_t my_n = blockIdx.x < n_tiles ? (n_tiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  uint32_t issued = 0;  // thread 0: tiles of this block whose copies were issued
  if (tid == 0) {
    for (uint32_t s = 0; s < n_stages; ++s) mbar_init(&full[s], 1);
    s_abort[0] = s_abort[1] = 0;
    mbar_fence_init();
    for (; issued < n_stages && issued < my_n; ++issued)
      bulk_issue(p, nr, blockIdx.x + issued * gridDim.x, stages + issued * stage_i4, &full[issued]);
  }
  if (kSmem) {
    for (uint32_t g = tid; g < 2 * p.n_groups; g += blockDim.x) sacc[g] = 0;
  }
  __syncthreads();
  unsigned long long surv = 0;
  uint32_t s = 0, phase = 0, par = 0, k = 0;
  for (; k < my_n; ++k) {
    const uint32_t t = blockIdx.x + k * gridDim.x;
    const bool ok = mbar_wait(&full[s], phase);
    if (!ok) {
      atomicOr(p.err, ERR_WAIT);
      s_abort[par] = 1u;
    }
    const uint32_t r0 = t * kBulkTile + 4u * tid;
    StageVals vals{stages + s * stage_i4 + tid, kBulkTile / 4};
    if (r0 < n && r0 + 3 >= n) {  // rows past the chunk's last whole group: from global memory
      for (uint32_t c = 0; c < nr; ++c) {
        const int32_t *col = p.staged[p.rowrole[c]];
        s_tail[c] = make_int4(__ldg(col + r0), r0 + 1 < n ? __ldg(col + r0 + 1) : 0,
                              r0 + 2 < n ? __ldg(col + r0 + 2) : 0, 0);
      }
      vals = StageVals{s_tail, 1};
    }
    bool alive[4] = {false, false, false, false};
    uint32_t g[4] = {0, 0, 0, 0};
    if constexpr (kSplit) {
      if (ok) star_eval4<1>(p, r0, vals, alive, g);
    } else {
      if (ok) star_rows4<kSmem, false, 1>(p, r0, vals, ssum, scnt, surv, static_cast<SurvTile *>(nullptr));
    }
    uint32_t b[4] = {0, 0, 0, 0}, wtot = 0;
    if constexpr (kSplit) {
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        b[j] = __ballot_sync(0xffffffffu, alive[j]);
        wtot += __popc(b[j]);
      }
      if (lane == 0) s_wcnt[par][warp] = wtot;
    }
    __syncthreads();  // every read of stage s done; warp counts and abort flags visible
    const bool abort = s_abort[par] != 0;
    if (tid == 0 && !abort && issued < my_n) {
      bulk_issue(p, nr, blockIdx.x + issued * gridDim.x, stages + s * stage_i4, &full[s]);
      ++issued;
    }
    if constexpr (kSplit) {
      uint32_t total = 0, woff = 0;
#pragma unroll
      for (uint32_t w = 0; w < 8; ++w) {
        const uint32_t c = s_wcnt[par][w];
        woff += w < warp ? c : 0u;
        total += c;
      }
      if (p.chunk_surv && lane == 0) surv += wtot;
      if (total) {
        if (tid == 0) s_base[par] = atomicAdd(p.surv_cnt, total);
        __syncthreads();
        const uint32_t lt = (1u << lane) - 1u;
        uint32_t o = s_base[par] + woff;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          if (alive[j] && o + __popc(b[j] & lt) < p.surv_cap)
            p.surv_list[o + __popc(b[j] & lt)] = make_uint2(r0 + (uint32_t)j, g[j]);
          o += __popc(b[j]);
        }
      }
    }
    par ^= 1u;
    if (++s == n_stages) {
      s = 0;
      phase ^= 1u;
    }
    if (abort) break;
  }
  if (tid == 0) {  // copies issued for tiles the block did not consume (a wait gave up) land first
    for (uint32_t j = k; j < issued; ++j)
      if (!mbar_wait(&full[j % n_stages], (j / n_stages) & 1u)) atomicOr(p.err, ERR_WAIT);
  }
  if (kSmem) {
    __syncthreads();
    for (uint32_t q = tid; q < p.n_groups; q += blockDim.x) {
      if (scnt[q]) {
        atomicAdd(&p.g_sum[q], ssum[q]);
        atomicAdd(&p.g_cnt[q], scnt[q]);
      }
    }
  }
  if (p.chunk_surv) {
    for (int off = 16; off > 0; off >>= 1) surv += __shfl_down_sync(0xffffffffu, surv, off);
    if (lane == 0 && surv) atomicAdd(&p.chunk_surv[p.chunk_idx], surv);
  }
}
// ---- end of the fused chunk kernel's device code

template <bool kSmem, bool kSplit, int kR>
static int vec_resident(size_t smem) {
  // resident blocks per SM of one instantiation at a dynamic shared-memory size
  static std::mutex mu;
  static std::map<size_t, int> cache;
  std::lock_guard<std::mutex> g(mu);
  auto it = cache.find(smem);
  if (it != cache.end()) return it->second;
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, star_vec_kernel<kSmem, kSplit, kR>, 256,
                                                    smem) != cudaSuccess || occ < 1)
    occ = 1;
  cudaGetLastError();
  cache[smem] = occ;
  return occ;
}

// tiles of n rows; a resident grid when groups accumulate in shared memory.
// acc_smem = the group accumulators' bytes (0 unless kSmem).
template <bool kSmem, bool kSplit, int kR>
static vx_status launch_vec_w(const vx_ctx *ctx, const ChunkParams &p, uint64_t n, size_t acc_smem,
                              cudaStream_t s) {
  static bool attr = false;  // the largest dynamic size this instantiation takes
  if (!attr) {
    VX_CUDA_TRY(cudaFuncSetAttribute(star_vec_kernel<kSmem, kSplit, kR>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)((kSmem ? 16 * kSmemGroups : 0) + vec_col_bytes(kSplit, kR))));
    attr = true;
  }
  const size_t smem = acc_smem + vec_col_bytes(kSplit, kR);
  constexpr uint64_t kTile = (uint64_t)vec_groups(kSplit, kR) * kVecTileRows;
  uint64_t grid = (n + kTile - 1) / kTile;
  // group accumulators in shared memory want a resident grid: each block
  // then merges its groups into global memory once per chunk, not once per tile
  if (kSmem)
    grid = std::min<uint64_t>(grid, (uint64_t)ctx->num_sms * vec_resident<kSmem, kSplit, kR>(smem));
  grid = std::max<uint64_t>(1, std::min<uint64_t>(grid, 1u << 30));
  star_vec_kernel<kSmem, kSplit, kR><<<(unsigned)grid, 256, smem, s>>>(p);
  return VX_OK;
}

template <bool kSmem, bool kSplit>
static vx_status launch_vec(const vx_ctx *ctx, const ChunkParams &p, int kr, size_t acc_smem, cudaStream_t s) {
  switch (kr) {
    case 2: return launch_vec_w<kSmem, kSplit, 2>(ctx, p, p.n, acc_smem, s);
    case 4: return launch_vec_w<kSmem, kSplit, 4>(ctx, p, p.n, acc_smem, s);
    case 6: return launch_vec_w<kSmem, kSplit, 6>(ctx, p, p.n, acc_smem, s);
    default: return launch_vec_w<kSmem, kSplit, 8>(ctx, p, p.n, acc_smem, s);
  }
}


// The bulk-copy pipeline: a resident grid of at most blocks_per_sm blocks per
// SM; the stages fill the shared memory that blocks_per_sm blocks leave after
// the group accumulators (acc_smem bytes), 2 to kBulkMaxStages stages.
template <bool kSmem, bool kSplit>
static vx_status launch_bulk(const vx_ctx *ctx, const ChunkParams &p, size_t acc_smem, cudaStream_t s) {
  static int smem_optin = 0, smem_sm = 0;
  static std::once_flag once;
  std::call_once(once, [] {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    cudaGetLastError();
  });
  static bool attr = false;
  constexpr size_t kStatic = 1024;  // the kernel's static shared memory, rounded up
  if (smem_optin <= (int)kStatic || smem_sm <= 0) {
    set_error("launch_bulk: shared-memory limits unavailable");
    return VX_E_CUDA;
  }
  if (!attr) {
    VX_CUDA_TRY(cudaFuncSetAttribute(star_bulk_kernel<kSmem, kSplit>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     smem_optin - (int)kStatic));
    attr = true;
  }
  const uint32_t nr = (uint32_t)p.n_rowroles;
  const size_t stage = (size_t)nr * kBulkColBytes;
  const int bps = std::max(1, std::min(8, ctx->cfg.blocks_per_sm));
  // per block: its share of the SM's shared memory less the static part and
  // the 1 KB the hardware reserves per block
  const size_t share = (size_t)smem_sm / bps > 2 * kStatic ? (size_t)smem_sm / bps - 2 * kStatic : 0;
  size_t n_st = share > acc_smem ? (share - acc_smem) / stage : 0;
  n_st = std::max<size_t>(2, std::min<size_t>(kBulkMaxStages, n_st));
  while (n_st > 2 && acc_smem + n_st * stage > (size_t)smem_optin - kStatic) --n_st;
  const size_t smem = acc_smem + n_st * stage;
  if (smem > (size_t)smem_optin - kStatic) {
    set_error("launch_bulk: accumulators and two stages exceed a block's shared memory");
    return VX_E_UNSUPPORTED;
  }
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, star_bulk_kernel<kSmem, kSplit>, 256, smem) !=
          cudaSuccess ||
      occ < 1)
    occ = 1;
  cudaGetLastError();
  const uint64_t tiles = (p.n + kBulkTile - 1) / kBulkTile;
  const uint64_t grid =
      std::max<uint64_t>(1, std::min<uint64_t>(tiles, (uint64_t)ctx->num_sms * (uint64_t)std::min(occ, bps)));
  star_bulk_kernel<kSmem, kSplit><<<(unsigned)grid, 256, smem, s>>>(p, (uint32_t)n_st);
  return VX_OK;
}

// width (2, 4, 6 or 8 loaded columns) of the vector path for a chunk, or 0
// for the scalar path (no row-logic column, more than 8, or a staged column
// not 16-byte aligned)
// kernel_rows 0 (automatic: one tile per block) and 2 (the bulk-copy
// pipeline) take the vector path where a chunk allows it; 8 and 16 the scalar
// kernel
static bool vec_path(const vx_ctx *ctx) { return ctx->cfg.kernel_rows == 0 || ctx->cfg.kernel_rows == 2; }
// the bulk-copy pipeline indexes a chunk's rows in 32 bits
static bool bulk_ok(const vx_ctx *ctx, const ChunkParams &p) {
  return ctx->cfg.kernel_rows == 2 && p.n < (1ull << 31);
}

static int vec_width(const ChunkParams &p) {
  if (p.n_rowroles < 1 || p.n_rowroles > 8) return 0;
  for (int k = 0; k < p.n_rowroles; ++k) {
    const int32_t *c = p.staged[p.rowrole[k]];
    if (!c || ((uintptr_t)c & 15)) return 0;
  }
  return p.n_rowroles <= 2 ? 2 : p.n_rowroles <= 4 ? 4 : p.n_rowroles <= 6 ? 6 : 8;
}

// Split mode, pass 1: filter, probe and group id per row; survivors of each
// block tile go to the chunk's survivor list (one global atomic per tile).
// The loop runs over whole block tiles so that every thread reaches the
// barriers.
__global__ void __launch_bounds__(256) star_split_kernel(const ChunkParams p) {
  __shared__ SurvTile st;
  if (threadIdx.x == 0) st.n = 0;
  __syncthreads();
  unsigned long long surv = 0;
  for (uint64_t t0 = (uint64_t)blockIdx.x * kStarTileRows; t0 < p.n; t0 += (uint64_t)gridDim.x * kStarTileRows) {
    star_rows<false, kStarTileRows / 256, true>(p, t0 + threadIdx.x, nullptr, nullptr, surv, &st);
    __syncthreads();
    const unsigned int n = st.n;
    if (n) {
      if (threadIdx.x == 0) st.base = atomicAdd(p.surv_cnt, n);
      __syncthreads();
      for (unsigned int k = threadIdx.x; k < n; k += blockDim.x)
        if (st.base + k < p.surv_cap) p.surv_list[st.base + k] = st.e[k];
      __syncthreads();
      if (threadIdx.x == 0) st.n = 0;
      __syncthreads();
    }
  }
  if (p.chunk_surv) {
    for (int off = 16; off > 0; off >>= 1) surv += __shfl_down_sync(0xffffffffu, surv, off);
    if ((threadIdx.x & 31) == 0 && surv) atomicAdd(&p.chunk_surv[p.chunk_idx], surv);
  }
}

// Split mode, pass 2: late payload columns of every survivor, read through
// mapped host memory with one independent load per survivor in flight, and
// aggregated into the group accumulators.  A chunk whose survivors did not
// fit the list is not aggregated at all: it is flagged for an exact rerun.
template <bool kSmem>
__global__ void __launch_bounds__(256) star_gather_kernel(const ChunkParams p) {
  extern __shared__ unsigned long long sacc[];
  unsigned long long *ssum = sacc, *scnt = sacc + p.n_groups;
  const unsigned int n = *p.surv_cnt;
  if (n > p.surv_cap) {  // the same for every thread of every block
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      if (p.chunk_ovf) p.chunk_ovf[p.chunk_idx] = 1u;
      else atomicOr(p.err, ERR_OVERFLOW);
    }
    return;
  }
  if (kSmem) {
    for (uint32_t g = threadIdx.x; g < 2 * p.n_groups; g += blockDim.x) sacc[g] = 0;
    __syncthreads();
  }
  for (unsigned int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const uint2 e = p.surv_list[i];
    const int64_t a = p.agg_a_role >= 0 ? load_role(p, p.agg_a_role, e.x) : 0;
    const int64_t b = p.agg_b_role >= 0 ? load_role(p, p.agg_b_role, e.x) : 0;
    const int64_t v = p.agg_op == VX_AGG_SUM ? a : p.agg_op == VX_AGG_MUL ? a * b : p.agg_op == VX_AGG_SUB ? a - b : 0;
    if (kSmem) {
      atomicAdd(&ssum[e.y], (unsigned long long)v);
      atomicAdd(&scnt[e.y], 1ull);
    } else {
      atomicAdd(&p.g_sum[e.y], (unsigned long long)v);
      atomicAdd(&p.g_cnt[e.y], 1ull);
    }
  }
  if (kSmem) {
    __syncthreads();
    for (uint32_t q = threadIdx.x; q < p.n_groups; q += blockDim.x) {
      if (scnt[q]) {
        atomicAdd(&p.g_sum[q], ssum[q]);
        atomicAdd(&p.g_cnt[q], scnt[q]);
      }
    }
  }
}

template <bool kSmem, int kRows>
__global__ void __launch_bounds__(256) star_chunk_kernel(const ChunkParams p) {
  extern __shared__ unsigned long long sacc[];  // [2 * n_groups]
  unsigned long long *ssum = sacc, *scnt = sacc + p.n_groups;
  if (kSmem) {
    for (uint32_t g = threadIdx.x; g < 2 * p.n_groups; g += blockDim.x) sacc[g] = 0;
    __syncthreads();
  }
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x * kRows;
  unsigned long long surv = 0;
  for (uint64_t base = (uint64_t)blockIdx.x * blockDim.x * kRows + threadIdx.x; base < p.n; base += stride)
    star_rows<kSmem, kRows>(p, base, ssum, scnt, surv);
  if (kSmem) {
    __syncthreads();
    for (uint32_t q = threadIdx.x; q < p.n_groups; q += blockDim.x) {
      if (scnt[q]) {
        atomicAdd(&p.g_sum[q], ssum[q]);
        atomicAdd(&p.g_cnt[q], scnt[q]);
      }
    }
  }
  if (p.chunk_surv) {
    for (int off = 16; off > 0; off >>= 1) surv += __shfl_down_sync(0xffffffffu, surv, off);
    if ((threadIdx.x & 31) == 0 && surv) atomicAdd(&p.chunk_surv[p.chunk_idx], surv);
  }
}

// Persistent multi-query kernel of the serving engine: one launch per staged
// chunk; resident blocks pull (query, tile) work items from a device counter,
// so queries covering uneven parts of the chunk share the launch.  A tile is
// kMultiTile rows of one query; accumulation goes straight to that query's
// global accumulators.
__global__ void __launch_bounds__(256) star_multi_kernel(const ChunkParams *__restrict__ ps,
                                                          const MultiItem *__restrict__ items, uint32_t n_items,
                                                          unsigned int *next) {
  __shared__ unsigned int s_item;
  __shared__ ChunkParams sp;
  unsigned long long surv = 0;
  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(next, 1u);
    __syncthreads();
    const unsigned int it = s_item;
    if (it >= n_items) break;
    const MultiItem m = items[it];
    const uint32_t *src = reinterpret_cast<const uint32_t *>(&ps[m.q]);
    uint32_t *dst = reinterpret_cast<uint32_t *>(&sp);
    for (uint32_t k = threadIdx.x; k < sizeof(ChunkParams) / 4; k += blockDim.x) dst[k] = src[k];
    __syncthreads();
    star_rows<false, 8>(sp, (uint64_t)m.tile * kMultiTile + threadIdx.x, nullptr, nullptr, surv);
    __syncthreads();  // sp and s_item are rewritten by the next item
  }
}

// union column slots of the shared-scan kernel: column u, thread t at sv[u * 256 + t]
struct UnionVals {
  const int4 *sv;
  const int8_t *ucol;  // the query's slot -> union column
  __device__ __forceinline__ int32_t operator()(int slot, int j) const {
    return lane4(sv[ucol[slot] * 256 + threadIdx.x], j & 3);
  }
};

__global__ void __launch_bounds__(256) star_scan_kernel(const ChunkParams *__restrict__ ps, uint32_t n_q,
                                                         const char *__restrict__ dcols, uint64_t col_stride,
                                                         uint32_t n_cols, uint64_t n_rows, unsigned int *next) {
  extern __shared__ __align__(16) int4 ucols[];  // [n_cols][256] 16-byte slots
  __shared__ unsigned int s_tile;
  unsigned long long surv = 0;
  for (;;) {
    if (threadIdx.x == 0) s_tile = atomicAdd(next, 1u);
    __syncthreads();
    const uint64_t t0 = (uint64_t)s_tile * kVecTileRows;
    __syncthreads();  // s_tile is rewritten by the next tile
    if (t0 >= n_rows) break;
    const uint64_t r0 = t0 + 4ull * threadIdx.x;
    const bool full = r0 + 3 < n_rows;
    for (uint32_t u = 0; u < n_cols; ++u) {  // each thread stages and later reads only its own slots
      const int32_t *col = reinterpret_cast<const int32_t *>(dcols + u * col_stride);
      int4 *dst = &ucols[u * 256 + threadIdx.x];
      if (full) {
        const unsigned sa = (unsigned)__cvta_generic_to_shared(dst);
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(col + r0) : "memory");
      } else {
        *dst = make_int4(r0 < n_rows ? col[r0] : 0, r0 + 1 < n_rows ? col[r0 + 1] : 0,
                         r0 + 2 < n_rows ? col[r0 + 2] : 0, 0);
      }
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    for (uint32_t q = 0; q < n_q; ++q) {
      const ChunkParams &p = ps[q];
      if (!p.scan_kr || t0 >= p.n || t0 + kVecTileRows <= p.row_lo) continue;  // uniform over the block
      const UnionVals vals{ucols, p.ucol};
      star_rows4<false, false, 1>(p, r0, vals, nullptr, nullptr, surv, static_cast<SurvTile *>(nullptr));
    }
  }
}

vx_status launch_star_scan(vx_ctx *ctx, const ChunkParams *d_params, uint32_t n_q, const char *dcols,
                           uint64_t col_stride, uint32_t n_cols, uint64_t n_rows, unsigned int *d_next,
                           cudaStream_t s) {
  if (!n_q || !n_rows || !n_cols) return VX_OK;
  static int occ = 0;
  const size_t smem = (size_t)n_cols * 256 * sizeof(int4);
  if (!occ) {
    VX_CUDA_TRY(cudaFuncSetAttribute(star_scan_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)(12 * 256 * sizeof(int4))));
    VX_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, star_scan_kernel, 256, 12 * 256 * sizeof(int4)));
    occ = std::max(occ, 1);
  }
  if (n_cols > 12) {
    set_error("shared scan: %u union columns; at most 12", n_cols);
    return VX_E_UNSUPPORTED;
  }
  VX_CUDA_TRY(cudaMemsetAsync(d_next, 0, 4, s));
  const uint64_t tiles = (n_rows + kVecTileRows - 1) / kVecTileRows;
  const uint32_t grid = (uint32_t)std::min<uint64_t>(tiles, (uint64_t)ctx->num_sms * occ);
  star_scan_kernel<<<grid, 256, smem, s>>>(d_params, n_q, dcols, col_stride, n_cols, n_rows, d_next);
  VX_CUDA_TRY(cudaGetLastError());
  return VX_OK;
}

vx_status launch_star_multi(vx_ctx *ctx, const ChunkParams *d_params, const MultiItem *d_items, uint32_t n_items,
                            unsigned int *d_next, cudaStream_t s) {
  if (!n_items) return VX_OK;
  VX_CUDA_TRY(cudaMemsetAsync(d_next, 0, 4, s));
  const uint32_t grid = std::min<uint32_t>(n_items, (uint32_t)ctx->num_sms * 4);
  star_multi_kernel<<<grid, 256, 0, s>>>(d_params, d_items, n_items, d_next);
  VX_CUDA_TRY(cudaGetLastError());
  return VX_OK;
}

// Per-chunk features of the cardinality regressor (one block per chunk): 256
// sampled rows (4 runs of 64 consecutive rows) read through mapped host
// memory; f_fact = fraction passing the fact predicates, f_all = fraction
// passing everything (predicates, every probe, group-key ranges).  All roles
// of p are zero-copy; p.row0 is the plan's first row.
__global__ void __launch_bounds__(kChunkSampleRows) chunk_features_kernel(const ChunkParams p, uint64_t n_rows,
                                                                          uint64_t chunk_rows, float dim_sel,
                                                                          float *feats) {
  __shared__ unsigned int cf, ca, cs, cd[VX_MAX_DIMS];
  if (threadIdx.x == 0) cf = ca = cs = 0;
  if (threadIdx.x < VX_MAX_DIMS) cd[threadIdx.x] = 0;
  __syncthreads();
  (void)dim_sel;
  const uint64_t c0 = (uint64_t)blockIdx.x * chunk_rows;
  const uint64_t cn = c0 + chunk_rows <= n_rows ? chunk_rows : n_rows - c0;
  const uint32_t run = threadIdx.x / 64, k = threadIdx.x % 64;
  const uint64_t off = (uint64_t)run * cn / 4 + k;
  if (off < cn) {
    const uint64_t i = p.row0 + c0 + off;
    // every value of the row is read through mapped host memory up front (the
    // reads overlap instead of forming a chain of link round trips), then
    // every dimension is probed (all lookups in flight, for the marginals)
    int32_t fv[VX_MAX_PREDS], kv[VX_MAX_DIMS], gv[VX_MAX_GKEYS];
#pragma unroll
    for (int q = 0; q < VX_MAX_PREDS; ++q) fv[q] = q < p.n_fact_preds ? p.zc[p.fp_role[q]][i] : 0;
#pragma unroll
    for (int d = 0; d < VX_MAX_DIMS; ++d) kv[d] = d < p.n_dims ? p.zc[p.dim_role[d]][i] : 0;
#pragma unroll
    for (int q = 0; q < VX_MAX_GKEYS; ++q) gv[q] = q < p.n_fgk ? p.zc[p.fgk_role[q]][i] : 0;
    bool ok = true;
#pragma unroll
    for (int q = 0; q < VX_MAX_PREDS; ++q)
      if (q < p.n_fact_preds) ok = ok && pred_ok(fv[q], p.fp_op[q], p.fp_lo[q], p.fp_hi[q]);
    bool hit[VX_MAX_DIMS];
#pragma unroll
    for (int d = 0; d < VX_MAX_DIMS; ++d) {
      uint32_t v = 0;
      hit[d] = d < p.n_dims && dim_lookup(p, d, kv[d], v);
    }
    bool all = ok;
#pragma unroll
    for (int d = 0; d < VX_MAX_DIMS; ++d) {
      if (d >= p.n_dims) continue;
      if (hit[d]) atomicAdd(&cd[d], 1u);
      all = all && hit[d];
    }
#pragma unroll
    for (int q = 0; q < VX_MAX_GKEYS; ++q)
      if (q < p.n_fgk) all = all && gv[q] >= 0 && gv[q] < p.fgk_card[q];
    atomicAdd(&cs, 1u);
    if (ok) atomicAdd(&cf, 1u);
    if (all) atomicAdd(&ca, 1u);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const float n = cs ? (float)cs : 1.f;
    float *f = feats + (uint64_t)blockIdx.x * kChunkFeatures;
    float indep = cf / n;  // per-chunk independence estimate: fact fraction x dimension marginals
    for (int d = 0; d < p.n_dims; ++d) indep *= cd[d] / n;
    f[0] = 1.f;
    f[1] = cf / n;
    f[2] = ca / n;
    f[3] = indep;
  }
}

// Normal equations of ridge regression: acc[0 .. d*d) += X^T X, acc[d*d ..
// d*d+d) += X^T y, in fp64 (shared-memory partial sums, one global add per
// block and entry)
__global__ void ridge_accumulate_kernel(const float *X, const float *y, uint64_t n, int d, double *acc) {
  __shared__ double s[8 * 8 + 8];
  for (int k = threadIdx.x; k < d * d + d; k += blockDim.x) s[k] = 0.0;
  __syncthreads();
  for (uint64_t r = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; r < n; r += (uint64_t)gridDim.x * blockDim.x) {
    const float *x = X + r * d;
    for (int a = 0; a < d; ++a) {
      for (int b = 0; b < d; ++b) atomicAdd(&s[a * d + b], (double)x[a] * (double)x[b]);
      atomicAdd(&s[d * d + a], (double)x[a] * (double)y[r]);
    }
  }
  __syncthreads();
  for (int k = threadIdx.x; k < d * d + d; k += blockDim.x) atomicAdd(&acc[k], s[k]);
}

// (X^T X + lambda I) w = X^T y by Cholesky factorisation, one thread (d <= 8)
__global__ void ridge_solve_kernel(const double *acc, int d, double lambda, float *w, uint32_t *err) {
  if (threadIdx.x || blockIdx.x) return;
  double A[8][8], L[8][8], z[8], x[8];
  for (int a = 0; a < d; ++a)
    for (int b = 0; b < d; ++b) A[a][b] = acc[a * d + b] + (a == b ? lambda : 0.0);
  for (int j = 0; j < d; ++j) {
    double sum = A[j][j];
    for (int k = 0; k < j; ++k) sum -= L[j][k] * L[j][k];
    if (!(sum > 1e-10 * A[j][j])) {  // pivot lost to cancellation: (numerically) singular
      *err = 1;
      return;
    }
    L[j][j] = sqrt(sum);
    for (int i = j + 1; i < d; ++i) {
      double t = A[i][j];
      for (int k = 0; k < j; ++k) t -= L[i][k] * L[j][k];
      L[i][j] = t / L[j][j];
    }
  }
  for (int i = 0; i < d; ++i) {  // L z = X^T y
    double t = acc[d * d + i];
    for (int k = 0; k < i; ++k) t -= L[i][k] * z[k];
    z[i] = t / L[i][i];
  }
  for (int i = d - 1; i >= 0; --i) {  // L^T x = z
    double t = z[i];
    for (int k = i + 1; k < d; ++k) t -= L[k][i] * x[k];
    x[i] = t / L[i][i];
  }
  for (int i = 0; i < d; ++i) w[i] = (float)x[i];
  *err = 0;
}

// Fraction of sampled rows passing the fact predicates (planner estimate);
// reads the sampled rows through mapped host memory, in runs of kSampleRun
// consecutive rows so that a few host pages are touched.
constexpr uint32_t kSampleRun = 256;  // 32 runs for the 8,192-row sample
__global__ void sample_preds_kernel(const SampleParams p) {
  unsigned long long c = 0;
  const uint32_t n_seg = (p.n_samples + kSampleRun - 1) / kSampleRun;
  for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < p.n_samples; s += gridDim.x * blockDim.x) {
    const uint64_t seg = s / kSampleRun, k = s % kSampleRun;
    const uint64_t off = seg * p.n / n_seg + k;
    if (off >= p.n) continue;
    const uint64_t i = p.row_begin + off;
    bool ok = true;
    for (int q = 0; q < p.n_preds && ok; ++q) ok = pred_ok(p.col[q][i], p.op[q], p.lo[q], p.hi[q]);
    c += ok;
  }
  for (int off = 16; off > 0; off >>= 1) c += __shfl_down_sync(0xffffffffu, c, off);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(p.out, c);
}

// ---- filter with ordered compaction: count per tile, scan, write ----------
__device__ __forceinline__ bool filter_row(const FilterParams &p, uint64_t i) {
  for (int q = 0; q < p.n_preds; ++q)
    if (!pred_ok(__ldg(&p.col[q][i]), p.op[q], p.lo[q], p.hi[q])) return false;
  return true;
}

__global__ void __launch_bounds__(kFilterThreads) filter_count_kernel(const FilterParams p, uint32_t *tile_cnt) {
  const uint64_t t0 = (uint64_t)blockIdx.x * kFilterTile;
  uint32_t c = 0;
  for (uint32_t k = 0; k < kFilterItems; ++k) {
    uint64_t i = t0 + (uint64_t)k * kFilterThreads + threadIdx.x;
    if (i < p.n) c += filter_row(p, i);
  }
  c = __reduce_add_sync(0xffffffffu, c);
  __shared__ uint32_t ws[kFilterThreads / 32];
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t s = 0;
    for (int w = 0; w < kFilterThreads / 32; ++w) s += ws[w];
    tile_cnt[blockIdx.x] = s;
  }
}

// one block: exclusive scan of tile counts; total -> *count_out (mapped host)
__global__ void __launch_bounds__(1024) filter_scan_kernel(const uint32_t *tile_cnt, uint32_t n_tiles,
                                                           uint32_t *tile_off, uint64_t *count_out) {
  __shared__ uint32_t wsum[32];
  __shared__ uint32_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (uint32_t base = 0; base < n_tiles; base += blockDim.x) {
    uint32_t i = base + threadIdx.x;
    uint32_t v = i < n_tiles ? tile_cnt[i] : 0;
    uint32_t x = v;
    for (int off = 1; off < 32; off <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, x, off);
      if ((threadIdx.x & 31) >= (unsigned)off) x += y;
    }
    if ((threadIdx.x & 31) == 31) wsum[threadIdx.x >> 5] = x;
    __syncthreads();
    if (threadIdx.x < 32) {
      uint32_t w = threadIdx.x < (blockDim.x >> 5) ? wsum[threadIdx.x] : 0;
      for (int off = 1; off < 32; off <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, w, off);
        if (threadIdx.x >= (unsigned)off) w += y;
      }
      wsum[threadIdx.x] = w;  // inclusive
    }
    __syncthreads();
    uint32_t wpre = (threadIdx.x >> 5) ? wsum[(threadIdx.x >> 5) - 1] : 0;
    if (i < n_tiles) tile_off[i] = carry + wpre + x - v;
    __syncthreads();
    if (threadIdx.x == 0) carry += wsum[(blockDim.x >> 5) - 1];
    __syncthreads();
  }
  if (threadIdx.x == 0) *count_out = carry;
}

__global__ void __launch_bounds__(kFilterThreads) filter_write_kernel(const FilterParams p, const uint32_t *tile_off,
                                                                      uint64_t *out) {
  __shared__ uint32_t wcnt[kFilterThreads / 32];
  const uint64_t t0 = (uint64_t)blockIdx.x * kFilterTile;
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t running = tile_off[blockIdx.x];
  for (uint32_t k = 0; k < kFilterItems; ++k) {
    uint64_t i = t0 + (uint64_t)k * kFilterThreads + threadIdx.x;
    bool keep = i < p.n && filter_row(p, i);
    uint32_t bal = __ballot_sync(0xffffffffu, keep);
    if (lane == 0) wcnt[warp] = __popc(bal);
    __syncthreads();
    uint32_t before = 0, total = 0;
    for (uint32_t w = 0; w < kFilterThreads / 32; ++w) {
      uint32_t c = wcnt[w];
      before += w < warp ? c : 0;
      total += c;
    }
    if (keep) out[running + before + __popc(bal & ((1u << lane) - 1u))] = p.row0 + i;
    running += total;
    __syncthreads();
  }
}

// ================================================================== host code

static uint32_t ceil_log2(uint64_t v) {
  uint32_t l = 0;
  while ((1ull << l) < v) ++l;
  return l;
}

static int grid_for(vx_ctx *ctx, uint64_t work_items, int threads) {
  uint64_t want = (work_items + threads - 1) / threads;
  uint64_t cap = (uint64_t)ctx->num_sms * (uint64_t)ctx->cfg.blocks_per_sm;
  if (want > cap) want = cap;
  return want < 1 ? 1 : (int)want;
}

// a 4-byte direct map repacked to vb = 1 or 2 bytes per key (the markers
// become the width's two largest values)
__global__ void pack_dmap_kernel(const uint32_t *in, uint64_t n, void *out, uint32_t vb) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t v = in[i];
    if (vb == 1)
      reinterpret_cast<uint8_t *>(out)[i] = v == HT_EMPTY_VAL ? 0xFFu : v == HT_FILTERED ? 0xFEu : (uint8_t)v;
    else
      reinterpret_cast<uint16_t *>(out)[i] = v == HT_EMPTY_VAL ? 0xFFFFu : v == HT_FILTERED ? 0xFFFEu : (uint16_t)v;
  }
}

__global__ void key_minmax_kernel(const int32_t *key, uint64_t n, int *out) {
  int lo = INT_MAX, hi = INT_MIN;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
    const int k = key[i];
    lo = min(lo, k);
    hi = max(hi, k);
  }
  for (int off = 16; off > 0; off >>= 1) {
    lo = min(lo, __shfl_down_sync(0xffffffffu, lo, off));
    hi = max(hi, __shfl_down_sync(0xffffffffu, hi, off));
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMin(&out[0], lo);
    atomicMax(&out[1], hi);
  }
}

vx_status build_dim_table(vx_ctx *ctx, const DimSpec &d, BuiltDim *out, uint32_t *d_err, uint64_t *d_passed) {
  const uint64_t rows = d.rows;
  cudaStream_t s = ctx->s_compute;
  out->rows = rows;
  out->buf.arena = &ctx->arena;
  // dense keys (span <= 2 x rows) get a direct map of 4-byte values
  if (rows) {
    DevBuf mm;
    mm.arena = &ctx->arena;
    mm.p = ctx->arena.alloc(256);
    if (!mm.p) {
      set_error("arena exhausted");
      return VX_E_NOMEM;
    }
    const int init[2] = {INT_MAX, INT_MIN};
    int h[2];
    VX_CUDA_TRY(cudaMemcpyAsync(mm.p, init, 8, cudaMemcpyHostToDevice, s));
    key_minmax_kernel<<<grid_for(ctx, rows, 256), 256, 0, s>>>(d.key, rows, mm.as<int>());
    VX_CUDA_TRY(cudaGetLastError());
    VX_CUDA_TRY(cudaMemcpyAsync(h, mm.p, 8, cudaMemcpyDeviceToHost, s));
    VX_CUDA_TRY(cudaStreamSynchronize(s));
    const uint64_t span = (uint64_t)((int64_t)h[1] - (int64_t)h[0]) + 1;
    if (span <= 2 * rows && span < (1ull << 31)) {
      out->kmin = h[0];
      out->span = (uint32_t)span;
    }
  }
  uint32_t log2cap = 0;
  if (out->span) {
    out->buf.p = ctx->arena.alloc(4ull * out->span);
    if (!out->buf.p) {
      set_error("dimension map of %llu bytes does not fit the arena", (unsigned long long)(4ull * out->span));
      return VX_E_NOMEM;
    }
    VX_CUDA_TRY(cudaMemsetAsync(out->buf.p, 0xFF, 4ull * out->span, s));  // every value empty
  } else {
    log2cap = ceil_log2(std::max<uint64_t>(2 * rows, 16));
    if (log2cap > 31) {
      set_error("dimension of %llu rows is too large for a 32-bit-indexed table", (unsigned long long)rows);
      return VX_E_UNSUPPORTED;
    }
    out->log2cap = log2cap;
    out->buf.p = ctx->arena.alloc((1ull << log2cap) * sizeof(uint64_t));
    if (!out->buf.p) {
      set_error("dimension hash table of %llu bytes does not fit the arena", (unsigned long long)(8ull << log2cap));
      return VX_E_NOMEM;
    }
    uint64_t cap = 1ull << log2cap;
    fill_u64_kernel<<<grid_for(ctx, cap, 256), 256, 0, s>>>(out->buf.as<uint64_t>(), cap, HT_EMPTY);
    VX_CUDA_TRY(cudaGetLastError());
  }
  DimBuildParams bp{};
  bp.key = d.key;
  bp.rows = rows;
  bp.n_attr = d.n_attr;
  for (int a = 0; a < d.n_attr; ++a) {
    bp.attr[a] = d.attr[a];
    bp.stride[a] = d.stride[a];
    bp.card[a] = d.card[a];
  }
  bp.n_preds = d.n_preds;
  for (int q = 0; q < d.n_preds; ++q) {
    bp.pred_attr[q] = d.pred_attr[q];
    bp.pred_op[q] = d.pred_op[q];
    bp.pred_lo[q] = d.pred_lo[q];
    bp.pred_hi[q] = d.pred_hi[q];
  }
  bp.slots = out->span ? nullptr : out->buf.as<uint64_t>();
  bp.log2cap = log2cap;
  bp.err = d_err;
  bp.passed = (unsigned long long *)d_passed;
  bp.dmap = out->span ? out->buf.as<uint32_t>() : nullptr;
  bp.kmin = out->kmin;
  bp.span = out->span;
  if (rows) {
    ht_build_kernel<<<grid_for(ctx, rows, 256), 256, 0, s>>>(bp);
    VX_CUDA_TRY(cudaGetLastError());
  }
  // a direct map whose largest group-code contribution fits a narrower value
  // (below that width's two markers) is repacked to 1 or 2 bytes per key
  if (out->span && rows) {
    uint64_t vmax = 0;
    for (int a = 0; a < d.n_attr; ++a)
      if (d.stride[a] && d.card[a] > 0) vmax += (uint64_t)(d.card[a] - 1) * d.stride[a];
    const uint32_t vb = vmax < 0xFEu ? 1 : vmax < 0xFFFEu ? 2 : 4;
    if (vb < 4) {
      DevBuf packed;
      packed.arena = &ctx->arena;
      packed.p = ctx->arena.alloc((uint64_t)vb * out->span);
      if (packed.p) {  // else the 4-byte map stays
        pack_dmap_kernel<<<grid_for(ctx, out->span, 256), 256, 0, s>>>(out->buf.as<uint32_t>(), out->span,
                                                                         packed.p, vb);
        VX_CUDA_TRY(cudaGetLastError());
        // the 4-byte map goes back to the arena only once the packing has read it
        VX_CUDA_TRY(cudaStreamSynchronize(s));
        out->buf = std::move(packed);
        out->vbytes = vb;
      }
    }
  }
  return VX_OK;
}

vx_status check_err_word(vx_ctx *ctx, const uint32_t *d_err) {
  uint32_t e = 0;
  VX_CUDA_TRY(cudaMemcpyAsync(&e, d_err, 4, cudaMemcpyDeviceToHost, ctx->s_compute));
  VX_CUDA_TRY(cudaStreamSynchronize(ctx->s_compute));
  if (e & ERR_DUPKEY) {
    set_error("duplicate key on the build side");
    return VX_E_DUPKEY;
  }
  if (e & ERR_RANGE) {
    set_error("group-key code outside [0, card)");
    return VX_E_RANGE;
  }
  if (e & ERR_HT_FULL) {
    set_error("hash table full");
    return VX_E_NOMEM;
  }
  if (e & ERR_OVERFLOW) {
    set_error("a survivor list overflowed with no rerun to catch it");
    return VX_E_CUDA;
  }
  if (e & ERR_WAIT) {
    set_error("a chunk kernel's wait for its staged tiles ran past its limit");
    return VX_E_TIMEOUT;
  }
  return VX_OK;
}

// ------------------------------------------------------------------ star ExKernel
struct StarExKernel : ExKernel {
  vx_ctx *ctx;
  ChunkParams proto{};
  std::vector<const Column *> staged_cols;  // staged role r -> column
  std::vector<int> staged_role;             // index of role in proto.staged
  uint64_t row_begin = 0, n_rows = 0, chunk_rows = 0;
  bool smem = true;
  size_t smem_bytes = 0;
  int grid = 1;
  // per-chunk late materialization: staged columns k with switchable[k] are
  // read through mapped host memory in chunks with chunk_late[it] set
  std::vector<uint8_t> switchable, chunk_late;

  // split mode (late roles): survivor list region after the staged columns,
  // surv_rows entries (0: chunk_rows, which no chunk can overflow)
  bool any_late = false;
  uint64_t surv_rows = 0;
  // a subset of the chunks (their indices), e.g. the overflowed ones rerun
  std::vector<uint64_t> only;
  // per-slot events around the fused kernel (its own duration, immediate schedule)
  std::vector<cudaEvent_t> ev_a, ev_b, ev_c;  // fused kernel [a, b), gather [b, c)
  std::vector<uint8_t> ev_used;
  bool graph_events = false;  // capturing: one event triple per chunk, recorded as graph nodes
  double ms_main = 0, ms_gather = 0;
  uint64_t main_launches = 0, launches = 0;
  ~StarExKernel() override {
    for (auto e : ev_a) cudaEventDestroy(e);
    for (auto e : ev_b) cudaEventDestroy(e);
    for (auto e : ev_c) cudaEventDestroy(e);
  }

  uint64_t size() override { return only.empty() ? (n_rows + chunk_rows - 1) / chunk_rows : only.size(); }
  uint64_t cid(uint64_t it) const { return only.empty() ? it : only[it]; }
  uint64_t surv_region() const { return surv_rows ? std::min(surv_rows, chunk_rows) : chunk_rows; }
  uint64_t cols_bytes() const { return (uint64_t)staged_cols.size() * ((chunk_rows * 4 + 255) & ~255ull); }
  uint64_t slot_bytes() override { return cols_bytes() + (any_late ? surv_region() * 8 + 256 : 0); }
  uint64_t col_off(size_t k) const { return k * ((chunk_rows * 4 + 255) & ~255ull); }
  bool chunk_has_late(uint64_t it) const {
    if (!any_late) return false;
    if (chunk_late.empty()) return true;  // one decision for the whole plan
    return chunk_late[cid(it)] != 0;
  }
  void on_retire(uint64_t it) override {
    const size_t k = it % ev_a.size();
    if (ev_a.empty() || !ev_used[k]) return;
    float ms = 0;
    if (cudaEventElapsedTime(&ms, ev_a[k], ev_b[k]) == cudaSuccess) {
      ms_main += ms;
      main_launches += 1;
    }
    if (ev_used[k] == 2 && cudaEventElapsedTime(&ms, ev_b[k], ev_c[k]) == cudaSuccess) ms_gather += ms;
    cudaGetLastError();
    ev_used[k] = 0;
  }
  uint64_t rows_of(uint64_t it) const { return std::min(chunk_rows, n_rows - cid(it) * chunk_rows); }
  bool late_in(size_t k, uint64_t it) const {
    const uint64_t c = cid(it);
    return k < switchable.size() && switchable[k] && c < chunk_late.size() && chunk_late[c];
  }

  void inputs(uint64_t it, char *slot, std::vector<CopyOp> &h2d) override {
    const uint64_t r0 = row_begin + cid(it) * chunk_rows, n = rows_of(it);
    for (size_t k = 0; k < staged_cols.size(); ++k)
      if (!late_in(k, it)) h2d.push_back({(const char *)staged_cols[k]->host + r0 * 4, slot + col_off(k), n * 4});
  }
  vx_status kernel(char *slot, uint64_t it, cudaStream_t s) override {
    ChunkParams p = proto;
    p.row0 = row_begin + cid(it) * chunk_rows;
    p.n = rows_of(it);
    p.chunk_idx = cid(it);
    for (size_t k = 0; k < staged_cols.size(); ++k)
      p.staged[staged_role[k]] = late_in(k, it) ? nullptr : (const int32_t *)(slot + col_off(k));
    int threads = ctx->cfg.block_threads > 256 ? 256 : ctx->cfg.block_threads;
    int g = grid_for(ctx, (p.n + 7) / 8, threads);
    const size_t ek = ev_a.empty() ? 0 : it % ev_a.size();
    const bool timed = !ev_a.empty() && (graph_events || ctx->cfg.sched == VX_SCHED_IMMEDIATE);
    auto rec = [&](cudaEvent_t e) {
      return graph_events ? cudaEventRecordWithFlags(e, s, cudaEventRecordExternal) : cudaEventRecord(e, s);
    };
    if (chunk_has_late(it)) {  // filter/probe pass, then the late-column gather
      p.surv_list = (uint2 *)(slot + cols_bytes());
      p.surv_cnt = (unsigned int *)(slot + cols_bytes() + surv_region() * 8);
      p.surv_cap = (unsigned int)surv_region();
      VX_CUDA_TRY(cudaMemsetAsync(p.surv_cnt, 0, 4, s));
      if (timed) VX_CUDA_TRY(rec(ev_a[ek]));
      const int kr = vec_path(ctx) ? vec_width(p) : 0;
      if (kr && bulk_ok(ctx, p)) {
        VX_TRY((launch_bulk<false, true>(ctx, p, 0, s)));
      } else if (kr) {
        VX_TRY((launch_vec<false, true>(ctx, p, kr, 0, s)));
      } else {
        const int gs = grid_for(ctx, (p.n + kStarTileRows - 1) / kStarTileRows, 1);
        star_split_kernel<<<gs, 256, 0, s>>>(p);
      }
      if (timed) VX_CUDA_TRY(rec(ev_b[ek]));
      const int gg = ctx->num_sms * 4;
      if (smem) {
        static bool attr_g = false;
        if (!attr_g) {
          VX_CUDA_TRY(cudaFuncSetAttribute(star_gather_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)(16 * kSmemGroups)));
          attr_g = true;
        }
        star_gather_kernel<true><<<gg, 256, smem_bytes, s>>>(p);
      } else {
        star_gather_kernel<false><<<gg, 256, 0, s>>>(p);
      }
      VX_CUDA_TRY(cudaGetLastError());
      launches += 2;
      if (timed) {
        VX_CUDA_TRY(rec(ev_c[ek]));
        if (!graph_events) ev_used[ek] = 2;
      }
      return VX_OK;
    }
    launches += 1;
    if (timed) VX_CUDA_TRY(rec(ev_a[ek]));
    const int kr = vec_path(ctx) ? vec_width(p) : 0;
    if (kr && bulk_ok(ctx, p)) {  // bulk-copy pipeline
      if (smem) {
        VX_TRY((launch_bulk<true, false>(ctx, p, smem_bytes, s)));
      } else {
        VX_TRY((launch_bulk<false, false>(ctx, p, 0, s)));
      }
    } else if (kr) {  // one tile per block
      if (smem) {
        VX_TRY((launch_vec<true, false>(ctx, p, kr, smem_bytes, s)));
      } else {
        VX_TRY((launch_vec<false, false>(ctx, p, kr, 0, s)));
      }
    } else if (ctx->cfg.kernel_rows == 16) {  // scalar kernel, 16 rows per thread
      g = grid_for(ctx, (p.n + 15) / 16, threads);
      if (smem) {
        static bool attr16 = false;
        if (!attr16) {
          VX_CUDA_TRY(cudaFuncSetAttribute(star_chunk_kernel<true, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)(16 * kSmemGroups)));
          attr16 = true;
        }
        star_chunk_kernel<true, 16><<<g, threads, smem_bytes, s>>>(p);
      } else {
        star_chunk_kernel<false, 16><<<g, threads, 0, s>>>(p);
      }
    } else if (smem) {
      static bool attr_set = false;
      if (!attr_set) {
        VX_CUDA_TRY(cudaFuncSetAttribute(star_chunk_kernel<true, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(16 * kSmemGroups)));
        attr_set = true;
      }
      star_chunk_kernel<true, 8><<<g, threads, smem_bytes, s>>>(p);
    } else {
      star_chunk_kernel<false, 8><<<g, threads, 0, s>>>(p);
    }
    VX_CUDA_TRY(cudaGetLastError());
    if (timed) {
      VX_CUDA_TRY(rec(ev_b[ek]));
      if (!graph_events) ev_used[ek] = 1;
    }
    return VX_OK;
  }
};

// Finds or captures the CUDA graph of a star pipeline (batching).  The key is
// everything the captured work depends on: the kernel parameters (tables,
// predicates, roles), the staged host columns, the chunking and the launch
// shape.  On a full arena the other cached graphs are released and the
// capture retried once; if it still does not fit, *out stays null and the
// caller runs the executor instead.
vx_status star_graph(vx_ctx *ctx, StarExKernel &ek, const std::vector<std::shared_ptr<ResidentHT>> &tables,
                     uint64_t G, std::shared_ptr<GraphEntry> *out) {
  ChunkParams kp = ek.proto;
  kp.g_sum = kp.g_cnt = nullptr;
  kp.err = nullptr;
  kp.chunk_ovf = nullptr;
  kp.row0 = kp.n = 0;
  std::string key((const char *)&kp, sizeof kp);
  for (const Column *c : ek.staged_cols) key.append((const char *)&c->host, sizeof(void *));
  const uint64_t dims[8] = {ek.row_begin, ek.n_rows, ek.chunk_rows, (uint64_t)ctx->cfg.n_slots,
                            (uint64_t)ctx->cfg.block_threads, (uint64_t)ctx->cfg.blocks_per_sm, ek.surv_rows,
                            (uint64_t)ctx->cfg.kernel_rows};
  key.append((const char *)dims, sizeof dims);
  key.append(ek.switchable.begin(), ek.switchable.end());
  key.append(ek.chunk_late.begin(), ek.chunk_late.end());
  auto it = ctx->graphs.find(key);
  if (it != ctx->graphs.end()) {
    *out = it->second;
    return VX_OK;
  }
  const int S = std::max(2, ctx->cfg.n_slots);
  const uint64_t slot = (ek.slot_bytes() + 255) & ~255ull;
  auto e = std::make_shared<GraphEntry>();
  e->tables = tables;
  const uint64_t n_ch = ek.size();
  const bool want_ovf = ek.proto.chunk_ovf != nullptr;
  for (int attempt = 0; attempt < 2; ++attempt) {
    e->ring.arena = e->acc.arena = e->err.arena = e->ovf.arena = &ctx->arena;
    e->ring.p = ctx->arena.alloc(slot * S);
    e->acc.p = ctx->arena.alloc(16 * G);
    e->err.p = ctx->arena.alloc(256);
    if (want_ovf) e->ovf.p = ctx->arena.alloc(4 * n_ch);
    if (e->ring.p && e->acc.p && e->err.p && (!want_ovf || e->ovf.p)) break;
    e->ring.release();
    e->acc.release();
    e->err.release();
    e->ovf.release();
    ctx->graphs.clear();
  }
  if (!e->ring.p || !e->acc.p || !e->err.p || (want_ovf && !e->ovf.p)) return VX_OK;  // no room: run without a graph
  ChunkParams gp = ek.proto;
  gp.g_sum = e->acc.as<unsigned long long>();
  gp.g_cnt = gp.g_sum + G;
  gp.err = e->err.as<uint32_t>();
  gp.chunk_ovf = want_ovf ? e->ovf.as<unsigned int>() : nullptr;
  StarExKernel gk = ek;
  gk.proto = gp;
  gk.ev_used.clear();
  // the graph's own timing events (the entry owns them; gk only borrows them
  // while capturing, and ek's belong to ek)
  const uint64_t N = gk.size();
  for (auto v : {&e->ev_a, &e->ev_b, &e->ev_c}) {
    v->resize(N, nullptr);
    for (uint64_t c = 0; c < N; ++c) VX_CUDA_TRY(cudaEventCreate(&(*v)[c]));
  }
  e->split.resize(N);
  for (uint64_t c = 0; c < N; ++c) e->split[c] = gk.chunk_has_late(c) ? 1 : 0;
  gk.ev_a = e->ev_a;
  gk.ev_b = e->ev_b;
  gk.ev_c = e->ev_c;
  gk.graph_events = true;
  struct Unborrow {
    StarExKernel &k;
    ~Unborrow() {
      k.ev_a.clear();
      k.ev_b.clear();
      k.ev_c.clear();
    }
  } unborrow{gk};
  cudaStream_t s = ctx->s_compute;
  VX_CUDA_TRY(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
  ExecStats est;
  vx_status st = VX_OK;
  if (cudaMemsetAsync(e->acc.p, 0, 16 * G, s) != cudaSuccess || cudaMemsetAsync(e->err.p, 0, 4, s) != cudaSuccess ||
      (want_ovf && cudaMemsetAsync(e->ovf.p, 0, 4 * n_ch, s) != cudaSuccess)) {
    set_error("graph capture: memset failed");
    st = VX_E_CUDA;
  }
  if (st == VX_OK) st = enqueue_pipeline_for_capture(ctx, gk, e->ring.as<char>(), S, &est);
  cudaGraph_t g = nullptr;
  cudaError_t ce = cudaStreamEndCapture(s, &g);
  if (st != VX_OK) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    return st;
  }
  VX_CUDA_TRY(ce);
  // per-node priorities, so that the copy kernels' high priority holds in
  // the replayed graph too (without the flag it runs at the stream's)
  ce = cudaGraphInstantiate(&e->exec, g, cudaGraphInstantiateFlagUseNodePriority);
  cudaGraphDestroy(g);
  VX_CUDA_TRY(ce);
  e->chunks = est.chunks;
  e->bytes_h2d = est.bytes_h2d;
  e->launches = est.kernel_launches;
  ctx->graphs[key] = e;
  *out = e;
  return VX_OK;
}

// planner: resolves a plan into dimension specs and chunk-kernel parameters
vx_status run_star(vx_ctx *ctx, const vx_plan *plan, vx_result *out, bool use_resident, PreparedStar *prep) {
  const double t_start = now_ms();
  vx_query_stats qs{};
  if (!plan || (!out && !prep)) {
    set_error("vx_run_plan: null argument");
    return VX_E_INVAL;
  }
  if (plan->n_dims < 0 || plan->n_dims > VX_MAX_DIMS || plan->n_fact_preds < 0 ||
      plan->n_fact_preds > VX_MAX_PREDS || plan->n_group_keys < 0 || plan->n_group_keys > VX_MAX_GKEYS ||
      plan->agg_op < VX_AGG_COUNT || plan->agg_op > VX_AGG_SUB) {
    set_error("vx_run_plan: counts out of range");
    return VX_E_INVAL;
  }
  // ---- fact columns and roles
  std::vector<int32_t> role_col;  // role -> column id
  auto role_of = [&](int32_t col) -> int {
    for (size_t r = 0; r < role_col.size(); ++r)
      if (role_col[r] == col) return (int)r;
    role_col.push_back(col);
    return (int)role_col.size() - 1;
  };
  uint64_t n_fact = UINT64_MAX;
  auto fact_col = [&](int32_t id) -> const Column * {
    const Column *c = get_col(ctx, id, VX_I32);
    if (c) {
      if (n_fact == UINT64_MAX) n_fact = c->n_rows;
      if (c->n_rows != n_fact) {
        set_error("fact columns differ in length");
        return nullptr;
      }
    }
    return c;
  };
  ChunkParams P{};
  for (int r = 0; r < kMaxRoles; ++r) {
    P.staged[r] = nullptr;
    P.zc[r] = nullptr;
  }
  P.n_fact_preds = plan->n_fact_preds;
  for (int q = 0; q < plan->n_fact_preds; ++q) {
    const vx_pred &fp = plan->fact_preds[q];
    if (!fact_col(fp.col)) return VX_E_INVAL;
    if (fp.op < VX_BETWEEN || fp.op > VX_GE) {
      set_error("bad predicate op %d", fp.op);
      return VX_E_INVAL;
    }
    P.fp_role[q] = role_of(fp.col);
    P.fp_op[q] = fp.op;
    P.fp_lo[q] = fp.lo;
    P.fp_hi[q] = fp.hi;
  }
  // group strides: first key most significant
  uint64_t G = 1;
  uint64_t stride_of[VX_MAX_GKEYS];
  for (int k = plan->n_group_keys - 1; k >= 0; --k) {
    const vx_plan_gkey &gk = plan->group_keys[k];
    if (gk.card < 1) {
      set_error("group key cardinality must be >= 1");
      return VX_E_INVAL;
    }
    stride_of[k] = G;
    G *= (uint64_t)gk.card;
    if (G > (1ull << 26)) {
      set_error("too many groups (%llu)", (unsigned long long)G);
      return VX_E_UNSUPPORTED;
    }
  }
  P.n_groups = (uint32_t)G;
  // dimensions
  std::vector<DimSpec> dspec(plan->n_dims);
  P.n_dims = plan->n_dims;
  for (int d = 0; d < plan->n_dims; ++d) {
    const vx_plan_dim &pd = plan->dims[d];
    const Column *kc = get_col(ctx, pd.key_col, VX_I32);
    if (!kc || !fact_col(pd.fact_fk_col)) return VX_E_INVAL;
    if (pd.n_attr < 0 || pd.n_attr > 4 || pd.n_preds < 0 || pd.n_preds > 4) {
      set_error("dimension %d: attribute/predicate count out of range", d);
      return VX_E_INVAL;
    }
    DimSpec &ds = dspec[d];
    ds.key = (const int32_t *)kc->dev;
    ds.key_col = pd.key_col;
    ds.rows = kc->n_rows;
    ds.n_attr = pd.n_attr;
    for (int a = 0; a < pd.n_attr; ++a) {
      const Column *ac = get_col(ctx, pd.attr_col[a], VX_I32);
      if (!ac || ac->n_rows != kc->n_rows) {
        set_error("dimension %d attribute %d: bad column", d, a);
        return VX_E_INVAL;
      }
      ds.attr[a] = (const int32_t *)ac->dev;
      ds.attr_col[a] = pd.attr_col[a];
      ds.stride[a] = 0;
      ds.card[a] = 0;
    }
    ds.n_preds = pd.n_preds;
    for (int q = 0; q < pd.n_preds; ++q) {
      if (pd.pred_attr[q] < 0 || pd.pred_attr[q] >= pd.n_attr || pd.pred_op[q] < 0 || pd.pred_op[q] > VX_GE) {
        set_error("dimension %d predicate %d: bad attribute or op", d, q);
        return VX_E_INVAL;
      }
      ds.pred_attr[q] = pd.pred_attr[q];
      ds.pred_op[q] = pd.pred_op[q];
      ds.pred_lo[q] = pd.pred_lo[q];
      ds.pred_hi[q] = pd.pred_hi[q];
    }
    P.dim_role[d] = role_of(pd.fact_fk_col);
  }
  P.n_fgk = 0;
  for (int k = 0; k < plan->n_group_keys; ++k) {
    const vx_plan_gkey &gk = plan->group_keys[k];
    if (gk.dim >= 0) {
      if (gk.dim >= plan->n_dims || gk.attr < 0 || gk.attr >= dspec[gk.dim].n_attr) {
        set_error("group key %d: bad dimension attribute", k);
        return VX_E_INVAL;
      }
      if (dspec[gk.dim].stride[gk.attr]) {
        set_error("group key %d repeats an attribute", k);
        return VX_E_INVAL;
      }
      dspec[gk.dim].stride[gk.attr] = (uint32_t)stride_of[k];
      dspec[gk.dim].card[gk.attr] = gk.card;
    } else {
      if (!fact_col(gk.fact_col)) return VX_E_INVAL;
      P.fgk_role[P.n_fgk] = role_of(gk.fact_col);
      P.fgk_card[P.n_fgk] = gk.card;
      P.fgk_stride[P.n_fgk] = (uint32_t)stride_of[k];
      ++P.n_fgk;
    }
  }
  if (n_fact == UINT64_MAX) {
    set_error("plan references no fact column");
    return VX_E_INVAL;
  }
  const uint64_t row_begin = std::min(plan->row_begin, n_fact);
  const uint64_t row_end = plan->row_end == 0 ? n_fact : std::min(plan->row_end, n_fact);
  const uint64_t n_rows = row_end > row_begin ? row_end - row_begin : 0;
  const size_t n_row_roles = role_col.size();  // roles needed for every row
  // aggregate columns
  P.agg_op = plan->agg_op;
  P.agg_a_role = P.agg_b_role = -1;
  int agg_cols[2] = {plan->agg_op == VX_AGG_COUNT ? -1 : plan->agg_a,
                     (plan->agg_op == VX_AGG_MUL || plan->agg_op == VX_AGG_SUB) ? plan->agg_b : -1};
  for (int j = 0; j < 2; ++j)
    if (agg_cols[j] >= 0 && !fact_col(agg_cols[j])) return VX_E_INVAL;

  // ---- device scratch: error word + counters
  DevBuf scratch;
  scratch.arena = &ctx->arena;
  scratch.p = ctx->arena.alloc(256 + 16 * 8);
  if (!scratch.p) {
    set_error("arena exhausted");
    return VX_E_NOMEM;
  }
  uint32_t *d_err = scratch.as<uint32_t>();
  uint64_t *d_cnt = (uint64_t *)(scratch.as<char>() + 256);
  VX_CUDA_TRY(cudaMemsetAsync(scratch.p, 0, 256 + 16 * 8, ctx->s_compute));

  // ---- dimension tables (Section 7.1: filtered, hashed, kept on the device)
  std::vector<std::shared_ptr<ResidentHT>> tables(plan->n_dims);
  for (int d = 0; d < plan->n_dims; ++d) {
    std::string sig = dim_signature(dspec[d]);
    auto it = use_resident ? ctx->resident.find(sig) : ctx->resident.end();
    if (it != ctx->resident.end()) {
      tables[d] = it->second;
      continue;
    }
    auto t = std::make_shared<ResidentHT>();
    VX_TRY(build_dim_table(ctx, dspec[d], &t->dim, d_err, d_cnt + d));
    tables[d] = t;
  }
  {
    uint64_t passed[VX_MAX_DIMS] = {0};
    VX_CUDA_TRY(cudaMemcpyAsync(passed, d_cnt, 8 * VX_MAX_DIMS, cudaMemcpyDeviceToHost, ctx->s_compute));
    VX_TRY(check_err_word(ctx, d_err));
    for (int d = 0; d < plan->n_dims; ++d) {
      if (!tables[d]->built) {
        tables[d]->dim.passed = passed[d];
        tables[d]->built = true;
        if (use_resident) ctx->resident[dim_signature(dspec[d])] = tables[d];
      }
      P.ht[d] = tables[d]->dim.buf.as<uint64_t>();
      P.ht_log2[d] = tables[d]->dim.log2cap;
      P.dmin[d] = tables[d]->dim.kmin;
      P.dspan[d] = tables[d]->dim.span;
      P.dvb[d] = (uint8_t)tables[d]->dim.vbytes;
    }
  }
  // ---- selectivity estimate: dimension pass fractions x sampled fact predicates
  double est = 1.0;
  for (int d = 0; d < plan->n_dims; ++d)
    est *= tables[d]->dim.rows ? (double)tables[d]->dim.passed / (double)tables[d]->dim.rows : 0.0;
  if (plan->n_fact_preds > 0 && n_rows > 0) {
    SampleParams sp{};
    sp.n_preds = plan->n_fact_preds;
    for (int q = 0; q < plan->n_fact_preds; ++q) {
      sp.col[q] = (const int32_t *)ctx->cols[plan->fact_preds[q].col].dev;
      sp.op[q] = plan->fact_preds[q].op;
      sp.lo[q] = plan->fact_preds[q].lo;
      sp.hi[q] = plan->fact_preds[q].hi;
    }
    sp.row_begin = row_begin;
    sp.n = n_rows;
    sp.n_samples = (uint32_t)std::min<uint64_t>(n_rows, 8192);
    sp.n_samples = sp.n_samples / kSampleRun * kSampleRun;
    if (sp.n_samples == 0) sp.n_samples = (uint32_t)n_rows;  // fewer rows than one run: all rows
    sp.out = (unsigned long long *)(d_cnt + 15);
    sample_preds_kernel<<<16, 256, 0, ctx->s_compute>>>(sp);
    VX_CUDA_TRY(cudaGetLastError());
    uint64_t hit = 0;
    VX_CUDA_TRY(cudaMemcpyAsync(&hit, d_cnt + 15, 8, cudaMemcpyDeviceToHost, ctx->s_compute));
    VX_CUDA_TRY(cudaStreamSynchronize(ctx->s_compute));
    est *= (double)hit / (double)sp.n_samples;
  }
  qs.est_selectivity = est;
  const double TH = ctx->cfg.zc_threshold > 0 ? ctx->cfg.zc_threshold : kDefaultZeroCopyTH;
  const bool per_chunk = plan->late_mat == VX_LATE_PER_CHUNK;
  bool late = plan->late_mat == VX_LATE_FORCE_LATE || (plan->late_mat == VX_LATE_AUTO && est < TH);
  // aggregate roles: a column already staged for the row logic stays staged
  uint32_t late_mask = 0, switch_mask = 0;
  for (int j = 0; j < 2; ++j) {
    if (agg_cols[j] < 0) continue;
    size_t before = role_col.size();
    int r = role_of(agg_cols[j]);
    bool is_new = role_col.size() > before;
    if (j == 0) P.agg_a_role = r; else P.agg_b_role = r;
    if (is_new && late) late_mask |= 1u << j;
    if (is_new && per_chunk) switch_mask |= 1u << j;
  }
  if (role_col.size() > (size_t)kMaxRoles) {
    set_error("plan references %zu fact columns; at most %d", role_col.size(), kMaxRoles);
    return VX_E_UNSUPPORTED;
  }
  {  // vector path: the row-logic roles (always staged) and each reader's slot
    std::vector<int> rr;
    auto slot = [&](int role) -> int8_t {
      for (size_t k = 0; k < rr.size(); ++k)
        if (rr[k] == role) return (int8_t)k;
      rr.push_back(role);
      return (int8_t)(rr.size() - 1);
    };
    for (int q = 0; q < P.n_fact_preds; ++q) P.fp_slot[q] = slot(P.fp_role[q]);
    for (int d = 0; d < P.n_dims; ++d) P.dim_slot[d] = slot(P.dim_role[d]);
    for (int k = 0; k < P.n_fgk; ++k) P.fgk_slot[k] = slot(P.fgk_role[k]);
    // an aggregate column staged in every chunk joins the up-front loads, so a
    // survivor's values need no load after its probe chain
    // (only while the vector path's eight columns suffice)
    const int agg_role[2] = {P.agg_a_role, P.agg_b_role};
    const size_t n_logic = rr.size();
    size_t n_new = 0;
    for (int j = 0; j < 2; ++j)
      if (agg_role[j] >= 0 && std::find(rr.begin(), rr.end(), agg_role[j]) == rr.end()) ++n_new;
    for (int j = 0; j < 2; ++j)
      P.agg_slot[j] = agg_role[j] >= 0 && !((late_mask | switch_mask) >> j & 1u) && n_logic >= 1 &&
                              n_logic + n_new <= 8
                          ? slot(agg_role[j])
                          : (int8_t)-1;
    P.n_rowroles = rr.size() <= 8 ? (int)rr.size() : 0;  // 0: scalar path
    for (size_t k = 0; k < rr.size() && k < 8; ++k) P.rowrole[k] = (int8_t)rr[k];
  }
  // ---- accumulators
  DevBuf acc;
  acc.arena = &ctx->arena;
  acc.p = ctx->arena.alloc(16 * G);
  if (!acc.p) {
    set_error("group accumulators do not fit the arena");
    return VX_E_NOMEM;
  }
  P.g_sum = acc.as<unsigned long long>();
  P.g_cnt = P.g_sum + G;
  P.err = d_err;
  VX_CUDA_TRY(cudaMemsetAsync(acc.p, 0, 16 * G, ctx->s_compute));

  StarExKernel ek;
  ek.ctx = ctx;
  ek.row_begin = row_begin;
  ek.n_rows = n_rows;
  for (size_t r = 0; r < role_col.size(); ++r) {
    const Column *c = &ctx->cols[role_col[r]];
    bool is_late = false, is_switch = false;
    if ((int)r == P.agg_a_role && (late_mask & 1u)) is_late = true;
    if ((int)r == P.agg_b_role && (late_mask & 2u)) is_late = true;
    if ((int)r == P.agg_a_role && (switch_mask & 1u)) is_switch = true;
    if ((int)r == P.agg_b_role && (switch_mask & 2u)) is_switch = true;
    if (is_late) {
      P.zc[r] = (const int32_t *)c->dev;
    } else {
      if (is_switch) P.zc[r] = (const int32_t *)c->dev;
      ek.staged_cols.push_back(c);
      ek.staged_role.push_back((int)r);
      ek.switchable.push_back(is_switch ? 1 : 0);
    }
  }
  (void)n_row_roles;
  // rows per chunk follow from all referenced columns, so the chunking does not
  // depend on the late/early decision
  const uint64_t per_row = 4 * std::max<size_t>(1, role_col.size());
  uint64_t cr = ctx->cfg.chunk_bytes / per_row;
  cr = cr / 1024 * 1024;
  if (cr < 1024) cr = 1024;
  if (cr > n_rows) cr = std::max<uint64_t>(n_rows, 1);
  ek.chunk_rows = cr;
  ek.smem = G <= kSmemGroups;
  ek.smem_bytes = ek.smem ? 16 * G : 0;
  ek.any_late = late_mask != 0 || switch_mask != 0;
  if (!ctx->cfg.use_graphs && ctx->cfg.sched == VX_SCHED_IMMEDIATE && !prep) {
    const int S = std::max(2, ctx->cfg.n_slots);
    ek.ev_a.resize(S);
    ek.ev_b.resize(S);
    ek.ev_c.resize(S);
    ek.ev_used.assign(S, 0);
    for (int i = 0; i < S; ++i) {
      VX_CUDA_TRY(cudaEventCreate(&ek.ev_a[i]));
      VX_CUDA_TRY(cudaEventCreate(&ek.ev_b[i]));
      VX_CUDA_TRY(cudaEventCreate(&ek.ev_c[i]));
    }
  }
  const uint64_t n_chunks = n_rows ? (n_rows + cr - 1) / cr : 0;

  if (prep) {  // planning only: hand the query to another executor
    prep->P = P;
    prep->acc = std::move(acc);
    prep->scratch = std::move(scratch);
    prep->tables = tables;
    prep->role_col = role_col;
    prep->staged_cols = ek.staged_cols;
    prep->staged_role = ek.staged_role;
    prep->G = G;
    prep->row_begin = row_begin;
    prep->n_rows = n_rows;
    prep->late_mask = late_mask;
    prep->est = est;
    return VX_OK;
  }
  // ---- per-chunk statistics (logged for the regressor) and per-chunk
  // late/early decisions from the regressor's predicted selectivity
  const bool want_log = ctx->cfg.log_chunk_stats && !ctx->cfg.use_graphs;
  std::vector<float> feats;
  DevBuf fbuf;
  uint32_t late_chunks = 0;
  double ms_features = 0;
  if ((per_chunk || want_log) && n_chunks) {
    const double tf0 = now_ms();
    fbuf.arena = &ctx->arena;
    fbuf.p = ctx->arena.alloc(n_chunks * (4 * kChunkFeatures + 8) + 512);
    if (!fbuf.p) {
      set_error("per-chunk statistics do not fit the arena");
      return VX_E_NOMEM;
    }
    float *d_feats = fbuf.as<float>();
    unsigned long long *d_surv =
        (unsigned long long *)(fbuf.as<char>() + ((n_chunks * 4 * kChunkFeatures + 255) & ~255ull));
    ChunkParams pz = P;
    for (size_t r = 0; r < role_col.size(); ++r) {
      pz.staged[r] = nullptr;
      pz.zc[r] = (const int32_t *)ctx->cols[role_col[r]].dev;
    }
    pz.row0 = row_begin;
    double dsel = 1.0;
    for (int d = 0; d < plan->n_dims; ++d)
      dsel *= tables[d]->dim.rows ? (double)tables[d]->dim.passed / (double)tables[d]->dim.rows : 0.0;
    chunk_features_kernel<<<(unsigned)n_chunks, kChunkSampleRows, 0, ctx->s_compute>>>(pz, n_rows, cr, (float)dsel,
                                                                                       d_feats);
    VX_CUDA_TRY(cudaGetLastError());
    feats.resize(n_chunks * kChunkFeatures);
    VX_CUDA_TRY(cudaMemcpyAsync(feats.data(), d_feats, 4 * feats.size(), cudaMemcpyDeviceToHost, ctx->s_compute));
    if (want_log) {
      VX_CUDA_TRY(cudaMemsetAsync(d_surv, 0, 8 * n_chunks, ctx->s_compute));
      P.chunk_surv = d_surv;
    }
    VX_CUDA_TRY(cudaStreamSynchronize(ctx->s_compute));
    if (per_chunk) {
      ek.chunk_late.resize(n_chunks);
      uint64_t cap_rows = 0;
      for (uint64_t c = 0; c < n_chunks; ++c) {
        const float *f = &feats[c * kChunkFeatures];
        double yhat = f[2];  // sampled selectivity when no regressor is trained
        if (ctx->reg_trained) {
          yhat = 0;
          for (int k = 0; k < kChunkFeatures; ++k) yhat += (double)ctx->reg_w[k] * f[k];
        }
        ek.chunk_late[c] = yhat < TH ? 1 : 0;
        late_chunks += ek.chunk_late[c];
        if (ek.chunk_late[c]) {
          // survivor-list entries a late chunk gets: the predicted survivors
          // with a quarter and four standard deviations of headroom (a chunk
          // beyond it is rerun exactly)
          const double pred = std::max(0.0, yhat) * (double)std::min(cr, n_rows - c * cr);
          cap_rows = std::max<uint64_t>(cap_rows, (uint64_t)std::ceil(1.25 * pred + 4.0 * std::sqrt(pred + 1.0)) +
                                                      2 * kStarTileRows);
        }
      }
      ek.surv_rows = std::max<uint64_t>(cap_rows, kStarTileRows);
    }
    ms_features = now_ms() - tf0;
  }
  // per-chunk survivor-list overflow flags (survivor lists sized from predictions)
  DevBuf ovf;
  if (per_chunk && late_chunks && n_chunks) {
    ovf.arena = &ctx->arena;
    ovf.p = ctx->arena.alloc(4 * n_chunks);
    if (!ovf.p) {
      set_error("overflow flags do not fit the arena");
      return VX_E_NOMEM;
    }
    VX_CUDA_TRY(cudaMemsetAsync(ovf.p, 0, 4 * n_chunks, ctx->s_compute));
    P.chunk_ovf = ovf.as<unsigned int>();
  }
  ek.proto = P;

  ExecStats es;
  void *res_acc = acc.p;
  uint32_t *res_err = d_err;
  const unsigned int *res_ovf = P.chunk_ovf;
  std::shared_ptr<GraphEntry> ge;
  if (n_rows && ctx->cfg.use_graphs) {
    VX_TRY(star_graph(ctx, ek, tables, G, &ge));
    if (ge) {
      VX_CUDA_TRY(cudaGraphLaunch(ge->exec, ctx->s_compute));
      es.chunks = ge->chunks;
      es.bytes_h2d = ge->bytes_h2d;
      es.kernel_launches = ge->launches;
      res_acc = ge->acc.p;
      res_err = ge->err.as<uint32_t>();
      res_ovf = ge->ovf.p ? ge->ovf.as<unsigned int>() : nullptr;
    }
  }
  if (!ge && n_rows) VX_TRY(run_pipeline(ctx, ek, &es));
  VX_CUDA_TRY(cudaStreamSynchronize(ctx->s_compute));
  VX_TRY(check_err_word(ctx, res_err));
  uint32_t overflow_retries = 0;
  if (res_ovf) {  // chunks whose survivors outgrew the predicted list: rerun them exactly
    std::vector<unsigned int> fl(n_chunks);
    VX_CUDA_TRY(cudaMemcpy(fl.data(), res_ovf, 4 * n_chunks, cudaMemcpyDeviceToHost));
    StarExKernel rk;
    for (uint64_t c = 0; c < n_chunks; ++c)
      if (fl[c]) rk.only.push_back(c);
    if (!rk.only.empty()) {
      rk.ctx = ctx;
      rk.proto = ek.proto;
      rk.proto.g_sum = (unsigned long long *)res_acc;
      rk.proto.g_cnt = rk.proto.g_sum + G;
      rk.proto.err = res_err;
      rk.proto.chunk_ovf = nullptr;
      rk.proto.chunk_surv = nullptr;
      rk.staged_cols = ek.staged_cols;
      rk.staged_role = ek.staged_role;
      rk.row_begin = ek.row_begin;
      rk.n_rows = ek.n_rows;
      rk.chunk_rows = ek.chunk_rows;
      rk.smem = ek.smem;
      rk.smem_bytes = ek.smem_bytes;
      rk.switchable = ek.switchable;
      rk.chunk_late = ek.chunk_late;
      rk.any_late = ek.any_late;
      rk.surv_rows = 0;  // worst case: every row of the chunk
      ExecStats er;
      VX_TRY(run_pipeline(ctx, rk, &er));
      VX_CUDA_TRY(cudaStreamSynchronize(ctx->s_compute));
      VX_TRY(check_err_word(ctx, res_err));
      es.bytes_h2d += er.bytes_h2d;
      overflow_retries = (uint32_t)rk.only.size();
      ek.launches += rk.launches;
    }
  }
  if (ge) {  // the replay's fused-kernel and gather times, from its event nodes
    for (size_t c = 0; c < ge->ev_a.size(); ++c) {
      float ms = 0;
      if (cudaEventElapsedTime(&ms, ge->ev_a[c], ge->ev_b[c]) == cudaSuccess) {
        ek.ms_main += ms;
        ek.main_launches += 1;
      }
      if (ge->split[c] && cudaEventElapsedTime(&ms, ge->ev_b[c], ge->ev_c[c]) == cudaSuccess) ek.ms_gather += ms;
    }
    cudaGetLastError();
  }
  if (want_log && n_chunks && !ge) {  // statistics log: features and the exact survivor fraction per chunk
    std::vector<unsigned long long> sv(n_chunks);
    VX_CUDA_TRY(cudaMemcpy(sv.data(), P.chunk_surv, 8 * n_chunks, cudaMemcpyDeviceToHost));
    for (uint64_t c = 0; c < n_chunks; ++c) {
      const uint64_t rows_c = std::min(cr, n_rows - c * cr);
      ctx->chunk_log_x.insert(ctx->chunk_log_x.end(), feats.begin() + c * kChunkFeatures,
                              feats.begin() + (c + 1) * kChunkFeatures);
      ctx->chunk_log_y.push_back((float)((double)sv[c] / (double)rows_c));
    }
  }

  // ---- results: non-empty groups in ascending id
  std::vector<uint64_t> h(2 * G);
  VX_CUDA_TRY(cudaMemcpy(h.data(), res_acc, 16 * G, cudaMemcpyDeviceToHost));
  uint64_t n_out = 0, surv = 0;
  vx_status st = VX_OK;
  for (uint64_t g = 0; g < G; ++g) {
    uint64_t c = h[G + g];
    if (!c) continue;
    surv += c;
    if (n_out < out->cap) {
      if (out->gid) out->gid[n_out] = g;
      if (out->sum) out->sum[n_out] = (int64_t)h[g];
      if (out->cnt) out->cnt[n_out] = c;
    }
    ++n_out;
  }
  out->n_out = n_out;
  if (n_out > out->cap) {
    set_error("result has %llu groups; capacity %llu", (unsigned long long)n_out, (unsigned long long)out->cap);
    st = VX_E_CAPACITY;
  }
  qs.rows = n_rows;
  qs.survivors = surv;
  qs.chunks = es.chunks;
  qs.bytes_h2d = es.bytes_h2d;
  qs.bytes_d2h = es.bytes_d2h + 16 * G;
  qs.late_mask = late_mask | (late_chunks ? switch_mask : 0);
  qs.bytes_zero_copy = surv * 64ull * (uint64_t)__builtin_popcount(late_mask);
  if (late_chunks) {  // survivors of late chunks, estimated from the per-chunk sample
    double zs = 0;
    for (uint64_t c = 0; c < n_chunks; ++c)
      if (ek.chunk_late[c]) zs += feats[c * kChunkFeatures + 2] * (double)std::min(cr, n_rows - c * cr);
    qs.bytes_zero_copy += (uint64_t)(zs * 64.0 * __builtin_popcount(switch_mask));
  }
  qs.late_chunks = late_chunks;
  qs.overflow_retries = overflow_retries;
  qs.surv_list_bytes = ek.any_late ? ek.surv_region() * 8 : 0;
  qs.bytes_logical = n_rows * 4ull * role_col.size();
  qs.ms_kernel = ek.main_launches ? ek.ms_main : es.ms_kernel;  // the fused kernel's own time when timed
  qs.ms_gather = ek.ms_gather;
  qs.ms_features = ms_features;
  qs.kernel_launches = ge ? es.kernel_launches : ek.launches;
  qs.ms_total = now_ms() - t_start;
  out->stats = qs;
  ctx->last = qs;
  return st;
}

// ------------------------------------------------------------------ filter ExKernel
struct FilterExKernel : ExKernel {
  vx_ctx *ctx;
  FilterParams proto{};
  std::vector<const Column *> cols;
  uint64_t row_begin = 0, n_rows = 0, chunk_rows = 0;
  uint64_t *out_rows = nullptr, cap = 0, written = 0, total = 0;
  int S = 2;

  uint64_t size() override { return (n_rows + chunk_rows - 1) / chunk_rows; }
  uint64_t in_bytes() const { return cols.size() * ((chunk_rows * 4 + 255) & ~255ull); }
  uint64_t n_tiles() const { return (chunk_rows + kFilterTile - 1) / kFilterTile; }
  uint64_t tile_bytes() const { return ((n_tiles() * 4 + 255) & ~255ull); }
  uint64_t slot_bytes() override { return in_bytes() + 2 * tile_bytes() + chunk_rows * 8; }
  uint64_t rows_of(uint64_t it) const { return std::min(chunk_rows, n_rows - it * chunk_rows); }
  void inputs(uint64_t it, char *slot, std::vector<CopyOp> &h2d) override {
    const uint64_t r0 = row_begin + it * chunk_rows, n = rows_of(it);
    for (size_t k = 0; k < cols.size(); ++k)
      h2d.push_back({(const char *)cols[k]->host + r0 * 4, slot + k * ((chunk_rows * 4 + 255) & ~255ull), n * 4});
  }
  vx_status kernel(char *slot, uint64_t it, cudaStream_t s) override {
    FilterParams p = proto;
    p.row0 = row_begin + it * chunk_rows;
    p.n = rows_of(it);
    for (int q = 0; q < p.n_preds; ++q)
      p.col[q] = (const int32_t *)(slot + (uint64_t)p.colidx[q] * ((chunk_rows * 4 + 255) & ~255ull));
    uint32_t *tcnt = (uint32_t *)(slot + in_bytes());
    uint32_t *toff = (uint32_t *)(slot + in_bytes() + tile_bytes());
    uint64_t *outb = (uint64_t *)(slot + in_bytes() + 2 * tile_bytes());
    uint32_t nt = (uint32_t)((p.n + kFilterTile - 1) / kFilterTile);
    filter_count_kernel<<<nt, kFilterThreads, 0, s>>>(p, tcnt);
    filter_scan_kernel<<<1, 1024, 0, s>>>(tcnt, nt, toff, ctx->d_scalars + 8 + (it % S));
    filter_write_kernel<<<nt, kFilterThreads, 0, s>>>(p, toff, outb);
    VX_CUDA_TRY(cudaGetLastError());
    return VX_OK;
  }
  bool has_outputs() override { return true; }
  vx_status outputs(uint64_t it, char *slot, std::vector<CopyOp> &d2h) override {
    uint64_t c = ((volatile uint64_t *)ctx->h_scalars)[8 + (it % S)];
    uint64_t *outb = (uint64_t *)(slot + in_bytes() + 2 * tile_bytes());
    uint64_t fit = written < cap ? std::min(c, cap - written) : 0;
    if (fit && out_rows) d2h.push_back({outb, out_rows + written, fit * 8});
    written += fit;
    total += c;
    return VX_OK;
  }
};

}  // namespace vx

using namespace vx;

namespace vx {
// Frees captured graphs and the resident dimension tables that nothing else
// references (the cache holds the only reference); returns whether anything
// was freed.  Callers retry an allocation that failed.
bool evict_unused_resident(vx_ctx *ctx) {
  bool freed = !ctx->graphs.empty();
  cudaStreamSynchronize(ctx->s_compute);
  ctx->graphs.clear();
  for (auto it = ctx->resident.begin(); it != ctx->resident.end();) {
    if (it->second.use_count() == 1) {
      it = ctx->resident.erase(it);
      freed = true;
    } else {
      ++it;
    }
  }
  return freed;
}
}  // namespace vx

VX_API vx_status vx_run_plan(vx_ctx *ctx, const vx_plan *plan, vx_result *out) {
  clear_error();
  VX_TRY(check_ctx(ctx));
  std::lock_guard<std::recursive_mutex> g(ctx->mu);
  vx_status st = run_star(ctx, plan, out, true);
  if (st == VX_E_NOMEM && evict_unused_resident(ctx)) {  // device budget: make room, once
    clear_error();
    st = run_star(ctx, plan, out, true);
  }
  return st;
}

static vx_status regressor_fit(vx_ctx *ctx, const float *X, const float *y, uint64_t n, int32_t d, float lambda,
                               float *w_out) {
  if (!X || !y || !w_out || n == 0 || d < 1 || d > 8 || !(lambda >= 0.f)) {
    set_error("regressor fit: need n > 0 rows, 1 <= d <= 8 features, lambda >= 0");
    return VX_E_INVAL;
  }
  DevBuf b;
  b.arena = &ctx->arena;
  const uint64_t xb = (4 * n * d + 255) & ~255ull, yb = (4 * n + 255) & ~255ull;
  b.p = ctx->arena.alloc(xb + yb + 8 * 80 + 256);
  if (!b.p) {
    set_error("regressor fit: %llu rows do not fit the arena", (unsigned long long)n);
    return VX_E_NOMEM;
  }
  float *dX = b.as<float>();
  float *dy = (float *)(b.as<char>() + xb);
  double *acc = (double *)(b.as<char>() + xb + yb);
  float *dw = (float *)(acc + 72);
  uint32_t *derr = (uint32_t *)(dw + 8);
  cudaStream_t s = ctx->s_compute;
  VX_CUDA_TRY(cudaMemcpyAsync(dX, X, 4 * n * d, cudaMemcpyHostToDevice, s));
  VX_CUDA_TRY(cudaMemcpyAsync(dy, y, 4 * n, cudaMemcpyHostToDevice, s));
  VX_CUDA_TRY(cudaMemsetAsync(acc, 0, 8 * 72, s));
  const int grid = (int)std::max<uint64_t>(1, std::min<uint64_t>((n + 255) / 256, (uint64_t)ctx->num_sms * 4));
  ridge_accumulate_kernel<<<grid, 256, 0, s>>>(dX, dy, n, d, acc);
  ridge_solve_kernel<<<1, 32, 0, s>>>(acc, d, (double)lambda, dw, derr);
  VX_CUDA_TRY(cudaGetLastError());
  uint32_t err = 0;
  VX_CUDA_TRY(cudaMemcpyAsync(w_out, dw, 4 * d, cudaMemcpyDeviceToHost, s));
  VX_CUDA_TRY(cudaMemcpyAsync(&err, derr, 4, cudaMemcpyDeviceToHost, s));
  VX_CUDA_TRY(cudaStreamSynchronize(s));
  if (err) {
    set_error("regressor fit: normal equations are singular (add lambda > 0)");
    return VX_E_INVAL;
  }
  return VX_OK;
}

VX_API vx_status vx_regressor_fit(vx_ctx *ctx, const float *X, const float *y, uint64_t n, int32_t d, float lambda,
                                  float *w_out) {
  clear_error();
  VX_TRY(check_ctx(ctx));
  std::lock_guard<std::recursive_mutex> g(ctx->mu);
  return regressor_fit(ctx, X, y, n, d, lambda, w_out);
}

VX_API vx_status vx_regressor_train(vx_ctx *ctx, float lambda, float *w_out, uint64_t *n_used) {
  clear_error();
  VX_TRY(check_ctx(ctx));
  std::lock_guard<std::recursive_mutex> g(ctx->mu);
  const uint64_t n = ctx->chunk_log_y.size();
  if (n_used) *n_used = n;
  if (n < (uint64_t)kChunkFeatures) {
    set_error("vx_regressor_train: %llu logged chunks; at least %d needed", (unsigned long long)n, kChunkFeatures);
    return VX_E_INVAL;
  }
  float w[kChunkFeatures];
  VX_TRY(regressor_fit(ctx, ctx->chunk_log_x.data(), ctx->chunk_log_y.data(), n, kChunkFeatures, lambda, w));
  for (int k = 0; k < kChunkFeatures; ++k) ctx->reg_w[k] = w[k];
  ctx->reg_trained = true;
  if (w_out) memcpy(w_out, w, sizeof w);
  return VX_OK;
}

VX_API vx_status vx_regressor_set(vx_ctx *ctx, const float *w, int32_t d) {
  clear_error();
  VX_TRY(check_ctx(ctx));
  if (!w || d != kChunkFeatures) {
    set_error("vx_regressor_set: %d weights expected", kChunkFeatures);
    return VX_E_INVAL;
  }
  std::lock_guard<std::recursive_mutex> g(ctx->mu);
  for (int k = 0; k < kChunkFeatures; ++k) ctx->reg_w[k] = w[k];
  ctx->reg_trained = true;
  return VX_OK;
}

VX_API vx_status vx_chunk_log(vx_ctx *ctx, float *X, float *y, uint64_t cap, uint64_t *n) {
  clear_error();
  if (!ctx || !n) return VX_E_INVAL;
  std::lock_guard<std::recursive_mutex> g(ctx->mu);
  const uint64_t m = ctx->chunk_log_y.size();
  *n = m;
  const uint64_t k = std::min(m, cap);
  if (X && k) memcpy(X, ctx->chunk_log_x.data(), 4 * k * kChunkFeatures);
  if (y && k) memcpy(y, ctx->chunk_log_y.data(), 4 * k);
  return m > cap && (X || y) ? VX_E_CAPACITY : VX_OK;
}

VX_API vx_status vx_chunk_log_clear(vx_ctx *ctx) {
  if (!ctx) return VX_E_INVAL;
  std::lock_guard<std::recursive_mutex> g(ctx->mu);
  ctx->chunk_log_x.clear();
  ctx->chunk_log_y.clear();
  ctx->reg_trained = false;
  return VX_OK;
}

VX_API vx_status vx_autotune(vx_ctx *ctx, const vx_plan *plan, uint64_t sample_rows, vx_config *best) {
  clear_error();
  VX_TRY(check_ctx(ctx));
  if (!plan || !best || sample_rows == 0) {
    set_error("vx_autotune: need a plan, an output and sample_rows > 0");
    return VX_E_INVAL;
  }
  std::lock_guard<std::recursive_mutex> g(ctx->mu);
  const vx_config base = ctx->cfg;
  vx_plan p = *plan;
  p.row_end = p.row_begin + sample_rows;
  const uint64_t chunks_mb[] = {8, 16, 32, 64, 128, 256};
  const int slots[] = {2, 3, 4};
  double best_ms = 1e300, best_kms = 1e300;
  vx_config best_cfg = base;
  // a candidate wins when it is more than 1 % faster, or within 1 % (a tie on
  // a link-bound query) with less fused-kernel time, which leaves the device
  // more headroom under the same link
  auto better = [&](double ms, double kms) {
    return ms < 0.99 * best_ms || (ms <= 1.01 * best_ms && kms < best_kms);
  };
  for (uint64_t mb : chunks_mb) {
    for (int S : slots) {
      vx_config c = base;
      c.chunk_bytes = mb << 20;
      c.n_slots = S;
      if ((uint64_t)S * c.chunk_bytes * 2 > ctx->arena.capacity()) continue;
      ctx->cfg = c;
      ctx->graphs.clear();
      double ms = 1e300, kms = 1e300;
      for (int rep = 0; rep < 3; ++rep) {  // first run warms tables and graphs
        vx_result r{};
        r.cap = UINT64_MAX;
        vx_status st = run_star(ctx, &p, &r, true);
        if (st != VX_OK) {
          ms = 1e300;
          break;
        }
        if (rep > 0) {
          ms = std::min(ms, r.stats.ms_total);
          kms = std::min(kms, r.stats.ms_kernel);
        }
      }
      if (ms < 1e300 && better(ms, kms)) {
        best_ms = ms;
        best_kms = kms;
        best_cfg = c;
      }
    }
  }
  // launch shape of the fused kernel at the best chunking: one tile per block,
  // the bulk-copy pipeline at 4 or 6 blocks per SM (a ring of 3 or 2 stages),
  // and the scalar kernel at 8 or 16 rows per thread and 4 or 8 resident
  // blocks per SM
  const int shapes[7][2] = {{0, 0}, {2, 4}, {2, 6}, {8, 4}, {8, 8}, {16, 4}, {16, 8}};
  const vx_config chunked = best_cfg;
  for (const auto &sh : shapes) {
    vx_config c = chunked;
    c.kernel_rows = sh[0];
    if (sh[1]) c.blocks_per_sm = sh[1];
    if (c.kernel_rows == chunked.kernel_rows && c.blocks_per_sm == chunked.blocks_per_sm) continue;
    ctx->cfg = c;
    ctx->graphs.clear();
    double ms = 1e300, kms = 1e300;
    for (int rep = 0; rep < 3; ++rep) {
      vx_result r{};
      r.cap = UINT64_MAX;
      if (run_star(ctx, &p, &r, true) != VX_OK) {
        ms = 1e300;
        break;
      }
      if (rep > 0) {
        ms = std::min(ms, r.stats.ms_total);
        kms = std::min(kms, r.stats.ms_kernel);
      }
    }
    if (ms < 1e300 && better(ms, kms)) {
      best_ms = ms;
      best_kms = kms;
      best_cfg = c;
    }
  }
  // host-to-device staging at that chunking and shape: the copy engine
  // against a copy kernel of 32 blocks.  On some hosts the copy engine's rate
  // drops (measured: 116-156 GB/s on a host where a copy kernel staged at
  // 183-191); where it holds, it ties or wins (the copy kernel takes SMs from
  // the fused kernel) and a tie keeps it, its fused-kernel time being lower.
  if (ctx->host_ptr_ok) {
    vx_config c = best_cfg;
    c.h2d_copy_blocks = best_cfg.h2d_copy_blocks ? 0 : 32;
    ctx->cfg = c;
    ctx->graphs.clear();
    double ms = 1e300, kms = 1e300;
    for (int rep = 0; rep < 3; ++rep) {
      vx_result r{};
      r.cap = UINT64_MAX;
      if (run_star(ctx, &p, &r, true) != VX_OK) {
        ms = 1e300;
        break;
      }
      if (rep > 0) {
        ms = std::min(ms, r.stats.ms_total);
        kms = std::min(kms, r.stats.ms_kernel);
      }
    }
    if (ms < 1e300 && better(ms, kms)) {
      best_ms = ms;
      best_kms = kms;
      best_cfg = c;
    }
  }
  ctx->graphs.clear();
  ctx->cfg = best_cfg;
  *best = best_cfg;
  if (best_ms >= 1e300) {
    set_error("vx_autotune: no candidate configuration ran");
    ctx->cfg = base;
    return VX_E_NOMEM;
  }
  return VX_OK;
}

VX_API vx_status vx_groupby(vx_ctx *ctx, const vx_plan_gkey *keys, int32_t n_keys, int32_t agg_op, int32_t agg_a,
                            int32_t agg_b, const vx_pred *preds, int32_t n_preds, vx_result *out) {
  clear_error();
  VX_TRY(check_ctx(ctx));
  if (n_keys < 0 || n_keys > VX_MAX_GKEYS || n_preds < 0 || n_preds > VX_MAX_PREDS || (n_keys && !keys) ||
      (n_preds && !preds)) {
    set_error("vx_groupby: bad argument");
    return VX_E_INVAL;
  }
  vx_plan p{};
  p.n_dims = 0;
  p.n_fact_preds = n_preds;
  for (int i = 0; i < n_preds; ++i) p.fact_preds[i] = preds[i];
  p.n_group_keys = n_keys;
  for (int i = 0; i < n_keys; ++i) {
    p.group_keys[i] = keys[i];
    if (keys[i].dim != -1) {
      set_error("vx_groupby: keys must be fact columns (dim = -1)");
      return VX_E_INVAL;
    }
  }
  p.agg_op = agg_op;
  p.agg_a = agg_a;
  p.agg_b = agg_b;
  p.late_mat = VX_LATE_FORCE_EARLY;
  std::lock_guard<std::recursive_mutex> g(ctx->mu);
  return run_star(ctx, &p, out, false);
}

VX_API vx_status vx_filter(vx_ctx *ctx, const vx_pred *preds, int32_t n_preds, uint64_t row_begin, uint64_t row_end,
                           uint64_t *out_rows, uint64_t cap, uint64_t *out_count) {
  clear_error();
  VX_TRY(check_ctx(ctx));
  if (n_preds < 1 || n_preds > VX_MAX_PREDS || !preds || !out_count) {
    set_error("vx_filter: need 1..%d predicates and out_count", VX_MAX_PREDS);
    return VX_E_INVAL;
  }
  std::lock_guard<std::recursive_mutex> g(ctx->mu);
  const double t0 = now_ms();
  FilterExKernel fk;
  fk.ctx = ctx;
  uint64_t n = UINT64_MAX;
  for (int q = 0; q < n_preds; ++q) {
    const Column *c = get_col(ctx, preds[q].col, VX_I32);
    if (!c) return VX_E_INVAL;
    if (n == UINT64_MAX) n = c->n_rows;
    if (c->n_rows != n || preds[q].op < VX_BETWEEN || preds[q].op > VX_GE) {
      set_error("vx_filter: columns differ in length or bad op");
      return VX_E_INVAL;
    }
    int k = -1;
    for (size_t j = 0; j < fk.cols.size(); ++j)
      if (fk.cols[j] == c) k = (int)j;
    if (k < 0) {
      fk.cols.push_back(c);
      k = (int)fk.cols.size() - 1;
    }
    fk.proto.op[q] = preds[q].op;
    fk.proto.lo[q] = preds[q].lo;
    fk.proto.hi[q] = preds[q].hi;
    fk.proto.colidx[q] = k;
  }
  fk.proto.n_preds = n_preds;
  const uint64_t rb = std::min(row_begin, n);
  const uint64_t re = row_end == 0 ? n : std::min(row_end, n);
  fk.row_begin = rb;
  fk.n_rows = re > rb ? re - rb : 0;
  uint64_t cr = ctx->cfg.chunk_bytes / (4 * fk.cols.size());
  cr = std::max<uint64_t>(cr / kFilterTile * kFilterTile, kFilterTile);
  cr = std::min<uint64_t>(cr, (uint64_t)kFilterTile * 65535);
  fk.chunk_rows = cr;
  fk.out_rows = out_rows;
  fk.cap = out_rows ? cap : 0;
  fk.S = ctx->cfg.n_slots;
  HostReg out_reg;  // the per-chunk stores of row ids then run asynchronously
  if (out_rows && cap) VX_TRY(out_reg.add(out_rows, 8 * cap));
  ExecStats es;
  if (fk.n_rows) VX_TRY(run_pipeline(ctx, fk, &es));
  *out_count = fk.total;
  vx_query_stats qs{};
  qs.rows = fk.n_rows;
  qs.survivors = fk.total;
  qs.chunks = es.chunks;
  qs.bytes_h2d = es.bytes_h2d;
  qs.bytes_d2h = es.bytes_d2h;
  qs.bytes_logical = fk.n_rows * 4 * fk.cols.size();
  qs.ms_kernel = es.ms_kernel;
  qs.kernel_launches = es.kernel_launches * 3;
  qs.ms_total = now_ms() - t0;
  ctx->last = qs;
  if (out_rows && fk.total > cap) {
    set_error("vx_filter: %llu rows qualify; capacity %llu", (unsigned long long)fk.total, (unsigned long long)cap);
    return VX_E_CAPACITY;
  }
  return VX_OK;
}
