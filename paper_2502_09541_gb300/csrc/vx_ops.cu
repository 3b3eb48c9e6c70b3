// Operator-at-a-time execution of a star plan with host intermediates (the
// paper's Section 6.4 discussion: chaining operators extended with the IO
// decoupling instead of one fused kernel, with CPU memory holding the
// intermediate results).
//
// The plan is resolved by the star planner (dimension tables built and kept
// on the device, accumulators zeroed).  Then each operator is its own
// pipelined ExKernel over the fact chunks:
//   filter     - fact predicates (and fact group keys) of every row of the
//                chunk; survivors (chunk-local row, partial group code) are
//                stored to a host intermediate;
//   probe d    - per dimension in plan order: the intermediate's entries of
//                the chunk are loaded, the foreign key of each is looked up,
//                hits (with the dimension's code added) are stored to the next
//                intermediate;
//   aggregate  - the last intermediate's entries accumulate agg(a, b) into the
//                group sums and counts.
// An operator reads the fact columns it needs either as the chunk's column
// slice copied by the copy engine or, when its input is sparse (entries /
// rows below TH, Section 6.3), through mapped host memory for its entries
// only.  Entries inside an intermediate are in no particular order; the
// aggregate is a sum, so the result is exact and equal to the fused plan's.
#include <algorithm>
#include <cmath>

#include "vx_internal.h"
#include "vx_probe.cuh"
#include "vx_star.cuh"

namespace vx {

namespace {

enum { kOpFilter = 0, kOpProbe = 1, kOpAggregate = 2 };
constexpr int kOpThreads = 256, kOpItems = 8, kOpTile = kOpThreads * kOpItems;

struct OpStage {
  int kind, d;
  const uint32_t *in_rows, *in_g;  // input entries (probe, aggregate)
  uint64_t m;                      // entries (filter: rows of the chunk)
  uint32_t *out_rows, *out_g;      // output entries (filter, probe)
  unsigned int *out_cnt;
  bool smem_acc;                   // aggregate: groups accumulated in shared memory first
};

__global__ void __launch_bounds__(kOpThreads) op_stage_kernel(const ChunkParams p, const OpStage s) {
  extern __shared__ unsigned long long oacc[];  // aggregate with smem_acc: [2 * n_groups]
  __shared__ uint32_t tr[kOpTile], tg[kOpTile];
  __shared__ unsigned int tn, tbase;
  if (s.smem_acc)
    for (uint32_t g = threadIdx.x; g < 2 * p.n_groups; g += blockDim.x) oacc[g] = 0;
  if (threadIdx.x == 0) tn = 0;
  __syncthreads();
  for (uint64_t t0 = (uint64_t)blockIdx.x * kOpTile; t0 < s.m; t0 += (uint64_t)gridDim.x * kOpTile) {
#pragma unroll 2
    for (int j = 0; j < kOpItems; ++j) {
      const uint64_t e = t0 + (uint64_t)j * kOpThreads + threadIdx.x;
      if (e >= s.m) continue;
      const uint32_t row = s.kind == kOpFilter ? (uint32_t)e : s.in_rows[e];
      uint32_t g = s.kind == kOpFilter ? 0u : s.in_g[e];
      bool keep = true;
      if (s.kind == kOpFilter) {
        for (int q = 0; q < p.n_fact_preds && keep; ++q)
          keep = pred_in(pred_range(p.fp_op[q], p.fp_lo[q], p.fp_hi[q]), load_role(p, p.fp_role[q], row));
        for (int k = 0; k < p.n_fgk && keep; ++k) {
          const int32_t code = load_role(p, p.fgk_role[k], row);
          if (code < 0 || code >= p.fgk_card[k]) {
            atomicOr(p.err, ERR_RANGE);
            keep = false;
          } else {
            g += (uint32_t)code * p.fgk_stride[k];
          }
        }
      } else if (s.kind == kOpProbe) {
        uint32_t v = 0;
        keep = dim_lookup(p, s.d, load_role(p, p.dim_role[s.d], row), v);
        g += keep ? v : 0u;
      } else {
        const int64_t a = p.agg_a_role >= 0 ? load_role(p, p.agg_a_role, row) : 0;
        const int64_t b = p.agg_b_role >= 0 ? load_role(p, p.agg_b_role, row) : 0;
        const int64_t v = p.agg_op == VX_AGG_SUM ? a : p.agg_op == VX_AGG_MUL ? a * b : p.agg_op == VX_AGG_SUB ? a - b : 0;
        if (s.smem_acc) {
          atomicAdd(&oacc[g], (unsigned long long)v);
          atomicAdd(&oacc[p.n_groups + g], 1ull);
        } else {
          atomicAdd(&p.g_sum[g], (unsigned long long)v);
          atomicAdd(&p.g_cnt[g], 1ull);
        }
        keep = false;
      }
      if (keep) {
        const unsigned int k = atomicAdd(&tn, 1u);
        tr[k] = row;
        tg[k] = g;
      }
    }
    __syncthreads();
    const unsigned int n = tn;
    if (n) {
      if (threadIdx.x == 0) tbase = atomicAdd(s.out_cnt, n);
      __syncthreads();
      for (unsigned int k = threadIdx.x; k < n; k += blockDim.x) {
        s.out_rows[tbase + k] = tr[k];
        s.out_g[tbase + k] = tg[k];
      }
      __syncthreads();
      if (threadIdx.x == 0) tn = 0;
    }
    __syncthreads();
  }
  if (s.smem_acc) {
    for (uint32_t q = threadIdx.x; q < p.n_groups; q += blockDim.x)
      if (oacc[p.n_groups + q]) {
        atomicAdd(&p.g_sum[q], oacc[q]);
        atomicAdd(&p.g_cnt[q], oacc[p.n_groups + q]);
      }
  }
}

__global__ void op_publish_kernel(const unsigned int *cnt, uint64_t *host_word) { *host_word = *cnt; }

// one operator over all fact chunks
struct OpPass : ExKernel {
  vx_ctx *ctx;
  ChunkParams P;
  int kind = kOpFilter, d = 0, S = 3;
  std::vector<int> roles;               // fact roles the operator reads
  std::vector<const Column *> role_cols;
  uint64_t row_begin = 0, n_rows = 0, R = 0;
  double TH = 0;
  const uint32_t *in_rows = nullptr, *in_g = nullptr;  // host intermediate in: chunk c at c * R
  const uint64_t *in_cnt = nullptr;
  uint32_t *out_rows = nullptr, *out_g = nullptr;      // host intermediate out
  uint64_t *out_cnt = nullptr;
  uint64_t zc_values = 0, entries = 0;
  int grid = 1;

  uint64_t size() override { return n_rows ? (n_rows + R - 1) / R : 0; }
  int n_slots() override { return S; }
  uint64_t rows(uint64_t c) const { return std::min(R, n_rows - c * R); }
  uint64_t m(uint64_t c) const { return kind == kOpFilter ? rows(c) : in_cnt[c]; }
  bool dense(uint64_t c) const { return kind == kOpFilter || (double)m(c) >= TH * (double)rows(c); }
  uint64_t eb() const { return (4 * R + 255) & ~255ull; }
  uint64_t slot_bytes() override { return (4 + roles.size()) * eb() + 256; }
  char *in_r(char *slot) const { return slot; }
  char *in_gp(char *slot) const { return slot + eb(); }
  char *col(char *slot, size_t k) const { return slot + (2 + k) * eb(); }
  char *out_r(char *slot) const { return slot + (2 + roles.size()) * eb(); }
  char *out_gp(char *slot) const { return slot + (3 + roles.size()) * eb(); }
  unsigned int *cnt(char *slot) const { return (unsigned int *)(slot + (4 + roles.size()) * eb()); }
  void inputs(uint64_t c, char *slot, std::vector<CopyOp> &h2d) override {
    const uint64_t e = m(c);
    if (kind != kOpFilter && e) {
      h2d.push_back({in_rows + c * R, in_r(slot), 4 * e});
      h2d.push_back({in_g + c * R, in_gp(slot), 4 * e});
    }
    if (e && dense(c))
      for (size_t k = 0; k < roles.size(); ++k)
        h2d.push_back({(const char *)role_cols[k]->host + 4 * (row_begin + c * R), col(slot, k), 4 * rows(c)});
  }
  vx_status kernel(char *slot, uint64_t c, cudaStream_t s) override {
    ChunkParams p = P;
    p.row0 = row_begin + c * R;
    p.n = rows(c);
    const bool dn = dense(c);
    for (size_t k = 0; k < roles.size(); ++k) p.staged[roles[k]] = dn ? (const int32_t *)col(slot, k) : nullptr;
    OpStage st{};
    st.kind = kind;
    st.d = d;
    st.in_rows = (const uint32_t *)in_r(slot);
    st.in_g = (const uint32_t *)in_gp(slot);
    st.m = m(c);
    st.out_rows = (uint32_t *)out_r(slot);
    st.out_g = (uint32_t *)out_gp(slot);
    st.out_cnt = cnt(slot);
    st.smem_acc = kind == kOpAggregate && P.n_groups <= kSmemGroups;
    entries += st.m;
    if (!dn) zc_values += st.m * roles.size();
    VX_CUDA_TRY(cudaMemsetAsync(st.out_cnt, 0, 4, s));
    if (st.m) {
      const uint64_t tiles = (st.m + kOpTile - 1) / kOpTile;
      const size_t smem = st.smem_acc ? 16ull * P.n_groups : 0;
      op_stage_kernel<<<(unsigned)std::min<uint64_t>(tiles, (uint64_t)grid), kOpThreads, smem, s>>>(p, st);
      VX_CUDA_TRY(cudaGetLastError());
    }
    if (kind != kOpAggregate) {
      op_publish_kernel<<<1, 1, 0, s>>>(st.out_cnt, ctx->d_scalars + 64 + (c % S));
      VX_CUDA_TRY(cudaGetLastError());
    }
    return VX_OK;
  }
  bool has_outputs() override { return kind != kOpAggregate; }
  vx_status outputs(uint64_t c, char *slot, std::vector<CopyOp> &d2h) override {
    const uint64_t n = ((volatile uint64_t *)ctx->h_scalars)[64 + (c % S)];
    out_cnt[c] = n;
    if (n) {
      d2h.push_back({out_r(slot), out_rows + c * R, 4 * n});
      d2h.push_back({out_gp(slot), out_g + c * R, 4 * n});
    }
    return VX_OK;
  }
};

}  // namespace

vx_status run_star_operators(vx_ctx *ctx, const vx_plan *plan, vx_result *out) {
  const double t0 = now_ms();
  if (!out) {
    set_error("vx_run_plan_operators: null result");
    return VX_E_INVAL;
  }
  PreparedStar prep;
  VX_TRY(run_star(ctx, plan, nullptr, true, &prep));
  ChunkParams P = prep.P;
  for (size_t r = 0; r < prep.role_col.size(); ++r) {
    P.staged[r] = nullptr;
    P.zc[r] = (const int32_t *)ctx->cols[prep.role_col[r]].dev;
  }
  const uint64_t n_rows = prep.n_rows, G = prep.G;
  // fact chunk: chunk_bytes over the widest operator's columns, rows a multiple of 1024 below 2^32
  size_t widest = 1;
  widest = std::max<size_t>(widest, (size_t)P.n_fact_preds + P.n_fgk);
  widest = std::max<size_t>(widest, 2);
  uint64_t R = ctx->cfg.chunk_bytes / (4 * (widest + 4));
  R = std::max<uint64_t>(1024, std::min<uint64_t>(R, 1ull << 31) / 1024 * 1024);
  const uint64_t n_chunks = n_rows ? (n_rows + R - 1) / R : 0;
  const int S = std::max(2, ctx->cfg.n_slots);
  const double TH = ctx->cfg.zc_threshold > 0 ? ctx->cfg.zc_threshold : kDefaultZeroCopyTH;

  // host intermediates: two ping-pong buffers of (row, code) entries, chunk c
  // at c * R, in the context's page-locked block (grown on demand)
  const uint64_t cap = std::max<uint64_t>(n_chunks * R, 1);
  if (ctx->op_host_bytes < 16 * cap) {
    if (ctx->op_host) cudaFreeHost(ctx->op_host);
    ctx->op_host = nullptr;
    ctx->op_host_bytes = 0;
    if (cudaHostAlloc((void **)&ctx->op_host, 16 * cap, cudaHostAllocMapped) != cudaSuccess) {
      cudaGetLastError();
      ctx->op_host = nullptr;
      set_error("vx_run_plan_operators: no page-locked host memory for the %llu-entry intermediates",
                (unsigned long long)cap);
      return VX_E_NOMEM;
    }
    ctx->op_host_bytes = 16 * cap;
  }
  char *base = ctx->op_host;
  uint32_t *rows_buf[2] = {(uint32_t *)base, (uint32_t *)(base + 8 * cap)};
  uint32_t *g_buf[2] = {(uint32_t *)(base + 4 * cap), (uint32_t *)(base + 12 * cap)};
  std::vector<uint64_t> counts[2] = {std::vector<uint64_t>(n_chunks, 0), std::vector<uint64_t>(n_chunks, 0)};

  vx_query_stats qs{};
  uint64_t launches = 0;
  int cur = 0;
  // operators in order: filter, a probe per dimension, aggregate
  std::vector<std::pair<int, int>> ops{{kOpFilter, 0}};
  for (int d = 0; d < P.n_dims; ++d) ops.push_back({kOpProbe, d});
  ops.push_back({kOpAggregate, 0});
  for (size_t i = 0; i < ops.size() && n_chunks; ++i) {
    OpPass op;
    op.ctx = ctx;
    op.P = P;
    op.kind = ops[i].first;
    op.d = ops[i].second;
    op.S = S;
    op.row_begin = prep.row_begin;
    op.n_rows = n_rows;
    op.R = R;
    op.TH = TH;
    op.grid = ctx->num_sms * 8;
    auto add_role = [&](int r) {
      if (r < 0 || std::find(op.roles.begin(), op.roles.end(), r) != op.roles.end()) return;
      op.roles.push_back(r);
      op.role_cols.push_back(&ctx->cols[prep.role_col[r]]);
    };
    if (op.kind == kOpFilter) {
      for (int q = 0; q < P.n_fact_preds; ++q) add_role(P.fp_role[q]);
      for (int k = 0; k < P.n_fgk; ++k) add_role(P.fgk_role[k]);
    } else if (op.kind == kOpProbe) {
      add_role(P.dim_role[op.d]);
    } else {
      add_role(P.agg_a_role);
      add_role(P.agg_b_role);
    }
    op.in_rows = rows_buf[cur];
    op.in_g = g_buf[cur];
    op.in_cnt = counts[cur].data();
    op.out_rows = rows_buf[1 - cur];
    op.out_g = g_buf[1 - cur];
    op.out_cnt = counts[1 - cur].data();
    if (op.kind == kOpAggregate && P.n_groups <= kSmemGroups) {
      static bool attr = false;
      if (!attr) {
        VX_CUDA_TRY(cudaFuncSetAttribute(op_stage_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(16 * kSmemGroups)));
        attr = true;
      }
    }
    ExecStats es;
    VX_TRY(run_pipeline(ctx, op, &es));
    VX_CUDA_TRY(cudaStreamSynchronize(ctx->s_compute));
    qs.bytes_h2d += es.bytes_h2d;
    qs.bytes_d2h += es.bytes_d2h;
    qs.bytes_zero_copy += op.zc_values * 64;
    launches += es.kernel_launches * 3;
    if (op.kind != kOpAggregate) cur = 1 - cur;
  }
  VX_TRY(check_err_word(ctx, P.err));

  // ---- results: non-empty groups in ascending id
  std::vector<uint64_t> h(2 * G);
  VX_CUDA_TRY(cudaMemcpy(h.data(), prep.acc.p, 16 * G, cudaMemcpyDeviceToHost));
  uint64_t n_out = 0, surv = 0;
  for (uint64_t g = 0; g < G; ++g) {
    const uint64_t c = h[G + g];
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
  vx_status st = VX_OK;
  if (n_out > out->cap) {
    set_error("result has %llu groups; capacity %llu", (unsigned long long)n_out, (unsigned long long)out->cap);
    st = VX_E_CAPACITY;
  }
  qs.rows = n_rows;
  qs.survivors = surv;
  qs.chunks = n_chunks * ops.size();
  qs.bytes_d2h += 16 * G;
  qs.bytes_logical = n_rows * 4ull * prep.role_col.size();
  qs.est_selectivity = prep.est;
  qs.kernel_launches = launches;
  qs.ms_total = now_ms() - t0;
  out->stats = qs;
  ctx->last = qs;
  return st;
}

}  // namespace vx

using namespace vx;

VX_API vx_status vx_run_plan_operators(vx_ctx *ctx, const vx_plan *plan, vx_result *out) {
  clear_error();
  VX_TRY(check_ctx(ctx));
  std::lock_guard<std::recursive_mutex> g(ctx->mu);
  vx_status st = run_star_operators(ctx, plan, out);
  if (st == VX_E_NOMEM && evict_unused_resident(ctx)) {
    clear_error();
    st = run_star_operators(ctx, plan, out);
  }
  return st;
}
