// Serving: continuous batching of star queries over shared host-resident
// fact tables.
//
// An engine thread runs one shared, circular scan.  Each cycle it picks the
// next chunk (in scan order) that some attached query still needs, stages
// the union of the columns those queries read (one copy per column, shared by
// all of them) into a slot of the staging ring, and launches one persistent
// multi-query kernel whose blocks pull (query, tile) work items.  A query is
// admitted (its dimension tables found or built and kept resident, its
// accumulators allocated) as soon as it fits the device budget and a slot of
// the attached set is free; it attaches at the current chunk and completes
// after it has seen every chunk of its row range, wherever the scan started —
// requests that arrive while others run join the work already on the device.
// Results are exact aggregates, so a query's result is the same alone and in
// any mix.
#include <algorithm>
#include <condition_variable>
#include <deque>
#include <thread>

#include "vx_internal.h"
#include "vx_sort.cuh"
#include "vx_star.cuh"

namespace vx {

struct ServeQuery {
  uint64_t id = 0;
  int kind = VX_QUERY_STAR;
  vx_op_request op{};     // sort / join queries
  vx_op_result op_res{};
  vx_plan plan{};
  double t_submit = 0, t_admit = 0, t_done = 0;
  PreparedStar prep;
  uint64_t c_first = 0, c_last = 0, left = 0;
  std::vector<uint8_t> seen;
  int state = 0;  // 0 pending, 1 attached, 2 draining, 3 done
  vx_status status = VX_OK;
  std::string error;  // message of a failed query (errors are thread-local to the engine)
  int rslot = -1;  // pinned result slot
  cudaEvent_t ev_done = nullptr;
  std::vector<uint64_t> gid, cnt;
  std::vector<int64_t> sum;
  vx_query_stats stats{};
};

struct ServeEngine {
  vx_ctx *ctx = nullptr;
  vx_serve_opts opts{};
  std::thread th;
  std::mutex mu;
  std::condition_variable cv, cv_done;
  bool stop = false;
  std::deque<ServeQuery *> pending;
  std::vector<ServeQuery *> active;
  std::map<uint64_t, std::unique_ptr<ServeQuery>> all;
  uint64_t next_id = 1;
  uint64_t n_chunks = 0, cursor = 0, cycles = 0, bytes_h2d = 0, active_peak = 0, failed = 0;
  uint64_t work_rows = 0;           // query rows the multi-query kernels evaluated
  double ms_kernel = 0, ms_admit = 0;  // their device time; host time spent admitting
  double ms_cycle = 0;                 // host time spent in scan cycles (issuing chunks)
  double ms_wait = 0;                  // of which waiting for a slot's previous kernel
  double t_start = 0;
  std::vector<double> latencies;
  std::vector<double> lat_kind[3];
  // sort / join queries: their own worker thread and device budgets
  std::thread op_th;
  std::deque<ServeQuery *> op_pending;
  bool op_running = false;
  // staging ring
  int S = 3;
  uint32_t max_cols = 12, max_items = 0;
  DevBuf ring;
  uint64_t slot_bytes = 0;
  struct Slot {
    cudaEvent_t ev_in = nullptr, ev_k0 = nullptr, ev_k = nullptr;  // ev_k0..ev_k: the multi-query kernel
    bool busy = false;
    char *host = nullptr;  // pinned staging for params and items
  };
  std::vector<Slot> slots;
  cudaStream_t s_plan = nullptr;  // admission's planning work, apart from the scan's kernels
  // pinned result slots
  std::vector<uint64_t *> rbuf;
  std::vector<int> rfree;
  vx_status fatal = VX_OK;
};

static constexpr uint64_t kServeMaxGroups = 4096;

static uint64_t serve_chunk_rows(const ServeEngine &e) { return e.opts.chunk_rows; }

// offsets inside one ring slot: [params | items | next | columns...]
static uint64_t params_bytes(const ServeEngine &e) { return ((uint64_t)e.opts.max_active * sizeof(ChunkParams) + 255) & ~255ull; }
static uint64_t items_bytes(const ServeEngine &e) { return ((uint64_t)e.max_items * sizeof(MultiItem) + 255) & ~255ull; }
static uint64_t col_bytes(const ServeEngine &e) { return (serve_chunk_rows(e) * 4 + 255) & ~255ull; }

static void finalize(ServeEngine &e, ServeQuery *q) {
  const uint64_t G = q->prep.G;
  const uint64_t *h = e.rbuf[q->rslot];
  for (uint64_t g = 0; g < G; ++g) {
    if (!h[G + g]) continue;
    q->gid.push_back(g);
    q->sum.push_back((int64_t)h[g]);
    q->cnt.push_back(h[G + g]);
    q->stats.survivors += h[G + g];
  }
  q->t_done = now_ms();
  q->stats.ms_total = q->t_done - q->t_submit;
  e.rfree.push_back(q->rslot);
  q->rslot = -1;
  q->prep = PreparedStar();  // releases accumulators; tables stay resident in the context
  if (q->ev_done) cudaEventDestroy(q->ev_done);
  q->ev_done = nullptr;
  q->state = 3;
  e.latencies.push_back(q->stats.ms_total);
  e.lat_kind[VX_QUERY_STAR].push_back(q->stats.ms_total);
}

static void fail(ServeEngine &e, ServeQuery *q, vx_status st) {
  q->status = st;
  q->error = vx_last_error();
  q->t_done = now_ms();
  q->stats.ms_total = q->t_done - q->t_submit;
  if (q->rslot >= 0) e.rfree.push_back(q->rslot);
  q->rslot = -1;
  q->prep = PreparedStar();
  q->state = 3;
  e.failed += 1;
}

// plans pending queries while result slots and device memory allow (FIFO)
static void admit(ServeEngine &e) {
  while (!e.pending.empty() && e.active.size() < e.opts.max_active && !e.rfree.empty()) {
    ServeQuery *q = e.pending.front();
    vx_status st;
    const double t_adm = now_ms();
    {
      std::lock_guard<std::recursive_mutex> g(e.ctx->mu);
      // planning (sampling, dimension builds, accumulator set-up) runs and
      // synchronises on its own stream, so it does not wait for the scan
      // kernels queued on the compute stream; it ends synchronised, before
      // the query attaches
      std::swap(e.ctx->s_compute, e.s_plan);
      st = run_star(e.ctx, &q->plan, nullptr, true, &q->prep);
      if (st == VX_E_NOMEM && evict_unused_resident(e.ctx)) {  // tables of finished queries make room
        q->prep = PreparedStar();
        st = run_star(e.ctx, &q->plan, nullptr, true, &q->prep);
      }
      cudaStreamSynchronize(e.ctx->s_compute);
      std::swap(e.ctx->s_compute, e.s_plan);
    }
    e.ms_admit += now_ms() - t_adm;
    if (st == VX_E_NOMEM && (!e.active.empty() || e.op_running)) return;  // wait for memory to free up
    e.pending.pop_front();
    if (st == VX_OK && q->prep.G > kServeMaxGroups) {
      set_error("serving: at most %llu groups per query", (unsigned long long)kServeMaxGroups);
      st = VX_E_UNSUPPORTED;
    }
    if (st == VX_OK && q->prep.staged_cols.size() > e.max_cols) st = VX_E_UNSUPPORTED;
    if (st != VX_OK) {
      fail(e, q, st);
      continue;
    }
    q->t_admit = now_ms();
    q->rslot = e.rfree.back();
    e.rfree.pop_back();
    const uint64_t cr = serve_chunk_rows(e);
    const uint64_t rb = q->prep.row_begin, re = q->prep.row_begin + q->prep.n_rows;
    q->c_first = rb / cr;
    q->c_last = q->prep.n_rows ? (re + cr - 1) / cr : q->c_first;
    q->left = q->c_last - q->c_first;
    q->seen.assign(q->left, 0);
    q->stats.rows = q->prep.n_rows;
    q->stats.late_mask = q->prep.late_mask;
    q->stats.est_selectivity = q->prep.est;
    q->stats.bytes_logical = q->prep.n_rows * 4ull * q->prep.role_col.size();
    e.n_chunks = std::max(e.n_chunks, q->c_last);
    q->state = 1;
    if (q->left == 0) {  // empty range: the zeroed accumulators are the result
      cudaMemcpy(e.rbuf[q->rslot], q->prep.acc.p, 16 * q->prep.G, cudaMemcpyDeviceToHost);
      finalize(e, q);
      continue;
    }
    e.active.push_back(q);
    e.active_peak = std::max<uint64_t>(e.active_peak, e.active.size());
  }
}

// one cycle of the shared scan; returns false when nothing is attached
static vx_status cycle(ServeEngine &e, bool *did) {
  *did = false;
  if (e.active.empty()) return VX_OK;
  // next chunk in scan order that an attached query still needs
  uint64_t c = UINT64_MAX;
  for (uint64_t k = 0; k < e.n_chunks && c == UINT64_MAX; ++k) {
    const uint64_t cand = (e.cursor + k) % e.n_chunks;
    for (ServeQuery *q : e.active)
      if (q->state == 1 && cand >= q->c_first && cand < q->c_last && !q->seen[cand - q->c_first]) {
        c = cand;
        break;
      }
  }
  if (c == UINT64_MAX) return VX_OK;
  vx_ctx *ctx = e.ctx;
  const int k = (int)(e.cycles % e.S);
  ServeEngine::Slot &sl = e.slots[k];
  if (sl.busy) {  // slot reuse waits for its previous kernel (bounded)
    const double t_w = now_ms();
    const double dl = t_w + ctx->cfg.wait_timeout_ms;
    for (;;) {
      cudaError_t qe = cudaEventQuery(sl.ev_k);
      if (qe == cudaSuccess) {
        float ms = 0;
        if (cudaEventElapsedTime(&ms, sl.ev_k0, sl.ev_k) == cudaSuccess) e.ms_kernel += ms;
        cudaGetLastError();
        e.ms_wait += now_ms() - t_w;
        break;
      }
      if (qe != cudaErrorNotReady) VX_CUDA_TRY(qe);
      if (now_ms() > dl) {
        set_error("serving: wait limit expired");
        return VX_E_TIMEOUT;
      }
      std::this_thread::sleep_for(std::chrono::microseconds(10));
    }
  }
  const uint64_t cr = serve_chunk_rows(e);
  const uint64_t c0 = c * cr;
  char *slot = e.ring.as<char>() + (uint64_t)k * e.slot_bytes;
  ChunkParams *dparams = (ChunkParams *)slot;
  MultiItem *ditems = (MultiItem *)(slot + params_bytes(e));
  unsigned int *dnext = (unsigned int *)(slot + params_bytes(e) + items_bytes(e));
  char *dcols = slot + params_bytes(e) + items_bytes(e) + 256;
  ChunkParams *hparams = (ChunkParams *)sl.host;
  MultiItem *hitems = (MultiItem *)(sl.host + params_bytes(e));
  // union of staged columns -> buffer index
  std::vector<const Column *> cols;
  auto buf_of = [&](const Column *col) -> int {
    for (size_t i = 0; i < cols.size(); ++i)
      if (cols[i] == col) return (int)i;
    if (cols.size() >= e.max_cols) return -1;
    cols.push_back(col);
    return (int)cols.size() - 1;
  };
  std::vector<ServeQuery *> qs;
  uint32_t n_items = 0;
  uint64_t n_scan_rows = 0;  // chunk rows the shared-scan queries reach
  for (ServeQuery *q : e.active) {
    if (q->state != 1 || c < q->c_first || c >= q->c_last || q->seen[c - q->c_first]) continue;
    const uint64_t lo = std::max(c0, q->prep.row_begin) - c0;
    const uint64_t hi = std::min(c0 + cr, q->prep.row_begin + q->prep.n_rows) - c0;
    bool fits = true;
    std::vector<int> bufs;
    size_t saved = cols.size();
    for (const Column *col : q->prep.staged_cols) {
      int b = buf_of(col);
      if (b < 0) fits = false;
      bufs.push_back(b);
    }
    if (!fits) {  // this query waits for a later cycle over the chunk
      cols.resize(saved);
      continue;
    }
    ChunkParams p = q->prep.P;
    p.chunk_surv = nullptr;
    // shared scan: row-logic slots read from the tile's union columns; staged
    // pointers at the chunk's base; the query's rows are [lo, hi) of the chunk
    int8_t ucol[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    bool scan = p.n_rowroles >= 1 && p.n_rowroles <= 8;
    for (int k = 0; scan && k < p.n_rowroles; ++k) {
      int b = -1;
      for (size_t i = 0; i < q->prep.staged_role.size(); ++i)
        if (q->prep.staged_role[i] == p.rowrole[k]) b = bufs[i];
      if (b < 0) scan = false;
      ucol[k] = (int8_t)b;
    }
    uint32_t tiles = 0;
    if (scan) {
      for (size_t i = 0; i < q->prep.staged_cols.size(); ++i)
        p.staged[q->prep.staged_role[i]] = (const int32_t *)(dcols + (uint64_t)bufs[i] * col_bytes(e));
      for (int k = 0; k < 8; ++k) p.ucol[k] = k < p.n_rowroles ? ucol[k] : ucol[0];
      p.scan_kr = (int8_t)(p.n_rowroles <= 2 ? 2 : p.n_rowroles <= 4 ? 4 : p.n_rowroles <= 6 ? 6 : 8);
      p.row0 = c0;
      p.row_lo = lo;
      p.n = hi;
    } else {  // the (query, tile) kernel over the query's part of the chunk
      tiles = (uint32_t)((hi - lo + kMultiTile - 1) / kMultiTile);
      if (n_items + tiles > e.max_items) {
        cols.resize(saved);
        continue;
      }
      for (size_t i = 0; i < q->prep.staged_cols.size(); ++i)
        p.staged[q->prep.staged_role[i]] = (const int32_t *)(dcols + (uint64_t)bufs[i] * col_bytes(e)) + lo;
      p.scan_kr = 0;
      p.row0 = c0 + lo;
      p.row_lo = 0;
      p.n = hi - lo;
    }
    e.work_rows += hi - lo;
    const uint32_t qi = (uint32_t)qs.size();
    hparams[qi] = p;
    for (uint32_t t = 0; t < tiles; ++t) hitems[n_items + t] = MultiItem{qi, t};
    n_items += tiles;
    n_scan_rows = std::max<uint64_t>(n_scan_rows, scan ? hi : 0);
    qs.push_back(q);
  }
  if (qs.empty()) return VX_OK;
  std::lock_guard<std::recursive_mutex> g(ctx->mu);
  std::vector<CopyOp> ops;
  for (size_t i = 0; i < cols.size(); ++i) {
    const uint64_t len = cols[i]->n_rows > c0 ? std::min(cr, cols[i]->n_rows - c0) : 0;
    if (len) ops.push_back({(const char *)cols[i]->host + c0 * 4, dcols + i * col_bytes(e), 4 * len});
  }
  VX_TRY(issue_copies(ops, cudaMemcpyHostToDevice, ctx->s_h2d, &e.bytes_h2d, h2d_sm_blocks(ctx)));
  VX_CUDA_TRY(cudaMemcpyAsync(dparams, hparams, sizeof(ChunkParams) * qs.size(), cudaMemcpyHostToDevice, ctx->s_h2d));
  if (n_items)
    VX_CUDA_TRY(cudaMemcpyAsync(ditems, hitems, sizeof(MultiItem) * n_items, cudaMemcpyHostToDevice, ctx->s_h2d));
  VX_CUDA_TRY(cudaEventRecord(sl.ev_in, ctx->s_h2d));
  VX_CUDA_TRY(cudaStreamWaitEvent(ctx->s_compute, sl.ev_in, 0));
  VX_CUDA_TRY(cudaEventRecord(sl.ev_k0, ctx->s_compute));
  VX_TRY(launch_star_scan(ctx, dparams, (uint32_t)qs.size(), dcols, col_bytes(e), (uint32_t)cols.size(), n_scan_rows,
                          dnext + 1, ctx->s_compute));
  VX_TRY(launch_star_multi(ctx, dparams, ditems, n_items, dnext, ctx->s_compute));
  VX_CUDA_TRY(cudaEventRecord(sl.ev_k, ctx->s_compute));
  sl.busy = true;
  for (ServeQuery *q : qs) {
    q->seen[c - q->c_first] = 1;
    q->stats.chunks += 1;
    q->stats.kernel_launches += 1;
    if (--q->left == 0) {  // last chunk: read the accumulators back after this kernel
      VX_CUDA_TRY(cudaMemcpyAsync(e.rbuf[q->rslot], q->prep.acc.p, 16 * q->prep.G, cudaMemcpyDeviceToHost,
                                  ctx->s_compute));
      VX_CUDA_TRY(cudaEventCreateWithFlags(&q->ev_done, cudaEventDisableTiming));
      VX_CUDA_TRY(cudaEventRecord(q->ev_done, ctx->s_compute));
      q->state = 2;
    }
  }
  e.cursor = (c + 1) % std::max<uint64_t>(e.n_chunks, 1);
  e.cycles += 1;
  *did = true;
  return VX_OK;
}

static void reap(ServeEngine &e) {
  for (size_t i = 0; i < e.active.size();) {
    ServeQuery *q = e.active[i];
    if (q->state == 2 && cudaEventQuery(q->ev_done) == cudaSuccess) {
      finalize(e, q);
      e.active.erase(e.active.begin() + i);
      continue;
    }
    ++i;
  }
}

static void engine_loop(ServeEngine *e) {
  cudaSetDevice(e->ctx->device);
  std::unique_lock<std::mutex> lk(e->mu);
  while (!e->stop) {
    admit(*e);
    bool did = false;
    vx_status st = VX_OK;
    if (e->fatal == VX_OK) {
      lk.unlock();
      const double t_cyc = now_ms();
      st = cycle(*e, &did);
      e->ms_cycle += now_ms() - t_cyc;
      lk.lock();
    }
    if (st != VX_OK && e->fatal == VX_OK) {
      e->fatal = st;
      for (ServeQuery *q : e->active) fail(*e, q, st);
      e->active.clear();
    }
    reap(*e);
    e->cv_done.notify_all();
    if (!did) {
      if (e->pending.empty() && e->active.empty())
        e->cv.wait_for(lk, std::chrono::milliseconds(5));
      else if (!did) {
        lk.unlock();
        std::this_thread::sleep_for(std::chrono::microseconds(20));
        lk.lock();
      }
    }
  }
}

// runs one sort or join query in a child context over its own device budget
static vx_status run_op(vx_ctx *child, ServeQuery *q) {
  const vx_op_request &r = q->op;
  if (r.kind == VX_QUERY_SORT) {
    const Column *kc = get_col(child, r.key_col, VX_U64);
    const Column *vc = get_col(child, r.val_col, VX_U32);
    if (!kc || !vc || kc->n_rows != vc->n_rows) {
      set_error("sort query: key and row-id columns must be uint64 / uint32 of equal length");
      return VX_E_INVAL;
    }
    const uint64_t re = r.row_end ? std::min(r.row_end, kc->n_rows) : kc->n_rows;
    const uint64_t rb = std::min(r.row_begin, re), n = re - rb;
    if (n && (!r.out_keys || !r.out_rowids)) {
      set_error("sort query: null output");
      return VX_E_INVAL;
    }
    HostReg r1, r2;
    VX_TRY(r1.add(r.out_keys, 8 * n));
    VX_TRY(r2.add(r.out_rowids, 4 * n));
    vx_sort_stats ss{};
    const double t0 = now_ms();
    const uint64_t *k = (const uint64_t *)kc->host + rb;
    const uint32_t *v = (const uint32_t *)vc->host + rb;
    vx_status st = r.sort.plan == VX_SORT_MERGE
                       ? merge_sort_plan(child, k, v, (const uint64_t *)kc->dev + rb, n, r.out_keys, r.out_rowids,
                                         r.sort, ss)
                       : sort_contiguous(child, k, v, (const uint64_t *)kc->dev + rb, n, r.out_keys, r.out_rowids,
                                         r.sort, ss, 0);
    ss.ms_total = now_ms() - t0;
    q->op_res.sort = ss;
    return st;
  }
  const Column *bk = get_col(child, r.key_col, -1);
  const Column *bp = get_col(child, r.val_col, -1);
  const Column *pk = get_col(child, r.probe_col, -1);
  if (!bk || !bp || !pk) return VX_E_INVAL;
  if (r.join.algorithm != VX_JOIN_DIRECT) {
    set_error("join query: serving runs the direct join");
    return VX_E_UNSUPPORTED;
  }
  return join_columns(child, bk, bp, pk, r.row_begin, r.row_end ? r.row_end : pk->n_rows, &r.join, &q->op_res.join);
}

// Sort / join worker: first come, first served; a query is admitted once its
// device budget can be carved from the arena (star queries finishing free it)
static void op_loop(ServeEngine *e) {
  cudaSetDevice(e->ctx->device);
  std::unique_lock<std::mutex> lk(e->mu);
  while (!e->stop) {
    if (e->op_pending.empty()) {
      e->cv.wait_for(lk, std::chrono::milliseconds(5));
      continue;
    }
    ServeQuery *q = e->op_pending.front();
    const uint64_t cap = e->ctx->arena.capacity();
    const uint64_t budget = q->op.device_budget ? q->op.device_budget : cap / 4;
    e->op_running = true;
    lk.unlock();
    vx_ctx *child = nullptr;
    vx_status st = budget > cap ? VX_E_NOMEM : open_child(e->ctx, budget, &child);
    if (st == VX_E_NOMEM && budget <= cap) {  // wait for memory to free up
      lk.lock();
      e->op_running = false;
      lk.unlock();
      std::this_thread::sleep_for(std::chrono::microseconds(500));
      lk.lock();
      continue;
    }
    lk.lock();
    e->op_pending.pop_front();
    q->t_admit = now_ms();
    q->state = 1;
    lk.unlock();
    if (st == VX_OK) st = run_op(child, q);
    std::string err = st == VX_OK ? std::string() : std::string(vx_last_error());
    if (child) close_child(e->ctx, child);
    lk.lock();
    e->op_running = false;
    q->status = st;
    q->error = err;
    q->t_done = now_ms();
    q->op_res.ms_total = q->t_done - q->t_submit;
    q->op_res.ms_queued = q->t_admit - q->t_submit;
    q->stats.ms_total = q->op_res.ms_total;
    q->state = 3;
    if (st == VX_OK) {
      e->latencies.push_back(q->op_res.ms_total);
      e->lat_kind[q->kind].push_back(q->op_res.ms_total);
    } else {
      e->failed += 1;
    }
    e->cv_done.notify_all();
  }
}

static ServeEngine *engine_of(vx_ctx *ctx) { return reinterpret_cast<ServeEngine *>(ctx->serve); }

void serve_shutdown(vx_ctx *ctx) {
  ServeEngine *e = engine_of(ctx);
  if (!e) return;
  {
    std::lock_guard<std::mutex> g(e->mu);
    e->stop = true;
  }
  e->cv.notify_all();
  if (e->th.joinable()) e->th.join();
  if (e->op_th.joinable()) e->op_th.join();
  cudaStreamSynchronize(ctx->s_compute);
  cudaStreamSynchronize(ctx->s_h2d);
  for (auto &kv : e->all)
    if (kv.second->ev_done) cudaEventDestroy(kv.second->ev_done);
  for (auto &s : e->slots) {
    if (s.ev_in) cudaEventDestroy(s.ev_in);
    if (s.ev_k) cudaEventDestroy(s.ev_k);
    if (s.ev_k0) cudaEventDestroy(s.ev_k0);
    if (s.host) cudaFreeHost(s.host);
  }
  for (uint64_t *p : e->rbuf) cudaFreeHost(p);
  if (e->s_plan) {
    cudaStreamSynchronize(e->s_plan);
    cudaStreamDestroy(e->s_plan);
  }
  delete e;
  ctx->serve = nullptr;
}

}  // namespace vx

using namespace vx;

VX_API vx_status vx_serve_start(vx_ctx *ctx, const vx_serve_opts *opts) {
  clear_error();
  VX_TRY(check_ctx(ctx));
  if (ctx->serve) {
    set_error("vx_serve_start: already serving");
    return VX_E_BUSY;
  }
  std::unique_ptr<ServeEngine> e(new ServeEngine());
  e->ctx = ctx;
  if (opts) e->opts = *opts;
  if (!e->opts.chunk_rows) e->opts.chunk_rows = 1u << 20;
  if (!e->opts.max_active) e->opts.max_active = 32;
  if (!e->opts.n_slots) e->opts.n_slots = 3;
  if (e->opts.chunk_rows % 1024 || e->opts.max_active > 256 || e->opts.n_slots < 2 || e->opts.n_slots > 8) {
    set_error("vx_serve_start: chunk_rows must be a multiple of 1024, max_active <= 256, 2 <= n_slots <= 8");
    return VX_E_INVAL;
  }
  e->S = (int)e->opts.n_slots;
  e->max_items = (uint32_t)(e->opts.max_active * ((e->opts.chunk_rows + kMultiTile - 1) / kMultiTile));
  e->slot_bytes = params_bytes(*e) + items_bytes(*e) + 256 + (uint64_t)e->max_cols * col_bytes(*e);
  std::lock_guard<std::recursive_mutex> g(ctx->mu);
  e->ring.arena = &ctx->arena;
  e->ring.p = ctx->arena.alloc(e->slot_bytes * e->S);
  if (!e->ring.p) {
    set_error("vx_serve_start: staging ring of %llu bytes does not fit the arena",
              (unsigned long long)(e->slot_bytes * e->S));
    return VX_E_NOMEM;
  }
  VX_CUDA_TRY(cudaStreamCreateWithFlags(&e->s_plan, cudaStreamNonBlocking));
  e->slots.resize(e->S);
  for (auto &s : e->slots) {
    VX_CUDA_TRY(cudaEventCreateWithFlags(&s.ev_in, cudaEventDisableTiming));
    VX_CUDA_TRY(cudaEventCreate(&s.ev_k0));
    VX_CUDA_TRY(cudaEventCreate(&s.ev_k));
    VX_CUDA_TRY(cudaHostAlloc((void **)&s.host, params_bytes(*e) + items_bytes(*e), cudaHostAllocDefault));
  }
  for (uint32_t i = 0; i < e->opts.max_active; ++i) {
    uint64_t *p = nullptr;
    VX_CUDA_TRY(cudaHostAlloc((void **)&p, 16 * kServeMaxGroups, cudaHostAllocDefault));
    e->rbuf.push_back(p);
    e->rfree.push_back((int)i);
  }
  e->t_start = now_ms();
  ServeEngine *raw = e.release();
  ctx->serve = raw;
  raw->th = std::thread(engine_loop, raw);
  raw->op_th = std::thread(op_loop, raw);
  return VX_OK;
}

VX_API vx_status vx_submit_op(vx_ctx *ctx, const vx_op_request *req, uint64_t *ticket) {
  clear_error();
  if (!ctx || !req || !ticket || (req->kind != VX_QUERY_SORT && req->kind != VX_QUERY_JOIN)) {
    set_error("vx_submit_op: bad argument");
    return VX_E_INVAL;
  }
  ServeEngine *e = engine_of(ctx);
  if (!e) {
    set_error("vx_submit_op: serving not started");
    return VX_E_INVAL;
  }
  std::unique_ptr<ServeQuery> q(new ServeQuery());
  q->kind = req->kind;
  q->op = *req;
  q->t_submit = now_ms();
  {
    std::lock_guard<std::mutex> g(e->mu);
    if (e->fatal != VX_OK) return e->fatal;
    q->id = e->next_id++;
    *ticket = q->id;
    e->op_pending.push_back(q.get());
    e->all[q->id] = std::move(q);
  }
  e->cv.notify_all();
  return VX_OK;
}

VX_API vx_status vx_wait_op(vx_ctx *ctx, uint64_t ticket, vx_op_result *out, uint32_t timeout_ms) {
  clear_error();
  if (!ctx) return VX_E_INVAL;
  ServeEngine *e = engine_of(ctx);
  if (!e) return VX_E_INVAL;
  std::unique_lock<std::mutex> lk(e->mu);
  auto it = e->all.find(ticket);
  if (it == e->all.end() || it->second->kind == VX_QUERY_STAR) {
    set_error("vx_wait_op: unknown op ticket");
    return VX_E_INVAL;
  }
  ServeQuery *q = it->second.get();
  if (!e->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), [&] { return q->state == 3; })) {
    set_error("vx_wait_op: query %llu not done within %u ms", (unsigned long long)ticket, timeout_ms);
    return VX_E_TIMEOUT;
  }
  if (out) *out = q->op_res;
  if (q->status != VX_OK) set_error("query %llu failed: %s", (unsigned long long)q->id, q->error.c_str());
  return q->status;
}

VX_API vx_status vx_submit(vx_ctx *ctx, const vx_plan *plan, uint64_t *ticket) {
  clear_error();
  if (!ctx || !plan || !ticket) return VX_E_INVAL;
  ServeEngine *e = engine_of(ctx);
  if (!e) {
    set_error("vx_submit: serving not started");
    return VX_E_INVAL;
  }
  std::unique_ptr<ServeQuery> q(new ServeQuery());
  q->plan = *plan;
  q->t_submit = now_ms();
  {
    std::lock_guard<std::mutex> g(e->mu);
    if (e->fatal != VX_OK) return e->fatal;
    q->id = e->next_id++;
    *ticket = q->id;
    e->pending.push_back(q.get());
    e->all[q->id] = std::move(q);
  }
  e->cv.notify_all();
  return VX_OK;
}

static vx_status copy_result(ServeQuery *q, vx_result *out) {
  if (q->status != VX_OK) {
    set_error("query %llu failed: %s", (unsigned long long)q->id, q->error.c_str());
    return q->status;
  }
  if (!out) return VX_OK;
  if (q->kind != VX_QUERY_STAR) {
    out->n_out = 0;
    out->stats = q->stats;
    return VX_OK;
  }
  const uint64_t n = q->gid.size();
  for (uint64_t i = 0; i < n && i < out->cap; ++i) {
    if (out->gid) out->gid[i] = q->gid[i];
    if (out->sum) out->sum[i] = q->sum[i];
    if (out->cnt) out->cnt[i] = q->cnt[i];
  }
  out->n_out = n;
  out->stats = q->stats;
  return n > out->cap ? VX_E_CAPACITY : VX_OK;
}

VX_API vx_status vx_poll(vx_ctx *ctx, uint64_t ticket, vx_result *out, int32_t *done) {
  clear_error();
  if (!ctx || !done) return VX_E_INVAL;
  ServeEngine *e = engine_of(ctx);
  if (!e) return VX_E_INVAL;
  std::lock_guard<std::mutex> g(e->mu);
  auto it = e->all.find(ticket);
  if (it == e->all.end()) {
    set_error("vx_poll: unknown ticket");
    return VX_E_INVAL;
  }
  ServeQuery *q = it->second.get();
  *done = q->state == 3;
  if (!*done) return VX_OK;
  return copy_result(q, out);
}

VX_API vx_status vx_wait(vx_ctx *ctx, uint64_t ticket, vx_result *out, uint32_t timeout_ms) {
  clear_error();
  if (!ctx) return VX_E_INVAL;
  ServeEngine *e = engine_of(ctx);
  if (!e) return VX_E_INVAL;
  std::unique_lock<std::mutex> lk(e->mu);
  auto it = e->all.find(ticket);
  if (it == e->all.end()) {
    set_error("vx_wait: unknown ticket");
    return VX_E_INVAL;
  }
  ServeQuery *q = it->second.get();
  if (!e->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), [&] { return q->state == 3; })) {
    set_error("vx_wait: query %llu not done within %u ms", (unsigned long long)ticket, timeout_ms);
    return VX_E_TIMEOUT;
  }
  return copy_result(q, out);
}

VX_API vx_status vx_serve_stats_get(vx_ctx *ctx, vx_serve_stats *out) {
  if (!ctx || !out) return VX_E_INVAL;
  ServeEngine *e = engine_of(ctx);
  if (!e) return VX_E_INVAL;
  std::lock_guard<std::mutex> g(e->mu);
  vx_serve_stats s{};
  s.submitted = e->next_id - 1;
  s.completed = e->latencies.size();
  s.failed = e->failed;
  s.cycles = e->cycles;
  s.work_rows = e->work_rows;
  s.ms_kernel = e->ms_kernel;
  s.ms_admit = e->ms_admit;
  s.ms_cycle = e->ms_cycle;
  s.ms_wait = e->ms_wait;
  s.bytes_h2d = e->bytes_h2d;
  s.active_peak = e->active_peak;
  s.wall_ms = now_ms() - e->t_start;
  auto pct = [](std::vector<double> l, double p) {  // nearest-rank percentile
    if (l.empty()) return 0.0;
    std::sort(l.begin(), l.end());
    const size_t i = (size_t)std::ceil(p * l.size());
    return l[std::min(l.size() - 1, i ? i - 1 : 0)];
  };
  if (!e->latencies.empty()) {
    s.p50_ms = pct(e->latencies, 0.50);
    s.p99_ms = pct(e->latencies, 0.99);
    s.max_ms = *std::max_element(e->latencies.begin(), e->latencies.end());
    double t = 0;
    for (double v : e->latencies) t += v;
    s.mean_ms = t / e->latencies.size();
  }
  for (int k = 0; k < 3; ++k) {
    s.completed_kind[k] = e->lat_kind[k].size();
    s.p50_kind_ms[k] = pct(e->lat_kind[k], 0.50);
    s.p99_kind_ms[k] = pct(e->lat_kind[k], 0.99);
  }
  *out = s;
  return VX_OK;
}

VX_API vx_status vx_serve_stop(vx_ctx *ctx) {
  if (!ctx) return VX_E_INVAL;
  serve_shutdown(ctx);
  return VX_OK;
}
