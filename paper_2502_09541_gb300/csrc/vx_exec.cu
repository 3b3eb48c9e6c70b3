// Pipelined executor (Section 5.3) over a ring of staging slots.
//
// In cycle n the kernel of chunk n-1 runs on the compute stream while the
// copy engine loads chunk n into a free slot and saves the output of chunk n-2
// on the device-to-host stream.  Two schedules:
//   VX_SCHED_IMMEDIATE — a host loop issues a copy only when it can start at
//     once (its slot is free and the previous user of the slot has finished),
//     following the first design principle of Section 4.3.  A chunk's store is
//     issued only once its kernel has completed, which in turn waited for its
//     load, so the device-to-host queue can never drain ahead of the
//     host-to-device queue (the flow-control policy of Section 4.3) and at
//     most max_in_flight() chunks occupy the link at once.  The loop polls
//     with a 10 us back-off (Section 4.3's retry period); the wall-clock limit
//     wait_timeout_ms applies to the time since the last completed step, so a
//     long operator that keeps making progress never times out.
//   VX_SCHED_DAG — every copy and kernel is enqueued up front with stream and
//     event dependencies (the baseline of Section 4.2).  Only operators whose
//     outputs stay on the device use it.
#include <algorithm>
#include <thread>

#include "vx_internal.h"

namespace vx {

namespace {

struct SlotState {
  int64_t chunk = -1;
  int phase = 0;  // 0 free, 1 kernel issued, 2 storing
  cudaEvent_t ev_in = nullptr, ev_k0 = nullptr, ev_k = nullptr, ev_out = nullptr;
  // timeline (log_timeline): timed events around the chunk's copies
  cudaEvent_t ev_h0 = nullptr, ev_h1 = nullptr, ev_d0 = nullptr, ev_d1 = nullptr;
  float issue_ms = 0;
};

struct EventSet {
  std::vector<SlotState> s;
  cudaEvent_t ref = nullptr;  // timeline origin
  ~EventSet() {
    for (auto &x : s)
      for (cudaEvent_t e : {x.ev_in, x.ev_k0, x.ev_k, x.ev_out, x.ev_h0, x.ev_h1, x.ev_d0, x.ev_d1})
        if (e) cudaEventDestroy(e);
    if (ref) cudaEventDestroy(ref);
  }
};

float since(cudaEvent_t ref, cudaEvent_t e) {
  float ms = -1;
  if (cudaEventElapsedTime(&ms, ref, e) != cudaSuccess) {
    cudaGetLastError();
    return -1;
  }
  return ms;
}

// A copy over the host link runs at full rate only when its host address
// starts on a 512-byte boundary: measured on this link, 12 GB each way with
// the host offsets 8- or 64-byte aligned took 85-96 ms, 512-byte aligned 70
// ms, whatever the device address.  A large copy whose host address is off
// such a boundary is issued as a short head up to it and an aligned body.
constexpr uintptr_t kHostCopyAlign = 512;
constexpr uint64_t kSplitMinBytes = 64 << 10;

vx_status issue_copies(const std::vector<CopyOp> &ops, cudaMemcpyKind kind, cudaStream_t s, uint64_t *bytes) {
  for (const CopyOp &c : ops) {
    if (!c.bytes) continue;
    const uintptr_t host = (uintptr_t)(kind == cudaMemcpyHostToDevice ? c.src : (const void *)c.dst);
    uint64_t head = (kHostCopyAlign - (host & (kHostCopyAlign - 1))) & (kHostCopyAlign - 1);
    if (c.bytes < kSplitMinBytes) head = 0;
    if (head) VX_CUDA_TRY(cudaMemcpyAsync(c.dst, c.src, head, kind, s));
    VX_CUDA_TRY(cudaMemcpyAsync((char *)c.dst + head, (const char *)c.src + head, c.bytes - head, kind, s));
    *bytes += c.bytes;
  }
  return VX_OK;
}

}  // namespace

bool drain_streams(vx_ctx *ctx) {
  cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
  cudaStream_t ss[3] = {ctx->s_compute, ctx->s_h2d, ctx->s_d2h};
  bool ok = true;
  for (int i = 0; i < 3; ++i)
    if (cudaEventCreateWithFlags(&ev[i], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventRecord(ev[i], ss[i]) != cudaSuccess)
      ok = false;
  const double limit = std::max<double>(ctx->cfg.wait_timeout_ms, kDrainLimitMs);
  const double t0 = now_ms();
  for (int i = 0; i < 3 && ok; ++i) {
    while (true) {
      cudaError_t q = cudaEventQuery(ev[i]);
      if (q == cudaSuccess) break;
      if (q != cudaErrorNotReady || now_ms() - t0 > limit) {
        ok = false;
        break;
      }
      std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
  }
  for (cudaEvent_t e : ev)
    if (e) cudaEventDestroy(e);
  cudaGetLastError();
  if (!ok) ctx->poisoned = true;
  return ok;
}

vx_status run_pipeline(vx_ctx *ctx, ExKernel &k, ExecStats *st) {
  const uint64_t N = k.size();
  if (N == 0) return VX_OK;
  const int S = k.n_slots() >= 2 ? k.n_slots() : ctx->cfg.n_slots < 2 ? 2 : ctx->cfg.n_slots;
  const uint64_t slot_bytes = (k.slot_bytes() + 255) & ~255ull;
  DevBuf ring;
  ring.arena = &ctx->arena;
  ring.p = ctx->arena.alloc(slot_bytes * (uint64_t)S);
  if (!ring.p) {
    set_error("executor: %d slots of %llu bytes do not fit the arena (%llu of %llu bytes free)", S,
              (unsigned long long)slot_bytes, (unsigned long long)ctx->arena.largest_free(),
              (unsigned long long)ctx->arena.capacity());
    return VX_E_NOMEM;
  }
  char *base = ring.as<char>();
  EventSet es;
  es.s.resize(S);
  for (auto &x : es.s) {
    VX_CUDA_TRY(cudaEventCreateWithFlags(&x.ev_in, cudaEventDisableTiming));
    VX_CUDA_TRY(cudaEventCreate(&x.ev_k0));
    VX_CUDA_TRY(cudaEventCreate(&x.ev_k));
    VX_CUDA_TRY(cudaEventCreateWithFlags(&x.ev_out, cudaEventDisableTiming));
  }
  std::vector<CopyOp> ops;
  const bool dag = ctx->cfg.sched == VX_SCHED_DAG && !k.has_outputs();
  const bool tl = ctx->cfg.log_timeline && !dag;
  double t_origin = 0;
  if (tl) {
    ctx->timeline.clear();
    for (auto &x : es.s)
      for (cudaEvent_t *e : {&x.ev_h0, &x.ev_h1, &x.ev_d0, &x.ev_d1}) VX_CUDA_TRY(cudaEventCreate(e));
    VX_CUDA_TRY(cudaEventCreate(&es.ref));
    VX_CUDA_TRY(cudaEventRecord(es.ref, ctx->s_h2d));
    t_origin = now_ms();
  }

  if (dag) {
    for (uint64_t it = 0; it < N; ++it) {
      SlotState &sl = es.s[it % S];
      char *slot = base + (it % S) * slot_bytes;
      if (it >= (uint64_t)S) VX_CUDA_TRY(cudaStreamWaitEvent(ctx->s_h2d, sl.ev_k, 0));
      ops.clear();
      k.inputs(it, slot, ops);
      VX_TRY(issue_copies(ops, cudaMemcpyHostToDevice, ctx->s_h2d, &st->bytes_h2d));
      VX_CUDA_TRY(cudaEventRecord(sl.ev_in, ctx->s_h2d));
      VX_CUDA_TRY(cudaStreamWaitEvent(ctx->s_compute, sl.ev_in, 0));
      VX_TRY(k.kernel(slot, it, ctx->s_compute));
      st->kernel_launches += 1;
      VX_CUDA_TRY(cudaEventRecord(sl.ev_k, ctx->s_compute));
    }
    st->chunks += N;
    // the caller synchronises the compute stream; the h2d stream must not run
    // ahead of the next operator's use of the arena either
    VX_CUDA_TRY(cudaStreamWaitEvent(ctx->s_h2d, es.s[(N - 1) % S].ev_k, 0));
    VX_CUDA_TRY(cudaStreamSynchronize(ctx->s_compute));
    VX_CUDA_TRY(cudaStreamSynchronize(ctx->s_h2d));
    return VX_OK;
  }

  double last_progress = now_ms();
  uint64_t next_load = 0, next_retire = 0;
  const uint64_t max_in_flight = (uint64_t)std::max(1, k.max_in_flight());
  while (next_retire < N) {
    bool progress = false;
    // retire in chunk order
    while (next_retire < next_load) {
      SlotState &sl = es.s[next_retire % S];
      if (sl.phase == 1) {
        cudaError_t q = cudaEventQuery(sl.ev_k);
        if (q == cudaErrorNotReady) break;
        VX_CUDA_TRY(q);
        float ms = 0;
        if (cudaEventElapsedTime(&ms, sl.ev_k0, sl.ev_k) == cudaSuccess) st->ms_kernel += ms;
        cudaGetLastError();
        k.on_retire(next_retire);
        if (tl) {
          const float row[VX_TIMELINE_COLS] = {(float)next_retire, sl.issue_ms, since(es.ref, sl.ev_h0),
                                               since(es.ref, sl.ev_h1), since(es.ref, sl.ev_k0),
                                               since(es.ref, sl.ev_k), -1.f, -1.f};
          ctx->timeline.insert(ctx->timeline.end(), row, row + VX_TIMELINE_COLS);
        }
        if (k.has_outputs()) {
          ops.clear();
          VX_TRY(k.outputs(next_retire, base + (next_retire % S) * slot_bytes, ops));
          if (tl) VX_CUDA_TRY(cudaEventRecord(sl.ev_d0, ctx->s_d2h));
          VX_TRY(issue_copies(ops, cudaMemcpyDeviceToHost, ctx->s_d2h, &st->bytes_d2h));
          if (tl) VX_CUDA_TRY(cudaEventRecord(sl.ev_d1, ctx->s_d2h));
          VX_CUDA_TRY(cudaEventRecord(sl.ev_out, ctx->s_d2h));
          sl.phase = 2;
        } else {
          sl.phase = 0;
          ++next_retire;
        }
        progress = true;
      } else if (sl.phase == 2) {
        cudaError_t q = cudaEventQuery(sl.ev_out);
        if (q == cudaErrorNotReady) break;
        VX_CUDA_TRY(q);
        if (tl) {  // this chunk's row is the last one recorded so far
          float *row = &ctx->timeline[ctx->timeline.size() - VX_TIMELINE_COLS];
          row[6] = since(es.ref, sl.ev_d0);
          row[7] = since(es.ref, sl.ev_d1);
        }
        sl.phase = 0;
        ++next_retire;
        progress = true;
      } else {
        break;
      }
    }
    // load the next chunk when its slot is free and fewer than max_in_flight
    // chunks are loaded, computing or storing
    if (next_load < N && next_load - next_retire < (uint64_t)S) {
      SlotState &sl = es.s[next_load % S];
      if (sl.phase == 0 && next_load - next_retire < max_in_flight) {
        char *slot = base + (next_load % S) * slot_bytes;
        ops.clear();
        k.inputs(next_load, slot, ops);
        if (tl) {
          sl.issue_ms = (float)(now_ms() - t_origin);
          VX_CUDA_TRY(cudaEventRecord(sl.ev_h0, ctx->s_h2d));
        }
        VX_TRY(issue_copies(ops, cudaMemcpyHostToDevice, ctx->s_h2d, &st->bytes_h2d));
        if (tl) VX_CUDA_TRY(cudaEventRecord(sl.ev_h1, ctx->s_h2d));
        VX_CUDA_TRY(cudaEventRecord(sl.ev_in, ctx->s_h2d));
        VX_CUDA_TRY(cudaStreamWaitEvent(ctx->s_compute, sl.ev_in, 0));
        VX_CUDA_TRY(cudaEventRecord(sl.ev_k0, ctx->s_compute));
        VX_TRY(k.kernel(slot, next_load, ctx->s_compute));
        st->kernel_launches += 1;
        VX_CUDA_TRY(cudaEventRecord(sl.ev_k, ctx->s_compute));
        sl.chunk = (int64_t)next_load;
        sl.phase = 1;
        ++next_load;
        progress = true;
      }
    }
    if (progress) {
      last_progress = now_ms();
    } else {
      if (now_ms() - last_progress > ctx->cfg.wait_timeout_ms) {
        set_error("executor: no chunk completed a step within the wait limit of %u ms (at chunk %llu of %llu)",
                  ctx->cfg.wait_timeout_ms, (unsigned long long)next_retire, (unsigned long long)N);
        // the ring goes back to the arena only once the work already issued
        // into it has finished; that drain is bounded too
        if (!drain_streams(ctx)) ring.arena = nullptr;
        return VX_E_TIMEOUT;
      }
      std::this_thread::sleep_for(std::chrono::microseconds(10));
    }
  }
  st->chunks += N;
  VX_CUDA_TRY(cudaStreamSynchronize(ctx->s_d2h));
  return VX_OK;
}

vx_status enqueue_pipeline_for_capture(vx_ctx *ctx, ExKernel &k, char *ring, int S, ExecStats *st) {
  const uint64_t N = k.size();
  const uint64_t slot_bytes = (k.slot_bytes() + 255) & ~255ull;
  EventSet es;
  es.s.resize(S);
  for (auto &x : es.s) {
    VX_CUDA_TRY(cudaEventCreateWithFlags(&x.ev_in, cudaEventDisableTiming));
    VX_CUDA_TRY(cudaEventCreateWithFlags(&x.ev_k, cudaEventDisableTiming));
  }
  cudaEvent_t fork = nullptr, join = nullptr;
  VX_CUDA_TRY(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
  VX_CUDA_TRY(cudaEventCreateWithFlags(&join, cudaEventDisableTiming));
  struct Free {
    cudaEvent_t a, b;
    ~Free() {
      cudaEventDestroy(a);
      cudaEventDestroy(b);
    }
  } fr{fork, join};
  VX_CUDA_TRY(cudaEventRecord(fork, ctx->s_compute));
  VX_CUDA_TRY(cudaStreamWaitEvent(ctx->s_h2d, fork, 0));
  std::vector<CopyOp> ops;
  for (uint64_t it = 0; it < N; ++it) {
    SlotState &sl = es.s[it % S];
    char *slot = ring + (it % S) * slot_bytes;
    if (it >= (uint64_t)S) VX_CUDA_TRY(cudaStreamWaitEvent(ctx->s_h2d, sl.ev_k, 0));
    ops.clear();
    k.inputs(it, slot, ops);
    VX_TRY(issue_copies(ops, cudaMemcpyHostToDevice, ctx->s_h2d, &st->bytes_h2d));
    VX_CUDA_TRY(cudaEventRecord(sl.ev_in, ctx->s_h2d));
    VX_CUDA_TRY(cudaStreamWaitEvent(ctx->s_compute, sl.ev_in, 0));
    VX_TRY(k.kernel(slot, it, ctx->s_compute));
    st->kernel_launches += 1;
    VX_CUDA_TRY(cudaEventRecord(sl.ev_k, ctx->s_compute));
  }
  VX_CUDA_TRY(cudaEventRecord(join, ctx->s_h2d));
  VX_CUDA_TRY(cudaStreamWaitEvent(ctx->s_compute, join, 0));
  st->chunks += N;
  return VX_OK;
}

}  // namespace vx
