// Pipelined executor (Section 5.3) over a ring of staging slots.
//
// In cycle n the kernel of chunk n-1 runs on the compute stream while the
// copy engine loads chunk n into a free slot and saves the output of chunk n-2
// on the device-to-host stream.  Two schedules:
//   VX_SCHED_IMMEDIATE — a host loop issues a copy only when it can start at
//     once (vx_sched.h holds the decisions; this file gives them the
//     context's streams and events).
//   VX_SCHED_DAG — every copy and kernel is enqueued up front with stream and
//     event dependencies (the baseline of Section 4.2).  Only operators whose
//     outputs stay on the device use it.
#include <algorithm>
#include <thread>

#include "vx_internal.h"
#include "vx_sched.h"

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

// The immediate schedule's device: the context's copy and compute streams,
// one event set per staging slot (vx_sched.h makes the decisions)
struct CudaDev {
  vx_ctx *ctx;
  ExKernel &k;
  ExecStats *st;
  EventSet &es;
  char *base;
  uint64_t slot_bytes;
  bool tl;
  double t_origin;
  DevBuf *ring;
  std::vector<CopyOp> ops;

  char *slot(int s) const { return base + (uint64_t)s * slot_bytes; }
  static int state(cudaEvent_t e) {
    const cudaError_t q = cudaEventQuery(e);
    if (q == cudaErrorNotReady) return 0;
    if (q == cudaSuccess) return 1;
    set_error("executor: %s", cudaGetErrorString(q));
    return VX_E_CUDA;
  }
  bool has_outputs() { return k.has_outputs(); }
  vx_status load(uint64_t it, int s) {
    SlotState &sl = es.s[s];
    ops.clear();
    k.inputs(it, slot(s), ops);
    if (tl) {
      sl.issue_ms = (float)(now_ms() - t_origin);
      VX_CUDA_TRY(cudaEventRecord(sl.ev_h0, ctx->s_h2d));
    }
    VX_TRY(issue_copies(ops, cudaMemcpyHostToDevice, ctx->s_h2d, &st->bytes_h2d, h2d_sm_blocks(ctx)));
    if (tl) VX_CUDA_TRY(cudaEventRecord(sl.ev_h1, ctx->s_h2d));
    VX_CUDA_TRY(cudaEventRecord(sl.ev_in, ctx->s_h2d));
    VX_CUDA_TRY(cudaStreamWaitEvent(ctx->s_compute, sl.ev_in, 0));
    VX_CUDA_TRY(cudaEventRecord(sl.ev_k0, ctx->s_compute));
    VX_TRY(k.kernel(slot(s), it, ctx->s_compute));
    st->kernel_launches += 1;
    VX_CUDA_TRY(cudaEventRecord(sl.ev_k, ctx->s_compute));
    sl.chunk = (int64_t)it;
    return VX_OK;
  }
  int kernel_state(int s) { return state(es.s[s].ev_k); }
  vx_status retire(uint64_t it, int s) {
    SlotState &sl = es.s[s];
    float ms = 0;
    if (cudaEventElapsedTime(&ms, sl.ev_k0, sl.ev_k) == cudaSuccess) st->ms_kernel += ms;
    cudaGetLastError();
    k.on_retire(it);
    if (tl) {
      const float row[VX_TIMELINE_COLS] = {(float)it, sl.issue_ms, since(es.ref, sl.ev_h0), since(es.ref, sl.ev_h1),
                                           since(es.ref, sl.ev_k0), since(es.ref, sl.ev_k), -1.f, -1.f};
      ctx->timeline.insert(ctx->timeline.end(), row, row + VX_TIMELINE_COLS);
    }
    return VX_OK;
  }
  vx_status store(uint64_t it, int s) {
    SlotState &sl = es.s[s];
    ops.clear();
    VX_TRY(k.outputs(it, slot(s), ops));
    if (tl) VX_CUDA_TRY(cudaEventRecord(sl.ev_d0, ctx->s_d2h));
    VX_TRY(issue_copies(ops, cudaMemcpyDeviceToHost, ctx->s_d2h, &st->bytes_d2h, 0));
    if (tl) VX_CUDA_TRY(cudaEventRecord(sl.ev_d1, ctx->s_d2h));
    VX_CUDA_TRY(cudaEventRecord(sl.ev_out, ctx->s_d2h));
    return VX_OK;
  }
  int store_state(int s) { return state(es.s[s].ev_out); }
  vx_status stored(uint64_t, int s) {
    if (tl) {  // this chunk's row is the last one recorded so far (chunks retire in order)
      float *row = &ctx->timeline[ctx->timeline.size() - VX_TIMELINE_COLS];
      row[6] = since(es.ref, es.s[s].ev_d0);
      row[7] = since(es.ref, es.s[s].ev_d1);
    }
    return VX_OK;
  }
  vx_status timed_out(uint64_t it) {
    set_error("executor: no chunk completed a step within the wait limit of %u ms (at chunk %llu of %llu)",
              ctx->cfg.wait_timeout_ms, (unsigned long long)it, (unsigned long long)k.size());
    // the ring goes back to the arena only once the work already issued into
    // it has finished; that drain is bounded too
    if (!drain_streams(ctx)) ring->arena = nullptr;
    return VX_E_TIMEOUT;
  }
  double now_ms() { return vx::now_ms(); }
  void pause() { std::this_thread::sleep_for(std::chrono::microseconds(10)); }
};

}  // namespace

// Host -> HBM copies made by the SMs instead of the copy engine
// (vx_config.h2d_copy_blocks > 0): loads of pinned host memory through its
// device-visible address (the same address on this platform), stores into
// HBM.  Alone on the link, a copy engine's 2 GB transfers now and then ran at
// 80-190 GB/s where SM-driven transfers in between kept 207-211 GB/s (32
// blocks of 256 threads reach the link's rate); inside a pipeline the copy
// kernel takes SMs from the chunk kernels, so the copy engine is the default.
// Its launches carry the device's highest priority: the next chunk's copy
// becomes ready when the current chunk's kernel does, and at equal priority
// the copy's blocks would wait behind that kernel's pending blocks while the
// link idles (186 against 198-204 GB/s per star query in captured pipelines).
constexpr int kCopyBatch = 16;
struct HostCopyBatch {
  const void *src[kCopyBatch];
  void *dst[kCopyBatch];
  uint64_t bytes[kCopyBatch];
  int n;
};

// each op in turn, the grid striding over it: when source and destination
// agree modulo 16, the 16-byte-aligned body as 16-byte words (eight loads in
// flight per thread before their stores) and the ends as 4-byte words; else
// 4-byte words throughout (sixteen in flight).  Every op is 4-byte aligned at
// both ends with a length that is a multiple of 4 (checked by the caller).
__global__ void __launch_bounds__(256) host_copy_kernel(const HostCopyBatch b) {
  const uint64_t tid = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x, nt = (uint64_t)gridDim.x * blockDim.x;
  for (int o = 0; o < b.n; ++o) {
    const char *s = (const char *)b.src[o];
    char *d = (char *)b.dst[o];
    const uint64_t n = b.bytes[o];
    if (((uintptr_t)s & 15) == ((uintptr_t)d & 15)) {
      uint64_t head = (16 - ((uintptr_t)s & 15)) & 15;
      if (head > n) head = n;
      const uint64_t n16 = (n - head) / 16, tail0 = head + 16 * n16;
      for (uint64_t i = 4 * tid; i < head; i += 4 * nt) *(uint32_t *)(d + i) = __ldg((const uint32_t *)(s + i));
      const int4 *s4 = (const int4 *)(s + head);
      int4 *d4 = (int4 *)(d + head);
      uint64_t i = tid;
      for (; i + 7 * nt < n16; i += 8 * nt) {
        int4 v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = __ldg(s4 + i + u * nt);
#pragma unroll
        for (int u = 0; u < 8; ++u) d4[i + u * nt] = v[u];
      }
      for (; i < n16; i += nt) d4[i] = __ldg(s4 + i);
      for (uint64_t j = tail0 + 4 * tid; j < n; j += 4 * nt) *(uint32_t *)(d + j) = __ldg((const uint32_t *)(s + j));
    } else {
      const uint32_t *s1 = (const uint32_t *)s;
      uint32_t *d1 = (uint32_t *)d;
      const uint64_t n4 = n / 4;
      uint64_t i = tid;
      for (; i + 15 * nt < n4; i += 16 * nt) {
        uint32_t v[16];
#pragma unroll
        for (int u = 0; u < 16; ++u) v[u] = __ldg(s1 + i + u * nt);
#pragma unroll
        for (int u = 0; u < 16; ++u) d1[i + u * nt] = v[u];
      }
      for (; i < n4; i += nt) d1[i] = __ldg(s1 + i);
    }
  }
}

// the greatest (numerically lowest) stream priority of the current device
static int copy_priority() {
  static int prio = 0;
  static std::once_flag once;
  std::call_once(once, [] {
    int lo = 0, hi = 0;
    if (cudaDeviceGetStreamPriorityRange(&lo, &hi) == cudaSuccess) prio = hi;
    cudaGetLastError();
  });
  return prio;
}

int h2d_sm_blocks(const vx_ctx *ctx) { return ctx->host_ptr_ok ? ctx->cfg.h2d_copy_blocks : 0; }

vx_status issue_copies(const std::vector<CopyOp> &ops, cudaMemcpyKind kind, cudaStream_t s, uint64_t *bytes,
                       int sm_blocks) {
  HostCopyBatch batch{};
  auto flush = [&]() -> vx_status {
    if (batch.n) {
      cudaLaunchConfig_t lc = {};
      lc.gridDim = dim3((unsigned)sm_blocks);
      lc.blockDim = dim3(256);
      lc.stream = s;
      cudaLaunchAttribute at[1];
      at[0].id = cudaLaunchAttributePriority;
      at[0].val.priority = copy_priority();
      lc.attrs = at;
      lc.numAttrs = 1;
      VX_CUDA_TRY(cudaLaunchKernelEx(&lc, host_copy_kernel, batch));
      batch.n = 0;
    }
    return VX_OK;
  };
  for (const CopyOp &c : ops) {
    if (!c.bytes) continue;
    *bytes += c.bytes;
    if (kind == cudaMemcpyHostToDevice && sm_blocks > 0 && !(((uintptr_t)c.src | (uintptr_t)c.dst | c.bytes) & 3)) {
      batch.src[batch.n] = c.src;
      batch.dst[batch.n] = c.dst;
      batch.bytes[batch.n] = c.bytes;
      if (++batch.n == kCopyBatch) VX_TRY(flush());
      continue;
    }
    const uintptr_t host = (uintptr_t)(kind == cudaMemcpyHostToDevice ? c.src : (const void *)c.dst);
    uint64_t head = (kHostCopyAlign - (host & (kHostCopyAlign - 1))) & (kHostCopyAlign - 1);
    if (c.bytes < kSplitMinBytes) head = 0;
    if (head) VX_CUDA_TRY(cudaMemcpyAsync(c.dst, c.src, head, kind, s));
    VX_CUDA_TRY(cudaMemcpyAsync((char *)c.dst + head, (const char *)c.src + head, c.bytes - head, kind, s));
  }
  return flush();
}


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
      VX_TRY(issue_copies(ops, cudaMemcpyHostToDevice, ctx->s_h2d, &st->bytes_h2d, h2d_sm_blocks(ctx)));
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

  CudaDev dev{ctx, k, st, es, base, slot_bytes, tl, t_origin, &ring, {}};
  VX_TRY(immediate_schedule(dev, N, S, (uint64_t)std::max(1, k.max_in_flight()), (double)ctx->cfg.wait_timeout_ms));
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
    VX_TRY(issue_copies(ops, cudaMemcpyHostToDevice, ctx->s_h2d, &st->bytes_h2d, h2d_sm_blocks(ctx)));
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
