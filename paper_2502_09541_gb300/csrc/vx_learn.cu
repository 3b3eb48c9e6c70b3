// Learned range partitioner: a monotone CDF MLP (1 -> H -> 1, fp32) trained on
// the device with a hand-written forward/backward kernel whose last block
// applies the Adam step (one launch per step, captured in one CUDA
// graph per 25 steps), then inverted by bisection to give integer
// splitters.  The model only decides where partitions are cut; every cut gives
// the same sorted output.
//
//   y(x) = gamma + sum_j softplus(alpha_j) * sigmoid(softplus(omega_j) x + beta_j)
//
// Both weight layers pass through softplus, so y is non-decreasing in x and
// its inverse is well defined for bisection.
#include <algorithm>
#include <cmath>

#include "vx_internal.h"
#include "vx_sort.cuh"

namespace vx {

__device__ __forceinline__ float softplusf(float v) { return v > 20.f ? v : log1pf(expf(v)); }
__device__ __forceinline__ float sigmoidf(float v) { return 1.f / (1.f + expf(-v)); }

constexpr int kMlpMaxH = 64;
constexpr int kMlpThreads = 256;

struct AdamState {
  float m1[3 * kMlpMaxH + 1], m2[3 * kMlpMaxH + 1];
  int t;
};

// one Adam update (Kingma & Ba 2015) of parameter k at step `step`
__device__ __forceinline__ void adam_update(float *theta, float g, AdamState *st, int k, int step, float lr, float b1,
                                            float b2, float eps) {
  const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
  const float m1 = b1 * st->m1[k] + (1.f - b1) * g;
  const float m2 = b2 * st->m2[k] + (1.f - b2) * g * g;
  st->m1[k] = m1;
  st->m2[k] = m2;
  theta[k] -= lr * (m1 / c1) / (sqrtf(m2 / c2) + eps);
}

// Adam settings of a fused training step (adam == nullptr: gradient only)
struct StepArgs {
  AdamState *adam;
  unsigned int *done;  // blocks that have added their gradient; the last one steps
  float lr, b1, b2, eps;
};

// dL/dtheta and L over m points; grad/loss are accumulated with atomics
// (caller zeroes them).  theta = [omega(H), beta(H), alpha(H), gamma].  Lane
// j of a warp owns hidden unit j (H <= 32): a warp evaluates one point at a
// time, every lane its unit, a butterfly sum gives y, and each lane keeps its
// unit's three partial derivatives in registers.  With sa.adam set, the
// last block to finish applies the Adam step to theta from the summed
// gradient and zeroes grad, loss and the block counter for the next step, so
// one launch is one training step.
template <int H>
__global__ void __launch_bounds__(kMlpThreads, 2) mlp_fwd_bwd_kernel(float *__restrict__ theta,
                                                                   const float *__restrict__ x,
                                                                   const float *__restrict__ t, uint64_t m,
                                                                   float *grad, float *loss, StepArgs sa) {
  static_assert(H >= 1 && H <= 32, "one hidden unit per lane");
  __shared__ float sg[3 * H + 2];
  for (int k = threadIdx.x; k < 3 * H + 2; k += blockDim.x) sg[k] = 0.f;
  __syncthreads();
  const unsigned lane = threadIdx.x & 31;
  const bool on = lane < (unsigned)H;
  const float w = on ? softplusf(theta[lane]) : 0.f, dw = on ? sigmoidf(theta[lane]) : 0.f;
  const float b = on ? theta[H + lane] : 0.f;
  const float a = on ? softplusf(theta[2 * H + lane]) : 0.f, da = on ? sigmoidf(theta[2 * H + lane]) : 0.f;
  const float gamma = theta[3 * H];
  const float inv_m = 1.f / (float)m;
  float g_om = 0.f, g_be = 0.f, g_al = 0.f, g_ga = 0.f, l = 0.f;
  // a warp takes 32 consecutive points at a time: one coalesced load of x and
  // t, then the points one by one, broadcast from the lane that loaded them
  const uint64_t n_warps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t base = (((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 32; base < m;
       base += n_warps * 32) {
    const uint64_t mine = base + lane;
    const float xl = mine < m ? x[mine] : 0.f, tl = mine < m ? t[mine] : 0.f;
    const int cnt = m - base < 32 ? (int)(m - base) : 32;
    for (int k = 0; k < cnt; ++k) {
      const float xi = __shfl_sync(0xffffffffu, xl, k), ti = __shfl_sync(0xffffffffu, tl, k);
      const float si = on ? sigmoidf(w * xi + b) : 0.f;
      float v = a * si;
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
      const float r = gamma + v - ti;
      const float dy = 2.f * r * inv_m;
      l += r * r;  // the same in every lane; lane 0's copy is kept
      g_ga += dy;
      const float q = dy * a * si * (1.f - si);
      g_be += q;
      g_om += q * xi * dw;
      g_al += dy * da * si;
    }
  }
  if (on) {
    atomicAdd(&sg[lane], g_om);
    atomicAdd(&sg[H + lane], g_be);
    atomicAdd(&sg[2 * H + lane], g_al);
  }
  if (lane == 0) {
    atomicAdd(&sg[3 * H], g_ga);
    atomicAdd(&sg[3 * H + 1], l);
  }
  __syncthreads();
  for (int k = threadIdx.x; k < 3 * H + 1; k += blockDim.x) atomicAdd(&grad[k], sg[k]);
  if (threadIdx.x == 0) atomicAdd(loss, sg[3 * H + 1] * inv_m);
  if (!sa.adam) return;
  // the last block to finish: every other block's atomics are done
  __shared__ bool last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(sa.done, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!last) return;
  __threadfence();
  const int step = sa.adam->t + 1;
  for (int k = threadIdx.x; k < 3 * H + 1; k += blockDim.x) {
    adam_update(theta, __ldcg(&grad[k]), sa.adam, k, step, sa.lr, sa.b1, sa.b2, sa.eps);
    grad[k] = 0.f;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    sa.adam->t = step;
    *loss = 0.f;
    *sa.done = 0u;
  }
}

// data-driven initial parameters from the (sorted) training points: unit j is
// a sigmoid step of height 1/H centred at the (j + 0.5)/H quantile of x, with a
// slope inverse to the width of its quantile bin, so the untrained network is
// already a smoothed H-segment quantile model that training then refines
__global__ void mlp_init_from_points_kernel(const float *x, uint32_t M, float *theta, int H) {
  for (int j = threadIdx.x; j < H; j += blockDim.x) {
    const uint32_t a = (uint32_t)((uint64_t)j * M / H), b = (uint32_t)((uint64_t)(j + 1) * M / H);
    const uint32_t c = (uint32_t)(((uint64_t)2 * j + 1) * M / (2 * H));
    const float lo = x[a < M ? a : M - 1], hi = x[b < M ? b : M - 1], mid = x[c < M ? c : M - 1];
    const float width = fmaxf(hi - lo, 1e-7f);
    const float slope = fminf(4.f / width, 1e7f);
    theta[j] = slope > 20.f ? slope : logf(expm1f(slope));  // softplus^-1(slope)
    theta[H + j] = -slope * mid;
    theta[2 * H + j] = logf(expm1f(1.f / H));  // softplus^-1(1/H)
  }
  if (threadIdx.x == 0) theta[3 * H] = 0.f;
}

// training points from the sorted sample: M evenly spaced order statistics,
// x = (key - kmin) / (kmax - kmin), target = empirical CDF (idx + 0.5) / m
__global__ void mlp_points_kernel(const uint64_t *sorted, uint64_t m, uint32_t M, float *x, float *t) {
  const uint64_t kmin = sorted[0], kmax = sorted[m - 1];
  const double span = kmax > kmin ? (double)(kmax - kmin) : 1.0;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < M; i += gridDim.x * blockDim.x) {
    const uint64_t idx = M > 1 ? (uint64_t)i * (m - 1) / (M - 1) : 0;
    x[i] = (float)((double)(sorted[idx] - kmin) / span);
    t[i] = (float)(((double)idx + 0.5) / (double)m);
  }
}

template <int H>
__device__ float mlp_eval(const float *theta, float x) {
  float y = theta[3 * H];
  for (int j = 0; j < H; ++j) y += softplusf(theta[2 * H + j]) * sigmoidf(softplusf(theta[j]) * x + theta[H + j]);
  return y;
}

// splitter p: bisection of y(x) = p/P on [0, 1], mapped back to the key
// domain and snapped to the first sample key >= it (so that a heavy key, a
// vertical step of the CDF, yields repeated splitters that isolate it)
template <int H>
__global__ void mlp_splitters_kernel(const float *theta, const uint64_t *sorted, uint64_t m, uint32_t P,
                                     uint64_t *spl) {
  const uint64_t kmin = sorted[0], kmax = sorted[m - 1];
  const double span = (double)(kmax - kmin);
  for (uint32_t p = 1 + blockIdx.x * blockDim.x + threadIdx.x; p < P; p += gridDim.x * blockDim.x) {
    const float q = (float)p / (float)P;
    float lo = 0.f, hi = 1.f;
    for (int it = 0; it < 40; ++it) {
      const float mid = 0.5f * (lo + hi);
      if (mlp_eval<H>(theta, mid) < q) lo = mid;
      else hi = mid;
    }
    double kf = (double)kmin + (double)hi * span;
    uint64_t key = kf >= (double)kmax ? kmax : (kf <= (double)kmin ? kmin : (uint64_t)kf);
    uint64_t a = 0, b = m;  // first index with sorted[i] >= key
    while (a < b) {
      const uint64_t mid = (a + b) >> 1;
      if (sorted[mid] < key) a = mid + 1;
      else b = mid;
    }
    spl[p - 1] = sorted[a < m ? a : m - 1];
  }
}

// ------------------------------------------------------------------ host

struct MlpWork {
  DevBuf buf;
  float *theta, *grad, *loss, *x, *t;
  unsigned int *done;
  AdamState *adam;
};

static vx_status mlp_alloc(vx_ctx *ctx, uint64_t M, MlpWork &w) {
  const uint64_t bytes = 4096 + sizeof(AdamState) + 2 * ((4 * M + 255) & ~255ull) + 1024;
  w.buf.arena = &ctx->arena;
  w.buf.p = ctx->arena.alloc(bytes);
  if (!w.buf.p) {
    set_error("MLP work area of %llu bytes does not fit the arena", (unsigned long long)bytes);
    return VX_E_NOMEM;
  }
  char *p = w.buf.as<char>();
  w.theta = (float *)p;
  w.grad = (float *)(p + 1024);
  w.loss = (float *)(p + 2048);
  w.done = (unsigned int *)(p + 2048 + 64);
  w.adam = (AdamState *)(p + 4096);
  char *q = p + 4096 + ((sizeof(AdamState) + 255) & ~255ull);
  w.x = (float *)q;
  w.t = (float *)(q + ((4 * M + 255) & ~255ull));
  return VX_OK;
}

// blocks of the forward/backward kernel: 32 points per warp, at most two
// blocks per SM (each block adds 3H + 2 atomics to the global gradient)
static int mlp_grid(const vx_ctx *ctx, uint64_t m) {
  const uint64_t per_block = 32 * (kMlpThreads / 32);
  return (int)std::max<uint64_t>(1, std::min<uint64_t>((m + per_block - 1) / per_block, 2ull * ctx->num_sms));
}

static vx_status launch_fwd_bwd(int H, float *theta, const float *x, const float *t, uint64_t m, float *grad,
                                float *loss, int grid, cudaStream_t s, StepArgs a = StepArgs{}) {
  if (H == 32)
    mlp_fwd_bwd_kernel<32><<<grid, kMlpThreads, 0, s>>>(theta, x, t, m, grad, loss, a);
  else if (H == 16)
    mlp_fwd_bwd_kernel<16><<<grid, kMlpThreads, 0, s>>>(theta, x, t, m, grad, loss, a);
  else if (H == 8)
    mlp_fwd_bwd_kernel<8><<<grid, kMlpThreads, 0, s>>>(theta, x, t, m, grad, loss, a);
  else if (H == 1)
    mlp_fwd_bwd_kernel<1><<<grid, kMlpThreads, 0, s>>>(theta, x, t, m, grad, loss, a);
  else {
    set_error("MLP width %d not built (1, 8, 16, 32)", H);
    return VX_E_UNSUPPORTED;
  }
  VX_CUDA_TRY(cudaGetLastError());
  return VX_OK;
}

// trains with `steps` Adam steps: every step is one launch (forward,
// backward, and the Adam update in the last block to finish); up to
// kStepsPerGraph consecutive steps are captured in one CUDA graph, which is
// launched as often as needed (one more graph for a remainder), so capture and
// instantiation stay short
constexpr uint32_t kStepsPerGraph = 25;

static vx_status launch_steps(int H, MlpWork &w, uint64_t m, uint32_t n, int grid, const StepArgs &a,
                              cudaStream_t s, uint32_t times) {
  if (n == 0 || times == 0) return VX_OK;
  cudaGraph_t g = nullptr;
  cudaGraphExec_t ge = nullptr;
  VX_CUDA_TRY(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
  vx_status st = VX_OK;
  for (uint32_t i = 0; i < n && st == VX_OK; ++i) st = launch_fwd_bwd(H, w.theta, w.x, w.t, m, w.grad, w.loss, grid, s, a);
  cudaError_t ce = cudaStreamEndCapture(s, &g);
  if (st != VX_OK) {
    if (g) cudaGraphDestroy(g);
    return st;
  }
  VX_CUDA_TRY(ce);
  ce = cudaGraphInstantiate(&ge, g, 0);
  cudaGraphDestroy(g);
  VX_CUDA_TRY(ce);
  for (uint32_t r = 0; r < times && ce == cudaSuccess; ++r) ce = cudaGraphLaunch(ge, s);
  cudaGraphExecDestroy(ge);
  VX_CUDA_TRY(ce);
  return VX_OK;
}

static vx_status train(vx_ctx *ctx, int H, MlpWork &w, uint64_t m, uint32_t steps, float lr) {
  cudaStream_t s = ctx->s_compute;
  const int grid = mlp_grid(ctx, m);
  VX_CUDA_TRY(cudaMemsetAsync(w.adam, 0, sizeof(AdamState), s));
  VX_CUDA_TRY(cudaMemsetAsync(w.grad, 0, 2048, s));  // grad[0..3H], loss, block counter
  const StepArgs a{w.adam, w.done, lr, 0.9f, 0.999f, 1e-8f};
  const uint32_t per = std::min(steps, kStepsPerGraph);
  if (per == 0) return VX_OK;
  VX_TRY(launch_steps(H, w, m, per, grid, a, s, steps / per));
  VX_TRY(launch_steps(H, w, m, steps % per, grid, a, s, 1));
  return VX_OK;
}

vx_status mlp_splitters(vx_ctx *ctx, const uint64_t *sorted, uint64_t m, uint32_t P, uint32_t steps, uint64_t *d_spl,
                        double *ms_train) {
  const uint32_t M = (uint32_t)std::min<uint64_t>(m, 65536);
  MlpWork w;
  VX_TRY(mlp_alloc(ctx, M, w));
  cudaStream_t s = ctx->s_compute;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0, s);
  mlp_points_kernel<<<(M + 255) / 256, 256, 0, s>>>(sorted, m, M, w.x, w.t);
  mlp_init_from_points_kernel<<<1, 64, 0, s>>>(w.x, M, w.theta, kMlpHidden);
  VX_CUDA_TRY(cudaGetLastError());
  VX_TRY(train(ctx, kMlpHidden, w, M, steps ? steps : 300, 1e-2f));
  mlp_splitters_kernel<kMlpHidden><<<1, 256, 0, s>>>(w.theta, sorted, m, P, d_spl);
  VX_CUDA_TRY(cudaGetLastError());
  cudaEventRecord(e1, s);
  VX_CUDA_TRY(cudaEventSynchronize(e1));
  float ms = 0;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (ms_train) *ms_train = ms;
  return VX_OK;
}

}  // namespace vx

using namespace vx;

static vx_status mlp_host_setup(vx_ctx *ctx, int32_t H, const float *x, const float *t, uint64_t m, MlpWork &w) {
  if (H < 1 || H > kMlpMaxH || m == 0 || !x || !t) {
    set_error("MLP: need 1 <= H <= %d, m > 0 and points", kMlpMaxH);
    return VX_E_INVAL;
  }
  VX_TRY(mlp_alloc(ctx, m, w));
  cudaStream_t s = ctx->s_compute;
  VX_CUDA_TRY(cudaMemcpyAsync(w.x, x, 4 * m, cudaMemcpyHostToDevice, s));
  VX_CUDA_TRY(cudaMemcpyAsync(w.t, t, 4 * m, cudaMemcpyHostToDevice, s));
  return VX_OK;
}

VX_API vx_status vx_mlp_loss_grad(vx_ctx *ctx, const float *theta, int32_t H, const float *x, const float *t,
                                  uint64_t m, float *grad_out, float *loss_out) {
  clear_error();
  VX_TRY(check_ctx(ctx));
  if (!theta || !grad_out || !loss_out) return VX_E_INVAL;
  std::lock_guard<std::recursive_mutex> g(ctx->mu);
  MlpWork w;
  VX_TRY(mlp_host_setup(ctx, H, x, t, m, w));
  cudaStream_t s = ctx->s_compute;
  VX_CUDA_TRY(cudaMemcpyAsync(w.theta, theta, 4 * (3 * H + 1), cudaMemcpyHostToDevice, s));
  VX_CUDA_TRY(cudaMemsetAsync(w.grad, 0, 2048, s));
  const int grid = mlp_grid(ctx, m);
  VX_TRY(launch_fwd_bwd(H, w.theta, w.x, w.t, m, w.grad, w.loss, grid, s));
  VX_CUDA_TRY(cudaMemcpyAsync(grad_out, w.grad, 4 * (3 * H + 1), cudaMemcpyDeviceToHost, s));
  VX_CUDA_TRY(cudaMemcpyAsync(loss_out, w.loss, 4, cudaMemcpyDeviceToHost, s));
  VX_CUDA_TRY(cudaStreamSynchronize(s));
  return VX_OK;
}

VX_API vx_status vx_mlp_train(vx_ctx *ctx, float *theta, int32_t H, const float *x, const float *t, uint64_t m,
                              uint32_t steps, float lr, float *loss_out) {
  clear_error();
  VX_TRY(check_ctx(ctx));
  if (!theta || !loss_out || !(lr > 0.f)) return VX_E_INVAL;
  std::lock_guard<std::recursive_mutex> g(ctx->mu);
  MlpWork w;
  VX_TRY(mlp_host_setup(ctx, H, x, t, m, w));
  cudaStream_t s = ctx->s_compute;
  VX_CUDA_TRY(cudaMemcpyAsync(w.theta, theta, 4 * (3 * H + 1), cudaMemcpyHostToDevice, s));
  VX_TRY(train(ctx, H, w, m, steps, lr));
  // loss of the final parameters
  VX_CUDA_TRY(cudaMemsetAsync(w.grad, 0, 2048, s));
  const int grid = mlp_grid(ctx, m);
  VX_TRY(launch_fwd_bwd(H, w.theta, w.x, w.t, m, w.grad, w.loss, grid, s));
  VX_CUDA_TRY(cudaMemcpyAsync(theta, w.theta, 4 * (3 * H + 1), cudaMemcpyDeviceToHost, s));
  VX_CUDA_TRY(cudaMemcpyAsync(loss_out, w.loss, 4, cudaMemcpyDeviceToHost, s));
  VX_CUDA_TRY(cudaStreamSynchronize(s));
  return VX_OK;
}
