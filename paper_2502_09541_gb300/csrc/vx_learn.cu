// Learned range partitioner: a monotone CDF MLP (1 -> H -> 1, fp32) trained on
// the device with hand-written forward/backward and Adam kernels, replayed
// from a captured CUDA graph, then inverted by bisection to give integer
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

// dL/dtheta and L over m points; grad/loss are accumulated with atomics
// (caller zeroes them).  theta = [omega(H), beta(H), alpha(H), gamma].
template <int H>
__global__ void __launch_bounds__(kMlpThreads) mlp_fwd_bwd_kernel(const float *__restrict__ theta,
                                                                   const float *__restrict__ x,
                                                                   const float *__restrict__ t, uint64_t m,
                                                                   float *grad, float *loss) {
  __shared__ float w[H], b[H], a[H], dw[H], da[H];
  __shared__ float sg[3 * H + 2];
  for (int j = threadIdx.x; j < H; j += blockDim.x) {
    w[j] = softplusf(theta[j]);
    dw[j] = sigmoidf(theta[j]);
    b[j] = theta[H + j];
    a[j] = softplusf(theta[2 * H + j]);
    da[j] = sigmoidf(theta[2 * H + j]);
  }
  for (int k = threadIdx.x; k < 3 * H + 2; k += blockDim.x) sg[k] = 0.f;
  __syncthreads();
  const float gamma = theta[3 * H];
  const float inv_m = 1.f / (float)m;
  float g_om[H], g_be[H], g_al[H];
#pragma unroll
  for (int j = 0; j < H; ++j) g_om[j] = g_be[j] = g_al[j] = 0.f;
  float g_ga = 0.f, l = 0.f;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < m; i += (uint64_t)gridDim.x * blockDim.x) {
    const float xi = x[i];
    float s[H];
    float y = gamma;
#pragma unroll
    for (int j = 0; j < H; ++j) {
      s[j] = sigmoidf(w[j] * xi + b[j]);
      y += a[j] * s[j];
    }
    const float r = y - t[i];
    l += r * r;
    const float dy = 2.f * r * inv_m;
    g_ga += dy;
#pragma unroll
    for (int j = 0; j < H; ++j) {
      const float ds = s[j] * (1.f - s[j]);
      const float q = dy * a[j] * ds;
      g_be[j] += q;
      g_om[j] += q * xi * dw[j];
      g_al[j] += dy * da[j] * s[j];
    }
  }
  // warp reductions, then one shared atomic per warp and value
  const unsigned lane = threadIdx.x & 31;
#pragma unroll
  for (int j = 0; j < H; ++j) {
    float v0 = g_om[j], v1 = g_be[j], v2 = g_al[j];
    for (int off = 16; off > 0; off >>= 1) {
      v0 += __shfl_down_sync(0xffffffffu, v0, off);
      v1 += __shfl_down_sync(0xffffffffu, v1, off);
      v2 += __shfl_down_sync(0xffffffffu, v2, off);
    }
    if (lane == 0) {
      atomicAdd(&sg[j], v0);
      atomicAdd(&sg[H + j], v1);
      atomicAdd(&sg[2 * H + j], v2);
    }
  }
  for (int off = 16; off > 0; off >>= 1) {
    g_ga += __shfl_down_sync(0xffffffffu, g_ga, off);
    l += __shfl_down_sync(0xffffffffu, l, off);
  }
  if (lane == 0) {
    atomicAdd(&sg[3 * H], g_ga);
    atomicAdd(&sg[3 * H + 1], l);
  }
  __syncthreads();
  for (int k = threadIdx.x; k < 3 * H + 1; k += blockDim.x) atomicAdd(&grad[k], sg[k]);
  if (threadIdx.x == 0) atomicAdd(loss, sg[3 * H + 1] * inv_m);
}

struct AdamState {
  float m1[3 * kMlpMaxH + 1], m2[3 * kMlpMaxH + 1];
  int t;
};

// one Adam step (Kingma & Ba 2015) on n parameters
__global__ void adam_kernel(float *theta, const float *grad, AdamState *st, int n, float lr, float b1, float b2,
                            float eps) {
  __shared__ int step;
  if (threadIdx.x == 0) step = st->t + 1;
  __syncthreads();
  const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    const float g = grad[k];
    const float m1 = b1 * st->m1[k] + (1.f - b1) * g;
    const float m2 = b2 * st->m2[k] + (1.f - b2) * g * g;
    st->m1[k] = m1;
    st->m2[k] = m2;
    theta[k] -= lr * (m1 / c1) / (sqrtf(m2 / c2) + eps);
  }
  __syncthreads();
  if (threadIdx.x == 0) st->t = step;
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
  w.adam = (AdamState *)(p + 4096);
  char *q = p + 4096 + ((sizeof(AdamState) + 255) & ~255ull);
  w.x = (float *)q;
  w.t = (float *)(q + ((4 * M + 255) & ~255ull));
  return VX_OK;
}

static vx_status launch_fwd_bwd(int H, const float *theta, const float *x, const float *t, uint64_t m, float *grad,
                                float *loss, int grid, cudaStream_t s) {
  if (H == 32)
    mlp_fwd_bwd_kernel<32><<<grid, kMlpThreads, 0, s>>>(theta, x, t, m, grad, loss);
  else if (H == 16)
    mlp_fwd_bwd_kernel<16><<<grid, kMlpThreads, 0, s>>>(theta, x, t, m, grad, loss);
  else if (H == 8)
    mlp_fwd_bwd_kernel<8><<<grid, kMlpThreads, 0, s>>>(theta, x, t, m, grad, loss);
  else if (H == 1)
    mlp_fwd_bwd_kernel<1><<<grid, kMlpThreads, 0, s>>>(theta, x, t, m, grad, loss);
  else {
    set_error("MLP width %d not built (1, 8, 16, 32)", H);
    return VX_E_UNSUPPORTED;
  }
  VX_CUDA_TRY(cudaGetLastError());
  return VX_OK;
}

// one training step: zero grad/loss, forward+backward, Adam
static vx_status enqueue_step(int H, MlpWork &w, uint64_t m, float lr, int grid, cudaStream_t s) {
  VX_CUDA_TRY(cudaMemsetAsync(w.grad, 0, 2048, s));  // grad[0..3H] and loss
  VX_TRY(launch_fwd_bwd(H, w.theta, w.x, w.t, m, w.grad, w.loss, grid, s));
  adam_kernel<<<1, 256, 0, s>>>(w.theta, w.grad, w.adam, 3 * H + 1, lr, 0.9f, 0.999f, 1e-8f);
  VX_CUDA_TRY(cudaGetLastError());
  return VX_OK;
}

// trains with `steps` Adam steps; the step is captured once in a CUDA graph
// and replayed
static vx_status train(vx_ctx *ctx, int H, MlpWork &w, uint64_t m, uint32_t steps, float lr) {
  cudaStream_t s = ctx->s_compute;
  const int grid = (int)std::max<uint64_t>(1, std::min<uint64_t>((m + kMlpThreads * 4 - 1) / (kMlpThreads * 4),
                                                                  (uint64_t)ctx->num_sms));
  VX_CUDA_TRY(cudaMemsetAsync(w.adam, 0, sizeof(AdamState), s));
  if (steps == 0) return VX_OK;
  cudaGraph_t g = nullptr;
  cudaGraphExec_t ge = nullptr;
  VX_CUDA_TRY(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
  vx_status st = enqueue_step(H, w, m, lr, grid, s);
  cudaError_t ce = cudaStreamEndCapture(s, &g);
  if (st != VX_OK) {
    if (g) cudaGraphDestroy(g);
    return st;
  }
  VX_CUDA_TRY(ce);
  ce = cudaGraphInstantiate(&ge, g, 0);
  cudaGraphDestroy(g);
  VX_CUDA_TRY(ce);
  for (uint32_t i = 0; i < steps; ++i) {
    ce = cudaGraphLaunch(ge, s);
    if (ce != cudaSuccess) break;
  }
  cudaGraphExecDestroy(ge);
  VX_CUDA_TRY(ce);
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
  const int grid = (int)std::max<uint64_t>(1, std::min<uint64_t>((m + 1023) / 1024, (uint64_t)ctx->num_sms));
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
  const int grid = (int)std::max<uint64_t>(1, std::min<uint64_t>((m + 1023) / 1024, (uint64_t)ctx->num_sms));
  VX_TRY(launch_fwd_bwd(H, w.theta, w.x, w.t, m, w.grad, w.loss, grid, s));
  VX_CUDA_TRY(cudaMemcpyAsync(theta, w.theta, 4 * (3 * H + 1), cudaMemcpyDeviceToHost, s));
  VX_CUDA_TRY(cudaMemcpyAsync(loss_out, w.loss, 4, cudaMemcpyDeviceToHost, s));
  VX_CUDA_TRY(cudaStreamSynchronize(s));
  return VX_OK;
}
