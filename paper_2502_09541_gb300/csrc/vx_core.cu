// Context lifetime, device arena, host column registry, errors, link probe.
#include <algorithm>
#include <cstdarg>
#include <cstdio>

#include "vx_internal.h"

namespace vx {

static thread_local char g_err[1024];

void set_error(const char *fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof g_err, fmt, ap);
  va_end(ap);
}
void clear_error() { g_err[0] = 0; }

double now_ms() {
  using namespace std::chrono;
  return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

// ------------------------------------------------------------------ arena
static constexpr uint64_t kAlign = 256;

void Arena::init(char *base, uint64_t bytes) {
  base_ = base;
  uint64_t b = bytes & ~(kAlign - 1);
  bytes_ = b;
  used_ = 0;
  free_.clear();
  live_.clear();
  if (b) free_[0] = b;
}

void *Arena::alloc(uint64_t bytes) {
  uint64_t need = (bytes + kAlign - 1) & ~(kAlign - 1);
  if (need == 0) need = kAlign;
  for (auto it = free_.begin(); it != free_.end(); ++it) {
    if (it->second >= need) {
      uint64_t off = it->first, sz = it->second;
      free_.erase(it);
      if (sz > need) free_[off + need] = sz - need;
      live_[off] = need;
      used_ += need;
      return base_ + off;
    }
  }
  return nullptr;
}

void Arena::free(void *p) {
  if (!p) return;
  uint64_t off = (uint64_t)((char *)p - base_);
  auto it = live_.find(off);
  if (it == live_.end()) return;
  uint64_t sz = it->second;
  live_.erase(it);
  used_ -= sz;
  auto nx = free_.lower_bound(off);
  if (nx != free_.end() && nx->first == off + sz) {  // merge with next
    sz += nx->second;
    free_.erase(nx);
  }
  auto pv = free_.lower_bound(off);
  if (pv != free_.begin()) {
    --pv;
    if (pv->first + pv->second == off) {  // merge with previous
      pv->second += sz;
      return;
    }
  }
  free_[off] = sz;
}

uint64_t Arena::largest_free() const {
  uint64_t m = 0;
  for (auto &kv : free_) m = kv.second > m ? kv.second : m;
  return m;
}

vx_status check_ctx(vx_ctx *ctx) {
  if (!ctx) {
    set_error("null context");
    return VX_E_INVAL;
  }
  if (ctx->poisoned) {
    set_error("context unusable: device work of an earlier call did not finish within its wait limit");
    return VX_E_TIMEOUT;
  }
  VX_CUDA_TRY(cudaSetDevice(ctx->device));
  return VX_OK;
}

const Column *get_col(vx_ctx *ctx, int32_t id, int32_t want) {
  if (id < 0 || id >= (int32_t)ctx->cols.size() || !ctx->cols[id].live) {
    set_error("invalid column id %d", id);
    return nullptr;
  }
  const Column &c = ctx->cols[id];
  if (want >= 0 && c.dtype != want) {
    set_error("column %d (%s) has dtype %d, expected %d", id, c.name.c_str(), c.dtype, want);
    return nullptr;
  }
  return &c;
}

static void default_config(vx_config *c) {
  memset(c, 0, sizeof *c);
  c->chunk_bytes = 64ull << 20;
  c->n_slots = 3;
  c->sched = VX_SCHED_IMMEDIATE;
  c->late_mat = VX_LATE_AUTO;
  c->zc_threshold = 0.0;
  c->use_graphs = 0;
  c->block_threads = 256;
  c->blocks_per_sm = 4;
  c->wait_timeout_ms = 60000;
}

static vx_status init_common(vx_ctx *ctx) {
  VX_CUDA_TRY(cudaGetDevice(&ctx->device));
  VX_CUDA_TRY(cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, ctx->device));
  int hp = 0;
  VX_CUDA_TRY(cudaDeviceGetAttribute(&hp, cudaDevAttrCanUseHostPointerForRegisteredMem, ctx->device));
  ctx->host_ptr_ok = hp != 0;
  if (!ctx->s_compute) {
    VX_CUDA_TRY(cudaStreamCreateWithFlags(&ctx->s_compute, cudaStreamNonBlocking));
    ctx->own_compute = true;
  }
  VX_CUDA_TRY(cudaStreamCreateWithFlags(&ctx->s_h2d, cudaStreamNonBlocking));
  VX_CUDA_TRY(cudaStreamCreateWithFlags(&ctx->s_d2h, cudaStreamNonBlocking));
  VX_CUDA_TRY(cudaHostAlloc((void **)&ctx->h_scalars, sizeof(uint64_t) * vx_ctx::kScalars,
                            cudaHostAllocMapped));
  memset(ctx->h_scalars, 0, sizeof(uint64_t) * vx_ctx::kScalars);
  VX_CUDA_TRY(cudaHostGetDevicePointer((void **)&ctx->d_scalars, ctx->h_scalars, 0));
  ctx->arena.init(ctx->arena_base, ctx->arena_bytes);
  default_config(&ctx->cfg);
  return VX_OK;
}

vx_status open_child(vx_ctx *parent, uint64_t bytes, vx_ctx **out) {
  *out = nullptr;
  std::unique_ptr<vx_ctx> c(new vx_ctx());
  {
    std::lock_guard<std::recursive_mutex> g(parent->mu);
    c->arena_base = (char *)parent->arena.alloc(bytes);
    if (!c->arena_base) {
      set_error("no room for a %llu-byte operator budget (%llu of %llu bytes free)", (unsigned long long)bytes,
                (unsigned long long)parent->arena.largest_free(), (unsigned long long)parent->arena.capacity());
      return VX_E_NOMEM;
    }
    c->arena_bytes = bytes;
    c->own_arena = false;
    c->cols = parent->cols;
    for (auto &col : c->cols) col.we_registered = false;  // the parent owns the registrations
  }
  vx_status st = init_common(c.get());
  if (st == VX_OK) {
    c->cfg = parent->cfg;
    // staging slots in proportion to the block: at most a sixteenth of it per chunk
    c->cfg.chunk_bytes = std::min<uint64_t>(parent->cfg.chunk_bytes, std::max<uint64_t>(bytes / 16, 1ull << 20));
    c->cfg.use_graphs = 0;
    c->cfg.log_timeline = 0;
    c->cfg.log_chunk_stats = 0;
  }
  if (st != VX_OK) {
    close_child(parent, c.release());
    return st;
  }
  *out = c.release();
  return VX_OK;
}

void close_child(vx_ctx *parent, vx_ctx *child) {
  if (!child) return;
  char *block = child->arena_base;
  const bool leak = child->poisoned && !drain_streams(child);
  if (leak) {  // work still running in the block: neither the block nor the streams are given back
    child->cols.clear();
    delete child;
    return;
  }
  child->arena_base = nullptr;  // borrowed from the parent
  vx_close(child);
  std::lock_guard<std::recursive_mutex> g(parent->mu);
  if (block) parent->arena.free(block);
}

}  // namespace vx

using namespace vx;

VX_API const char *vx_last_error(void) { return g_err; }

VX_API vx_status vx_open(uint64_t budget, vx_ctx **out) {
  clear_error();
  if (!out || budget < (1u << 20)) {
    set_error("vx_open: budget must be >= 1 MiB");
    return VX_E_INVAL;
  }
  std::unique_ptr<vx_ctx> ctx(new vx_ctx());
  void *p = nullptr;
  cudaError_t e = cudaMalloc(&p, budget);
  if (e != cudaSuccess) {
    cudaGetLastError();
    set_error("vx_open: cudaMalloc(%llu) failed: %s", (unsigned long long)budget, cudaGetErrorString(e));
    return VX_E_NOMEM;
  }
  ctx->arena_base = (char *)p;
  ctx->arena_bytes = budget;
  ctx->own_arena = true;
  vx_status st = init_common(ctx.get());
  if (st != VX_OK) {
    vx_close(ctx.release());
    return st;
  }
  *out = ctx.release();
  return VX_OK;
}

VX_API vx_status vx_open_ex(void *dev_arena, uint64_t bytes, void *stream, vx_ctx **out) {
  clear_error();
  if (!out || !dev_arena || bytes < (1u << 20)) {
    set_error("vx_open_ex: need a device arena of >= 1 MiB");
    return VX_E_INVAL;
  }
  std::unique_ptr<vx_ctx> ctx(new vx_ctx());
  ctx->arena_base = (char *)dev_arena;
  ctx->arena_bytes = bytes;
  ctx->own_arena = false;
  ctx->s_compute = (cudaStream_t)stream;
  vx_status st = init_common(ctx.get());
  if (st != VX_OK) {
    vx_close(ctx.release());
    return st;
  }
  *out = ctx.release();
  return VX_OK;
}

VX_API vx_status vx_close(vx_ctx *ctx) {
  if (!ctx) return VX_OK;
  cudaSetDevice(ctx->device);
  serve_shutdown(ctx);  // the engine thread takes the context lock: stop it first
  bool leak = false;
  {
    std::lock_guard<std::recursive_mutex> g(ctx->mu);
    leak = ctx->poisoned && !drain_streams(ctx);
  }
  if (leak) {
    // device work that gave up on its wait is still running: the arena, the
    // page-locked columns and the streams it may use are left as they are
    // (never blocked on); only the host-side context is released
    ctx->graphs.clear();
    ctx->resident.clear();
    ctx->cols.clear();
    delete ctx;
    return VX_E_TIMEOUT;
  }
  {
    std::lock_guard<std::recursive_mutex> g(ctx->mu);
    if (ctx->s_compute) cudaStreamSynchronize(ctx->s_compute);
    if (ctx->s_h2d) cudaStreamSynchronize(ctx->s_h2d);
    if (ctx->s_d2h) cudaStreamSynchronize(ctx->s_d2h);
    ctx->graphs.clear();
    ctx->resident.clear();
    for (auto &c : ctx->cols)
      if (c.live && c.we_registered) cudaHostUnregister((void *)c.host);
    ctx->cols.clear();
    if (ctx->h_scalars) cudaFreeHost(ctx->h_scalars);
    if (ctx->op_host) cudaFreeHost(ctx->op_host);
    if (ctx->own_compute && ctx->s_compute) cudaStreamDestroy(ctx->s_compute);
    if (ctx->s_h2d) cudaStreamDestroy(ctx->s_h2d);
    if (ctx->s_d2h) cudaStreamDestroy(ctx->s_d2h);
    if (ctx->own_arena && ctx->arena_base) cudaFree(ctx->arena_base);
  }
  delete ctx;
  return VX_OK;
}

VX_API vx_status vx_get_config(vx_ctx *ctx, vx_config *out) {
  if (!ctx || !out) return VX_E_INVAL;
  *out = ctx->cfg;
  return VX_OK;
}

VX_API vx_status vx_set_config(vx_ctx *ctx, const vx_config *cfg) {
  clear_error();
  if (!ctx || !cfg) return VX_E_INVAL;
  if (cfg->n_slots < 2 || cfg->n_slots > 16 || cfg->chunk_bytes < 4096 || cfg->block_threads < 64 ||
      cfg->block_threads > 1024 || (cfg->block_threads & 31) || cfg->blocks_per_sm < 1 ||
      cfg->blocks_per_sm > 32 || (cfg->sched != VX_SCHED_IMMEDIATE && cfg->sched != VX_SCHED_DAG) ||
      cfg->wait_timeout_ms == 0 || cfg->zc_threshold < 0 || cfg->zc_threshold > 1 ||
      (cfg->kernel_rows != 0 && cfg->kernel_rows != 2 && cfg->kernel_rows != 8 && cfg->kernel_rows != 16) ||
      cfg->h2d_copy_blocks < 0 || cfg->h2d_copy_blocks > 1024 || cfg->reserved != 0) {
    set_error("vx_set_config: value out of range");
    return VX_E_INVAL;
  }
  std::lock_guard<std::recursive_mutex> g(ctx->mu);
  if (memcmp(&ctx->cfg, cfg, sizeof *cfg) != 0) {
    cudaStreamSynchronize(ctx->s_compute);
    ctx->graphs.clear();  // captured pipelines follow the old chunking and launch shape
  }
  ctx->cfg = *cfg;
  return VX_OK;
}

VX_API vx_status vx_register_host_column(vx_ctx *ctx, const char *name, int32_t dtype, const void *host,
                                         uint64_t n_rows, uint32_t flags, int32_t *col_id) {
  clear_error();
  VX_TRY(check_ctx(ctx));
  if (!col_id || (dtype < VX_I32 || dtype > VX_U64) || (!host && n_rows) || flags != 0) {
    set_error("vx_register_host_column: bad argument");
    return VX_E_INVAL;
  }
  std::lock_guard<std::recursive_mutex> g(ctx->mu);
  Column c;
  c.name = name ? name : "";
  c.dtype = dtype;
  c.elem = dtype_size(dtype);
  c.host = host;
  c.n_rows = n_rows;
  c.live = true;
  uint64_t bytes = n_rows * c.elem;
  if (bytes) {
    cudaPointerAttributes at{};
    cudaError_t e = cudaPointerGetAttributes(&at, host);
    bool pinned = (e == cudaSuccess && at.type == cudaMemoryTypeHost);
    cudaGetLastError();
    if (!pinned) {
      e = cudaHostRegister((void *)host, bytes, cudaHostRegisterMapped);
      if (e != cudaSuccess) {
        cudaGetLastError();
        set_error("cudaHostRegister(%llu bytes) failed: %s", (unsigned long long)bytes, cudaGetErrorString(e));
        return VX_E_CUDA;
      }
      c.we_registered = true;
    }
    void *dp = nullptr;
    e = cudaHostGetDevicePointer(&dp, (void *)host, 0);
    if (e != cudaSuccess) {
      cudaGetLastError();
      if (c.we_registered) cudaHostUnregister((void *)host);
      set_error("cudaHostGetDevicePointer failed: %s", cudaGetErrorString(e));
      return VX_E_CUDA;
    }
    c.dev = dp;
  }
  ctx->cols.push_back(c);
  *col_id = (int32_t)ctx->cols.size() - 1;
  return VX_OK;
}

VX_API vx_status vx_unregister_host_column(vx_ctx *ctx, int32_t col_id) {
  clear_error();
  VX_TRY(check_ctx(ctx));
  std::lock_guard<std::recursive_mutex> g(ctx->mu);
  if (!get_col(ctx, col_id, -1)) return VX_E_INVAL;
  Column &c = ctx->cols[col_id];
  cudaStreamSynchronize(ctx->s_compute);
  cudaStreamSynchronize(ctx->s_h2d);
  ctx->graphs.clear();  // captured pipelines and cached tables may refer to the column
  ctx->resident.clear();
  if (c.we_registered) cudaHostUnregister((void *)c.host);
  c.live = false;
  return VX_OK;
}

VX_API vx_status vx_drop_resident(vx_ctx *ctx) {
  clear_error();
  VX_TRY(check_ctx(ctx));
  std::lock_guard<std::recursive_mutex> g(ctx->mu);
  VX_CUDA_TRY(cudaStreamSynchronize(ctx->s_compute));
  ctx->graphs.clear();
  ctx->resident.clear();
  return VX_OK;
}

VX_API vx_status vx_last_stats(vx_ctx *ctx, vx_query_stats *out) {
  if (!ctx || !out) return VX_E_INVAL;
  *out = ctx->last;
  return VX_OK;
}

VX_API vx_status vx_last_timeline(vx_ctx *ctx, float *out, uint64_t cap, uint64_t *n) {
  clear_error();
  if (!ctx || !n || (cap && !out)) {
    set_error("vx_last_timeline: bad argument");
    return VX_E_INVAL;
  }
  std::lock_guard<std::recursive_mutex> g(ctx->mu);
  const uint64_t rows = ctx->timeline.size() / VX_TIMELINE_COLS;
  *n = rows;
  if (cap) memcpy(out, ctx->timeline.data(), sizeof(float) * VX_TIMELINE_COLS * std::min(cap, rows));
  return VX_OK;
}

// ------------------------------------------------------------------ zero-copy probe
// The Section 6.3 micro-benchmark: sum += pred[i % npred] % SEL == 0 ? v[i] : 0
// with pred in device memory and v in host memory, read either through mapped
// host memory (zero-copy) or after a copy-engine transfer into HBM.
namespace vx {
__global__ void zc_probe_kernel(const int *__restrict__ pred, uint64_t npred, const int *__restrict__ v, uint64_t n,
                                uint64_t v_off, int sel, unsigned long long *out) {
  unsigned long long s = 0;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t g = v_off + i;
    if (pred[g % npred] % sel == 0) s += (unsigned)v[i];
  }
  for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
  if ((threadIdx.x & 31) == 0 && s) atomicAdd(out, s);
}
__global__ void zc_fill_pred_kernel(int *p, uint64_t n) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
    uint64_t x = (i + 1) * 0x9E3779B97F4A7C15ull;
    x ^= x >> 31;
    x *= 0xBF58476D1CE4E5B9ull;
    x ^= x >> 29;
    p[i] = (int)(x & 0x7fffffff);
  }
}
// one 4-byte read of mapped host memory per index, summed (the access of the
// late-materialization gather without its aggregation)
__global__ void zc_gather_probe_kernel(const int *__restrict__ host, const uint32_t *__restrict__ idx, uint32_t n,
                                       unsigned long long *out) {
  unsigned long long s = 0;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    s += (unsigned)host[idx[i]];
  for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
  if ((threadIdx.x & 31) == 0 && s) atomicAdd(out, s);
}
}  // namespace vx

VX_API vx_status vx_probe_zero_copy_gather(vx_ctx *ctx, uint64_t window_bytes, uint32_t n_reads, uint64_t seed,
                                           double *us_first, double *us_warm, uint64_t *checksum) {
  clear_error();
  VX_TRY(check_ctx(ctx));
  if (window_bytes < 4 || window_bytes / 4 > 0xFFFFFFFFull || n_reads == 0 || !us_first || !us_warm) {
    set_error("vx_probe_zero_copy_gather: bad argument");
    return VX_E_INVAL;
  }
  std::lock_guard<std::recursive_mutex> g(ctx->mu);
  const uint64_t n_int = window_bytes / 4;
  DevBuf ib, ob;
  ib.arena = ob.arena = &ctx->arena;
  ib.p = ctx->arena.alloc(4ull * n_reads);
  ob.p = ctx->arena.alloc(256);
  if (!ib.p || !ob.p) {
    set_error("vx_probe_zero_copy_gather: %u indices do not fit the arena", n_reads);
    return VX_E_NOMEM;
  }
  int *hv = nullptr, *dv = nullptr;
  VX_CUDA_TRY(cudaHostAlloc((void **)&hv, 4 * n_int, cudaHostAllocMapped));
  struct FreeHost {
    void *p;
    ~FreeHost() { cudaFreeHost(p); }
  } fh{hv};
  for (uint64_t i = 0; i < n_int; ++i) hv[i] = (int)(i & 1023);
  VX_CUDA_TRY(cudaHostGetDevicePointer((void **)&dv, hv, 0));
  // sorted uniform indices over the window (a survivor list is in row order
  // within each tile); SplitMix64 of seed + i, reduced by multiply-shift
  std::vector<uint32_t> idx(n_reads);
  uint64_t expect = 0;
  for (uint32_t i = 0; i < n_reads; ++i) {
    uint64_t z = seed + 0x9E3779B97F4A7C15ull * (i + 1);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    idx[i] = (uint32_t)(((unsigned __int128)z * n_int) >> 64);
  }
  std::sort(idx.begin(), idx.end());
  for (uint32_t i = 0; i < n_reads; ++i) expect += (uint64_t)(idx[i] & 1023);
  cudaStream_t s = ctx->s_compute;
  VX_CUDA_TRY(cudaMemcpyAsync(ib.p, idx.data(), 4ull * n_reads, cudaMemcpyHostToDevice, s));
  unsigned long long *out = ob.as<unsigned long long>();
  cudaEvent_t e0, e1;
  VX_CUDA_TRY(cudaEventCreate(&e0));
  VX_CUDA_TRY(cudaEventCreate(&e1));
  struct Ev {
    cudaEvent_t a, b;
    ~Ev() {
      cudaEventDestroy(a);
      cudaEventDestroy(b);
    }
  } ev{e0, e1};
  double best = 1e300;
  for (int r = 0; r < 4; ++r) {  // the first launch touches the window's pages for the first time
    VX_CUDA_TRY(cudaMemsetAsync(out, 0, 8, s));
    VX_CUDA_TRY(cudaEventRecord(e0, s));
    zc_gather_probe_kernel<<<ctx->num_sms * 4, 256, 0, s>>>(dv, ib.as<uint32_t>(), n_reads, out);
    VX_CUDA_TRY(cudaGetLastError());
    VX_CUDA_TRY(cudaEventRecord(e1, s));
    VX_CUDA_TRY(cudaEventSynchronize(e1));
    float ms = 0;
    VX_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
    if (r == 0) *us_first = 1000.0 * ms;
    else best = std::min(best, 1000.0 * (double)ms);
    uint64_t got = 0;
    VX_CUDA_TRY(cudaMemcpy(&got, out, 8, cudaMemcpyDeviceToHost));
    if (got != expect) {
      set_error("vx_probe_zero_copy_gather: sum %llu, expected %llu", (unsigned long long)got,
                (unsigned long long)expect);
      return VX_E_CUDA;
    }
  }
  *us_warm = best;
  if (checksum) *checksum = expect;
  return VX_OK;
}

VX_API vx_status vx_probe_zero_copy(vx_ctx *ctx, uint64_t n, const int32_t *sels, int32_t n_sel, double *ms_zero_copy,
                                    double *ms_copy, uint64_t *checksums) {
  clear_error();
  VX_TRY(check_ctx(ctx));
  if (!n || !sels || n_sel < 1 || !ms_zero_copy || !ms_copy) {
    set_error("vx_probe_zero_copy: bad argument");
    return VX_E_INVAL;
  }
  for (int k = 0; k < n_sel; ++k)
    if (sels[k] < 1) {
      set_error("vx_probe_zero_copy: SEL must be >= 1");
      return VX_E_INVAL;
    }
  std::lock_guard<std::recursive_mutex> g(ctx->mu);
  const uint64_t npred = std::min<uint64_t>(n, 16ull << 20);
  const uint64_t chunk = 16ull << 20;  // ints per copy chunk (64 MiB)
  DevBuf pb, cb, ob;
  pb.arena = cb.arena = ob.arena = &ctx->arena;
  pb.p = ctx->arena.alloc(4 * npred);
  cb.p = ctx->arena.alloc(2 * 4 * chunk);
  ob.p = ctx->arena.alloc(256);
  if (!pb.p || !cb.p || !ob.p) {
    set_error("vx_probe_zero_copy: %llu bytes do not fit the arena", (unsigned long long)(4 * npred + 8 * 4 * chunk));
    return VX_E_NOMEM;
  }
  int *hv = nullptr, *dv = nullptr;
  VX_CUDA_TRY(cudaHostAlloc((void **)&hv, 4 * n, cudaHostAllocMapped));
  struct FreeHost {
    void *p;
    ~FreeHost() { cudaFreeHost(p); }
  } fh{hv};
  for (uint64_t i = 0; i < n; ++i) hv[i] = (int)(i & 1023);
  VX_CUDA_TRY(cudaHostGetDevicePointer((void **)&dv, hv, 0));
  cudaStream_t s = ctx->s_compute;
  zc_fill_pred_kernel<<<ctx->num_sms * 4, 256, 0, s>>>(pb.as<int>(), npred);
  unsigned long long *out = ob.as<unsigned long long>();
  cudaEvent_t e0, e1, ec[2], ek[2];
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  for (int i = 0; i < 2; ++i) {
    cudaEventCreateWithFlags(&ec[i], cudaEventDisableTiming);
    cudaEventCreateWithFlags(&ek[i], cudaEventDisableTiming);
  }
  const int grid = ctx->num_sms * 8;
  for (int k = 0; k < n_sel; ++k) {
    // zero-copy: the kernel reads v through mapped host memory
    VX_CUDA_TRY(cudaMemsetAsync(out, 0, 8, s));
    cudaEventRecord(e0, s);
    zc_probe_kernel<<<grid, 256, 0, s>>>(pb.as<int>(), npred, dv, n, 0, sels[k], out);
    cudaEventRecord(e1, s);
    VX_CUDA_TRY(cudaEventSynchronize(e1));
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    ms_zero_copy[k] = ms;
    unsigned long long zc_sum = 0;
    VX_CUDA_TRY(cudaMemcpy(&zc_sum, out, 8, cudaMemcpyDeviceToHost));
    // copy engine: double-buffered 64 MiB chunks into HBM, same kernel on HBM
    VX_CUDA_TRY(cudaMemsetAsync(out, 0, 8, s));
    VX_CUDA_TRY(cudaStreamSynchronize(s));
    cudaEventRecord(e0, s);
    cudaEventRecord(ek[0], s);
    cudaEventRecord(ek[1], s);
    for (uint64_t off = 0, c = 0; off < n; off += chunk, ++c) {
      const uint64_t m = std::min(chunk, n - off);
      int *buf = cb.as<int>() + (c & 1) * chunk;
      cudaStreamWaitEvent(ctx->s_h2d, ek[c & 1], 0);
      cudaMemcpyAsync(buf, hv + off, 4 * m, cudaMemcpyHostToDevice, ctx->s_h2d);
      cudaEventRecord(ec[c & 1], ctx->s_h2d);
      cudaStreamWaitEvent(s, ec[c & 1], 0);
      zc_probe_kernel<<<grid, 256, 0, s>>>(pb.as<int>(), npred, buf, m, off, sels[k], out);
      cudaEventRecord(ek[c & 1], s);
    }
    cudaEventRecord(e1, s);
    VX_CUDA_TRY(cudaEventSynchronize(e1));
    cudaEventElapsedTime(&ms, e0, e1);
    ms_copy[k] = ms;
    unsigned long long ce_sum = 0;
    VX_CUDA_TRY(cudaMemcpy(&ce_sum, out, 8, cudaMemcpyDeviceToHost));
    if (ce_sum != zc_sum) {
      set_error("vx_probe_zero_copy: the two reads disagree");
      return VX_E_CUDA;
    }
    if (checksums) checksums[k] = zc_sum;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  for (int i = 0; i < 2; ++i) {
    cudaEventDestroy(ec[i]);
    cudaEventDestroy(ek[i]);
  }
  VX_CUDA_TRY(cudaGetLastError());
  return VX_OK;
}

// ------------------------------------------------------------------ random-read probe
namespace {
__device__ __forceinline__ uint64_t rr_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// read i goes to bucket mix(i) mapped onto [0, nbk) by multiply-shift
__global__ void __launch_bounds__(256) rand_read_kernel(const ulonglong2 *__restrict__ t, uint64_t nbk, uint64_t n,
                                                        unsigned long long *sink) {
  constexpr int kR = 8;
  unsigned long long x = 0;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x * kR;
  for (uint64_t i = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) * kR; i < n; i += stride) {
    ulonglong2 v[kR];
#pragma unroll
    for (int j = 0; j < kR; ++j) v[j] = i + j < n ? __ldg(t + 2 * __umul64hi(rr_mix(i + j), nbk)) : make_ulonglong2(0, 0);
#pragma unroll
    for (int j = 0; j < kR; ++j) x ^= v[j].x;
  }
  if (x == 0x5EEDull) atomicAdd(sink, 1ull);  // keeps the reads live
}
}  // namespace

VX_API vx_status vx_probe_hbm_random(vx_ctx *ctx, uint64_t table_bytes, uint64_t n_reads, double *g_reads_per_s) {
  clear_error();
  VX_TRY(check_ctx(ctx));
  if (table_bytes < 32 || !n_reads || !g_reads_per_s) {
    set_error("vx_probe_hbm_random: need table_bytes >= 32, n_reads > 0 and an output");
    return VX_E_INVAL;
  }
  std::lock_guard<std::recursive_mutex> g(ctx->mu);
  const uint64_t nbk = table_bytes / 32;
  DevBuf tb;
  tb.arena = &ctx->arena;
  tb.p = ctx->arena.alloc(nbk * 32 + 256);
  if (!tb.p) {
    set_error("vx_probe_hbm_random: %llu bytes do not fit the arena", (unsigned long long)table_bytes);
    return VX_E_NOMEM;
  }
  unsigned long long *sink = (unsigned long long *)(tb.as<char>() + nbk * 32);
  cudaStream_t s = ctx->s_compute;
  VX_CUDA_TRY(cudaMemsetAsync(tb.p, 0, nbk * 32 + 256, s));
  int occ = 0;
  VX_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, rand_read_kernel, 256, 0));
  const int grid = std::max(1, occ) * ctx->num_sms;
  cudaEvent_t e0, e1;
  VX_CUDA_TRY(cudaEventCreate(&e0));
  VX_CUDA_TRY(cudaEventCreate(&e1));
  float best = 0;
  for (int it = 0; it < 4; ++it) {  // the first run warms up
    cudaEventRecord(e0, s);
    rand_read_kernel<<<grid, 256, 0, s>>>(tb.as<ulonglong2>(), nbk, n_reads, sink);
    cudaEventRecord(e1, s);
    cudaEventSynchronize(e1);
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    if (it && (best == 0 || ms < best)) best = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaError_t le = cudaGetLastError();
  if (le != cudaSuccess) {
    set_error("vx_probe_hbm_random: %s", cudaGetErrorString(le));
    return VX_E_CUDA;
  }
  *g_reads_per_s = best > 0 ? (double)n_reads / (best * 1e6) : 0.0;
  return VX_OK;
}

// ------------------------------------------------------------------ streaming probe
namespace {
// plain coalesced read of n16 16-byte values: four independent loads in
// flight per thread, one 1024-value tile per block
__global__ void __launch_bounds__(256) stream_read_kernel(const int4 *__restrict__ p, uint64_t n16,
                                                          unsigned long long *sink) {
  const uint64_t base = (uint64_t)blockIdx.x * 1024 + threadIdx.x;
  int4 v[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) v[j] = base + j * 256 < n16 ? __ldg(p + base + j * 256) : make_int4(0, 0, 0, 0);
  int x = 0;
#pragma unroll
  for (int j = 0; j < 4; ++j) x ^= v[j].x ^ v[j].y ^ v[j].z ^ v[j].w;
  if (x == 0x5EED5EED) atomicAdd(sink, 1ull);  // keeps the reads live
}
}  // namespace

// one coalesced read of `bytes` right after their host-to-device copy, timed
// with events on the compute stream (median of reps launches after one
// warm-up); with copy_bytes > 0 a copy of copy_bytes from pinned host memory
// into another device buffer is in flight on the host-to-device stream while
// the read runs, as the next chunk's copy is while a chunk's kernel runs
static vx_status probe_stream(vx_ctx *ctx, uint64_t bytes, int32_t reps, uint64_t copy_bytes, double *gbs,
                              const char *who) {
  clear_error();
  VX_TRY(check_ctx(ctx));
  if (bytes < 16 || reps < 1 || !gbs) {
    set_error("%s: need bytes >= 16, reps >= 1 and an output", who);
    return VX_E_INVAL;
  }
  std::lock_guard<std::recursive_mutex> g(ctx->mu);
  const uint64_t n16 = bytes / 16;
  bytes = n16 * 16;
  const uint64_t lead = copy_bytes ? std::min<uint64_t>(copy_bytes, 4ull << 20) : 0;  // starts the copy engine
  DevBuf db, cb;
  db.arena = cb.arena = &ctx->arena;
  db.p = ctx->arena.alloc(bytes + 256);
  if (copy_bytes) cb.p = ctx->arena.alloc(copy_bytes);
  if (!db.p || (copy_bytes && !cb.p)) {
    set_error("%s: %llu + %llu bytes do not fit the arena", who, (unsigned long long)bytes,
              (unsigned long long)copy_bytes);
    return VX_E_NOMEM;
  }
  unsigned long long *sink = (unsigned long long *)(db.as<char>() + bytes);
  char *hs = nullptr;
  VX_CUDA_TRY(cudaHostAlloc((void **)&hs, std::max(bytes, copy_bytes), cudaHostAllocDefault));
  memset(hs, 3, std::max(bytes, copy_bytes));
  cudaStream_t s = ctx->s_compute, sc = ctx->s_h2d;
  cudaEvent_t e0 = nullptr, e1 = nullptr, ec = nullptr;
  std::vector<float> t;
  cudaError_t ce = cudaEventCreate(&e0);
  if (ce == cudaSuccess) ce = cudaEventCreate(&e1);
  if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&ec, cudaEventDisableTiming);
  if (ce == cudaSuccess) ce = cudaMemsetAsync(sink, 0, 8, s);
  const uint64_t grid = (n16 + 1023) / 1024;
  for (int it = 0; ce == cudaSuccess && it <= reps; ++it) {  // the first launch warms up
    // the bytes arrive by copy engine first, as a staged chunk does
    ce = cudaMemcpyAsync(db.p, hs, bytes, cudaMemcpyHostToDevice, s);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
    if (ce == cudaSuccess && copy_bytes) {
      // a short lead copy, then the long one: the read starts once the lead
      // has landed, with the long copy streaming behind it
      ce = cudaMemcpyAsync(cb.p, hs, lead, cudaMemcpyHostToDevice, sc);
      if (ce == cudaSuccess) ce = cudaEventRecord(ec, sc);
      if (ce == cudaSuccess && copy_bytes > lead)
        ce = cudaMemcpyAsync(cb.as<char>() + lead, hs + lead, copy_bytes - lead, cudaMemcpyHostToDevice, sc);
      if (ce == cudaSuccess) ce = cudaStreamWaitEvent(s, ec, 0);
    }
    if (ce == cudaSuccess) ce = cudaEventRecord(e0, s);
    if (ce == cudaSuccess) {
      stream_read_kernel<<<(unsigned)std::min<uint64_t>(grid, 1u << 30), 256, 0, s>>>(db.as<int4>(), n16, sink);
      ce = cudaGetLastError();
    }
    if (ce == cudaSuccess) ce = cudaEventRecord(e1, s);
    if (ce == cudaSuccess) ce = cudaEventSynchronize(e1);
    if (ce == cudaSuccess && copy_bytes) ce = cudaStreamSynchronize(sc);
    float ms = 0;
    if (ce == cudaSuccess) ce = cudaEventElapsedTime(&ms, e0, e1);
    if (ce == cudaSuccess && it) t.push_back(ms);
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (ec) cudaEventDestroy(ec);
  cudaFreeHost(hs);
  VX_CUDA_TRY(ce);
  std::sort(t.begin(), t.end());
  const float med = t[t.size() / 2];
  *gbs = med > 0 ? (double)bytes / (med * 1e6) : 0.0;
  return VX_OK;
}

VX_API vx_status vx_probe_stream(vx_ctx *ctx, uint64_t bytes, int32_t reps, double *gbs) {
  return probe_stream(ctx, bytes, reps, 0, gbs, "vx_probe_stream");
}

VX_API vx_status vx_probe_stream_copying(vx_ctx *ctx, uint64_t bytes, int32_t reps, uint64_t copy_bytes,
                                         double *gbs) {
  if (copy_bytes < 16) {
    clear_error();
    set_error("vx_probe_stream_copying: need copy_bytes >= 16");
    return VX_E_INVAL;
  }
  return probe_stream(ctx, bytes, reps, copy_bytes, gbs, "vx_probe_stream_copying");
}

// ------------------------------------------------------------------ link probe
VX_API vx_status vx_probe_link(vx_ctx *ctx, uint64_t bytes, uint64_t chunk, double *h2d, double *d2h,
                               double *bidir) {
  clear_error();
  VX_TRY(check_ctx(ctx));
  if (!bytes || !chunk || chunk > bytes) {
    set_error("vx_probe_link: need 0 < chunk <= bytes");
    return VX_E_INVAL;
  }
  std::lock_guard<std::recursive_mutex> g(ctx->mu);
  bytes = bytes / chunk * chunk;
  DevBuf a, b;
  a.arena = b.arena = &ctx->arena;
  a.p = ctx->arena.alloc(bytes);
  b.p = ctx->arena.alloc(bytes);
  if (!a.p || !b.p) {
    set_error("vx_probe_link: %llu bytes x2 do not fit the arena", (unsigned long long)bytes);
    return VX_E_NOMEM;
  }
  char *hs = nullptr, *hd = nullptr;
  VX_CUDA_TRY(cudaHostAlloc((void **)&hs, bytes, cudaHostAllocDefault));
  cudaError_t e = cudaHostAlloc((void **)&hd, bytes, cudaHostAllocDefault);
  if (e != cudaSuccess) {
    cudaFreeHost(hs);
    VX_CUDA_TRY(e);
  }
  memset(hs, 1, bytes);
  memset(hd, 2, bytes);
  cudaEvent_t e0, e1, eh, ed;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventCreate(&eh);
  cudaEventCreate(&ed);
  double res[3] = {0, 0, 0};
  for (int warm = 0; warm < 2; ++warm) {
    for (int dir = 0; dir < 3; ++dir) {
      cudaStreamSynchronize(ctx->s_h2d);
      cudaStreamSynchronize(ctx->s_d2h);
      cudaEventRecord(e0, ctx->s_h2d);
      cudaStreamWaitEvent(ctx->s_d2h, e0, 0);
      for (uint64_t off = 0; off < bytes; off += chunk) {
        if (dir != 1) cudaMemcpyAsync((char *)a.p + off, hs + off, chunk, cudaMemcpyHostToDevice, ctx->s_h2d);
        if (dir != 0) cudaMemcpyAsync(hd + off, (char *)b.p + off, chunk, cudaMemcpyDeviceToHost, ctx->s_d2h);
      }
      cudaEventRecord(ed, ctx->s_d2h);
      cudaStreamWaitEvent(ctx->s_h2d, ed, 0);
      cudaEventRecord(e1, ctx->s_h2d);
      cudaEventSynchronize(e1);
      float ms = 0;
      cudaEventElapsedTime(&ms, e0, e1);
      res[dir] = (double)bytes * (dir == 2 ? 2 : 1) / (ms * 1e6);
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaEventDestroy(eh);
  cudaEventDestroy(ed);
  cudaFreeHost(hs);
  cudaFreeHost(hd);
  cudaError_t le = cudaGetLastError();
  if (le != cudaSuccess) {
    set_error("vx_probe_link: %s", cudaGetErrorString(le));
    return VX_E_CUDA;
  }
  if (h2d) *h2d = res[0];
  if (d2h) *d2h = res[1];
  if (bidir) *bidir = res[2];
  return VX_OK;
}
