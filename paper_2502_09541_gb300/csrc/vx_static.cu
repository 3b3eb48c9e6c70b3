// Allocation-free variant of the ordered filter (vx_filter_device_static).
//
// Some callers cannot let a library allocate device memory: code that runs
// inside another framework's memory manager, which owns all device memory and
// hands out only the input and output buffers of each call, and
// latency-critical paths where a cudaMalloc or cudaFree (which may synchronise
// the device) is not acceptable.  For them this entry point keeps its scratch
// — per-tile survivor counts, their exclusive prefix and the total — in one
// file-scope __device__ array of fixed size instead of an arena.  Every GPU
// that loads the library holds that array (kStaticScratchWords 32-bit words,
// 256 KiB + 256 B) until the process exits.
//
// Host code must not pass the array's name to a kernel: on the host the name
// is a stand-in object, not a device address, and a kernel given it would
// fault or, where the GPU can reach host memory, silently use the wrong
// memory.  The device address is looked up once per device with
// cudaGetSymbolAddress (with that device current) and passed to the kernels.
#include <mutex>

#include "vx_internal.h"

namespace vx {

constexpr uint64_t kStaticMaxRows = 1ull << 26;  // rows per call (67,108,864)
constexpr int kSfThreads = 256;
constexpr int kSfItems = 8;
constexpr int kSfTile = kSfThreads * kSfItems;  // rows per tile
constexpr uint32_t kStaticMaxTiles = (uint32_t)(kStaticMaxRows / kSfTile);  // 32,768
constexpr uint32_t kStaticScratchWords = 2 * kStaticMaxTiles + 64;  // counts | offsets | total

// Shared by every call on a device; holds the last call's contents.  Each
// call writes every word it reads before reading it (counts, then offsets and
// the total), so nothing has to be cleared between calls.
static __device__ __align__(256) uint32_t g_filter_scratch[kStaticScratchWords];

namespace {

struct SfParams {
  int n_preds;
  const int32_t *col[VX_MAX_PREDS];
  int32_t op[VX_MAX_PREDS], lo[VX_MAX_PREDS], hi[VX_MAX_PREDS];
  uint64_t row0, n, cap;
};

__device__ __forceinline__ bool sf_pred(int32_t v, int32_t op, int32_t lo, int32_t hi) {
  switch (op) {
    case VX_BETWEEN: return lo <= v && v <= hi;
    case VX_EQ: return v == lo;
    case VX_NE: return v != lo;
    case VX_LT: return v < lo;
    case VX_LE: return v <= lo;
    case VX_GT: return v > lo;
    case VX_GE: return v >= lo;
  }
  return false;
}

__device__ __forceinline__ bool sf_row(const SfParams &p, uint64_t i) {
  for (int q = 0; q < p.n_preds; ++q)
    if (!sf_pred(__ldg(&p.col[q][i]), p.op[q], p.lo[q], p.hi[q])) return false;
  return true;
}

// scratch layout: counts [0, kStaticMaxTiles), offsets [kStaticMaxTiles, 2*kStaticMaxTiles),
// total (two words, low first) at 2*kStaticMaxTiles
__global__ void __launch_bounds__(kSfThreads) sf_count_kernel(const SfParams p, uint32_t *scratch) {
  const uint64_t t0 = (uint64_t)blockIdx.x * kSfTile;
  uint32_t c = 0;
  for (int k = 0; k < kSfItems; ++k) {
    const uint64_t i = t0 + (uint64_t)k * kSfThreads + threadIdx.x;
    if (i < p.n) c += sf_row(p, i);
  }
  c = __reduce_add_sync(0xffffffffu, c);
  __shared__ uint32_t ws[kSfThreads / 32];
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t s = 0;
    for (int w = 0; w < kSfThreads / 32; ++w) s += ws[w];
    scratch[blockIdx.x] = s;
  }
}

__global__ void __launch_bounds__(1024) sf_scan_kernel(uint32_t n_tiles, uint32_t *scratch) {
  __shared__ uint32_t wsum[32];
  __shared__ uint32_t carry;
  const uint32_t *cnt = scratch;
  uint32_t *off = scratch + kStaticMaxTiles;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (uint32_t base = 0; base < n_tiles; base += blockDim.x) {
    const uint32_t i = base + threadIdx.x;
    const uint32_t v = i < n_tiles ? cnt[i] : 0;
    uint32_t x = v;
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if ((threadIdx.x & 31) >= (unsigned)o) x += y;
    }
    if ((threadIdx.x & 31) == 31) wsum[threadIdx.x >> 5] = x;
    __syncthreads();
    if (threadIdx.x < 32) {
      uint32_t w = wsum[threadIdx.x];
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
        if (threadIdx.x >= (unsigned)o) w += y;
      }
      wsum[threadIdx.x] = w;
    }
    __syncthreads();
    const uint32_t wpre = (threadIdx.x >> 5) ? wsum[(threadIdx.x >> 5) - 1] : 0;
    if (i < n_tiles) off[i] = carry + wpre + x - v;
    __syncthreads();
    if (threadIdx.x == 0) carry += wsum[31];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    scratch[2 * kStaticMaxTiles] = carry;
    scratch[2 * kStaticMaxTiles + 1] = 0;
  }
}

// ordered write of the ascending row ids; ids at positions >= cap are dropped
__global__ void __launch_bounds__(kSfThreads) sf_write_kernel(const SfParams p, const uint32_t *scratch,
                                                              uint64_t *out) {
  __shared__ uint32_t wcnt[kSfThreads / 32];
  const uint64_t t0 = (uint64_t)blockIdx.x * kSfTile;
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint64_t running = scratch[kStaticMaxTiles + blockIdx.x];
  for (int k = 0; k < kSfItems; ++k) {
    const uint64_t i = t0 + (uint64_t)k * kSfThreads + threadIdx.x;
    const bool keep = i < p.n && sf_row(p, i);
    const uint32_t bal = __ballot_sync(0xffffffffu, keep);
    if (lane == 0) wcnt[warp] = __popc(bal);
    __syncthreads();
    uint32_t before = 0, total = 0;
    for (uint32_t w = 0; w < kSfThreads / 32; ++w) {
      const uint32_t c = wcnt[w];
      before += w < warp ? c : 0;
      total += c;
    }
    const uint64_t pos = running + before + __popc(bal & ((1u << lane) - 1u));
    if (keep && pos < p.cap) out[pos] = p.row0 + i;
    running += total;
    __syncthreads();
  }
}

// device address of g_filter_scratch, looked up once per device
std::mutex g_addr_mu;
uint32_t *g_addr[64] = {};

vx_status scratch_address(uint32_t **out) {
  int dev = 0;
  VX_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) {
    set_error("vx_filter_device_static: device ordinal %d out of range", dev);
    return VX_E_UNSUPPORTED;
  }
  std::lock_guard<std::mutex> g(g_addr_mu);
  if (!g_addr[dev]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_filter_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      set_error("vx_filter_device_static: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
      return VX_E_CUDA;
    }
    g_addr[dev] = (uint32_t *)p;
  }
  *out = g_addr[dev];
  return VX_OK;
}

}  // namespace
}  // namespace vx

using namespace vx;

VX_API vx_status vx_filter_device_static(const int32_t *const *cols, int32_t n_cols, const vx_pred *preds,
                                         int32_t n_preds, uint64_t n_rows, uint64_t row0, uint64_t *out_rows,
                                         uint64_t cap, uint64_t *out_count, void *stream) {
  clear_error();
  if (!cols || !preds || !out_count || n_cols < 1 || n_preds < 1 || n_preds > VX_MAX_PREDS || (cap && !out_rows)) {
    set_error("vx_filter_device_static: bad argument");
    return VX_E_INVAL;
  }
  if (n_rows > kStaticMaxRows) {
    set_error("vx_filter_device_static: %llu rows exceed the static scratch limit of %llu rows per call",
              (unsigned long long)n_rows, (unsigned long long)kStaticMaxRows);
    return VX_E_INVAL;
  }
  SfParams p{};
  p.n_preds = n_preds;
  for (int q = 0; q < n_preds; ++q) {
    if (preds[q].col < 0 || preds[q].col >= n_cols || !cols[preds[q].col] || preds[q].op < VX_BETWEEN ||
        preds[q].op > VX_GE) {
      set_error("vx_filter_device_static: predicate %d: bad column index or op", q);
      return VX_E_INVAL;
    }
    p.col[q] = cols[preds[q].col];
    p.op[q] = preds[q].op;
    p.lo[q] = preds[q].lo;
    p.hi[q] = preds[q].hi;
  }
  p.row0 = row0;
  p.n = n_rows;
  p.cap = cap;
  *out_count = 0;
  if (n_rows == 0) return VX_OK;
  uint32_t *scratch = nullptr;
  VX_TRY(scratch_address(&scratch));
  cudaStream_t s = (cudaStream_t)stream;
  const uint32_t nt = (uint32_t)((n_rows + kSfTile - 1) / kSfTile);
  sf_count_kernel<<<nt, kSfThreads, 0, s>>>(p, scratch);
  sf_scan_kernel<<<1, 1024, 0, s>>>(nt, scratch);
  sf_write_kernel<<<nt, kSfThreads, 0, s>>>(p, scratch, out_rows);
  VX_CUDA_TRY(cudaGetLastError());
  uint32_t total[2] = {0, 0};
  VX_CUDA_TRY(cudaMemcpyAsync(total, scratch + 2 * kStaticMaxTiles, sizeof total, cudaMemcpyDeviceToHost, s));
  VX_CUDA_TRY(cudaStreamSynchronize(s));
  *out_count = total[0];
  if (total[0] > cap) {
    set_error("vx_filter_device_static: %u rows qualify; capacity %llu", total[0], (unsigned long long)cap);
    return VX_E_CAPACITY;
  }
  return VX_OK;
}
