// Out-of-core sort: range partition + per-partition LSD radix sort.
//
// Section 6.1 sorts chunks and merges them; here the partition step comes
// first (the two-phase layout of Section 6.2.1: per-chunk clustering with a
// boundary array, then per-group processing of the multi-extent partitions),
// with a monotone range function so that sorted partitions concatenate into
// the sorted output:
//   pass 1 (ExKernel over input chunks): stable scatter of each chunk by
//           partition id into a host intermediate at the chunk's own offset,
//           plus the chunk's P+1 boundary array;
//   pass 2 (ExKernel over partitions): gather partition p's extents (one per
//           chunk), LSD radix sort in HBM, store at the partition's final
//           offset.
// Both passes run on the pipelined executor, so host->device loads and
// device->host stores overlap with the kernels.  Partitions of one key value
// are already in input order and are copied through; a multi-key partition
// above the slot capacity is sorted recursively.
#include <algorithm>
#include <cstddef>
#include <deque>
#include <cmath>
#include <thread>

#include "vx_internal.h"
#include "vx_radix.cuh"
#include "vx_sort.cuh"

namespace vx {

// ================================================================== kernels

__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// digit of a key: an LSD byte (kRange = false) or the number of splitters <= key
template <bool kRange>
__device__ __forceinline__ uint32_t key_digit(uint64_t k, int shift, const uint64_t *s_spl, int n_spl) {
  if (!kRange) return (uint32_t)(k >> shift) & 0xFFu;
  int lo = 0, hi = n_spl;
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (s_spl[mid] <= k) lo = mid + 1;
    else hi = mid;
  }
  return (uint32_t)lo;
}

template <bool kRange>
__global__ void __launch_bounds__(kRxThreads) rx_upsweep(RadixBufs b, const RadixState *st, int pass, uint64_t n,
                                                         int shift, const uint64_t *spl, int n_spl, uint32_t *hist,
                                                         uint32_t ntiles) {
  if (!kRange && st->skip[pass]) return;
  __shared__ uint32_t wcnt[kRxWarps][kRxDigits];
  __shared__ uint64_t s_spl[kRxDigits];
  const int c = kRange ? 0 : st->cur[pass];
  const uint64_t *keys = b.keys[c];
  for (int i = threadIdx.x; i < kRxWarps * kRxDigits; i += blockDim.x) (&wcnt[0][0])[i] = 0;
  if (kRange)
    for (int i = threadIdx.x; i < n_spl; i += blockDim.x) s_spl[i] = spl[i];
  __syncthreads();
  const uint32_t lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const uint64_t wbase = (uint64_t)blockIdx.x * kRxTile + (uint64_t)w * (32 * kRxItems);
#pragma unroll 4
  for (int r = 0; r < kRxItems; ++r) {
    const uint64_t i = wbase + (uint64_t)r * 32 + lane;
    const uint32_t d = i < n ? key_digit<kRange>(keys[i], shift, s_spl, n_spl) : kRxInvalid;
    if (d != kRxInvalid) atomicAdd(&wcnt[w][d], 1u);  // counting needs no order
  }
  __syncthreads();
  for (int d = threadIdx.x; d < kRxDigits; d += blockDim.x) {
    uint32_t s = 0;
    for (int q = 0; q < kRxWarps; ++q) s += wcnt[q][d];
    hist[(uint64_t)d * ntiles + blockIdx.x] = s;
  }
}

// block d: exclusive scan of hist[d][0..ntiles) in place; row total -> totals[d]
__global__ void __launch_bounds__(1024) rx_scan_rows(uint32_t *hist, uint32_t ntiles, RadixState *st,
                                                     const int pass, const bool check_skip) {
  if (check_skip && st->skip[pass]) return;
  __shared__ uint32_t wsum[32];
  __shared__ uint64_t carry;
  uint32_t *row = hist + (uint64_t)blockIdx.x * ntiles;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (uint32_t base = 0; base < ntiles; base += blockDim.x) {
    const uint32_t i = base + threadIdx.x;
    const uint32_t v = i < ntiles ? row[i] : 0;
    uint32_t x = v;
    for (int off = 1; off < 32; off <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, x, off);
      if ((threadIdx.x & 31) >= (unsigned)off) x += y;
    }
    if ((threadIdx.x & 31) == 31) wsum[threadIdx.x >> 5] = x;
    __syncthreads();
    if (threadIdx.x < 32) {
      uint32_t wv = threadIdx.x < (blockDim.x >> 5) ? wsum[threadIdx.x] : 0;
      for (int off = 1; off < 32; off <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, wv, off);
        if (threadIdx.x >= (unsigned)off) wv += y;
      }
      wsum[threadIdx.x] = wv;
    }
    __syncthreads();
    const uint32_t wpre = (threadIdx.x >> 5) ? wsum[(threadIdx.x >> 5) - 1] : 0;
    if (i < ntiles) row[i] = (uint32_t)carry + wpre + x - v;
    __syncthreads();
    if (threadIdx.x == 0) carry += wsum[(blockDim.x >> 5) - 1];
    __syncthreads();
  }
  if (threadIdx.x == 0) st->totals[blockIdx.x] = carry;
}

// one block of 256 threads: digit bases (exclusive scan of totals, base[256] =
// n); for LSD passes, a digit holding all n pairs marks the pass skipped and
// the double-buffer marker advances only for executed passes
__global__ void __launch_bounds__(kRxDigits) rx_scan_totals(RadixState *st, int pass, uint64_t n, bool lsd) {
  __shared__ uint64_t s[kRxDigits];
  __shared__ int any_full;
  const int d = threadIdx.x;
  if (lsd && st->skip[pass]) {  // decided by the digit-histogram prepass
    if (d == 0) st->cur[pass + 1] = st->cur[pass];
    return;
  }
  if (d == 0) any_full = 0;
  __syncthreads();
  const uint64_t t = st->totals[d];
  s[d] = t;
  if (t == n) any_full = 1;
  __syncthreads();
  for (int off = 1; off < kRxDigits; off <<= 1) {
    uint64_t y = d >= off ? s[d - off] : 0;
    __syncthreads();
    s[d] += y;
    __syncthreads();
  }
  st->base[d] = s[d] - t;
  if (d == 0) st->base[kRxDigits] = n;
  if (lsd && d == 0) {
    st->skip[pass] = any_full;
    st->cur[pass + 1] = any_full ? st->cur[pass] : 1 - st->cur[pass];
  }
}

// full-range histogram of all eight key bytes in one read: marks constant
// digits so that their passes are skipped (upsweep, scan and scatter)
__global__ void __launch_bounds__(kRxThreads) rx_byte_hist(const RadixBufs b, uint64_t n, unsigned long long *bh) {
  __shared__ uint32_t h[8][kRxDigits];
  for (int i = threadIdx.x; i < 8 * kRxDigits; i += blockDim.x) (&h[0][0])[i] = 0;
  __syncthreads();
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t k = b.keys[0][i];
#pragma unroll
    for (int p = 0; p < 8; ++p) atomicAdd(&h[p][(k >> (8 * p)) & 0xFF], 1u);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 8 * kRxDigits; i += blockDim.x)
    if ((&h[0][0])[i]) atomicAdd(&bh[i], (unsigned long long)(&h[0][0])[i]);
}

__global__ void rx_init_state(RadixState *st, const unsigned long long *bh, uint64_t n, uint32_t spin_limit) {
  const int p = threadIdx.x;  // 8 threads
  if (p == 0) {
    st->cur[0] = 0;
    st->err = 0;
    st->spin_limit = spin_limit;
  }
  if (p < 8) {
    int full = 0;
    for (int d = 0; d < kRxDigits; ++d) full |= bh[p * kRxDigits + d] == n;
    st->skip[p] = full;
  }
}

// dynamic shared memory of the scatter: the tile's pairs regrouped by digit
// (keys, values, digits), per-warp digit counters, per-digit offsets
struct RxScatterSmem {
  uint64_t k[kRxTile];
  uint32_t v[kRxTile];
  uint32_t wcnt[kRxWarps][kRxDigits];
  uint64_t off[kRxDigits];  // global position of local position 0 of each digit
  uint32_t tstart[kRxDigits];
  uint32_t wsum[kRxWarps];
  uint8_t d[kRxTile];
};

// One-sweep LSD passes: per-(tile, digit) status words carry a flag (0 not
// ready, 1 the tile's own count, 2 the inclusive prefix over tiles 0..t), the
// pass number (so one clearing serves all eight passes) and the value.
constexpr uint64_t kRxFlagAgg = 1ull << 62, kRxFlagIncl = 2ull << 62;
constexpr uint64_t kRxValueMask = (1ull << 59) - 1;
constexpr uint32_t kRxSpinLimit = 1u << 20;  // polls of one predecessor word before giving up

__device__ __forceinline__ uint64_t rx_status_word(uint64_t flag, int pass, uint64_t value) {
  return flag | (uint64_t)pass << 59 | value;
}

// 8 blocks x 256 threads: exclusive scan of each digit histogram = the global
// position of each digit's first pair in every LSD pass
__global__ void __launch_bounds__(kRxDigits) rx_init_bases(const unsigned long long *bh, uint64_t *bases) {
  __shared__ uint64_t s[kRxDigits];
  const int p = blockIdx.x, d = threadIdx.x;
  const uint64_t t = bh[p * kRxDigits + d];
  s[d] = t;
  __syncthreads();
  for (int off = 1; off < kRxDigits; off <<= 1) {
    const uint64_t y = d >= off ? s[d - off] : 0;
    __syncthreads();
    s[d] += y;
    __syncthreads();
  }
  bases[p * kRxDigits + d] = s[d] - t;
}

// Stable scatter of one tile: rank every pair inside its warp (match_any over
// 16 rounds of 32 consecutive pairs), regroup the tile by digit in shared
// memory, then write each digit's run with consecutive threads on consecutive
// output positions, so stores leave the SM as contiguous runs.
// kOneSweep (LSD passes): the tile is the block's ticket, and its digit offsets
// come from the one-read histogram (bases) plus a look-back over the status
// words of the tiles before it; otherwise the tile is blockIdx.x and its
// offsets come from the scanned per-tile histograms.
template <bool kRange, bool kOneSweep>
__global__ void __launch_bounds__(kRxThreads, 2) rx_downsweep(RadixBufs b, RadixState *st, int pass, uint64_t n,
                                                              int shift, const uint64_t *spl, int n_spl,
                                                              const uint32_t *hist, uint32_t ntiles,
                                                              const uint64_t *bases, unsigned int *tickets,
                                                              unsigned long long *status) {
  if (!kRange && st->skip[pass]) {
    if (kOneSweep && blockIdx.x == 0 && threadIdx.x == 0) st->cur[pass + 1] = st->cur[pass];
    return;
  }
  extern __shared__ __align__(16) unsigned char rx_smem[];
  RxScatterSmem &sm = *reinterpret_cast<RxScatterSmem *>(rx_smem);
  __shared__ uint64_t s_spl[kRxDigits];
  __shared__ uint32_t s_tile;
  const int c = kRange ? 0 : st->cur[pass];
  const uint64_t *kin = b.keys[c];
  const uint32_t *vin = b.vals[c];
  uint64_t *kout = b.keys[1 - c];
  uint32_t *vout = b.vals[1 - c];
  if (kOneSweep && threadIdx.x == 0) s_tile = atomicAdd(&tickets[pass], 1u);
  for (int i = threadIdx.x; i < kRxWarps * kRxDigits; i += blockDim.x) (&sm.wcnt[0][0])[i] = 0;
  if (kRange)
    for (int i = threadIdx.x; i < n_spl; i += blockDim.x) s_spl[i] = spl[i];
  __syncthreads();
  const uint32_t tile = kOneSweep ? s_tile : blockIdx.x;
  if (kOneSweep && tile == 0 && threadIdx.x == 0) st->cur[pass + 1] = 1 - c;  // read by the next pass only
  const uint32_t lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const uint64_t tbase = (uint64_t)tile * kRxTile;
  const uint64_t wbase = tbase + (uint64_t)w * (32 * kRxItems);
  uint64_t k[kRxItems];
  uint32_t v[kRxItems], dr[kRxItems];  // dr = rank inside the warp << 9 | digit
#pragma unroll
  for (int r = 0; r < kRxItems; ++r) {
    const uint64_t i = wbase + (uint64_t)r * 32 + lane;
    k[r] = i < n ? kin[i] : 0;
    v[r] = i < n ? vin[i] : 0;
  }
#pragma unroll
  for (int r = 0; r < kRxItems; ++r) {
    const uint64_t i = wbase + (uint64_t)r * 32 + lane;
    const uint32_t d = i < n ? key_digit<kRange>(k[r], shift, s_spl, n_spl) : kRxInvalid;
    const uint32_t peers = __match_any_sync(0xffffffffu, d);
    uint32_t before = 0;
    if (d != kRxInvalid) before = sm.wcnt[w][d];
    __syncwarp();
    dr[r] = (before + __popc(peers & lanemask_lt())) << 9 | d;
    if (d != kRxInvalid && lane == (uint32_t)(__ffs(peers) - 1)) sm.wcnt[w][d] = before + __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  {  // thread d: warp offsets within digit d, then the tile's digit starts (exclusive scan over digits)
    const int d = threadIdx.x;
    uint32_t run = 0;
#pragma unroll
    for (int q = 0; q < kRxWarps; ++q) {
      const uint32_t cq = sm.wcnt[q][d];
      sm.wcnt[q][d] = run;
      run += cq;
    }
    uint64_t before_tile;  // position of the tile's first pair of digit d
    if (kOneSweep) {
      volatile unsigned long long *sw = status + (uint64_t)tile * kRxDigits + d;
      *sw = rx_status_word(tile == 0 ? kRxFlagIncl : kRxFlagAgg, pass, run);
      uint64_t prefix = 0;  // pairs of digit d in the tiles before this one
      const uint32_t limit = st->spin_limit;
      for (uint32_t t = tile; t > 0;) {  // look back over the predecessors' words
        --t;
        const volatile unsigned long long *pw = status + (uint64_t)t * kRxDigits + d;
        uint64_t word = *pw;
        uint32_t spins = 0;
        while ((word >> 62) == 0 || (int)((word >> 59) & 7u) != pass) {
          // give up after the limit, or at once when another tile already gave up
          if (++spins > limit || ((spins & 1023u) == 0 && *(volatile uint32_t *)&st->err)) {
            spins = limit + 1;
            break;
          }
          __nanosleep(32);
          word = *pw;
        }
        if (spins > limit) {  // a predecessor never published: report, keep going (a partial
                              // prefix only lowers this tile's positions, all inside the pass's n)
          atomicOr(&st->err, 1u);
          break;
        }
        prefix += word & kRxValueMask;
        if ((word >> 62) == 2) break;
      }
      if (tile > 0) *sw = rx_status_word(kRxFlagIncl, pass, prefix + run);
      before_tile = bases[pass * kRxDigits + d] + prefix;
    } else {
      before_tile = st->base[d] + hist[(uint64_t)d * ntiles + tile];
    }
    uint32_t x = run;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, x, off);
      if (lane >= (uint32_t)off) x += y;
    }
    if (lane == 31) sm.wsum[w] = x;
    __syncthreads();
    uint32_t wpre = 0;
#pragma unroll
    for (int q = 0; q < kRxWarps; ++q) wpre += q < (int)w ? sm.wsum[q] : 0u;
    const uint32_t excl = wpre + x - run;
    sm.tstart[d] = excl;
    sm.off[d] = before_tile - excl;  // wraps back when added to a position
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < kRxItems; ++r) {
    const uint32_t d = dr[r] & 0x1FFu;
    if (d == kRxInvalid) continue;
    const uint32_t lp = sm.tstart[d] + sm.wcnt[w][d] + (dr[r] >> 9);
    sm.k[lp] = k[r];
    sm.v[lp] = v[r];
    sm.d[lp] = (uint8_t)d;
  }
  __syncthreads();
  const uint32_t valid = n - tbase < (uint64_t)kRxTile ? (uint32_t)(n - tbase) : (uint32_t)kRxTile;
  for (uint32_t t = threadIdx.x; t < valid; t += blockDim.x) {
    const uint64_t pos = sm.off[sm.d[t]] + t;
    kout[pos] = sm.k[t];
    vout[pos] = sm.v[t];
  }
}

constexpr size_t kRxScatterSmem = sizeof(RxScatterSmem);

// the scatter's shared memory is above the 48 KB default: raise the limit once
static vx_status rx_scatter_attr() {
  static bool done = false;
  if (!done) {
    VX_CUDA_TRY(cudaFuncSetAttribute(rx_downsweep<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)kRxScatterSmem));
    VX_CUDA_TRY(cudaFuncSetAttribute(rx_downsweep<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)kRxScatterSmem));
    done = true;
  }
  return VX_OK;
}

// publishes the buffer holding the result (low byte), the number of
// executed (not skipped) passes (next byte) and the error word (bit 16) to a
// mapped host word
__global__ void rx_publish(const RadixState *st, int pass, uint64_t *host_word) {
  uint64_t executed = 0;
  for (int p = 0; p < pass; ++p) executed += st->skip[p] ? 0u : 1u;
  *host_word = (uint64_t)st->cur[pass] | executed << 8 | (uint64_t)(st->err != 0) << 16;
}

// ---- sampling and splitters -----------------------------------------------

// key of sample i at position mix64(base + i) mod n (the library's own
// counter-based positions), read through mapped host memory
__device__ __forceinline__ uint64_t mix64_dev(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__global__ void sample_keys_kernel(const uint64_t *keys, uint64_t n, uint64_t m, uint64_t seed, uint64_t *out,
                                   uint32_t *out_vals) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < m; i += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t pos = mix64_dev(seed * 0x9E3779B97F4A7C15ull + i) % n;
    out[i] = keys[pos];
    out_vals[i] = (uint32_t)i;
  }
}

// rank[i] = number of sample keys below splitter i (lower bound in the sorted
// sample): partition p (keys in [spl[p-1], spl[p])) holds rank[p] - rank[p-1]
// of the m sample keys
__global__ void sample_ranks_kernel(const uint64_t *sorted, uint64_t m, const uint64_t *spl, uint32_t n_spl,
                                    uint64_t *rank) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n_spl; i += gridDim.x * blockDim.x) {
    uint64_t lo = 0, hi = m;
    while (lo < hi) {
      const uint64_t mid = (lo + hi) >> 1;
      if (sorted[mid] < spl[i]) lo = mid + 1;
      else hi = mid;
    }
    rank[i] = lo;
  }
}

// splitters from the sorted sample: s_p = sample[p*m/P]
__global__ void sample_splitters_kernel(const uint64_t *sorted, uint64_t m, uint32_t P, uint64_t *spl) {
  for (uint32_t p = 1 + blockIdx.x * blockDim.x + threadIdx.x; p < P; p += gridDim.x * blockDim.x)
    spl[p - 1] = sorted[(uint64_t)p * m / P];
}

// piecewise-linear CDF model: knot j = sorted[j*(m-1)/S], CDF(knot j) = j/S;
// splitter p = model inverse at p/P, exact integer interpolation
__global__ void pl_knots_kernel(const uint64_t *sorted, uint64_t m, uint32_t S, uint64_t *knots) {
  for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j <= S; j += gridDim.x * blockDim.x)
    knots[j] = sorted[(uint64_t)j * (m - 1) / S];
}

__global__ void pl_splitters_kernel(const uint64_t *knots, uint32_t S, uint32_t P, uint64_t *spl) {
  for (uint32_t p = 1 + blockIdx.x * blockDim.x + threadIdx.x; p < P; p += gridDim.x * blockDim.x) {
    const uint64_t num = (uint64_t)p * S;
    const uint64_t j = num / P, rem = num % P;
    if (j >= S) {
      spl[p - 1] = knots[S];
      continue;
    }
    const uint64_t gap = knots[j + 1] - knots[j];
    // floor(gap * rem / P) without 128-bit arithmetic: gap = q*P + r
    spl[p - 1] = knots[j] + (gap / P) * rem + ((gap % P) * rem) / P;
  }
}

// Keys of the sorted sample that occur at least m / (2P) times (up to cap of
// them, in no particular order; *n counts them all).  Thread i looks at run
// starts only and finds the run's end by binary search.
__global__ void heavy_keys_kernel(const uint64_t *sorted, uint64_t m, uint32_t P, uint64_t *keys, uint32_t *n,
                                  uint32_t cap) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < m; i += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t v = sorted[i];
    if (i > 0 && sorted[i - 1] == v) continue;
    uint64_t a = i, b = m;  // first index with sorted[] > v
    while (a < b) {
      const uint64_t mid = (a + b) >> 1;
      if (sorted[mid] <= v) a = mid + 1;
      else b = mid;
    }
    if ((a - i) * 2 * (uint64_t)P >= m) {
      const uint32_t j = atomicAdd(n, 1u);
      if (j < cap) keys[j] = v;
    }
  }
}

// raw (n_raw non-decreasing splitters of a smooth model) merged with the heavy
// keys (sorted here, at most cap_heavy of them), duplicates dropped, at most
// cap_out entries: every heavy key becomes a splitter, so the isolation below
// gives it a partition of its own as the sample's quantiles do.  One thread.
__global__ void merge_heavy_kernel(const uint64_t *raw, uint32_t n_raw, uint64_t *heavy, const uint32_t *n_heavy,
                                   uint32_t cap_heavy, uint64_t *out, uint32_t *n_out, uint32_t cap_out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const uint32_t nh = *n_heavy < cap_heavy ? *n_heavy : cap_heavy;
  for (uint32_t i = 1; i < nh; ++i) {  // insertion sort of a few dozen keys
    const uint64_t x = heavy[i];
    uint32_t j = i;
    while (j > 0 && heavy[j - 1] > x) {
      heavy[j] = heavy[j - 1];
      --j;
    }
    heavy[j] = x;
  }
  uint32_t a = 0, b = 0, k = 0;
  // the model's splitters all stay; heavy keys fill what room is left
  uint32_t room = cap_out > n_raw ? cap_out - n_raw : 0;
  while ((a < n_raw || b < nh) && k < cap_out) {
    uint64_t v;
    if (b >= nh || (a < n_raw && raw[a] <= heavy[b])) {
      v = raw[a++];
    } else {
      v = heavy[b++];
      if (room == 0) continue;
      --room;
    }
    if (k > 0 && out[k - 1] == v) continue;
    out[k++] = v;
  }
  *n_out = k;
}

// Heavy keys.  A value repeated among consecutive splitters would leave empty
// partitions, and one partition [v, next) would hold all copies of v plus
// other keys.  Walking left to right, a splitter not above the last kept one
// becomes that one + 1 (dropped at UINT64_MAX); a kept value v that occurs at
// least m / (2P) times in the sorted sample (half a partition's share) is
// followed by the boundary v + 1, so [v, v + 1) holds v alone.  At most
// 2 n_raw splitters result; their count goes to *n_out.
__global__ void isolate_splitters_kernel(const uint64_t *raw, uint32_t n_raw, const uint64_t *sorted, uint64_t m,
                                         uint32_t P, uint64_t *out, uint32_t *n_out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  uint32_t k = 0;
  for (uint32_t j = 0; j < n_raw; ++j) {
    uint64_t v = raw[j];
    if (k > 0 && v <= out[k - 1]) {
      if (out[k - 1] == UINT64_MAX) continue;
      v = out[k - 1] + 1;
    }
    out[k++] = v;
    uint64_t a = 0, b = m;  // lower bound of v
    while (a < b) {
      const uint64_t mid = (a + b) >> 1;
      if (sorted[mid] < v) a = mid + 1;
      else b = mid;
    }
    uint64_t c = a, d = m;  // upper bound of v
    while (c < d) {
      const uint64_t mid = (c + d) >> 1;
      if (sorted[mid] <= v) c = mid + 1;
      else d = mid;
    }
    if ((c - a) * 2 * (uint64_t)P >= m && v != UINT64_MAX) out[k++] = v + 1;
  }
  *n_out = k;
}

// ================================================================== host helpers

vx_status radix_publish_enqueue(char *temp, uint64_t *host_word, cudaStream_t s, int npass) {
  rx_publish<<<1, 1, 0, s>>>(radix_state_of(temp), npass, host_word);
  VX_CUDA_TRY(cudaGetLastError());
  return VX_OK;
}

static uint32_t ntiles_of(uint64_t n) { return (uint32_t)((n + kRxTile - 1) / kRxTile); }

// temp layout: [RadixState | 8 byte histograms (u64) | per-tile region]; the
// per-tile region holds the range partition's per-tile histograms (u32), or
// for an LSD sort the 8 digit bases (u64), 8 tickets and the look-back status
// words (u64 per tile and digit)
constexpr uint64_t kStateBytes = (sizeof(RadixState) + 255) & ~255ull;
constexpr uint64_t kByteHistBytes = 8ull * kRxDigits * 8;
constexpr uint64_t kBasesBytes = 8ull * kRxDigits * 8;
constexpr uint64_t kTicketBytes = 256;

uint64_t radix_temp_bytes(uint64_t cap) {
  const uint64_t nt = std::max<uint32_t>(ntiles_of(cap), 1);
  return kStateBytes + kByteHistBytes + kBasesBytes + kTicketBytes + (uint64_t)kRxDigits * nt * 8 + 256;
}

RadixState *radix_state_of(char *temp) { return (RadixState *)temp; }

// after a radix sort on s: the buffer holding the result, or VX_E_TIMEOUT when
// a look-back wait gave up
static vx_status radix_result(char *temp, cudaStream_t s, int *cur) {
  RadixState h;
  VX_CUDA_TRY(cudaMemcpyAsync(&h, radix_state_of(temp), offsetof(RadixState, totals), cudaMemcpyDeviceToHost, s));
  VX_CUDA_TRY(cudaStreamSynchronize(s));
  if (h.err) {
    set_error("radix sort: a look-back wait gave up");
    return VX_E_TIMEOUT;
  }
  *cur = h.cur[8];
  return VX_OK;
}

// Enqueues a stable LSD radix sort of b.keys[0]/b.vals[0] (n pairs) on s by
// the low npass bytes of the key (8: the whole key).  The sorted pairs end in
// buffer st->cur[npass] (0 or 1).
vx_status radix_sort_enqueue(RadixBufs b, uint64_t n, char *temp, cudaStream_t s, int num_sms, int npass,
                             uint32_t spin_limit) {
  uint32_t nt = ntiles_of(n);
  RadixState *st = radix_state_of(temp);
  unsigned long long *bh = (unsigned long long *)(temp + kStateBytes);
  uint32_t *hist = (uint32_t *)(temp + kStateBytes + kByteHistBytes);
  VX_CUDA_TRY(cudaMemsetAsync(bh, 0, kByteHistBytes, s));
  if (n == 0) {
    VX_CUDA_TRY(cudaMemsetAsync(st, 0, sizeof(RadixState), s));
    return VX_OK;
  }
  VX_TRY(rx_scatter_attr());
  uint64_t *bases = (uint64_t *)hist;
  unsigned int *tickets = (unsigned int *)((char *)hist + kBasesBytes);
  unsigned long long *status = (unsigned long long *)((char *)hist + kBasesBytes + kTicketBytes);
  // tickets and status words: cleared once, the words carry their pass number
  VX_CUDA_TRY(cudaMemsetAsync(tickets, 0, kTicketBytes + (uint64_t)kRxDigits * nt * 8, s));
  int g = (int)std::min<uint64_t>((n + kRxThreads - 1) / kRxThreads, (uint64_t)num_sms * 4);
  rx_byte_hist<<<g, kRxThreads, 0, s>>>(b, n, bh);
  rx_init_state<<<1, 32, 0, s>>>(st, bh, n, spin_limit ? spin_limit : kRxSpinLimit);
  rx_init_bases<<<8, kRxDigits, 0, s>>>(bh, bases);
  for (int pass = 0; pass < npass; ++pass)  // a skipped pass returns at once and keeps the buffer
    rx_downsweep<false, true><<<nt, kRxThreads, kRxScatterSmem, s>>>(b, st, pass, n, 8 * pass, nullptr, 0, nullptr, nt,
                                                                      bases, tickets, status);
  VX_CUDA_TRY(cudaGetLastError());
  return VX_OK;
}

// Enqueues a stable scatter of b.keys[0]/b.vals[0] into b.keys[1]/b.vals[1] by
// partition id (splitters spl[0..P-2] on the device); the P+1 boundary array
// is left in st->base[0..P] with base[P] = n.
vx_status range_partition_enqueue(RadixBufs b, uint64_t n, const uint64_t *spl, uint32_t P, char *temp,
                                  cudaStream_t s) {
  uint32_t nt = std::max<uint32_t>(ntiles_of(n), 1);
  RadixState *st = radix_state_of(temp);
  uint32_t *hist = (uint32_t *)(temp + kStateBytes + kByteHistBytes);
  VX_TRY(rx_scatter_attr());
  VX_CUDA_TRY(cudaMemsetAsync(st, 0, sizeof(RadixState), s));
  if (n) {
    rx_upsweep<true><<<nt, kRxThreads, 0, s>>>(b, st, 0, n, 0, spl, (int)P - 1, hist, nt);
    rx_scan_rows<<<kRxDigits, 1024, 0, s>>>(hist, nt, st, 0, false);
  }
  rx_scan_totals<<<1, kRxDigits, 0, s>>>(st, 0, n, false);
  if (n)
    rx_downsweep<true, false><<<nt, kRxThreads, kRxScatterSmem, s>>>(b, st, 0, n, 0, spl, (int)P - 1, hist, nt,
                                                                      nullptr, nullptr, nullptr);
  VX_CUDA_TRY(cudaGetLastError());
  return VX_OK;
}


// Splitters for P requested partitions from the sorted sample (device), then
// heavy-key isolation.  spl_buf has kSplitterBufBytes: [out 256 | raw 256 |
// knots 1025 | count]; returns the number of splitters in *n_spl (at most 254).
vx_status splitters_from_sample(vx_ctx *ctx, int32_t kind, const uint64_t *sorted, uint64_t m, uint32_t P,
                                uint64_t *spl_buf, uint32_t mlp_steps, double *ms_train, uint32_t *n_spl) {
  cudaStream_t s = ctx->s_compute;
  *n_spl = 0;
  if (P < 2) return VX_OK;
  if (P > kMaxRequestedPartitions) {
    set_error("at most %u partitions per pass", kMaxRequestedPartitions);
    return VX_E_UNSUPPORTED;
  }
  uint64_t *d_out = spl_buf, *d_raw = spl_buf + 256, *d_knots = spl_buf + 512;
  uint32_t *d_n = (uint32_t *)(spl_buf + 512 + kPLSegments + 1);
  if (kind == VX_PART_SAMPLE) {
    sample_splitters_kernel<<<1, 256, 0, s>>>(sorted, m, P, d_raw);
  } else if (kind == VX_PART_LEARNED_PL) {
    pl_knots_kernel<<<(kPLSegments + 256) / 256, 256, 0, s>>>(sorted, m, kPLSegments, d_knots);
    pl_splitters_kernel<<<1, 256, 0, s>>>(d_knots, kPLSegments, P, d_raw);
  } else if (kind == VX_PART_LEARNED_MLP) {
    VX_TRY(mlp_splitters(ctx, sorted, m, P, mlp_steps, d_raw, ms_train));
  } else {
    set_error("unknown partitioner %d", kind);
    return VX_E_INVAL;
  }
  uint32_t n_raw = P - 1;
  if (kind == VX_PART_LEARNED_MLP) {
    // a smooth CDF model steps over a heavy key's jump instead of landing a
    // splitter on it: add the sample's heavy keys to its splitters (the
    // knots area is free here: heavy keys, then the merged list, then counts)
    constexpr uint32_t kHeavyCap = 64, kMergedCap = 127;  // isolation doubles at most: <= 254 cuts
    uint64_t *d_heavy = d_knots, *d_merged = d_knots + kHeavyCap;
    uint32_t *d_cnt = (uint32_t *)(d_knots + kHeavyCap + kMergedCap);
    VX_CUDA_TRY(cudaMemsetAsync(d_cnt, 0, 8, s));
    heavy_keys_kernel<<<(unsigned)std::min<uint64_t>((m + 255) / 256, 1024), 256, 0, s>>>(sorted, m, P, d_heavy, d_cnt,
                                                                                      kHeavyCap);
    merge_heavy_kernel<<<1, 1, 0, s>>>(d_raw, P - 1, d_heavy, d_cnt, kHeavyCap, d_merged, d_cnt + 1, kMergedCap);
    VX_CUDA_TRY(cudaGetLastError());
    VX_CUDA_TRY(cudaMemcpyAsync(&n_raw, d_cnt + 1, 4, cudaMemcpyDeviceToHost, s));
    VX_CUDA_TRY(cudaStreamSynchronize(s));
    VX_CUDA_TRY(cudaMemcpyAsync(d_raw, d_merged, 8ull * n_raw, cudaMemcpyDeviceToDevice, s));
  }
  isolate_splitters_kernel<<<1, 32, 0, s>>>(d_raw, n_raw, sorted, m, P, d_out, d_n);
  VX_CUDA_TRY(cudaGetLastError());
  VX_CUDA_TRY(cudaMemcpyAsync(n_spl, d_n, 4, cudaMemcpyDeviceToHost, s));
  VX_CUDA_TRY(cudaStreamSynchronize(s));
  return VX_OK;
}

// samples m keys of a mapped column and sorts them on the device; m shrinks to
// what the free arena holds
vx_status sample_and_sort(vx_ctx *ctx, const uint64_t *dev_keys, uint64_t n, uint64_t &m, uint64_t seed,
                          DevBuf &sorted_out, uint64_t **sorted_ptr) {
  cudaStream_t s = ctx->s_compute;
  const uint64_t freeb = ctx->arena.largest_free();
  const uint64_t m_fit = freeb > (64u << 10) ? (freeb - (64u << 10)) / 25 : 0;
  m = std::min(m, m_fit);
  if (m == 0) {
    set_error("no room in the arena for a key sample");
    return VX_E_NOMEM;
  }
  uint64_t bytes = 2 * m * 12 + radix_temp_bytes(m) + 1024;
  sorted_out.arena = &ctx->arena;
  sorted_out.p = ctx->arena.alloc(bytes);
  if (!sorted_out.p) {
    set_error("sample of %llu keys does not fit the arena", (unsigned long long)m);
    return VX_E_NOMEM;
  }
  char *p = sorted_out.as<char>();
  RadixBufs b;
  b.keys[0] = (uint64_t *)p;
  b.keys[1] = (uint64_t *)(p + ((8 * m + 255) & ~255ull));
  char *q = p + 2 * ((8 * m + 255) & ~255ull);
  b.vals[0] = (uint32_t *)q;
  b.vals[1] = (uint32_t *)(q + ((4 * m + 255) & ~255ull));
  char *temp = q + 2 * ((4 * m + 255) & ~255ull);
  sample_keys_kernel<<<ctx->num_sms * 2, 256, 0, s>>>(dev_keys, n, m, seed, b.keys[0], b.vals[0]);
  VX_CUDA_TRY(cudaGetLastError());
  VX_TRY(radix_sort_enqueue(b, m, temp, s, ctx->num_sms, 8, ctx->cfg.lookback_spin_limit));
  int cur = 0;
  VX_TRY(radix_result(temp, s, &cur));
  *sorted_ptr = b.keys[cur];
  return VX_OK;
}

// ================================================================== out-of-core sort

namespace {

void parallel_copy(void *dst, const void *src, uint64_t bytes) {
  const uint64_t kMin = 64ull << 20;
  unsigned nt = std::max(1u, std::min(16u, (unsigned)(bytes / kMin)));
  if (nt == 1) {
    memcpy(dst, src, bytes);
    return;
  }
  std::vector<std::thread> th;
  for (unsigned t = 0; t < nt; ++t) {
    uint64_t b = bytes * t / nt, e = bytes * (t + 1) / nt;
    th.emplace_back([=] { memcpy((char *)dst + b, (const char *)src + b, e - b); });
  }
  for (auto &x : th) x.join();
}

// pass 1: per-chunk stable partition into the intermediate + boundary arrays
// a run of one partition's pairs in host memory, in input order
struct Extent {
  const uint64_t *k;
  const uint32_t *v;
  uint64_t len;
};

// host memory registered for the call that holds spilled partition segments
struct Spill {
  std::unique_ptr<char[]> mem;
  HostReg reg;
  uint64_t cap = 0, used = 0;
};

// pass 1: range-partition each chunk on the device and store its partition
// segments to the host intermediate.  Contiguous layout: partition p owns
// [reg_off[p], reg_off[p] + reg_cap[p]) of the intermediate and each chunk's
// segment of p is appended there, so the sort pass loads a partition with one
// copy per column; what does not fit goes to the overflow area after the
// regions, then to spill buffers.  Blocked layout (an intermediate without room
// for the regions): chunk c keeps rows [c R, c R + R) and partition p is one
// extent per chunk.
struct PartitionPass : ExKernel {
  vx_ctx *ctx;
  const uint64_t *keys;
  const uint32_t *vals;
  uint64_t n, R;
  uint32_t P;
  const uint64_t *d_spl;
  uint64_t *mid_keys;
  uint32_t *mid_vals;
  uint64_t *h_bnd;  // page-locked host, chunks x (P+1): chunk-local partition starts
  bool contig = false;
  uint64_t C = 0;                          // pairs of the intermediate
  std::vector<uint64_t> reg_off, reg_cap;  // contiguous layout
  std::vector<uint64_t> used;
  uint64_t ovf = 0;                        // next free pair of the overflow area
  std::deque<Spill> *spills = nullptr;
  std::vector<std::vector<Extent>> ext;    // per partition, in input order

  uint64_t size() override { return (n + R - 1) / R; }
  uint64_t rows(uint64_t it) const { return std::min(R, n - it * R); }
  uint64_t kb() const { return (8 * R + 255) & ~255ull; }
  uint64_t vb() const { return (4 * R + 255) & ~255ull; }
  uint64_t slot_bytes() override { return 2 * kb() + 2 * vb() + radix_temp_bytes(R); }
  RadixBufs bufs(char *slot) const {
    RadixBufs b;
    b.keys[0] = (uint64_t *)slot;
    b.keys[1] = (uint64_t *)(slot + kb());
    b.vals[0] = (uint32_t *)(slot + 2 * kb());
    b.vals[1] = (uint32_t *)(slot + 2 * kb() + vb());
    return b;
  }
  char *temp(char *slot) const { return slot + 2 * kb() + 2 * vb(); }
  void inputs(uint64_t it, char *slot, std::vector<CopyOp> &h2d) override {
    RadixBufs b = bufs(slot);
    uint64_t r0 = it * R, m = rows(it);
    h2d.push_back({keys + r0, b.keys[0], 8 * m});
    h2d.push_back({vals + r0, b.vals[0], 4 * m});
  }
  vx_status kernel(char *slot, uint64_t it, cudaStream_t s) override {
    VX_TRY(range_partition_enqueue(bufs(slot), rows(it), d_spl, P, temp(slot), s));
    // the chunk's boundary array goes to page-locked host memory (a copy into
    // pageable memory would hold the issuing thread until the store queue
    // drains); outputs() reads it once the kernel has completed
    VX_CUDA_TRY(cudaMemcpyAsync(h_bnd + it * (P + 1), radix_state_of(temp(slot))->base, 8ull * (P + 1),
                                cudaMemcpyDeviceToHost, s));
    return VX_OK;
  }
  bool has_outputs() override { return true; }
  void add_extent(uint32_t p, const uint64_t *k, const uint32_t *v, uint64_t len) {
    std::vector<Extent> &e = ext[p];
    if (!e.empty() && e.back().k + e.back().len == k && e.back().v + e.back().len == v)
      e.back().len += len;  // right after the partition's previous segment
    else
      e.push_back({k, v, len});
  }
  // room for up to len pairs of partition p: its region, the overflow area,
  // then a spill buffer; *take pairs of it are handed out
  vx_status place(uint32_t p, uint64_t len, uint64_t **dk, uint32_t **dv, uint64_t *take) {
    if (used[p] < reg_cap[p]) {
      *take = std::min(len, reg_cap[p] - used[p]);
      *dk = mid_keys + reg_off[p] + used[p];
      *dv = mid_vals + reg_off[p] + used[p];
      used[p] += *take;
      return VX_OK;
    }
    if (ovf < C) {
      *take = std::min(len, C - ovf);
      *dk = mid_keys + ovf;
      *dv = mid_vals + ovf;
      ovf += *take;
      return VX_OK;
    }
    if (spills->empty() || spills->back().used == spills->back().cap) {
      spills->emplace_back();
      Spill &sp = spills->back();
      sp.cap = std::max(len, R);
      sp.mem.reset(new (std::nothrow) char[12 * sp.cap]);
      if (!sp.mem) {
        set_error("vx_sort: no host memory for %llu spilled pairs", (unsigned long long)sp.cap);
        return VX_E_NOMEM;
      }
      VX_TRY(sp.reg.add(sp.mem.get(), 12 * sp.cap));
    }
    Spill &sp = spills->back();
    *take = std::min(len, sp.cap - sp.used);
    *dk = (uint64_t *)sp.mem.get() + sp.used;
    *dv = (uint32_t *)(sp.mem.get() + 8 * sp.cap) + sp.used;
    sp.used += *take;
    return VX_OK;
  }
  vx_status outputs(uint64_t it, char *slot, std::vector<CopyOp> &d2h) override {
    RadixBufs b = bufs(slot);
    const uint64_t r0 = it * R, m = rows(it);
    const uint64_t *bd = h_bnd + it * (P + 1);  // copied before the kernel's completion event
    if (!contig) {
      d2h.push_back({b.keys[1], mid_keys + r0, 8 * m});
      d2h.push_back({b.vals[1], mid_vals + r0, 4 * m});
      for (uint32_t p = 0; p < P; ++p)
        if (bd[p + 1] > bd[p]) add_extent(p, mid_keys + r0 + bd[p], mid_vals + r0 + bd[p], bd[p + 1] - bd[p]);
      return VX_OK;
    }
    for (uint32_t p = 0; p < P; ++p) {
      uint64_t s0 = bd[p], len = bd[p + 1] - bd[p];
      while (len) {
        uint64_t *dk;
        uint32_t *dv;
        uint64_t take;
        VX_TRY(place(p, len, &dk, &dv, &take));
        d2h.push_back({b.keys[1] + s0, dk, 8 * take});
        d2h.push_back({b.vals[1] + s0, dv, 4 * take});
        add_extent(p, dk, dv, take);
        s0 += take;
        len -= take;
      }
    }
    return VX_OK;
  }
};

// pass 2: per-partition gather + radix sort + store
struct SortPass : ExKernel {
  vx_ctx *ctx;
  uint64_t cap;
  std::vector<std::vector<Extent>> ext;  // per job
  std::vector<uint64_t> job_n, job_off;
  uint64_t *out_keys;
  uint32_t *out_vals;
  int S;                    // slots of the ring (one published result word per slot)
  uint64_t pass_pairs = 0;  // pairs x executed passes

  uint64_t size() override { return job_n.size(); }
  int n_slots() override { return S; }
  int max_in_flight() override { return S; }
  uint64_t kb() const { return (8 * cap + 255) & ~255ull; }
  uint64_t vb() const { return (4 * cap + 255) & ~255ull; }
  uint64_t slot_bytes() override { return 2 * kb() + 2 * vb() + radix_temp_bytes(cap); }
  RadixBufs bufs(char *slot) const {
    RadixBufs b;
    b.keys[0] = (uint64_t *)slot;
    b.keys[1] = (uint64_t *)(slot + kb());
    b.vals[0] = (uint32_t *)(slot + 2 * kb());
    b.vals[1] = (uint32_t *)(slot + 2 * kb() + vb());
    return b;
  }
  char *temp(char *slot) const { return slot + 2 * kb() + 2 * vb(); }
  void inputs(uint64_t it, char *slot, std::vector<CopyOp> &h2d) override {
    RadixBufs b = bufs(slot);
    uint64_t at = 0;
    for (const Extent &e : ext[it]) {
      if (!e.len) continue;
      h2d.push_back({e.k, b.keys[0] + at, 8 * e.len});
      h2d.push_back({e.v, b.vals[0] + at, 4 * e.len});
      at += e.len;
    }
  }
  vx_status kernel(char *slot, uint64_t it, cudaStream_t s) override {
    VX_TRY(radix_sort_enqueue(bufs(slot), job_n[it], temp(slot), s, ctx->num_sms, 8, ctx->cfg.lookback_spin_limit));
    rx_publish<<<1, 1, 0, s>>>(radix_state_of(temp(slot)), 8, ctx->d_scalars + 64 + (it % S));
    VX_CUDA_TRY(cudaGetLastError());
    return VX_OK;
  }
  bool has_outputs() override { return true; }
  vx_status outputs(uint64_t it, char *slot, std::vector<CopyOp> &d2h) override {
    RadixBufs b = bufs(slot);
    const uint64_t word = ((volatile uint64_t *)ctx->h_scalars)[64 + (it % S)];
    if (word >> 16 & 1) {
      set_error("radix sort of partition job %llu: a look-back wait gave up", (unsigned long long)it);
      return VX_E_TIMEOUT;
    }
    const int c = (int)(word & 0xFF);
    pass_pairs += job_n[it] * ((word >> 8) & 0xFF);
    if (job_n[it] == 0) return VX_OK;
    d2h.push_back({b.keys[c], out_keys + job_off[it], 8 * job_n[it]});
    d2h.push_back({b.vals[c], out_vals + job_off[it], 4 * job_n[it]});
    return VX_OK;
  }
};

}  // namespace

// sorts contiguous host pairs (keys/vals mapped or pinned) into out
vx_status sort_contiguous(vx_ctx *ctx, const uint64_t *keys, const uint32_t *vals, const uint64_t *dev_keys, uint64_t n,
                          uint64_t *out_keys, uint32_t *out_vals, const vx_sort_opts &o, vx_sort_stats &ss, int depth) {
  const int S = std::max(2, ctx->cfg.n_slots);
  const uint64_t avail = ctx->arena.largest_free();
  // pairs per slot: (2 x 12 B + histograms) per pair, S slots
  uint64_t cap = (uint64_t)((double)avail / (S * (24.0 + 256.0 * 8 / kRxTile)) * 0.97);
  cap = cap / kRxTile * kRxTile;
  if (o.max_slot_pairs) cap = std::min<uint64_t>(cap, o.max_slot_pairs / kRxTile * kRxTile);
  if (cap < kRxTile) {
    set_error("vx_sort: arena of %llu bytes too small", (unsigned long long)ctx->arena.capacity());
    return VX_E_NOMEM;
  }
  ss.slot_pairs = cap;
  if (n == 0) return VX_OK;
  double t0 = now_ms();
  // ---- P = 1: the input fits one slot
  if (n <= cap && o.n_partitions <= 1) {
    SortPass sp;
    sp.ctx = ctx;
    sp.cap = cap;
    sp.ext.push_back({{keys, vals, n}});
    sp.job_n.push_back(n);
    sp.job_off.push_back(0);
    sp.out_keys = out_keys;
    sp.out_vals = out_vals;
    sp.S = S;
    ExecStats es;
    VX_TRY(run_pipeline(ctx, sp, &es));
    ss.bytes_h2d += es.bytes_h2d;
    ss.bytes_d2h += es.bytes_d2h;
    ss.kernel_launches += es.kernel_launches;
    ss.ms_sort_kernel += es.ms_kernel;
    ss.radix_pass_pairs += sp.pass_pairs;
    ss.n_partitions = std::max<uint32_t>(ss.n_partitions, 1);
    ss.max_partition = std::max(ss.max_partition, n);
    ss.ms_sort += now_ms() - t0;
    return VX_OK;
  }
  // ---- splitters from a sample
  // requested partitions: 30% headroom at the top level, 2x inside a recursion
  const double over = depth == 0 ? 1.3 : 2.0;
  uint32_t P = o.n_partitions > 1 ? (uint32_t)o.n_partitions
                                  : (uint32_t)std::min<uint64_t>(kMaxRequestedPartitions,
                                                                 (uint64_t)std::ceil(over * (double)n / cap));
  if (P < 2) P = 2;
  // enough partitions that the sort pass pipelines (loads of partition p+1
  // and stores of p-1 overlap the sort of p) when the caller leaves P open
  if (depth == 0 && o.n_partitions <= 1 && n >= kPipelineRows * 4) P = std::max<uint32_t>(P, 16);
  if (P > kMaxRequestedPartitions) {
    set_error("vx_sort: at most %u partitions per pass", kMaxRequestedPartitions);
    return VX_E_UNSUPPORTED;
  }
  uint64_t m = std::min<uint64_t>(o.sample_size ? o.sample_size : (1ull << 20), n);
  DevBuf sbuf, splbuf;
  uint64_t *sorted = nullptr;
  double ts = now_ms();
  // the splitters outlive the sample: allocated first, they do not split the
  // arena's free space in two once the sample is released (the passes below
  // size their slots from the largest free block)
  splbuf.arena = &ctx->arena;
  splbuf.p = ctx->arena.alloc(kSplitterBufBytes);
  if (!splbuf.p) {
    set_error("vx_sort: no room for the splitters");
    return VX_E_NOMEM;
  }
  uint64_t *d_spl = splbuf.as<uint64_t>();
  VX_TRY(sample_and_sort(ctx, dev_keys, n, m, o.seed + (uint64_t)depth * 7919, sbuf, &sorted));
  double ms_train = 0;
  uint32_t n_spl = 0;
  VX_TRY(splitters_from_sample(ctx, o.partitioner, sorted, m, P, d_spl, o.mlp_steps, &ms_train, &n_spl));
  P = n_spl + 1;  // partitions after heavy-key isolation
  std::vector<uint64_t> spl(n_spl), srank(n_spl);
  if (n_spl) {
    DevBuf rbuf;
    rbuf.arena = &ctx->arena;
    rbuf.p = ctx->arena.alloc(8 * n_spl);
    if (!rbuf.p) return VX_E_NOMEM;
    sample_ranks_kernel<<<1, 128, 0, ctx->s_compute>>>(sorted, m, d_spl, n_spl, rbuf.as<uint64_t>());
    VX_CUDA_TRY(cudaGetLastError());
    VX_CUDA_TRY(cudaMemcpyAsync(spl.data(), d_spl, 8 * n_spl, cudaMemcpyDeviceToHost, ctx->s_compute));
    VX_CUDA_TRY(cudaMemcpyAsync(srank.data(), rbuf.p, 8 * n_spl, cudaMemcpyDeviceToHost, ctx->s_compute));
    VX_CUDA_TRY(cudaStreamSynchronize(ctx->s_compute));
  }
  VX_CUDA_TRY(cudaStreamSynchronize(ctx->s_compute));
  sbuf.release();
  ss.ms_sample += now_ms() - ts - ms_train;
  ss.ms_train += ms_train;
  if (depth == 0 && o.splitters_out) memcpy(o.splitters_out, spl.data(), 8 * n_spl);

  // partition-pass chunks of kPipelineRows pairs: long enough for efficient
  // copies (576 MB), short enough that the pass pipelines over many chunks
  const uint64_t R = std::min<uint64_t>(cap, kPipelineRows);
  const uint64_t n_chunks = (n + R - 1) / R;

  // ---- host intermediate: one region per partition, sized from the sample's
  // count c in it (estimate n c / m) plus 1 % and four binomial standard
  // deviations, then an overflow area of what the intermediate has left (at
  // least n / 256 pairs); the sort stays exact whatever the estimates, only the
  // number of extents grows
  std::vector<uint64_t> reg_off(P), reg_cap(P);
  uint64_t regions = 0;
  for (uint32_t p = 0; p < P; ++p) {
    const uint64_t r1 = p < n_spl ? srank[p] : m, r0 = p ? srank[p - 1] : 0;
    const double cnt = (double)(r1 - r0), scale = (double)n / (double)m;
    const double slack = o.region_slack_pct ? o.region_slack_pct / 100.0 : 0.01;
    const double sigmas = o.region_slack_pct ? 0.0 : 4.0;
    const double est = (1.0 + slack) * cnt * scale + sigmas * std::sqrt(cnt + 1.0) * scale + kRxTile;
    // regions start on 128-pair boundaries (1 KB of keys, 512 B of values), so
    // the sort pass loads each from an aligned host address
    reg_cap[p] = (std::min<uint64_t>(n, (uint64_t)std::ceil(est)) + 127) / 128 * 128;
    reg_off[p] = regions;
    regions += reg_cap[p];
  }
  const uint64_t want = regions + n / 256 + kRxTile;
  uint64_t *mid_keys = nullptr;
  uint32_t *mid_vals = nullptr;
  uint64_t C = 0;  // pairs the intermediate holds
  bool contig = true;
  std::unique_ptr<char[]> own;
  HostReg reg_mid;
  std::deque<Spill> spills;
  if (depth == 0 && o.host_scratch && o.host_scratch_bytes >= 12 * n) {
    C = o.host_scratch_bytes / 12 / 128 * 128;  // the value array then starts 1 KB-aligned too
    contig = C >= want;  // else the blocked layout in the first 12 n bytes
    if (!contig) C = n;
    mid_keys = (uint64_t *)o.host_scratch;
    mid_vals = (uint32_t *)((char *)o.host_scratch + 8 * C);
    VX_TRY(reg_mid.add(o.host_scratch, 12 * C));
  } else {
    C = (regions + n / 64 + kRxTile + 127) / 128 * 128;
    own.reset(new (std::nothrow) char[12 * C + 4096]);
    if (!own) {
      set_error("vx_sort: no host memory for the %llu-pair intermediate", (unsigned long long)C);
      return VX_E_NOMEM;
    }
    char *base = (char *)(((uintptr_t)own.get() + 4095) & ~(uintptr_t)4095);  // page-aligned
    mid_keys = (uint64_t *)base;
    mid_vals = (uint32_t *)(base + 8 * C);
    VX_TRY(reg_mid.add(base, 12 * C));
  }

  // ---- pass 1: partition
  double tp = now_ms();
  PartitionPass pp;
  {
    uint64_t *h_bnd = nullptr;
    VX_CUDA_TRY(cudaHostAlloc((void **)&h_bnd, 8 * n_chunks * (P + 1), cudaHostAllocDefault));
    struct FreeHost {
      void *p;
      ~FreeHost() { cudaFreeHost(p); }
    } free_bnd{h_bnd};
    pp.ctx = ctx;
    pp.keys = keys;
    pp.vals = vals;
    pp.n = n;
    pp.R = R;
    pp.P = P;
    pp.d_spl = d_spl;
    pp.mid_keys = mid_keys;
    pp.mid_vals = mid_vals;
    pp.h_bnd = h_bnd;
    pp.contig = contig;
    pp.C = C;
    pp.reg_off = reg_off;
    pp.reg_cap = reg_cap;
    pp.used.assign(P, 0);
    pp.ovf = regions;
    pp.spills = &spills;
    pp.ext.resize(P);
    ExecStats es;
    VX_TRY(run_pipeline(ctx, pp, &es));
    VX_CUDA_TRY(cudaStreamSynchronize(ctx->s_compute));
    ss.bytes_h2d += es.bytes_h2d;
    ss.bytes_d2h += es.bytes_d2h;
    ss.kernel_launches += es.kernel_launches * 4;  // upsweep, row scan, totals, downsweep
  }
  ss.ms_partition += now_ms() - tp;

  // ---- partition sizes and output offsets
  std::vector<uint64_t> psize(P, 0), poff(P, 0);
  for (uint32_t p = 0; p < P; ++p) {
    for (const Extent &e : pp.ext[p]) psize[p] += e.len;
    if (contig) ss.out_of_region_pairs += psize[p] - pp.used[p];
  }
  ss.spill_buffers += spills.size();
  if (depth == 0) ss.contiguous_layout = contig ? 1u : 0u;
  for (uint32_t p = 1; p < P; ++p) poff[p] = poff[p - 1] + psize[p - 1];
  auto extents = [&](uint32_t p) { return pp.ext[p]; };
  uint64_t mx = 0, mn = UINT64_MAX;
  for (uint32_t p = 0; p < P; ++p) {
    mx = std::max(mx, psize[p]);
    mn = std::min(mn, psize[p]);
  }
  if (depth == 0) {
    ss.n_partitions = P;
    ss.max_partition = mx;
    ss.min_partition = mn;
    ss.imbalance = (double)mx / ((double)n / P);
  }

  // ---- pass 2: sort the partitions that fit; copy through single-key ones;
  // recurse on the others
  double tq = now_ms();
  SortPass sp;
  sp.ctx = ctx;
  sp.cap = cap;
  sp.out_keys = out_keys;
  sp.out_vals = out_vals;
  sp.S = S;
  std::vector<uint32_t> big;
  for (uint32_t p = 0; p < P; ++p) {
    if (psize[p] == 0) continue;
    if (psize[p] <= cap) {
      sp.ext.push_back(extents(p));
      sp.job_n.push_back(psize[p]);
      sp.job_off.push_back(poff[p]);
    } else {
      big.push_back(p);
    }
  }
  {
    // Slots sized by the largest job, as many as fit (at most kMaxSortSlots):
    // a job's load, sort and store take about the same time, so with three
    // slots the next load waits for a store and every uneven partition leaves
    // the device idle; more slots let loads run ahead.  Never fewer than the
    // S slots of `cap` pairs the partition count was planned for.
    uint64_t jcap = 0;
    for (uint64_t x : sp.job_n) jcap = std::max(jcap, x);
    jcap = (jcap + kRxTile - 1) / kRxTile * kRxTile;
    if (jcap) {
      sp.cap = jcap;
      const uint64_t sb = (sp.slot_bytes() + 255) & ~255ull;
      sp.S = std::max<int>(S, (int)std::min<uint64_t>(kMaxSortSlots, ctx->arena.largest_free() / sb));
    }
    ExecStats es;
    VX_TRY(run_pipeline(ctx, sp, &es));
    ss.bytes_h2d += es.bytes_h2d;
    ss.bytes_d2h += es.bytes_d2h;
    ss.kernel_launches += es.kernel_launches * 35;  // byte histogram, state, 8 x 4 passes, publish
    ss.ms_sort_kernel += es.ms_kernel;
    ss.radix_pass_pairs += sp.pass_pairs;
  }
  for (uint32_t p : big) {
    const uint64_t lo = p == 0 ? 0 : spl[p - 1];
    const bool single_key = p + 1 < P ? (spl[p] > lo && spl[p] - lo == 1) : lo == UINT64_MAX;
    std::vector<Extent> ex = extents(p);
    if (single_key) {  // already in input order: copy through
      uint64_t at = poff[p];
      for (const Extent &e : ex) {
        parallel_copy(out_keys + at, e.k, 8 * e.len);
        parallel_copy(out_vals + at, e.v, 4 * e.len);
        at += e.len;
      }
      ss.passthrough_partitions += 1;
      continue;
    }
    if (depth >= 3) {
      set_error("vx_sort: partition of %llu pairs still exceeds the slot after 3 levels",
                (unsigned long long)psize[p]);
      return VX_E_CAPACITY;
    }
    ss.overflow_retries += 1;
    // gather the partition contiguously (in input order) and sort it recursively
    std::vector<char> tmp(psize[p] * 12);
    uint64_t *tk = (uint64_t *)tmp.data();
    uint32_t *tv = (uint32_t *)(tmp.data() + 8 * psize[p]);
    uint64_t at = 0;
    for (const Extent &e : ex) {
      parallel_copy(tk + at, e.k, 8 * e.len);
      parallel_copy(tv + at, e.v, 4 * e.len);
      at += e.len;
    }
    HostReg rt;
    VX_TRY(rt.add(tmp.data(), tmp.size()));
    void *dk = nullptr;
    VX_CUDA_TRY(cudaHostGetDevicePointer(&dk, tk, 0));
    vx_sort_opts o2 = o;
    o2.n_partitions = 0;
    VX_TRY(sort_contiguous(ctx, tk, tv, (const uint64_t *)dk, psize[p], out_keys + poff[p], out_vals + poff[p], o2,
                           ss, depth + 1));
  }
  ss.ms_sort += now_ms() - tq;
  return VX_OK;
}

}  // namespace vx

using namespace vx;

VX_API vx_status vx_sort(vx_ctx *ctx, int32_t key_col, int32_t rowid_col, uint64_t *out_keys, uint32_t *out_rowids,
                         const vx_sort_opts *opts, vx_sort_stats *stats) {
  clear_error();
  VX_TRY(check_ctx(ctx));
  std::lock_guard<std::recursive_mutex> g(ctx->mu);
  const Column *kc = get_col(ctx, key_col, VX_U64);
  const Column *vc = get_col(ctx, rowid_col, VX_U32);
  if (!kc || !vc) return VX_E_INVAL;
  if (kc->n_rows != vc->n_rows || ((!out_keys || !out_rowids) && kc->n_rows)) {
    set_error("vx_sort: columns differ in length or null output");
    return VX_E_INVAL;
  }
  vx_sort_opts o{};
  if (opts) o = *opts;
  if (o.partitioner < VX_PART_SAMPLE || o.partitioner > VX_PART_LEARNED_MLP || o.n_partitions < 0 ||
      o.n_partitions > 256 || (o.plan != VX_SORT_PARTITION && o.plan != VX_SORT_MERGE) || o.runs_mode < 0 ||
      o.runs_mode > 1) {
    set_error("vx_sort: bad options");
    return VX_E_INVAL;
  }
  const uint64_t n = kc->n_rows;
  HostReg r1, r2;
  VX_TRY(r1.add(out_keys, 8 * n));
  VX_TRY(r2.add(out_rowids, 4 * n));
  vx_sort_stats ss{};
  double t0 = now_ms();
  vx_status st = o.plan == VX_SORT_MERGE
                     ? merge_sort_plan(ctx, (const uint64_t *)kc->host, (const uint32_t *)vc->host,
                                       (const uint64_t *)kc->dev, n, out_keys, out_rowids, o, ss)
                     : sort_contiguous(ctx, (const uint64_t *)kc->host, (const uint32_t *)vc->host,
                                       (const uint64_t *)kc->dev, n, out_keys, out_rowids, o, ss, 0);
  ss.ms_total = now_ms() - t0;
  if (stats) *stats = ss;
  return st;
}

VX_API vx_status vx_radix_sort_pairs(vx_ctx *ctx, const uint64_t *keys, const uint32_t *vals, uint64_t n,
                                     uint64_t *out_keys, uint32_t *out_vals) {
  clear_error();
  VX_TRY(check_ctx(ctx));
  if (n && (!keys || !vals || !out_keys || !out_vals)) {
    set_error("vx_radix_sort_pairs: null buffer");
    return VX_E_INVAL;
  }
  std::lock_guard<std::recursive_mutex> g(ctx->mu);
  if (n == 0) return VX_OK;
  DevBuf buf;
  buf.arena = &ctx->arena;
  const uint64_t kb = (8 * n + 255) & ~255ull, vb = (4 * n + 255) & ~255ull;
  buf.p = ctx->arena.alloc(2 * kb + 2 * vb + radix_temp_bytes(n));
  if (!buf.p) {
    set_error("vx_radix_sort_pairs: %llu pairs do not fit the arena", (unsigned long long)n);
    return VX_E_NOMEM;
  }
  char *p = buf.as<char>();
  RadixBufs b;
  b.keys[0] = (uint64_t *)p;
  b.keys[1] = (uint64_t *)(p + kb);
  b.vals[0] = (uint32_t *)(p + 2 * kb);
  b.vals[1] = (uint32_t *)(p + 2 * kb + vb);
  char *temp = p + 2 * kb + 2 * vb;
  cudaStream_t s = ctx->s_compute;
  VX_CUDA_TRY(cudaMemcpyAsync(b.keys[0], keys, 8 * n, cudaMemcpyHostToDevice, s));
  VX_CUDA_TRY(cudaMemcpyAsync(b.vals[0], vals, 4 * n, cudaMemcpyHostToDevice, s));
  VX_TRY(radix_sort_enqueue(b, n, temp, s, ctx->num_sms, 8, ctx->cfg.lookback_spin_limit));
  int cur = 0;
  VX_TRY(radix_result(temp, s, &cur));
  VX_CUDA_TRY(cudaMemcpyAsync(out_keys, b.keys[cur], 8 * n, cudaMemcpyDeviceToHost, s));
  VX_CUDA_TRY(cudaMemcpyAsync(out_vals, b.vals[cur], 4 * n, cudaMemcpyDeviceToHost, s));
  VX_CUDA_TRY(cudaStreamSynchronize(s));
  return VX_OK;
}

VX_API vx_status vx_range_partition(vx_ctx *ctx, const uint64_t *keys, const uint32_t *vals, uint64_t n,
                                    const uint64_t *splitters, uint32_t n_partitions, uint64_t *out_keys,
                                    uint32_t *out_vals, uint64_t *boundary) {
  clear_error();
  VX_TRY(check_ctx(ctx));
  if (n_partitions < 1 || n_partitions > 256 || (n_partitions > 1 && !splitters) || !boundary ||
      (n && (!keys || !vals || !out_keys || !out_vals))) {
    set_error("vx_range_partition: bad argument");
    return VX_E_INVAL;
  }
  for (uint32_t i = 1; i + 1 < n_partitions; ++i)
    if (splitters[i] < splitters[i - 1]) {
      set_error("vx_range_partition: splitters must be non-decreasing");
      return VX_E_INVAL;
    }
  std::lock_guard<std::recursive_mutex> g(ctx->mu);
  DevBuf buf;
  buf.arena = &ctx->arena;
  const uint64_t kb = (8 * std::max<uint64_t>(n, 1) + 255) & ~255ull, vb = (4 * std::max<uint64_t>(n, 1) + 255) & ~255ull;
  buf.p = ctx->arena.alloc(2 * kb + 2 * vb + radix_temp_bytes(std::max<uint64_t>(n, 1)) + 8 * 256);
  if (!buf.p) {
    set_error("vx_range_partition: %llu pairs do not fit the arena", (unsigned long long)n);
    return VX_E_NOMEM;
  }
  char *p = buf.as<char>();
  RadixBufs b;
  b.keys[0] = (uint64_t *)p;
  b.keys[1] = (uint64_t *)(p + kb);
  b.vals[0] = (uint32_t *)(p + 2 * kb);
  b.vals[1] = (uint32_t *)(p + 2 * kb + vb);
  char *temp = p + 2 * kb + 2 * vb;
  uint64_t *d_spl = (uint64_t *)(temp + radix_temp_bytes(std::max<uint64_t>(n, 1)));
  cudaStream_t s = ctx->s_compute;
  if (n_partitions > 1) VX_CUDA_TRY(cudaMemcpyAsync(d_spl, splitters, 8 * (n_partitions - 1), cudaMemcpyHostToDevice, s));
  if (n) {
    VX_CUDA_TRY(cudaMemcpyAsync(b.keys[0], keys, 8 * n, cudaMemcpyHostToDevice, s));
    VX_CUDA_TRY(cudaMemcpyAsync(b.vals[0], vals, 4 * n, cudaMemcpyHostToDevice, s));
  }
  VX_TRY(range_partition_enqueue(b, n, d_spl, n_partitions, temp, s));
  RadixState *st = radix_state_of(temp);
  VX_CUDA_TRY(cudaMemcpyAsync(boundary, st->base, 8ull * (n_partitions + 1), cudaMemcpyDeviceToHost, s));
  if (n) {
    VX_CUDA_TRY(cudaMemcpyAsync(out_keys, b.keys[1], 8 * n, cudaMemcpyDeviceToHost, s));
    VX_CUDA_TRY(cudaMemcpyAsync(out_vals, b.vals[1], 4 * n, cudaMemcpyDeviceToHost, s));
  }
  VX_CUDA_TRY(cudaStreamSynchronize(s));
  boundary[n_partitions] = n;
  return VX_OK;
}

VX_API vx_status vx_sort_splitters(vx_ctx *ctx, int32_t key_col, int32_t partitioner, uint32_t n_partitions,
                                   uint64_t sample_size, uint64_t seed, uint64_t *splitters_out, uint32_t *n_out) {
  clear_error();
  VX_TRY(check_ctx(ctx));
  std::lock_guard<std::recursive_mutex> g(ctx->mu);
  const Column *kc = get_col(ctx, key_col, VX_U64);
  if (!kc) return VX_E_INVAL;
  if (n_partitions < 2 || n_partitions > kMaxRequestedPartitions || !splitters_out || !n_out || kc->n_rows == 0) {
    set_error("vx_sort_splitters: need 2..%u partitions, outputs, non-empty column", kMaxRequestedPartitions);
    return VX_E_INVAL;
  }
  uint64_t m = std::min<uint64_t>(sample_size ? sample_size : (1ull << 20), kc->n_rows);
  DevBuf sbuf, splbuf;
  uint64_t *sorted = nullptr;
  VX_TRY(sample_and_sort(ctx, (const uint64_t *)kc->dev, kc->n_rows, m, seed, sbuf, &sorted));
  splbuf.arena = &ctx->arena;
  splbuf.p = ctx->arena.alloc(kSplitterBufBytes);
  if (!splbuf.p) return VX_E_NOMEM;
  uint64_t *d_spl = splbuf.as<uint64_t>();
  double ms = 0;
  uint32_t k = 0;
  VX_TRY(splitters_from_sample(ctx, partitioner, sorted, m, n_partitions, d_spl, 0, &ms, &k));
  if (k) VX_CUDA_TRY(cudaMemcpyAsync(splitters_out, d_spl, 8ull * k, cudaMemcpyDeviceToHost, ctx->s_compute));
  VX_CUDA_TRY(cudaStreamSynchronize(ctx->s_compute));
  *n_out = k;
  return VX_OK;
}
