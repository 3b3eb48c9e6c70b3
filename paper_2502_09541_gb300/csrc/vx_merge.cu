// Sort by merging sorted runs (Section 6.1): a SortExKernel radix-sorts each
// contiguous chunk in HBM and stores it as a sorted run of a host
// intermediate; the MergeExKernel's data mapping regroups the runs into P
// partitions with max(partition p) <= min(partition p + 1) by an exact search
// over the runs; its kernel merges a partition's segments (one per run)
// pairwise in rounds, a tree over a double buffer, and the executor stores
// the result at the partition's final offset.
//
// Exact cuts.  The stable order is (key, position in the input); runs are
// consecutive pieces of the input, so it is (key, run, position in the run).
// The cut at rank k takes, from every run, the elements below the key v of
// rank k, and of the elements equal to v the first k - (elements below v),
// lowest runs first.  v is found by binary search over the 64-bit key value:
// each step counts, in every run, the keys <= the candidate with two searches
// - over the run's fences (every 4,096th key, kept in HBM since pass 1) and
// then inside one 4,096-key window of the run itself, read through mapped
// host memory - and sums the counts over the runs.
//
// Merge rounds.  Round r merges segments (2q, 2q + 1) of the current buffer
// into the other; a block owns 2,048 consecutive outputs, finds where they
// start and end in the two inputs by merge path (the first d outputs take i
// elements of A, the largest i with A[i-1] <= B[d-i]: ties go to A, the
// earlier run, which keeps the merge stable), stages both pieces in shared
// memory and merges 8 outputs per thread.
#include <algorithm>
#include <cmath>

#include "vx_internal.h"
#include "vx_sort.cuh"

namespace vx {

namespace {

constexpr uint64_t kFenceStride = kRxTile;  // keys per fence of a sorted run
constexpr int kMergeThreads = 256;
constexpr int kMergeItems = 8;
constexpr uint32_t kMergeTile = kMergeThreads * kMergeItems;
constexpr uint32_t kMaxRuns = 256;
constexpr int kSplitThreads = 256;  // thread r searches run r
static_assert(kSplitThreads >= (int)kMaxRuns, "one split thread per run");

// ------------------------------------------------------------------ fences
// fences[j] = key j * kFenceStride of the sorted run (keys = k, or the radix
// sort's result buffer when st is given)
__global__ void run_fences_kernel(const uint64_t *k0, const uint64_t *k1, const RadixState *st, uint64_t n,
                                  uint64_t *fences) {
  const uint64_t *k = st && st->cur[8] ? k1 : k0;
  const uint64_t nf = (n + kFenceStride - 1) / kFenceStride;
  for (uint64_t j = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; j < nf; j += (uint64_t)gridDim.x * blockDim.x)
    fences[j] = k[j * kFenceStride];
}

// ------------------------------------------------------------------ natural runs
// Descents of one staged chunk of keys (chunk rows row0 .. row0 + m): every i
// in [1, m) with k[i] < k[i - 1] starts an ascending run of the input; up to
// cap of their global rows go to pos (in no particular order), all of them are
// counted in *cnt.  A chunk's first row is compared on the host.
__global__ void descent_kernel(const uint64_t *__restrict__ k, uint64_t m, uint64_t row0, unsigned long long *cnt,
                               uint64_t *pos, uint32_t cap) {
  for (uint64_t i = 1 + blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < m; i += (uint64_t)gridDim.x * blockDim.x)
    if (k[i] < k[i - 1]) {
      const unsigned long long j = atomicAdd(cnt, 1ull);
      if (j < cap) pos[j] = row0 + i;
    }
}

// fences of ascending runs of the input read through mapped host memory:
// run r = blockIdx.y, fence j of it = key run_off[r] + j * kFenceStride
__global__ void natural_fences_kernel(const uint64_t *keys, const uint64_t *run_off, const uint64_t *fence_start,
                                      uint64_t *fences) {
  const uint32_t r = blockIdx.y;
  const uint64_t len = run_off[r + 1] - run_off[r], nf = (len + kFenceStride - 1) / kFenceStride;
  for (uint64_t j = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; j < nf; j += (uint64_t)gridDim.x * blockDim.x)
    fences[fence_start[r] + j] = keys[run_off[r] + j * kFenceStride];
}

// ------------------------------------------------------------------ exact cuts
struct SplitParams {
  const uint64_t *keys;         // run r at keys + run_off[r] (mapped host memory or HBM)
  const uint64_t *run_off;      // device, n_runs + 1
  const uint64_t *fence_start;  // device, n_runs: run r's fences at fences + fence_start[r]
  const uint64_t *fences;
  const uint64_t *ranks;        // device, one target rank per block
  uint32_t n_runs;
  uint64_t *out;                // device, gridDim.x x n_runs
};

// keys of run r that are <= v (le) or < v (!le)
__device__ uint64_t run_count(const SplitParams &p, uint32_t r, uint64_t v, bool le) {
  const uint64_t len = p.run_off[r + 1] - p.run_off[r];
  const uint64_t nf = (len + kFenceStride - 1) / kFenceStride;
  const uint64_t *f = p.fences + p.fence_start[r];
  uint64_t lo = 0, hi = nf;  // fences passing the test
  while (lo < hi) {
    const uint64_t mid = (lo + hi) / 2;
    const uint64_t x = f[mid];
    if (le ? x <= v : x < v) lo = mid + 1; else hi = mid;
  }
  if (lo == 0) return 0;
  // key (lo-1) * stride passes and key lo * stride (if any) fails: the first
  // failing position lies in ((lo-1) * stride, min(lo * stride, len)]
  const uint64_t *k = p.keys + p.run_off[r];
  uint64_t a = (lo - 1) * kFenceStride + 1, b = lo * kFenceStride < len ? lo * kFenceStride : len;
  while (a < b) {
    const uint64_t mid = (a + b) / 2;
    const uint64_t x = k[mid];
    if (le ? x <= v : x < v) a = mid + 1; else b = mid;
  }
  return a;
}

__device__ uint64_t block_sum(uint64_t x, uint64_t *red) {
  for (int off = 16; off > 0; off >>= 1) x += __shfl_down_sync(0xffffffffu, x, off);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = x;
  __syncthreads();
  uint64_t t = 0;
  for (int w = 0; w < kSplitThreads / 32; ++w) t += red[w];
  return t;
}

__global__ void __launch_bounds__(kSplitThreads) exact_split_kernel(const SplitParams p) {
  __shared__ uint64_t red[kSplitThreads / 32];
  __shared__ uint64_t eq_s[kSplitThreads];
  const uint32_t r = threadIdx.x;
  const bool mine = r < p.n_runs;
  const uint64_t k = p.ranks[blockIdx.x];
  const uint64_t len = mine ? p.run_off[r + 1] - p.run_off[r] : 0;
  const uint64_t total = block_sum(len, red);
  if (k >= total) {  // the whole input lies left of the cut
    if (mine) p.out[(uint64_t)blockIdx.x * p.n_runs + r] = len;
    return;
  }
  // v = the smallest key with more than k keys <= v (the key of rank k)
  uint64_t lo = 0, hi = ~0ull;
  while (lo < hi) {
    const uint64_t mid = lo + (hi - lo) / 2;
    const uint64_t c = block_sum(mine ? run_count(p, r, mid, true) : 0, red);
    if (c > k) hi = mid; else lo = mid + 1;
  }
  const uint64_t lt = mine ? run_count(p, r, lo, false) : 0;
  const uint64_t le = mine ? run_count(p, r, lo, true) : 0;
  const uint64_t below = block_sum(lt, red);
  // of the keys equal to v, the cut takes k - below, from the lowest runs first
  eq_s[r] = le - lt;
  __syncthreads();
  uint64_t before = 0;
  for (uint32_t q = 0; q < r && q < p.n_runs; ++q) before += eq_s[q];
  const uint64_t need = k - below;
  const uint64_t take = need > before ? (need - before < le - lt ? need - before : le - lt) : 0;
  if (mine) p.out[(uint64_t)blockIdx.x * p.n_runs + r] = lt + take;
}

// ------------------------------------------------------------------ merge rounds
struct MergeRound {
  const uint64_t *kin;
  const uint32_t *vin;
  uint64_t *kout;
  uint32_t *vout;
  uint64_t n;
  uint32_t nseg;
  uint64_t seg[kMaxRuns + 1];  // segment s = [seg[s], seg[s + 1]) of the input buffer
};

// elements of a among the first d outputs of the stable merge of a and b
template <class I>
__device__ __forceinline__ I merge_path(const uint64_t *a, I na, const uint64_t *b, I nb, I d) {
  I lo = d > nb ? d - nb : 0, hi = d < na ? d : na;
  while (lo < hi) {
    const I mid = (lo + hi) / 2;
    if (a[mid] <= b[d - 1 - mid]) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// pair of segments holding output position t, and its bounds
struct PairAt {
  uint64_t base, amid, pend;
};
__device__ __forceinline__ PairAt pair_at(const MergeRound &p, uint64_t t) {
  const uint32_t npairs = (p.nseg + 1) / 2;
  uint32_t qlo = 0, qhi = npairs - 1;
  while (qlo < qhi) {
    const uint32_t mid = (qlo + qhi + 1) / 2;
    if (p.seg[2 * mid] <= t) qlo = mid; else qhi = mid - 1;
  }
  return PairAt{p.seg[2 * qlo], p.seg[2 * qlo + 1], p.seg[2 * qlo + 2 < p.nseg ? 2 * qlo + 2 : p.nseg]};
}

// Merge-path cuts of a round, one thread per tile boundary: cut[b] = the
// elements of the first segment of its pair among the pair's outputs before
// output b * kMergeTile (searched in parallel for every tile, so a merge block
// starts at once instead of waiting on a serial search of global memory).
// A boundary that starts a pair has cut 0.
__global__ void merge_cuts_kernel(const MergeRound p, uint64_t *cut, uint64_t n_bounds) {
  for (uint64_t b = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; b < n_bounds; b += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t t = b * kMergeTile < p.n ? b * kMergeTile : p.n;
    if (t >= p.n) {
      cut[b] = 0;
      continue;
    }
    const PairAt q = pair_at(p, t);
    cut[b] = merge_path<uint64_t>(p.kin + q.base, q.amid - q.base, p.kin + q.amid, q.pend - q.amid, t - q.base);
  }
}

__global__ void __launch_bounds__(kMergeThreads) merge_round_kernel(const MergeRound p, const uint64_t *cut) {
  __shared__ uint64_t sk[kMergeTile];
  __shared__ uint32_t sv[kMergeTile];
  uint64_t t0 = (uint64_t)blockIdx.x * kMergeTile;
  const uint64_t t_end = t0 + kMergeTile < p.n ? t0 + kMergeTile : p.n;
  while (t0 < t_end) {  // the outputs of one pair at a time (a tile may span pairs)
    const PairAt q = pair_at(p, t0);
    const uint64_t base = q.base, amid = q.amid, pend = q.pend;
    const uint64_t t1 = t_end < pend ? t_end : pend;
    const uint64_t *A = p.kin + base, *B = p.kin + amid;
    const uint64_t na = amid - base, nb = pend - amid;
    const uint64_t d0 = t0 - base, d1 = t1 - base;
    // cuts at the tile's own boundaries come precomputed; a pair boundary
    // inside the tile is where a pair starts (cut 0) or ends (cut na)
    const uint64_t i0 = t0 == (uint64_t)blockIdx.x * kMergeTile ? cut[blockIdx.x] : 0;
    const uint64_t i1 = t1 == pend ? na : cut[blockIdx.x + 1];
    const uint64_t j0 = d0 - i0;
    const uint32_t la = (uint32_t)(i1 - i0), L = (uint32_t)(d1 - d0), lb = L - la;
    for (uint32_t x = threadIdx.x; x < L; x += kMergeThreads) {
      if (x < la) {
        sk[x] = A[i0 + x];
        sv[x] = p.vin[base + i0 + x];
      } else {
        sk[x] = B[j0 + x - la];
        sv[x] = p.vin[amid + j0 + x - la];
      }
    }
    __syncthreads();
    const uint32_t u0 = threadIdx.x * kMergeItems < L ? threadIdx.x * kMergeItems : L;
    uint32_t ia = merge_path<uint32_t>(sk, la, sk + la, lb, u0), ib = u0 - ia;
    uint64_t ok[kMergeItems];
    uint32_t ov[kMergeItems];
#pragma unroll
    for (int e = 0; e < kMergeItems; ++e) {
      if (u0 + e < L) {
        const bool take_a = ib >= lb || (ia < la && sk[ia] <= sk[la + ib]);
        const uint32_t at = take_a ? ia : la + ib;
        ok[e] = sk[at];
        ov[e] = sv[at];
        ia += take_a;
        ib += !take_a;
      }
    }
    __syncthreads();
#pragma unroll
    for (int e = 0; e < kMergeItems; ++e)
      if (u0 + e < L) {
        sk[u0 + e] = ok[e];
        sv[u0 + e] = ov[e];
      }
    __syncthreads();
    for (uint32_t x = threadIdx.x; x < L; x += kMergeThreads) {
      p.kout[t0 + x] = sk[x];
      p.vout[t0 + x] = sv[x];
    }
    __syncthreads();
    t0 = t1;
  }
}

// Enqueues the merge of the nseg segments seg[0..nseg] of b.keys[0]/b.vals[0]
// (n pairs) on s; returns the buffer that holds the result and adds the
// executed rounds to *rounds.
// cuts: device scratch of n / kMergeTile + 2 words
int merge_enqueue(RadixBufs b, uint64_t n, const std::vector<uint64_t> &seg, uint64_t *cuts, cudaStream_t s,
                  uint64_t *rounds) {
  int c = 0;
  std::vector<uint64_t> cur = seg;
  while (cur.size() > 2) {  // more than one segment
    MergeRound r{};
    r.kin = b.keys[c];
    r.vin = b.vals[c];
    r.kout = b.keys[1 - c];
    r.vout = b.vals[1 - c];
    r.n = n;
    r.nseg = (uint32_t)(cur.size() - 1);
    for (size_t i = 0; i < cur.size(); ++i) r.seg[i] = cur[i];
    const unsigned grid = (unsigned)((n + kMergeTile - 1) / kMergeTile);
    merge_cuts_kernel<<<(grid + 1 + 255) / 256, 256, 0, s>>>(r, cuts, (uint64_t)grid + 1);
    merge_round_kernel<<<grid, kMergeThreads, 0, s>>>(r, cuts);
    std::vector<uint64_t> nx;
    for (uint32_t q = 0; 2 * q < r.nseg; ++q) nx.push_back(cur[2 * q]);
    nx.push_back(n);
    cur.swap(nx);
    c = 1 - c;
    *rounds += 1;
  }
  return c;
}

// segment boundaries of the non-empty lengths, starting at 0
std::vector<uint64_t> segments_of(const std::vector<uint64_t> &lens) {
  std::vector<uint64_t> seg{0};
  for (uint64_t l : lens)
    if (l) seg.push_back(seg.back() + l);
  return seg;
}

// ------------------------------------------------------------------ pass 1: sorted runs
struct RunPass : ExKernel {
  vx_ctx *ctx;
  const uint64_t *keys;
  const uint32_t *vals;
  uint64_t n, R;
  uint64_t *mid_keys;
  uint32_t *mid_vals;
  uint64_t *d_fences;  // run it's fences at it * fences_per_run
  uint64_t fences_per_run;
  int S;
  uint64_t pass_pairs = 0;

  uint64_t size() override { return (n + R - 1) / R; }
  int n_slots() override { return S; }
  int max_in_flight() override { return S; }
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
    h2d.push_back({keys + it * R, b.keys[0], 8 * rows(it)});
    h2d.push_back({vals + it * R, b.vals[0], 4 * rows(it)});
  }
  vx_status kernel(char *slot, uint64_t it, cudaStream_t s) override {
    RadixBufs b = bufs(slot);
    const uint64_t m = rows(it);
    VX_TRY(radix_sort_enqueue(b, m, temp(slot), s, ctx->num_sms, 8, ctx->cfg.lookback_spin_limit));
    const uint64_t nf = (m + kFenceStride - 1) / kFenceStride;
    run_fences_kernel<<<(unsigned)std::max<uint64_t>(1, std::min<uint64_t>((nf + 255) / 256, 1024)), 256, 0, s>>>(
        b.keys[0], b.keys[1], radix_state_of(temp(slot)), m, d_fences + it * fences_per_run);
    VX_CUDA_TRY(cudaGetLastError());
    return radix_publish_enqueue(temp(slot), ctx->d_scalars + 64 + (it % S), s);
  }
  bool has_outputs() override { return true; }
  vx_status outputs(uint64_t it, char *slot, std::vector<CopyOp> &d2h) override {
    RadixBufs b = bufs(slot);
    const uint64_t word = ((volatile uint64_t *)ctx->h_scalars)[64 + (it % S)];
    if (word >> 16 & 1) {
      set_error("radix sort of run %llu: a look-back wait gave up", (unsigned long long)it);
      return VX_E_TIMEOUT;
    }
    const int c = (int)(word & 0xFF);
    pass_pairs += rows(it) * ((word >> 8) & 0xFF);
    d2h.push_back({b.keys[c], mid_keys + it * R, 8 * rows(it)});
    d2h.push_back({b.vals[c], mid_vals + it * R, 4 * rows(it)});
    return VX_OK;
  }
};

// ------------------------------------------------------------------ run detection
// Streams the keys through the device chunk by chunk and records where the
// input's ascending runs start (descent_kernel); nothing comes back but the
// positions.
struct RunDetectPass : ExKernel {
  const uint64_t *keys;
  uint64_t n, R;
  unsigned long long *d_cnt;
  uint64_t *d_pos;
  uint32_t cap;
  int num_sms;

  uint64_t size() override { return (n + R - 1) / R; }
  uint64_t rows(uint64_t it) const { return std::min(R, n - it * R); }
  uint64_t slot_bytes() override { return (8 * R + 255) & ~255ull; }
  void inputs(uint64_t it, char *slot, std::vector<CopyOp> &h2d) override {
    h2d.push_back({keys + it * R, slot, 8 * rows(it)});
  }
  vx_status kernel(char *slot, uint64_t it, cudaStream_t s) override {
    const uint64_t m = rows(it);
    const uint64_t grid = std::max<uint64_t>(1, std::min<uint64_t>((m + 255) / 256, (uint64_t)num_sms * 8));
    descent_kernel<<<(unsigned)grid, 256, 0, s>>>((const uint64_t *)slot, m, it * R, d_cnt, d_pos, cap);
    VX_CUDA_TRY(cudaGetLastError());
    return VX_OK;
  }
};

// Starts of the input's ascending runs when there are at most kMaxRuns of
// them (*found = true; starts[0] = 0), after a host-side sample of adjacent
// pairs has suggested so; else *found = false (and the detection pass did not
// run, or counted too many descents).
vx_status natural_runs(vx_ctx *ctx, const uint64_t *keys, uint64_t n, uint64_t max_rows,
                       std::vector<uint64_t> *starts, bool *found, uint64_t *bytes_h2d) {
  *found = false;
  starts->assign(1, 0);
  if (n < 2) {
    *found = true;
    return VX_OK;
  }
  // sample: descents among up to 65,536 adjacent pairs at pseudo-random rows
  const uint64_t ns = std::min<uint64_t>(65536, n - 1);
  uint64_t desc = 0;
  for (uint64_t j = 0; j < ns; ++j) {
    uint64_t z = 0x9E3779B97F4A7C15ull * (j + 1);
    z = (z ^ (z >> 31)) * 0xBF58476D1CE4E5B9ull;
    z ^= z >> 29;
    const uint64_t i = 1 + (uint64_t)(((unsigned __int128)z * (n - 1)) >> 64);
    desc += keys[i] < keys[i - 1];
  }
  if ((double)desc * (double)(n - 1) / (double)ns >= (double)kMaxRuns) return VX_OK;
  const int S = std::max(2, ctx->cfg.n_slots);
  uint64_t R = (uint64_t)((double)ctx->arena.largest_free() / S * 0.9) / 8;
  R = std::min<uint64_t>(R, kPipelineRows);
  if (max_rows) R = std::min<uint64_t>(R, max_rows);
  if (R < 2) return VX_OK;
  DevBuf b;
  b.arena = &ctx->arena;
  b.p = ctx->arena.alloc(8 * (kMaxRuns + 1));
  if (!b.p) return VX_OK;
  unsigned long long *d_cnt = b.as<unsigned long long>();
  uint64_t *d_pos = b.as<uint64_t>() + 1;
  VX_CUDA_TRY(cudaMemsetAsync(d_cnt, 0, 8, ctx->s_compute));
  RunDetectPass dp;
  dp.keys = keys;
  dp.n = n;
  dp.R = R;
  dp.d_cnt = d_cnt;
  dp.d_pos = d_pos;
  dp.cap = kMaxRuns;
  dp.num_sms = ctx->num_sms;
  ExecStats es;
  VX_TRY(run_pipeline(ctx, dp, &es));
  *bytes_h2d += es.bytes_h2d;
  uint64_t cnt = 0;
  VX_CUDA_TRY(cudaMemcpyAsync(&cnt, d_cnt, 8, cudaMemcpyDeviceToHost, ctx->s_compute));
  VX_CUDA_TRY(cudaStreamSynchronize(ctx->s_compute));
  std::vector<uint64_t> pos(std::min<uint64_t>(cnt, kMaxRuns));
  if (!pos.empty()) {
    VX_CUDA_TRY(cudaMemcpyAsync(pos.data(), d_pos, 8 * pos.size(), cudaMemcpyDeviceToHost, ctx->s_compute));
    VX_CUDA_TRY(cudaStreamSynchronize(ctx->s_compute));
  }
  // the chunks' first rows against the rows before them
  for (uint64_t c = R; c < n; c += R)
    if (keys[c] < keys[c - 1]) ++cnt, pos.push_back(c);
  if (cnt + 1 > kMaxRuns) return VX_OK;
  std::sort(pos.begin(), pos.end());
  starts->insert(starts->end(), pos.begin(), pos.end());
  *found = true;
  return VX_OK;
}

// ------------------------------------------------------------------ pass 2: merge partitions
struct MergePass : ExKernel {
  vx_ctx *ctx;
  uint64_t cap;  // pairs per slot
  const uint64_t *run_keys;
  const uint32_t *run_vals;
  std::vector<uint64_t> run_off;  // N + 1
  std::vector<uint64_t> cut;      // (P + 1) x N: cut[p * N + r] = elements of run r before partition p
  uint32_t N = 0, P = 0;
  uint64_t *out_keys;
  uint32_t *out_vals;
  int S;
  std::vector<int> result_buf;  // per slot: buffer holding the merged partition
  uint64_t rounds_pairs = 0;
  std::vector<cudaEvent_t> ev0, ev1;
  double ms_merge = 0;
  ~MergePass() override {
    for (auto e : ev0) cudaEventDestroy(e);
    for (auto e : ev1) cudaEventDestroy(e);
  }

  uint64_t size() override { return P; }
  int n_slots() override { return S; }
  int max_in_flight() override { return S; }
  uint64_t kb() const { return (8 * cap + 255) & ~255ull; }
  uint64_t vb() const { return (4 * cap + 255) & ~255ull; }
  uint64_t cb() const { return (8 * (cap / kMergeTile + 2) + 255) & ~255ull; }
  uint64_t slot_bytes() override { return 2 * kb() + 2 * vb() + cb(); }
  RadixBufs bufs(char *slot) const {
    RadixBufs b;
    b.keys[0] = (uint64_t *)slot;
    b.keys[1] = (uint64_t *)(slot + kb());
    b.vals[0] = (uint32_t *)(slot + 2 * kb());
    b.vals[1] = (uint32_t *)(slot + 2 * kb() + vb());
    return b;
  }
  uint64_t *cuts(char *slot) const { return (uint64_t *)(slot + 2 * kb() + 2 * vb()); }
  uint64_t seg_len(uint64_t p, uint32_t r) const { return cut[(p + 1) * N + r] - cut[p * N + r]; }
  uint64_t part_off(uint64_t p) const {
    uint64_t o = 0;
    for (uint32_t r = 0; r < N; ++r) o += cut[p * N + r];
    return o;
  }
  uint64_t part_len(uint64_t p) const {
    uint64_t o = 0;
    for (uint32_t r = 0; r < N; ++r) o += seg_len(p, r);
    return o;
  }
  void inputs(uint64_t p, char *slot, std::vector<CopyOp> &h2d) override {
    RadixBufs b = bufs(slot);
    uint64_t at = 0;
    for (uint32_t r = 0; r < N; ++r) {
      const uint64_t l = seg_len(p, r), from = run_off[r] + cut[p * N + r];
      if (!l) continue;
      h2d.push_back({run_keys + from, b.keys[0] + at, 8 * l});
      h2d.push_back({run_vals + from, b.vals[0] + at, 4 * l});
      at += l;
    }
  }
  vx_status kernel(char *slot, uint64_t p, cudaStream_t s) override {
    std::vector<uint64_t> lens(N);
    for (uint32_t r = 0; r < N; ++r) lens[r] = seg_len(p, r);
    const uint64_t n = part_len(p);
    const size_t e = p % S;
    if (!ev0.empty()) VX_CUDA_TRY(cudaEventRecord(ev0[e], s));
    uint64_t rounds = 0;
    result_buf[e] = merge_enqueue(bufs(slot), n, segments_of(lens), cuts(slot), s, &rounds);
    VX_CUDA_TRY(cudaGetLastError());
    if (!ev1.empty()) VX_CUDA_TRY(cudaEventRecord(ev1[e], s));
    rounds_pairs += rounds * n;
    return VX_OK;
  }
  void on_retire(uint64_t p) override {
    if (ev0.empty()) return;
    float ms = 0;
    if (cudaEventElapsedTime(&ms, ev0[p % S], ev1[p % S]) == cudaSuccess) ms_merge += ms;
    cudaGetLastError();
  }
  bool has_outputs() override { return true; }
  vx_status outputs(uint64_t p, char *slot, std::vector<CopyOp> &d2h) override {
    RadixBufs b = bufs(slot);
    const int c = result_buf[p % S];
    const uint64_t n = part_len(p), off = part_off(p);
    if (n) {
      d2h.push_back({b.keys[c], out_keys + off, 8 * n});
      d2h.push_back({b.vals[c], out_vals + off, 4 * n});
    }
    return VX_OK;
  }
};

// exact cuts of runs (keys: device-visible address of the runs) at the given
// ranks; fences: device, run r's at fence_start[r]
vx_status exact_cuts(vx_ctx *ctx, const uint64_t *keys, const std::vector<uint64_t> &run_off,
                     const std::vector<uint64_t> &fence_start, const uint64_t *d_fences,
                     const std::vector<uint64_t> &ranks, std::vector<uint64_t> *out) {
  const uint32_t N = (uint32_t)run_off.size() - 1, Q = (uint32_t)ranks.size();
  out->assign((uint64_t)Q * N, 0);
  if (!Q || !N) return VX_OK;
  DevBuf b;
  b.arena = &ctx->arena;
  const uint64_t words = (N + 1) + N + Q + (uint64_t)Q * N;
  b.p = ctx->arena.alloc(8 * words);
  if (!b.p) {
    set_error("exact cuts: %llu bytes do not fit the arena", (unsigned long long)(8 * words));
    return VX_E_NOMEM;
  }
  uint64_t *d = b.as<uint64_t>();
  std::vector<uint64_t> h(words - (uint64_t)Q * N);
  std::copy(run_off.begin(), run_off.end(), h.begin());
  std::copy(fence_start.begin(), fence_start.end(), h.begin() + N + 1);
  std::copy(ranks.begin(), ranks.end(), h.begin() + 2 * N + 1);
  cudaStream_t s = ctx->s_compute;
  VX_CUDA_TRY(cudaMemcpyAsync(d, h.data(), 8 * h.size(), cudaMemcpyHostToDevice, s));
  SplitParams sp{};
  sp.keys = keys;
  sp.run_off = d;
  sp.fence_start = d + N + 1;
  sp.fences = d_fences;
  sp.ranks = d + 2 * N + 1;
  sp.n_runs = N;
  sp.out = d + 2 * N + 1 + Q;
  exact_split_kernel<<<Q, kSplitThreads, 0, s>>>(sp);
  VX_CUDA_TRY(cudaGetLastError());
  VX_CUDA_TRY(cudaMemcpyAsync(out->data(), sp.out, 8ull * Q * N, cudaMemcpyDeviceToHost, s));
  VX_CUDA_TRY(cudaStreamSynchronize(s));
  return VX_OK;
}

}  // namespace

// The merge plan of vx_sort.  When a sample of adjacent pairs suggests the
// input is already made of few ascending runs, a detection pass finds them
// (at most kMaxRuns) and they serve as the sorted runs directly: pass 1 and its
// intermediate are skipped, and the merge pass loads the runs' segments from
// the input itself.
vx_status merge_sort_plan(vx_ctx *ctx, const uint64_t *keys, const uint32_t *vals, const uint64_t *dev_keys,
                          uint64_t n, uint64_t *out_keys, uint32_t *out_vals, const vx_sort_opts &o,
                          vx_sort_stats &ss) {
  const int S = std::max(2, ctx->cfg.n_slots);
  ss.plan = VX_SORT_MERGE;
  if (n == 0) return VX_OK;
  std::vector<uint64_t> run_off, fence_start;
  DevBuf fb;
  fb.arena = &ctx->arena;
  const uint64_t *run_keys = nullptr, *run_keys_dev = nullptr;
  const uint32_t *run_vals = nullptr;
  uint32_t N = 0;
  std::unique_ptr<char[]> own;
  HostReg reg_mid;

  // ---- natural runs of the input
  bool nat = false;
  if (o.runs_mode == 0 && dev_keys) {
    const double td = now_ms();
    std::vector<uint64_t> starts;
    VX_TRY(natural_runs(ctx, keys, n, o.max_slot_pairs, &starts, &nat, &ss.bytes_h2d));
    if (nat) {
      N = (uint32_t)starts.size();
      run_off = starts;
      run_off.push_back(n);
      fence_start.assign(N, 0);
      uint64_t nf = 0, mx_nf = 0;
      for (uint32_t r = 0; r < N; ++r) {
        fence_start[r] = nf;
        const uint64_t f = (run_off[r + 1] - run_off[r] + kFenceStride - 1) / kFenceStride;
        nf += f;
        mx_nf = std::max(mx_nf, f);
      }
      fb.p = ctx->arena.alloc(8 * (nf + 2 * (uint64_t)N + 1));
      if (!fb.p) {
        set_error("vx_sort: fences do not fit the arena");
        return VX_E_NOMEM;
      }
      uint64_t *d_fences = fb.as<uint64_t>(), *d_off = d_fences + nf, *d_fs = d_off + N + 1;
      VX_CUDA_TRY(cudaMemcpyAsync(d_off, run_off.data(), 8 * (N + 1), cudaMemcpyHostToDevice, ctx->s_compute));
      VX_CUDA_TRY(cudaMemcpyAsync(d_fs, fence_start.data(), 8 * N, cudaMemcpyHostToDevice, ctx->s_compute));
      const dim3 grid((unsigned)std::max<uint64_t>(1, std::min<uint64_t>((mx_nf + 255) / 256, 256)), N);
      natural_fences_kernel<<<grid, 256, 0, ctx->s_compute>>>(dev_keys, d_off, d_fs, d_fences);
      VX_CUDA_TRY(cudaGetLastError());
      VX_CUDA_TRY(cudaStreamSynchronize(ctx->s_compute));
      run_keys = keys;
      run_vals = vals;
      run_keys_dev = dev_keys;
      ss.natural_runs = 1;
    }
    ss.ms_partition += now_ms() - td;
  }

  if (!nat) {
    const uint64_t avail = ctx->arena.largest_free();
    // pass 1 runs: kPipelineRows pairs, fewer if S slots of them do not fit
    uint64_t cap1 = (uint64_t)((double)avail / (S * (24.0 + 256.0 * 8 / kRxTile)) * 0.9);
    cap1 = cap1 / kRxTile * kRxTile;
    if (o.max_slot_pairs) cap1 = std::min<uint64_t>(cap1, o.max_slot_pairs / kRxTile * kRxTile);
    const uint64_t R = std::min<uint64_t>(cap1, kPipelineRows);
    if (R < kRxTile) {
      set_error("vx_sort: arena of %llu bytes too small", (unsigned long long)ctx->arena.capacity());
      return VX_E_NOMEM;
    }
    const uint64_t N64 = (n + R - 1) / R;
    if (N64 > kMaxRuns) {
      set_error("vx_sort (merge plan): %llu runs; at most %u", (unsigned long long)N64, kMaxRuns);
      return VX_E_UNSUPPORTED;
    }
    N = (uint32_t)N64;

    // ---- host intermediate for the sorted runs: keys (8 n bytes), then values
    uint64_t *mid_keys = nullptr;
    uint32_t *mid_vals = nullptr;
    if (o.host_scratch && o.host_scratch_bytes >= 12 * n) {
      mid_keys = (uint64_t *)o.host_scratch;
      mid_vals = (uint32_t *)((char *)o.host_scratch + 8 * n);
      VX_TRY(reg_mid.add(o.host_scratch, 12 * n));
    } else {
      own.reset(new (std::nothrow) char[12 * n + 4096]);
      if (!own) {
        set_error("vx_sort: no host memory for the %llu-pair intermediate", (unsigned long long)n);
        return VX_E_NOMEM;
      }
      char *base = (char *)(((uintptr_t)own.get() + 4095) & ~(uintptr_t)4095);
      mid_keys = (uint64_t *)base;
      mid_vals = (uint32_t *)(base + 8 * n);
      VX_TRY(reg_mid.add(base, 12 * n));
    }
    void *dev_mid = nullptr;
    VX_CUDA_TRY(cudaHostGetDevicePointer(&dev_mid, mid_keys, 0));

    // ---- pass 1: sorted runs and their fences
    const uint64_t fpr = (R + kFenceStride - 1) / kFenceStride;
    fb.p = ctx->arena.alloc(8 * fpr * N);
    if (!fb.p) {
      set_error("vx_sort: fences do not fit the arena");
      return VX_E_NOMEM;
    }
    double t0 = now_ms();
    {
      RunPass rp;
      rp.ctx = ctx;
      rp.keys = keys;
      rp.vals = vals;
      rp.n = n;
      rp.R = R;
      rp.mid_keys = mid_keys;
      rp.mid_vals = mid_vals;
      rp.d_fences = fb.as<uint64_t>();
      rp.fences_per_run = fpr;
      rp.S = S;
      ExecStats es;
      VX_TRY(run_pipeline(ctx, rp, &es));
      VX_CUDA_TRY(cudaStreamSynchronize(ctx->s_compute));
      ss.bytes_h2d += es.bytes_h2d;
      ss.bytes_d2h += es.bytes_d2h;
      ss.kernel_launches += es.kernel_launches * 37;  // radix sort (35), fences, publish
      ss.ms_sort_kernel += es.ms_kernel;
      ss.radix_pass_pairs += rp.pass_pairs;
    }
    ss.ms_partition += now_ms() - t0;
    run_off.assign(N + 1, 0);
    fence_start.assign(N, 0);
    for (uint32_t r = 0; r <= N; ++r) run_off[r] = std::min<uint64_t>((uint64_t)r * R, n);
    for (uint32_t r = 0; r < N; ++r) fence_start[r] = (uint64_t)r * fpr;
    run_keys = mid_keys;
    run_vals = mid_vals;
    run_keys_dev = (const uint64_t *)dev_mid;
  }
  ss.n_runs = N;

  // ---- partitions: equal shares of the pairs, each within a merge slot;
  // enough of them that the merge pass pipelines
  const double ts = now_ms();
  uint64_t cap2 = (uint64_t)((double)ctx->arena.largest_free() / (S * 24.0) * 0.95);
  if (o.max_slot_pairs) cap2 = std::min<uint64_t>(cap2, o.max_slot_pairs);
  uint64_t P = o.n_partitions > 0 ? (uint64_t)o.n_partitions : (n + cap2 - 1) / std::max<uint64_t>(cap2, 1);
  if (o.n_partitions <= 0 && n >= kPipelineRows * 4) P = std::max<uint64_t>(P, 16);
  P = std::max<uint64_t>(P, 1);
  if ((n + P - 1) / P > cap2) {
    set_error("vx_sort (merge plan): partitions of %llu pairs exceed a slot of %llu",
              (unsigned long long)((n + P - 1) / P), (unsigned long long)cap2);
    return VX_E_NOMEM;
  }
  std::vector<uint64_t> ranks;
  for (uint64_t p = 1; p < P; ++p) ranks.push_back(p * n / P);
  std::vector<uint64_t> inner;
  VX_TRY(exact_cuts(ctx, run_keys_dev, run_off, fence_start, fb.as<uint64_t>(), ranks, &inner));
  fb.release();
  MergePass mp;
  mp.ctx = ctx;
  mp.run_keys = run_keys;
  mp.run_vals = run_vals;
  mp.run_off = run_off;
  mp.N = N;
  mp.P = (uint32_t)P;
  mp.cut.assign((P + 1) * N, 0);
  for (uint64_t p = 1; p < P; ++p)
    for (uint32_t r = 0; r < N; ++r) mp.cut[p * N + r] = inner[(p - 1) * N + r];
  for (uint32_t r = 0; r < N; ++r) mp.cut[P * N + r] = run_off[r + 1] - run_off[r];
  uint64_t mx = 0, mn = UINT64_MAX;
  for (uint64_t p = 0; p < P; ++p) {
    const uint64_t l = mp.part_len(p);
    mx = std::max(mx, l);
    mn = std::min(mn, l);
  }
  ss.ms_sample += now_ms() - ts;
  ss.n_partitions = (uint32_t)P;
  ss.max_partition = mx;
  ss.min_partition = mn;
  ss.imbalance = (double)mx / ((double)n / P);

  // ---- pass 2: merge each partition's segments
  const double tq = now_ms();
  mp.cap = (mx + kMergeTile - 1) / kMergeTile * kMergeTile;
  const uint64_t sb = (mp.slot_bytes() + 255) & ~255ull;
  mp.S = std::max<int>(S, (int)std::min<uint64_t>(kMaxSortSlots, ctx->arena.largest_free() / std::max<uint64_t>(sb, 1)));
  mp.result_buf.assign(mp.S, 0);
  mp.out_keys = out_keys;
  mp.out_vals = out_vals;
  if (ctx->cfg.sched == VX_SCHED_IMMEDIATE) {
    mp.ev0.resize(mp.S);
    mp.ev1.resize(mp.S);
    for (int i = 0; i < mp.S; ++i) {
      VX_CUDA_TRY(cudaEventCreate(&mp.ev0[i]));
      VX_CUDA_TRY(cudaEventCreate(&mp.ev1[i]));
    }
  }
  ExecStats es;
  VX_TRY(run_pipeline(ctx, mp, &es));
  ss.bytes_h2d += es.bytes_h2d;
  ss.bytes_d2h += es.bytes_d2h;
  ss.kernel_launches += es.kernel_launches;
  ss.ms_merge_kernel += mp.ms_merge;
  ss.merge_pass_pairs += mp.rounds_pairs;
  ss.slot_pairs = mp.cap;
  ss.ms_sort += now_ms() - tq;
  return VX_OK;
}

}  // namespace vx

using namespace vx;

VX_API vx_status vx_exact_splits(vx_ctx *ctx, const uint64_t *keys, const uint64_t *run_off, uint32_t n_runs,
                                 const uint64_t *ranks, uint32_t n_ranks, uint64_t *out) {
  clear_error();
  VX_TRY(check_ctx(ctx));
  if (n_runs == 0 || n_runs > kMaxRuns || !run_off || (n_ranks && (!ranks || !out)) || run_off[0] != 0) {
    set_error("vx_exact_splits: bad argument (1 <= n_runs <= %u, run_off[0] == 0)", kMaxRuns);
    return VX_E_INVAL;
  }
  for (uint32_t r = 0; r < n_runs; ++r)
    if (run_off[r + 1] < run_off[r]) {
      set_error("vx_exact_splits: run offsets decrease at run %u", r);
      return VX_E_INVAL;
    }
  const uint64_t n = run_off[n_runs];
  if (n && !keys) {
    set_error("vx_exact_splits: null keys");
    return VX_E_INVAL;
  }
  std::lock_guard<std::recursive_mutex> g(ctx->mu);
  HostReg reg;
  VX_TRY(reg.add((void *)keys, 8 * n));
  void *dk = nullptr;
  if (n) VX_CUDA_TRY(cudaHostGetDevicePointer(&dk, (void *)keys, 0));
  std::vector<uint64_t> ro(run_off, run_off + n_runs + 1), fs(n_runs);
  uint64_t nf = 0;
  for (uint32_t r = 0; r < n_runs; ++r) {
    fs[r] = nf;
    nf += (ro[r + 1] - ro[r] + kFenceStride - 1) / kFenceStride;
  }
  DevBuf fb;
  fb.arena = &ctx->arena;
  fb.p = ctx->arena.alloc(8 * std::max<uint64_t>(nf, 1));
  if (!fb.p) {
    set_error("vx_exact_splits: fences do not fit the arena");
    return VX_E_NOMEM;
  }
  cudaStream_t s = ctx->s_compute;
  for (uint32_t r = 0; r < n_runs; ++r) {
    const uint64_t len = ro[r + 1] - ro[r];
    if (!len) continue;
    const uint64_t f = (len + kFenceStride - 1) / kFenceStride;
    run_fences_kernel<<<(unsigned)std::min<uint64_t>((f + 255) / 256, 1024), 256, 0, s>>>(
        (const uint64_t *)dk + ro[r], nullptr, nullptr, len, fb.as<uint64_t>() + fs[r]);
  }
  VX_CUDA_TRY(cudaGetLastError());
  std::vector<uint64_t> rk(ranks, ranks + n_ranks), res;
  VX_TRY(exact_cuts(ctx, (const uint64_t *)dk, ro, fs, fb.as<uint64_t>(), rk, &res));
  if (n_ranks) memcpy(out, res.data(), 8ull * n_ranks * n_runs);
  return VX_OK;
}

VX_API vx_status vx_merge_runs(vx_ctx *ctx, const uint64_t *keys, const uint32_t *vals, const uint64_t *run_off,
                               uint32_t n_runs, uint64_t *out_keys, uint32_t *out_vals) {
  clear_error();
  VX_TRY(check_ctx(ctx));
  if (n_runs == 0 || n_runs > kMaxRuns || !run_off || run_off[0] != 0) {
    set_error("vx_merge_runs: bad argument (1 <= n_runs <= %u, run_off[0] == 0)", kMaxRuns);
    return VX_E_INVAL;
  }
  std::vector<uint64_t> lens(n_runs);
  for (uint32_t r = 0; r < n_runs; ++r) {
    if (run_off[r + 1] < run_off[r]) {
      set_error("vx_merge_runs: run offsets decrease at run %u", r);
      return VX_E_INVAL;
    }
    lens[r] = run_off[r + 1] - run_off[r];
  }
  const uint64_t n = run_off[n_runs];
  if (n == 0) return VX_OK;
  if (!keys || !vals || !out_keys || !out_vals) {
    set_error("vx_merge_runs: null buffer");
    return VX_E_INVAL;
  }
  std::lock_guard<std::recursive_mutex> g(ctx->mu);
  const uint64_t kb = (8 * n + 255) & ~255ull, vb = (4 * n + 255) & ~255ull;
  const uint64_t cb = (8 * (n / kMergeTile + 2) + 255) & ~255ull;
  DevBuf buf;
  buf.arena = &ctx->arena;
  buf.p = ctx->arena.alloc(2 * kb + 2 * vb + cb);
  if (!buf.p) {
    set_error("vx_merge_runs: %llu pairs do not fit the arena twice", (unsigned long long)n);
    return VX_E_NOMEM;
  }
  RadixBufs b;
  b.keys[0] = buf.as<uint64_t>();
  b.keys[1] = (uint64_t *)(buf.as<char>() + kb);
  b.vals[0] = (uint32_t *)(buf.as<char>() + 2 * kb);
  b.vals[1] = (uint32_t *)(buf.as<char>() + 2 * kb + vb);
  cudaStream_t s = ctx->s_compute;
  VX_CUDA_TRY(cudaMemcpyAsync(b.keys[0], keys, 8 * n, cudaMemcpyHostToDevice, s));
  VX_CUDA_TRY(cudaMemcpyAsync(b.vals[0], vals, 4 * n, cudaMemcpyHostToDevice, s));
  uint64_t rounds = 0;
  const int c = merge_enqueue(b, n, segments_of(lens), (uint64_t *)(buf.as<char>() + 2 * kb + 2 * vb), s, &rounds);
  VX_CUDA_TRY(cudaGetLastError());
  VX_CUDA_TRY(cudaMemcpyAsync(out_keys, b.keys[c], 8 * n, cudaMemcpyDeviceToHost, s));
  VX_CUDA_TRY(cudaMemcpyAsync(out_vals, b.vals[c], 4 * n, cudaMemcpyDeviceToHost, s));
  VX_CUDA_TRY(cudaStreamSynchronize(s));
  return VX_OK;
}
