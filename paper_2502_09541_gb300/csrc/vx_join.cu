// Partitioned hash join beyond the device budget (Section 6.2: equi-join of
// two tables larger than device memory; A.key == B.key with unique build
// keys), reporting count, wrapping payload sum and a pair fingerprint.
//
// The build side is cut into P key ranges by splitters (sample or learned CDF
// model over the build keys).  For each range p: the build side streams
// through the executor and keys of range p are inserted into an
// open-addressing table in HBM; then the probe side streams and keys of range
// p probe it.  No partition is materialised in host memory: with the host
// link as the only IO path and P small (P = 1 when the table fits), reading
// the inputs P times moves fewer bytes than a partition pass that writes and
// re-reads both sides.  Tables are sized either by an exact count pass over
// the build keys (plain form) or from the partition sizes the model predicts
// (learned form; an overflowing table is rebuilt larger).
#include <algorithm>
#include <cmath>

#include "vx_internal.h"
#include "vx_sort.cuh"

namespace vx {

constexpr uint64_t kJoinEmpty = ~0ull;  // empty-slot key; a build key equal to it is kept aside

struct JoinSlot {
  unsigned long long key;
  unsigned long long payload;
};

struct JoinAcc {
  unsigned long long count, psum, fp, inserted, sentinel_present, sentinel_payload;
  unsigned long long max_disp;  // longest probe distance of any inserted key
  uint32_t err;
};

// an insertion that needs more steps than this marks the table overflowed
constexpr uint64_t kMaxInsertSteps = 1ull << 16;

__device__ __forceinline__ uint64_t fmix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Linear probing whose walk starts at a bucket boundary: the home of a key is
// the first slot of bucket home_bucket(key) (multiply-shift range reduction of
// a mixed key onto the nbk = cap / kJoinBucket buckets), so the home bucket of
// two 16-byte slots is one aligned 32-byte sector.
constexpr int kJoinBucket = 2;
constexpr double kJoinMaxAutoLoad = 0.8, kJoinMinAutoLoad = 0.5;
__device__ __forceinline__ uint64_t home_bucket(uint64_t key, uint64_t nbk) {
  return __umul64hi(fmix64(key ^ 0x2545F4914F6CDD1Dull), nbk);
}

__device__ __forceinline__ bool in_range(uint64_t k, uint64_t lo, uint64_t hi, bool last) {
  return k >= lo && (last || k < hi);
}

__global__ void join_fill_kernel(JoinSlot *t, uint64_t cap) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < cap; i += (uint64_t)gridDim.x * blockDim.x) {
    t[i].key = kJoinEmpty;
    t[i].payload = 0;
  }
}

// counts build keys per partition (plain form's exact sizing pass)
__global__ void join_count_kernel(const uint64_t *keys, uint64_t n, const uint64_t *spl, int n_spl,
                                  unsigned long long *counts) {
  __shared__ uint64_t s_spl[256];
  __shared__ unsigned int c[257];
  for (int i = threadIdx.x; i < n_spl; i += blockDim.x) s_spl[i] = spl[i];
  for (int i = threadIdx.x; i <= n_spl; i += blockDim.x) c[i] = 0;
  __syncthreads();
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t k = keys[i];
    int lo = 0, hi = n_spl;
    while (lo < hi) {
      int mid = (lo + hi) >> 1;
      if (s_spl[mid] <= k) lo = mid + 1;
      else hi = mid;
    }
    atomicAdd(&c[lo], 1u);
  }
  __syncthreads();
  for (int i = threadIdx.x; i <= n_spl; i += blockDim.x)
    if (c[i]) atomicAdd(&counts[i], (unsigned long long)c[i]);
}

__global__ void join_build_kernel(const uint64_t *keys, const uint64_t *payload, uint64_t n, uint64_t lo, uint64_t hi,
                                  bool last, JoinSlot *t, uint64_t cap, JoinAcc *acc) {
  unsigned long long ins = 0, disp = 0;  // per-thread count and longest displacement
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t k = keys[i];
    if (!in_range(k, lo, hi, last)) continue;
    const uint64_t pay = payload[i];
    ++ins;
    if (k == kJoinEmpty) {
      if (atomicExch(&acc->sentinel_present, 1ull)) atomicOr(&acc->err, ERR_DUPKEY);
      acc->sentinel_payload = pay;
      continue;
    }
    uint64_t h = home_bucket(k, cap / kJoinBucket) * kJoinBucket;
    bool done = false;
    const uint64_t limit = cap < kMaxInsertSteps ? cap : kMaxInsertSteps;
    for (uint64_t step = 0; step < limit; ++step) {
      const unsigned long long old = atomicCAS(&t[h].key, kJoinEmpty, k);
      if (old == kJoinEmpty) {
        t[h].payload = pay;
        disp = step > disp ? step : disp;
        done = true;
        break;
      }
      if (old == k) {
        atomicOr(&acc->err, ERR_DUPKEY);
        done = true;
        break;
      }
      h = h + 1 == cap ? 0 : h + 1;
    }
    if (!done) atomicOr(&acc->err, ERR_HT_FULL);
  }
  for (int off = 16; off > 0; off >>= 1) {
    ins += __shfl_down_sync(0xffffffffu, ins, off);
    const unsigned long long o = __shfl_down_sync(0xffffffffu, disp, off);
    disp = o > disp ? o : disp;
  }
  if ((threadIdx.x & 31) == 0 && ins) {
    atomicAdd(&acc->inserted, ins);
    atomicMax(&acc->max_disp, disp);
  }
}

// probes the keys of range p; row0 = global row of keys[0].
// A table much larger than L2 makes every probe a random DRAM access, and the
// rate of random 32-byte sectors, not bandwidth or latency, bounds the kernel.
// So a probe reads its home bucket (two slots, one aligned sector) in one
// access, and each thread keeps kRows rows in flight in lock-step rounds: all
// unresolved rows issue their next bucket read together, so a row with a long
// chain costs rounds, not a serial walk after the rows before it.
template <int kRows>
__global__ void __launch_bounds__(256, 4) join_probe_kernel(const uint64_t *__restrict__ keys, uint64_t n,
                                                            uint64_t row0, uint64_t lo, uint64_t hi, bool last,
                                                            const JoinSlot *__restrict__ t, uint64_t cap,
                                                            JoinAcc *acc) {
  unsigned long long c = 0, s = 0, f = 0;
  const bool sp = acc->sentinel_present != 0;
  const uint64_t spay = acc->sentinel_payload;
  const uint64_t nbk = cap / kJoinBucket;
  // every key sits within max_disp slots of its (bucket-aligned) home
  const uint64_t max_rounds = acc->max_disp / kJoinBucket + 1;
  const ulonglong2 *tv = reinterpret_cast<const ulonglong2 *>(t);
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x * kRows;
  for (uint64_t base = (uint64_t)blockIdx.x * blockDim.x * kRows + threadIdx.x; base < n; base += stride) {
    uint64_t k[kRows], b[kRows];
    unsigned live = 0;
#pragma unroll
    for (int j = 0; j < kRows; ++j) {
      const uint64_t i = base + (uint64_t)j * blockDim.x;
      k[j] = i < n ? keys[i] : kJoinEmpty;
      if (i < n && in_range(k[j], lo, hi, last)) {
        if (k[j] != kJoinEmpty) {
          live |= 1u << j;
        } else if (sp) {  // the empty-slot key matches only the build row kept aside
          c += 1;
          s += spay;
          f += fmix64((row0 + i) ^ ((spay << 17) | (spay >> 47)));
        }
      }
      b[j] = home_bucket(k[j], nbk);
    }
    for (uint64_t round = 0; live && round < max_rounds; ++round) {
      ulonglong2 v[kRows][kJoinBucket];
#pragma unroll
      for (int j = 0; j < kRows; ++j)
        if (live >> j & 1)
#pragma unroll
          for (int q = 0; q < kJoinBucket; ++q) v[j][q] = __ldg(tv + b[j] * kJoinBucket + q);
#pragma unroll
      for (int j = 0; j < kRows; ++j) {
        if (!(live >> j & 1)) continue;
        bool hit = false, empty = false;
        uint64_t pay = 0;
#pragma unroll
        for (int q = 0; q < kJoinBucket; ++q) {
          if (v[j][q].x == k[j]) {
            hit = true;
            pay = v[j][q].y;
          }
          empty |= v[j][q].x == kJoinEmpty;
        }
        if (hit) {
          c += 1;
          s += pay;
          f += fmix64((row0 + base + (uint64_t)j * blockDim.x) ^ ((pay << 17) | (pay >> 47)));
        }
        // no deletions and bucket-aligned homes: a key lies before the first
        // empty slot of its walk, so an empty slot in the bucket ends it
        if (hit || empty) live &= ~(1u << j);
        else b[j] = b[j] + 1 == nbk ? 0 : b[j] + 1;
      }
    }
  }
  for (int off = 16; off > 0; off >>= 1) {
    c += __shfl_down_sync(0xffffffffu, c, off);
    s += __shfl_down_sync(0xffffffffu, s, off);
    f += __shfl_down_sync(0xffffffffu, f, off);
  }
  // one set of global atomics per block (wrapping sums are order-free)
  __shared__ unsigned long long bc[8], bs[8], bf[8];
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    bc[w] = c;
    bs[w] = s;
    bf[w] = f;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long tc = 0, ts = 0, tf = 0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
      tc += bc[i];
      ts += bs[i];
      tf += bf[i];
    }
    if (tc) {
      atomicAdd(&acc->count, tc);
      atomicAdd(&acc->psum, ts);
      atomicAdd(&acc->fp, tf);
    }
  }
}

// ------------------------------------------------------------------ host

namespace {

int grid_of(vx_ctx *ctx, uint64_t items, int threads, int per_sm) {
  uint64_t g = (items + threads - 1) / threads;
  uint64_t cap = (uint64_t)ctx->num_sms * per_sm;
  return (int)std::max<uint64_t>(1, std::min(g, cap));
}

// streams a key column (and optional payload column) in chunks
struct StreamPass : ExKernel {
  vx_ctx *ctx;
  const uint64_t *keys;
  const uint64_t *payload;  // null for the probe side
  uint64_t n, R;
  uint64_t row_base = 0;  // global row of keys[0] (the probe fingerprint uses global rows)
  std::function<vx_status(const uint64_t *, const uint64_t *, uint64_t, uint64_t, cudaStream_t)> fn;
  uint64_t size() override { return (n + R - 1) / R; }
  uint64_t rows(uint64_t it) const { return std::min(R, n - it * R); }
  uint64_t kb() const { return (8 * R + 255) & ~255ull; }
  uint64_t slot_bytes() override { return kb() * (payload ? 2 : 1); }
  void inputs(uint64_t it, char *slot, std::vector<CopyOp> &h2d) override {
    h2d.push_back({keys + it * R, slot, 8 * rows(it)});
    if (payload) h2d.push_back({payload + it * R, slot + kb(), 8 * rows(it)});
  }
  vx_status kernel(char *slot, uint64_t it, cudaStream_t s) override {
    return fn((const uint64_t *)slot, payload ? (const uint64_t *)(slot + kb()) : nullptr, rows(it), row_base + it * R,
              s);
  }
};

}  // namespace

}  // namespace vx

using namespace vx;

VX_API vx_status vx_join(vx_ctx *ctx, int32_t build_key, int32_t build_payload, int32_t probe_key,
                         const vx_join_opts *opts, vx_join_result *out) {
  clear_error();
  VX_TRY(check_ctx(ctx));
  if (!out) return VX_E_INVAL;
  std::lock_guard<std::recursive_mutex> g(ctx->mu);
  const Column *bk = get_col(ctx, build_key, -1);
  const Column *bp = get_col(ctx, build_payload, -1);
  const Column *pk = get_col(ctx, probe_key, -1);
  if (!bk || !bp || !pk) return VX_E_INVAL;
  return join_columns(ctx, bk, bp, pk, 0, pk->n_rows, opts, out);
}

namespace vx {

vx_status join_columns(vx_ctx *ctx, const Column *bk, const Column *bp, const Column *pk, uint64_t probe_begin,
                       uint64_t probe_end, const vx_join_opts *opts, vx_join_result *out) {
  const double t0 = now_ms();
  if (bk->elem != 8 || bp->elem != 8 || pk->elem != 8 || bk->n_rows != bp->n_rows) {
    set_error("vx_join: keys and payload must be 64-bit columns; build key and payload of equal length");
    return VX_E_INVAL;
  }
  probe_end = std::min(probe_end, pk->n_rows);
  probe_begin = std::min(probe_begin, probe_end);
  vx_join_opts o{};
  if (opts) o = *opts;
  // load factor 0 = automatic: partitions are counted at load 0.8, then each
  // table spreads over the free budget down to load 0.5 (fewer sectors per probe)
  const bool auto_load = o.load_factor <= 0;
  if (auto_load) o.load_factor = kJoinMaxAutoLoad;
  if (o.load_factor > 0.95 || o.n_partitions < 0 || o.n_partitions > 256 || o.partitioner < VX_PART_SAMPLE ||
      o.partitioner > VX_PART_LEARNED_MLP || (o.algorithm != VX_JOIN_DIRECT && o.algorithm != VX_JOIN_RADIX)) {
    set_error("vx_join: bad options");
    return VX_E_INVAL;
  }
  if (o.algorithm == VX_JOIN_RADIX) {
    if (probe_begin != 0 || probe_end != pk->n_rows) {
      set_error("vx_join: the radix join probes whole columns");
      return VX_E_UNSUPPORTED;
    }
    return radix_join(ctx, bk, bp, pk, o, out);
  }
  const uint64_t nb = bk->n_rows, np = probe_end - probe_begin;
  vx_join_result res{};
  cudaStream_t s = ctx->s_compute;
  DevBuf accb;
  accb.arena = &ctx->arena;
  accb.p = ctx->arena.alloc(256 + kSplitterBufBytes + 8 * 258 + 1024);
  if (!accb.p) {
    set_error("vx_join: arena exhausted");
    return VX_E_NOMEM;
  }
  JoinAcc *acc = accb.as<JoinAcc>();
  uint64_t *d_spl = (uint64_t *)(accb.as<char>() + 256);
  unsigned long long *d_counts = (unsigned long long *)((char *)d_spl + kSplitterBufBytes);
  VX_CUDA_TRY(cudaMemsetAsync(acc, 0, sizeof(JoinAcc), s));

  // staging per slot: build side 16 B/row; slots sized by chunk_bytes
  const int S = std::max(2, ctx->cfg.n_slots);
  uint64_t R = std::max<uint64_t>(ctx->cfg.chunk_bytes / 16, 1 << 16);
  const uint64_t staging = (uint64_t)S * (16 * R + 512);
  const uint64_t avail = ctx->arena.largest_free();
  if (avail < staging + (1 << 20)) {
    set_error("vx_join: budget too small for %d staging slots", S);
    return VX_E_NOMEM;
  }
  const uint64_t table_bytes_max = (uint64_t)((avail - staging) * 0.98);
  const uint64_t slots_max = table_bytes_max / sizeof(JoinSlot) / kJoinBucket * kJoinBucket;
  // ---- partitions: P such that each table (at the load factor) fits
  uint32_t P = o.n_partitions > 0 ? (uint32_t)o.n_partitions
                                  : (uint32_t)std::max<double>(1.0, std::ceil(nb / (o.load_factor * slots_max) * 1.05));
  if (P > kMaxRequestedPartitions) {
    set_error("vx_join: more than %u partitions needed", kMaxRequestedPartitions);
    return VX_E_UNSUPPORTED;
  }
  std::vector<uint64_t> spl;
  std::vector<uint64_t> part_n(P, nb);
  double tsp = now_ms();
  if (P > 1) {
    uint64_t m = std::min<uint64_t>(o.sample_size ? o.sample_size : (1ull << 20), nb);
    DevBuf sbuf;
    uint64_t *sorted = nullptr;
    VX_TRY(sample_and_sort(ctx, (const uint64_t *)bk->dev, nb, m, o.seed, sbuf, &sorted));
    double ms_train = 0;
    uint32_t n_spl = 0;
    VX_TRY(splitters_from_sample(ctx, o.partitioner, sorted, m, P, d_spl, 0, &ms_train, &n_spl));
    P = n_spl + 1;  // after heavy-key isolation
    part_n.assign(P, nb);
    spl.resize(n_spl);
    if (n_spl) VX_CUDA_TRY(cudaMemcpyAsync(spl.data(), d_spl, 8ull * n_spl, cudaMemcpyDeviceToHost, s));
    VX_CUDA_TRY(cudaStreamSynchronize(s));
    res.ms_train = ms_train;
    if (o.count_pass) {  // plain form: exact partition sizes from one pass over the build keys
      VX_CUDA_TRY(cudaMemsetAsync(d_counts, 0, 8 * 258, s));
      StreamPass cp;
      cp.ctx = ctx;
      cp.keys = (const uint64_t *)bk->host;
      cp.payload = nullptr;
      cp.n = nb;
      cp.R = 2 * R;
      cp.fn = [&](const uint64_t *k, const uint64_t *, uint64_t n, uint64_t, cudaStream_t st) -> vx_status {
        join_count_kernel<<<grid_of(ctx, n, 256, 4), 256, 0, st>>>(k, n, d_spl, (int)P - 1, d_counts);
        VX_CUDA_TRY(cudaGetLastError());
        return VX_OK;
      };
      ExecStats es;
      VX_TRY(run_pipeline(ctx, cp, &es));
      res.bytes_h2d += es.bytes_h2d;
      res.kernel_launches += es.kernel_launches;
      std::vector<unsigned long long> cnt(P);
      VX_CUDA_TRY(cudaMemcpy(cnt.data(), d_counts, 8 * P, cudaMemcpyDeviceToHost));
      for (uint32_t p = 0; p < P; ++p) part_n[p] = cnt[p];
    } else {  // learned form: the model cuts at quantiles p/P, so each range holds ~nb/P keys
      for (uint32_t p = 0; p < P; ++p) part_n[p] = (uint64_t)std::ceil((double)nb / P * 1.02) + 4096;
    }
  }
  res.ms_sample = now_ms() - tsp;
  res.n_partitions = P;

  // ---- per partition: build, then probe
  for (uint32_t p = 0; p < P; ++p) {
    const uint64_t lo = p == 0 ? 0 : spl[p - 1];
    const uint64_t hi = p + 1 < P ? spl[p] : ~0ull;
    const bool last = p + 1 == P;
    if (p > 0 && p + 1 < P && hi <= lo) continue;  // empty range
    uint64_t cap = std::max<uint64_t>((uint64_t)std::ceil(part_n[p] / o.load_factor), 1024);
    if (auto_load)
      cap = std::max(cap, std::min<uint64_t>((uint64_t)std::ceil(part_n[p] / kJoinMinAutoLoad), slots_max));
    cap = (cap + kJoinBucket - 1) / kJoinBucket * kJoinBucket;
    for (int attempt = 0;; ++attempt) {
      if (cap > slots_max) {
        set_error("vx_join: partition %u needs %llu slots; %llu fit", p, (unsigned long long)cap,
                  (unsigned long long)slots_max);
        return VX_E_NOMEM;
      }
      DevBuf tb;
      tb.arena = &ctx->arena;
      tb.p = ctx->arena.alloc(cap * sizeof(JoinSlot));
      if (!tb.p) {
        set_error("vx_join: table of %llu bytes does not fit", (unsigned long long)(cap * sizeof(JoinSlot)));
        return VX_E_NOMEM;
      }
      JoinSlot *t = tb.as<JoinSlot>();
      join_fill_kernel<<<grid_of(ctx, cap, 256, 8), 256, 0, s>>>(t, cap);
      VX_CUDA_TRY(cudaMemsetAsync(&acc->inserted, 0, 8, s));
      VX_CUDA_TRY(cudaMemsetAsync(&acc->err, 0, 4, s));
      VX_CUDA_TRY(cudaMemsetAsync(&acc->sentinel_present, 0, 24, s));  // sentinel flag, payload, max_disp
      double tb0 = now_ms();
      StreamPass bpass;
      bpass.ctx = ctx;
      bpass.keys = (const uint64_t *)bk->host;
      bpass.payload = (const uint64_t *)bp->host;
      bpass.n = nb;
      bpass.R = R;
      bpass.fn = [&](const uint64_t *k, const uint64_t *pay, uint64_t n, uint64_t, cudaStream_t st) -> vx_status {
        join_build_kernel<<<grid_of(ctx, n, 256, 8), 256, 0, st>>>(k, pay, n, lo, hi, last, t, cap, acc);
        VX_CUDA_TRY(cudaGetLastError());
        return VX_OK;
      };
      ExecStats es;
      VX_TRY(run_pipeline(ctx, bpass, &es));
      res.bytes_h2d += es.bytes_h2d;
      res.kernel_launches += es.kernel_launches + 1;
      VX_CUDA_TRY(cudaStreamSynchronize(s));
      res.ms_build += now_ms() - tb0;
      JoinAcc h{};
      VX_CUDA_TRY(cudaMemcpy(&h, acc, sizeof(JoinAcc), cudaMemcpyDeviceToHost));
      if (h.err & ERR_DUPKEY) {
        set_error("vx_join: duplicate build key");
        return VX_E_DUPKEY;
      }
      if ((h.err & ERR_HT_FULL) || h.inserted > (uint64_t)(0.95 * cap)) {
        // the table overflowed its load limit: rebuild larger (learned sizing's retry)
        res.overflow_retries += 1;
        // at least double: an overflow from the probe-walk limit (clustered
        // homes) is not cured by a table sized for the same load again; the
        // last attempt takes the largest table that fits
        const uint64_t need = (uint64_t)std::ceil(h.inserted / o.load_factor) + 4096;
        uint64_t grow = std::max<uint64_t>(2 * cap, need);
        if (grow > slots_max && need <= slots_max && cap < slots_max) grow = slots_max;
        cap = grow / kJoinBucket * kJoinBucket;
        if (attempt >= 3) {
          set_error("vx_join: table sizing did not converge");
          return VX_E_NOMEM;
        }
        continue;
      }
      res.max_partition = std::max<uint64_t>(res.max_partition, h.inserted);
      double tp0 = now_ms();
      StreamPass ppass;
      ppass.ctx = ctx;
      ppass.keys = (const uint64_t *)pk->host + probe_begin;
      ppass.payload = nullptr;
      ppass.n = np;
      ppass.R = 2 * R;
      ppass.row_base = probe_begin;
      ppass.fn = [&](const uint64_t *k, const uint64_t *, uint64_t n, uint64_t row0, cudaStream_t st) -> vx_status {
        join_probe_kernel<4><<<grid_of(ctx, (n + 3) / 4, 256, 4), 256, 0, st>>>(k, n, row0, lo, hi, last, t, cap,
                                                                               acc);
        VX_CUDA_TRY(cudaGetLastError());
        return VX_OK;
      };
      ExecStats ep;
      if (np) VX_TRY(run_pipeline(ctx, ppass, &ep));
      VX_CUDA_TRY(cudaStreamSynchronize(s));
      res.bytes_h2d += ep.bytes_h2d;
      res.kernel_launches += ep.kernel_launches;
      res.ms_probe += now_ms() - tp0;
      res.ms_kernel += es.ms_kernel + ep.ms_kernel;
      res.ms_probe_kernel += ep.ms_kernel;
      break;
    }
  }
  JoinAcc h{};
  VX_CUDA_TRY(cudaMemcpy(&h, acc, sizeof(JoinAcc), cudaMemcpyDeviceToHost));
  res.count = h.count;
  res.payload_sum = h.psum;
  res.pair_fp = h.fp;
  res.ms_total = now_ms() - t0;
  *out = res;
  return VX_OK;
}

}  // namespace vx
