// Radix-partitioned hash join (Section 6.2): the paper's RadixPartitionExKer
// and HashJoinExKer, for an equi-join of two tables larger than the budget.
//
// RadixPartitionExKer.  Each chunk of a table is clustered by the low b bits
// of the key (b = 24: 2^24 groups): a stable LSD radix sort over the low b/8
// key bytes of (key, chunk-local row) pairs, then find_boundary (Section
// 6.2.1, Fig. 9) — a boundary array of 2^b + 1 entries starts as
// placeholders, every position whose group differs from the previous
// position's records itself at its group's entry, the last entry is the
// chunk length, and each remaining placeholder takes the next valid entry to
// its right (a suffix minimum).  The clustered keys, the build side's
// payloads (gathered by the sorted local rows) or the probe side's local rows,
// and the boundary array go back to host memory.
//
// HashJoinExKer.  The data mapping cuts the 2^b groups into ranges whose
// tuples fit a staging slot, by binary search over the boundary arrays (the
// tuples of groups [g0, g1) in chunk c are [B_c[g0], B_c[g1]) of its
// clustered chunk).  A range's segments of every chunk of both tables and the
// slices B_c[g0 .. g1] of their boundary arrays are loaded; one warp joins one
// group in shared memory: lane c inserts chunk c's build tuples of the group
// into an open-addressing table sized to the group (at most 256 slots; a
// group with more build tuples is joined by a scan of its build tuples), then
// lane c probes with chunk c's probe tuples of the group.  Matches add to a
// count, a wrapping payload sum and the pair fingerprint
// mix64(probe_row ^ rotl(payload, 17)), probe_row = chunk * R + local row.
#include <algorithm>
#include <cmath>

#include "vx_internal.h"
#include "vx_sort.cuh"

namespace vx {

namespace {

constexpr uint32_t kRjNone = 0xFFFFFFFFu;  // boundary placeholder
constexpr int kRjSeg = 4096;               // boundary entries per block of the back-fill
constexpr int kRjWarps = 8;
constexpr int kRjTable = 256;              // slots of a warp's shared-memory table
constexpr uint64_t kRjEmpty = ~0ull;       // empty slot key; a build key equal to it is kept aside
// a group with more probe tuples than this (skewed probe keys) is joined by
// kRjHeavyParts blocks at once instead of one warp
constexpr uint64_t kRjHeavy = 8192;
constexpr uint32_t kRjHeavyCap = 1u << 16, kRjHeavyParts = 32;

__device__ __forceinline__ uint64_t rj_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__global__ void rj_iota_kernel(uint32_t *v, uint64_t n) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
    v[i] = (uint32_t)i;
}

// find_boundary, step 2: a position whose group differs from the previous
// position's records itself at its group's entry; the last entry is n
__global__ void rj_mark_kernel(const uint64_t *k0, const uint64_t *k1, const RadixState *st, int npass, uint64_t n,
                               uint64_t mask, uint32_t *bnd) {
  const uint64_t *k = st->cur[npass] ? k1 : k0;
  const uint64_t G = mask + 1;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t h = k[i] & mask;
    if (i == 0 || h != (k[i - 1] & mask)) bnd[h] = (uint32_t)i;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) bnd[G] = (uint32_t)n;
}

// find_boundary, step 3: each placeholder takes the next valid entry to its
// right.  Valid entries increase along the array, so that is the suffix
// minimum; per segment of kRjSeg entries first (its minimum to carry[seg]),
// then over the segments' carries, then applied.
__global__ void __launch_bounds__(256) rj_fill_local_kernel(uint32_t *bnd, uint64_t m, uint32_t *carry) {
  __shared__ uint32_t tmin[256];
  const uint64_t s0 = (uint64_t)blockIdx.x * kRjSeg;
  constexpr int kPer = kRjSeg / 256;
  const uint64_t a = s0 + (uint64_t)threadIdx.x * kPer;
  uint32_t v[kPer];
  uint32_t run = kRjNone;
#pragma unroll
  for (int j = kPer - 1; j >= 0; --j) {
    v[j] = a + j < m ? bnd[a + j] : kRjNone;
    run = v[j] < run ? v[j] : run;
    v[j] = run;
  }
  tmin[threadIdx.x] = run;
  __syncthreads();
  // minimum over the threads to the right (a suffix scan over 256 values)
  for (int off = 1; off < 256; off <<= 1) {
    const uint32_t y = threadIdx.x + off < 256 ? tmin[threadIdx.x + off] : kRjNone;
    __syncthreads();
    if (y < tmin[threadIdx.x]) tmin[threadIdx.x] = y;
    __syncthreads();
  }
  const uint32_t right = threadIdx.x + 1 < 256 ? tmin[threadIdx.x + 1] : kRjNone;
#pragma unroll
  for (int j = 0; j < kPer; ++j)
    if (a + j < m) bnd[a + j] = v[j] < right ? v[j] : right;
  if (threadIdx.x == 0) carry[blockIdx.x] = tmin[0];
}

__global__ void __launch_bounds__(1024) rj_fill_carry_kernel(uint32_t *carry, uint32_t nseg) {
  // one block: carry[s] becomes the minimum over segments after s (exclusive suffix minimum)
  __shared__ uint32_t sm[1024];
  uint32_t run = kRjNone;
  const uint32_t per = (nseg + 1023) / 1024;
  const uint32_t a = threadIdx.x * per;
  for (uint32_t j = 0; j < per; ++j)
    if (a + j < nseg && carry[a + j] < run) run = carry[a + j];
  sm[threadIdx.x] = run;
  __syncthreads();
  for (int off = 1; off < 1024; off <<= 1) {
    const uint32_t y = threadIdx.x + off < 1024 ? sm[threadIdx.x + off] : kRjNone;
    __syncthreads();
    if (y < sm[threadIdx.x]) sm[threadIdx.x] = y;
    __syncthreads();
  }
  uint32_t after = threadIdx.x + 1 < 1024 ? sm[threadIdx.x + 1] : kRjNone;
  for (int j = (int)per - 1; j >= 0; --j) {
    if (a + j >= nseg) continue;
    const uint32_t own = carry[a + j];
    carry[a + j] = after;
    if (own < after) after = own;
  }
}

__global__ void rj_fill_apply_kernel(uint32_t *bnd, uint64_t m, const uint32_t *carry) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < m; i += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t c = carry[i / kRjSeg];
    if (c < bnd[i]) bnd[i] = c;
  }
}

// payload of the clustered build tuples: out[i] = in[sorted local row i]
__global__ void rj_gather_kernel(const uint32_t *v0, const uint32_t *v1, const RadixState *st, int npass, uint64_t n,
                                 const uint64_t *in, uint64_t *out) {
  const uint32_t *v = st->cur[npass] ? v1 : v0;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
    out[i] = in[v[i]];
}

struct RjAcc {
  unsigned long long count, psum, fp;
  uint32_t err;
};

// one range of groups, all chunks of both tables loaded into the slot
struct RjJoinParams {
  const uint64_t *akeys, *apay;  // build tuples of the range, chunk after chunk
  const uint64_t *bkeys;         // probe tuples of the range, chunk after chunk
  const uint32_t *brows;         // their chunk-local rows
  const uint32_t *abnd, *bbnd;   // per chunk, boundary slice B_c[g0 .. g1] (ng + 1 entries)
  const uint64_t *abase, *bbase; // per chunk, first tuple of the chunk's segment in the slot
  uint32_t na, nb, ng;           // build chunks, probe chunks, groups of the range
  uint64_t probe_chunk_rows;     // R of the probe side's partition pass
  uint32_t key_shift;            // the group bits: the in-group hash uses the key above them
  RjAcc *acc;
  uint32_t *heavy;               // groups left to rj_heavy_kernel (at most kRjHeavyCap)
  unsigned int *heavy_n;
};

// Calls f(c, idx) for every tuple of group g in the chunks of one side, with
// the warp's lanes spread over the group's tuples in all chunks at once rather
// than chunk after chunk: lane c of each batch of 32 chunks loads chunk c's
// boundaries (one round of loads for the batch), a warp scan turns the
// segments' lengths into offsets, and tuple i of the batch goes to lane
// i mod 32, which finds its chunk by a binary search over the scan (five
// shuffles).  Every lane must call it (warp collectives); f runs only for real
// tuples.
template <class F>
__device__ __forceinline__ void rj_for_group_tuples(const uint32_t *bnd, const uint64_t *base, uint32_t nchunks,
                                                    uint64_t ng1, uint64_t g, uint32_t lane, F &&f) {
  for (uint32_t c0 = 0; c0 < nchunks; c0 += 32) {
    const uint32_t c = c0 + lane;
    uint32_t m = 0;
    uint64_t at = 0;
    if (c < nchunks) {
      const uint32_t *bd = bnd + (uint64_t)c * ng1;
      const uint32_t lo = bd[g];
      m = bd[g + 1] - lo;
      at = base[c] + (lo - bd[0]);
    }
    uint32_t incl = m;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, incl, off);
      if (lane >= (uint32_t)off) incl += y;
    }
    const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
    for (uint32_t i0 = 0; i0 < total; i0 += 32) {
      const uint32_t i = i0 + lane;
      uint32_t k = 0;  // lanes whose inclusive count is <= i: the chunk of tuple i
#pragma unroll
      for (uint32_t step = 16; step > 0; step >>= 1) {
        const uint32_t v = __shfl_sync(0xffffffffu, incl, (int)(k + step - 1));
        if (v <= i) k += step;
      }
      k = k < 31 ? k : 31;
      const uint32_t mk = __shfl_sync(0xffffffffu, m, (int)k), ik = __shfl_sync(0xffffffffu, incl, (int)k);
      const uint64_t ak = __shfl_sync(0xffffffffu, at, (int)k);
      if (i < total) f(c0 + k, ak + (i - (ik - mk)));
    }
  }
}

// the build tuples of group g into the warp's shared-memory table of cap
// slots, the lanes spread over the group's tuples of every chunk
__device__ __forceinline__ void rj_build_group_warp(const RjJoinParams &p, uint64_t g, uint32_t cap, uint32_t lane,
                                                    unsigned long long *tkey, unsigned long long *tpay,
                                                    unsigned long long *sent) {
  rj_for_group_tuples(p.abnd, p.abase, p.na, (uint64_t)p.ng + 1, g, lane, [&](uint32_t, uint64_t idx) {
    const uint64_t k = p.akeys[idx], pay = p.apay[idx];
    if (k == kRjEmpty) {
      if (atomicExch(&sent[0], 1ull)) atomicOr(&p.acc->err, ERR_DUPKEY);
      sent[1] = pay;
      return;
    }
    uint32_t h = (uint32_t)(rj_mix(k >> p.key_shift) & (cap - 1));
    for (uint32_t step = 0; step < cap; ++step) {
      const unsigned long long old = atomicCAS(&tkey[h], kRjEmpty, k);
      if (old == kRjEmpty) {
        tpay[h] = pay;
        break;
      }
      if (old == k) {
        atomicOr(&p.acc->err, ERR_DUPKEY);
        break;
      }
      h = (h + 1) & (cap - 1);
    }
  });
}

// the build tuples of group g into an open-addressing table of cap slots in
// shared memory (threads t = 0, stride of them cooperate); a build key equal
// to the empty marker goes to sent[0..1]
__device__ __forceinline__ void rj_build_group(const RjJoinParams &p, uint64_t g, uint32_t cap, uint32_t t,
                                               uint32_t stride, unsigned long long *tkey, unsigned long long *tpay,
                                               unsigned long long *sent) {
  for (uint32_t c = 0; c < p.na; ++c) {
    const uint32_t *bd = p.abnd + (uint64_t)c * (p.ng + 1);
    const uint64_t at = p.abase[c] + (bd[g] - bd[0]);
    const uint32_t m = bd[g + 1] - bd[g];
    for (uint32_t i = t; i < m; i += stride) {
      const uint64_t k = p.akeys[at + i], pay = p.apay[at + i];
      if (k == kRjEmpty) {
        if (atomicExch(&sent[0], 1ull)) atomicOr(&p.acc->err, ERR_DUPKEY);
        sent[1] = pay;
        continue;
      }
      uint32_t h = (uint32_t)(rj_mix(k >> p.key_shift) & (cap - 1));
      for (uint32_t step = 0; step < cap; ++step) {
        const unsigned long long old = atomicCAS(&tkey[h], kRjEmpty, k);
        if (old == kRjEmpty) {
          tpay[h] = pay;
          break;
        }
        if (old == k) {
          atomicOr(&p.acc->err, ERR_DUPKEY);
          break;
        }
        h = (h + 1) & (cap - 1);
      }
    }
  }
}

// one probe tuple against group g: the shared-memory table, or (in_smem
// false) a scan of the group's build tuples
__device__ __forceinline__ bool rj_probe_one(const RjJoinParams &p, uint64_t g, uint64_t k, bool in_smem,
                                             uint32_t cap, const unsigned long long *tkey,
                                             const unsigned long long *tpay, const unsigned long long *sent,
                                             uint64_t &pay) {
  if (in_smem) {
    if (k == kRjEmpty) {
      pay = sent[1];
      return sent[0] != 0;
    }
    uint32_t h = (uint32_t)(rj_mix(k >> p.key_shift) & (cap - 1));
    for (uint32_t step = 0; step < cap; ++step) {
      const unsigned long long kk = tkey[h];
      if (kk == k) {
        pay = tpay[h];
        return true;
      }
      if (kk == kRjEmpty) return false;
      h = (h + 1) & (cap - 1);
    }
    return false;
  }
  for (uint32_t ca = 0; ca < p.na; ++ca) {
    const uint32_t *ad = p.abnd + (uint64_t)ca * (p.ng + 1);
    const uint64_t aat = p.abase[ca] + (ad[g] - ad[0]);
    for (uint32_t j = 0; j < ad[g + 1] - ad[g]; ++j)
      if (p.akeys[aat + j] == k) {
        pay = p.apay[aat + j];
        return true;
      }
  }
  return false;
}

__global__ void __launch_bounds__(32 * kRjWarps) rj_join_kernel(const RjJoinParams p) {
  __shared__ unsigned long long tkey[kRjWarps][kRjTable];
  __shared__ unsigned long long tpay[kRjWarps][kRjTable];
  __shared__ unsigned long long sent[kRjWarps][2];  // a build key equal to kRjEmpty: present flag, payload
  const uint32_t lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  unsigned long long cnt = 0, psum = 0, fp = 0;
  const uint64_t warps = (uint64_t)gridDim.x * kRjWarps;
  for (uint64_t g = blockIdx.x * (uint64_t)kRjWarps + w; g < p.ng; g += warps) {
    // build and probe tuples of the group, over the chunks
    uint64_t nbuild = 0, nprobe = 0;
    for (uint32_t c = lane; c < p.na; c += 32) {
      const uint32_t *bd = p.abnd + (uint64_t)c * (p.ng + 1);
      nbuild += bd[g + 1] - bd[g];
    }
    for (uint32_t c = lane; c < p.nb; c += 32) {
      const uint32_t *bd = p.bbnd + (uint64_t)c * (p.ng + 1);
      nprobe += bd[g + 1] - bd[g];
    }
    for (int off = 16; off > 0; off >>= 1) {
      nbuild += __shfl_xor_sync(0xffffffffu, nbuild, off);
      nprobe += __shfl_xor_sync(0xffffffffu, nprobe, off);
    }
    if (nprobe > kRjHeavy) {  // many blocks take this group in the second kernel, if the list has room
      unsigned int slot = 0;
      if (lane == 0) slot = atomicAdd(p.heavy_n, 1u);
      slot = __shfl_sync(0xffffffffu, slot, 0);
      if (slot < kRjHeavyCap) {
        if (lane == 0) p.heavy[slot] = (uint32_t)g;
        continue;
      }
    }
    const bool in_smem = nbuild <= kRjTable / 2;
    uint32_t cap = 32;
    while (cap < 2 * nbuild && cap < kRjTable) cap <<= 1;
    if (in_smem) {
      for (uint32_t i = lane; i < cap; i += 32) tkey[w][i] = kRjEmpty;
      if (lane == 0) sent[w][0] = 0;
      __syncwarp();
      rj_build_group_warp(p, g, cap, lane, tkey[w], tpay[w], sent[w]);
      __syncwarp();
    }
    // the lanes spread over the group's probe tuples of every chunk
    rj_for_group_tuples(p.bbnd, p.bbase, p.nb, (uint64_t)p.ng + 1, g, lane, [&](uint32_t c, uint64_t idx) {
      uint64_t pay = 0;
      if (rj_probe_one(p, g, p.bkeys[idx], in_smem, cap, tkey[w], tpay[w], sent[w], pay)) {
        const uint64_t row = (uint64_t)c * p.probe_chunk_rows + p.brows[idx];
        cnt += 1;
        psum += pay;
        fp += rj_mix(row ^ ((pay << 17) | (pay >> 47)));
      }
    });
    __syncwarp();
  }
  for (int off = 16; off > 0; off >>= 1) {
    cnt += __shfl_down_sync(0xffffffffu, cnt, off);
    psum += __shfl_down_sync(0xffffffffu, psum, off);
    fp += __shfl_down_sync(0xffffffffu, fp, off);
  }
  if (lane == 0 && cnt) {
    atomicAdd(&p.acc->count, cnt);
    atomicAdd(&p.acc->psum, psum);
    atomicAdd(&p.acc->fp, fp);
  }
}

// groups with many probe tuples: work item (heavy group h, part q) of
// kRjHeavyParts per group; the block builds the group's table in shared
// memory and probes every kRjHeavyParts-th stripe of 256 tuples of each chunk
__global__ void __launch_bounds__(256) rj_heavy_kernel(const RjJoinParams p) {
  __shared__ unsigned long long tkey[kRjTable], tpay[kRjTable], sent[2];
  __shared__ unsigned long long red[3][8];
  const unsigned int nh = *p.heavy_n < kRjHeavyCap ? *p.heavy_n : kRjHeavyCap;
  unsigned long long cnt = 0, psum = 0, fp = 0;
  for (uint64_t wi = blockIdx.x; wi < (uint64_t)nh * kRjHeavyParts; wi += gridDim.x) {
    const uint64_t g = p.heavy[wi / kRjHeavyParts];
    const uint32_t part = (uint32_t)(wi % kRjHeavyParts);
    uint64_t nbuild = 0;
    for (uint32_t c = 0; c < p.na; ++c) {
      const uint32_t *bd = p.abnd + (uint64_t)c * (p.ng + 1);
      nbuild += bd[g + 1] - bd[g];
    }
    const bool in_smem = nbuild <= kRjTable / 2;
    uint32_t cap = 32;
    while (cap < 2 * nbuild && cap < kRjTable) cap <<= 1;
    __syncthreads();  // the previous item's probes are done with the table
    if (in_smem) {
      for (uint32_t i = threadIdx.x; i < cap; i += blockDim.x) tkey[i] = kRjEmpty;
      if (threadIdx.x == 0) sent[0] = 0;
      __syncthreads();
      rj_build_group(p, g, cap, threadIdx.x, blockDim.x, tkey, tpay, sent);
      __syncthreads();
    }
    for (uint32_t c = 0; c < p.nb; ++c) {
      const uint32_t *bd = p.bbnd + (uint64_t)c * (p.ng + 1);
      const uint64_t at = p.bbase[c] + (bd[g] - bd[0]);
      const uint32_t m = bd[g + 1] - bd[g];
      for (uint64_t i = (uint64_t)part * 256 + threadIdx.x; i < m; i += (uint64_t)kRjHeavyParts * 256) {
        uint64_t pay = 0;
        if (rj_probe_one(p, g, p.bkeys[at + i], in_smem, cap, tkey, tpay, sent, pay)) {
          const uint64_t row = (uint64_t)c * p.probe_chunk_rows + p.brows[at + i];
          cnt += 1;
          psum += pay;
          fp += rj_mix(row ^ ((pay << 17) | (pay >> 47)));
        }
      }
    }
  }
  for (int off = 16; off > 0; off >>= 1) {
    cnt += __shfl_down_sync(0xffffffffu, cnt, off);
    psum += __shfl_down_sync(0xffffffffu, psum, off);
    fp += __shfl_down_sync(0xffffffffu, fp, off);
  }
  const uint32_t lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) {
    red[0][w] = cnt;
    red[1][w] = psum;
    red[2][w] = fp;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long a = 0, b = 0, f = 0;
    for (int k = 0; k < 8; ++k) {
      a += red[0][k];
      b += red[1][k];
      f += red[2][k];
    }
    if (a) {
      atomicAdd(&p.acc->count, a);
      atomicAdd(&p.acc->psum, b);
      atomicAdd(&p.acc->fp, f);
    }
  }
}

int grid_for(vx_ctx *ctx, uint64_t items, int threads, int per_sm) {
  const uint64_t g = (items + threads - 1) / threads;
  return (int)std::max<uint64_t>(1, std::min<uint64_t>(g, (uint64_t)ctx->num_sms * per_sm));
}

// enqueues find_boundary of a clustered chunk (bnd: 2^bits + 1 entries)
vx_status find_boundary_enqueue(vx_ctx *ctx, RadixBufs b, const RadixState *st, int npass, uint64_t n, int bits,
                                uint32_t *bnd, uint32_t *carry, cudaStream_t s) {
  const uint64_t G = 1ull << bits, m = G + 1;
  VX_CUDA_TRY(cudaMemsetAsync(bnd, 0xFF, 4 * m, s));
  rj_mark_kernel<<<grid_for(ctx, n, 256, 8), 256, 0, s>>>(b.keys[0], b.keys[1], st, npass, n, G - 1, bnd);
  const uint32_t nseg = (uint32_t)((m + kRjSeg - 1) / kRjSeg);
  rj_fill_local_kernel<<<nseg, 256, 0, s>>>(bnd, m, carry);
  rj_fill_carry_kernel<<<1, 1024, 0, s>>>(carry, nseg);
  rj_fill_apply_kernel<<<grid_for(ctx, m, 256, 8), 256, 0, s>>>(bnd, m, carry);
  VX_CUDA_TRY(cudaGetLastError());
  return VX_OK;
}

// RadixPartitionExKer of one table: chunks of R tuples clustered into the host
// intermediate (keys, then payloads or local rows) plus a boundary array per chunk
struct RjPartitionPass : ExKernel {
  vx_ctx *ctx;
  const uint64_t *keys, *payload;  // payload null: the probe side (local rows are kept instead)
  uint64_t n, R;
  int bits, npass, S;
  uint64_t *mid_keys;
  uint64_t *mid_pay;    // build side
  uint32_t *mid_rows;   // probe side
  uint32_t *mid_bnd;    // chunk c at c * (2^bits + 1)
  uint64_t size() override { return (n + R - 1) / R; }
  int n_slots() override { return S; }
  int max_in_flight() override { return S; }
  uint64_t rows(uint64_t it) const { return std::min(R, n - it * R); }
  uint64_t G1() const { return (1ull << bits) + 1; }
  uint64_t kb() const { return (8 * R + 255) & ~255ull; }
  uint64_t vb() const { return (4 * R + 255) & ~255ull; }
  uint64_t bb() const { return (4 * G1() + 255) & ~255ull; }
  uint64_t cb() const { return (4 * ((G1() + kRjSeg - 1) / kRjSeg) + 255) & ~255ull; }
  uint64_t slot_bytes() override {
    return 2 * kb() + 2 * vb() + radix_temp_bytes(R) + bb() + cb() + (payload ? 2 * kb() : 0);
  }
  RadixBufs bufs(char *slot) const {
    RadixBufs b;
    b.keys[0] = (uint64_t *)slot;
    b.keys[1] = (uint64_t *)(slot + kb());
    b.vals[0] = (uint32_t *)(slot + 2 * kb());
    b.vals[1] = (uint32_t *)(slot + 2 * kb() + vb());
    return b;
  }
  char *temp(char *slot) const { return slot + 2 * kb() + 2 * vb(); }
  uint32_t *bnd(char *slot) const { return (uint32_t *)(temp(slot) + radix_temp_bytes(R)); }
  uint32_t *carry(char *slot) const { return (uint32_t *)((char *)bnd(slot) + bb()); }
  uint64_t *pay_in(char *slot) const { return (uint64_t *)((char *)carry(slot) + cb()); }
  uint64_t *pay_out(char *slot) const { return (uint64_t *)((char *)pay_in(slot) + kb()); }
  void inputs(uint64_t it, char *slot, std::vector<CopyOp> &h2d) override {
    h2d.push_back({keys + it * R, bufs(slot).keys[0], 8 * rows(it)});
    if (payload) h2d.push_back({payload + it * R, pay_in(slot), 8 * rows(it)});
  }
  vx_status kernel(char *slot, uint64_t it, cudaStream_t s) override {
    RadixBufs b = bufs(slot);
    const uint64_t m = rows(it);
    rj_iota_kernel<<<grid_for(ctx, m, 256, 8), 256, 0, s>>>(b.vals[0], m);
    VX_TRY(radix_sort_enqueue(b, m, temp(slot), s, ctx->num_sms, npass, ctx->cfg.lookback_spin_limit));
    const RadixState *st = radix_state_of(temp(slot));
    VX_TRY(find_boundary_enqueue(ctx, b, st, npass, m, bits, bnd(slot), carry(slot), s));
    if (payload)
      rj_gather_kernel<<<grid_for(ctx, m, 256, 8), 256, 0, s>>>(b.vals[0], b.vals[1], st, npass, m, pay_in(slot),
                                                                pay_out(slot));
    VX_CUDA_TRY(cudaGetLastError());
    return radix_publish_enqueue(temp(slot), ctx->d_scalars + 64 + (it % S), s, npass);
  }
  bool has_outputs() override { return true; }
  vx_status outputs(uint64_t it, char *slot, std::vector<CopyOp> &d2h) override {
    RadixBufs b = bufs(slot);
    const uint64_t word = ((volatile uint64_t *)ctx->h_scalars)[64 + (it % S)];
    if (word >> 16 & 1) {
      set_error("radix join: the clustering sort of chunk %llu gave up a look-back wait", (unsigned long long)it);
      return VX_E_TIMEOUT;
    }
    const int c = (int)(word & 0xFF);
    const uint64_t m = rows(it);
    d2h.push_back({b.keys[c], mid_keys + it * R, 8 * m});
    if (payload) d2h.push_back({pay_out(slot), mid_pay + it * R, 8 * m});
    else d2h.push_back({b.vals[c], mid_rows + it * R, 4 * m});
    d2h.push_back({bnd(slot), mid_bnd + it * G1(), 4 * G1()});
    return VX_OK;
  }
};

// one range of groups and where its pieces sit in a slot
struct RjRange {
  uint64_t g0, g1;
  uint64_t akeys, apay, bkeys, brows, abnd, bbnd, abase, bbase, heavy, bytes;  // byte offsets in the slot
  uint64_t na_tuples, nb_tuples;
};

// HashJoinExKer: ranges of groups, each joined in shared memory
struct RjJoinPass : ExKernel {
  vx_ctx *ctx;
  uint64_t slot_b;
  int S;
  uint32_t NA, NB;
  uint64_t G1, RA, RB;
  const uint64_t *akeys, *apay, *bkeys;
  const uint32_t *brows, *abnd_h, *bbnd_h;
  std::vector<RjRange> ranges;
  const uint64_t *base_h = nullptr;  // page-locked; per range NA + NB words: abase, then bbase
  int bits;
  RjAcc *acc;
  std::vector<cudaEvent_t> ev0, ev1;
  double ms_join = 0;
  ~RjJoinPass() override {
    for (auto e : ev0) cudaEventDestroy(e);
    for (auto e : ev1) cudaEventDestroy(e);
  }
  uint64_t size() override { return ranges.size(); }
  int n_slots() override { return S; }
  int max_in_flight() override { return S; }
  uint64_t slot_bytes() override { return slot_b; }
  void inputs(uint64_t it, char *slot, std::vector<CopyOp> &h2d) override {
    const RjRange &r = ranges[it];
    const uint64_t ng1 = r.g1 - r.g0 + 1;
    for (uint32_t c = 0; c < NA; ++c) {
      const uint32_t *bd = abnd_h + c * G1;
      const uint64_t lo = bd[r.g0], hi = bd[r.g1], at = base_h[it * (NA + NB) + c];
      if (hi > lo) {
        h2d.push_back({akeys + c * RA + lo, slot + r.akeys + 8 * at, 8 * (hi - lo)});
        h2d.push_back({apay + c * RA + lo, slot + r.apay + 8 * at, 8 * (hi - lo)});
      }
      h2d.push_back({bd + r.g0, slot + r.abnd + 4 * c * ng1, 4 * ng1});
    }
    for (uint32_t c = 0; c < NB; ++c) {
      const uint32_t *bd = bbnd_h + c * G1;
      const uint64_t lo = bd[r.g0], hi = bd[r.g1], at = base_h[it * (NA + NB) + NA + c];
      if (hi > lo) {
        h2d.push_back({bkeys + c * RB + lo, slot + r.bkeys + 8 * at, 8 * (hi - lo)});
        h2d.push_back({brows + c * RB + lo, slot + r.brows + 4 * at, 4 * (hi - lo)});
      }
      h2d.push_back({bd + r.g0, slot + r.bbnd + 4 * c * ng1, 4 * ng1});
    }
    h2d.push_back({base_h + it * (NA + NB), slot + r.abase, 8ull * (NA + NB)});
  }
  vx_status kernel(char *slot, uint64_t it, cudaStream_t s) override {
    const RjRange &r = ranges[it];
    RjJoinParams p{};
    p.akeys = (const uint64_t *)(slot + r.akeys);
    p.apay = (const uint64_t *)(slot + r.apay);
    p.bkeys = (const uint64_t *)(slot + r.bkeys);
    p.brows = (const uint32_t *)(slot + r.brows);
    p.abnd = (const uint32_t *)(slot + r.abnd);
    p.bbnd = (const uint32_t *)(slot + r.bbnd);
    p.abase = (const uint64_t *)(slot + r.abase);
    p.bbase = p.abase + NA;
    p.na = NA;
    p.nb = NB;
    p.ng = (uint32_t)(r.g1 - r.g0);
    p.probe_chunk_rows = RB;
    p.key_shift = (uint32_t)bits;
    p.acc = acc;
    p.heavy = (uint32_t *)(slot + r.heavy);
    p.heavy_n = (unsigned int *)(slot + r.heavy + 4ull * kRjHeavyCap);
    const size_t e = it % S;
    VX_CUDA_TRY(cudaMemsetAsync(p.heavy_n, 0, 4, s));
    if (!ev0.empty()) VX_CUDA_TRY(cudaEventRecord(ev0[e], s));
    const uint64_t blocks = (p.ng + kRjWarps - 1) / kRjWarps;
    rj_join_kernel<<<(unsigned)std::min<uint64_t>(blocks, (uint64_t)ctx->num_sms * 8), 32 * kRjWarps, 0, s>>>(p);
    rj_heavy_kernel<<<(unsigned)ctx->num_sms * 4, 256, 0, s>>>(p);
    VX_CUDA_TRY(cudaGetLastError());
    if (!ev1.empty()) VX_CUDA_TRY(cudaEventRecord(ev1[e], s));
    return VX_OK;
  }
  void on_retire(uint64_t it) override {
    if (ev0.empty()) return;
    float ms = 0;
    if (cudaEventElapsedTime(&ms, ev0[it % S], ev1[it % S]) == cudaSuccess) ms_join += ms;
    cudaGetLastError();
  }
};

struct HostBuf {
  std::unique_ptr<char[]> mem;
  HostReg reg;
  char *p = nullptr;
  vx_status alloc(uint64_t bytes) {
    mem.reset(new (std::nothrow) char[bytes + 4096]);
    if (!mem) {
      set_error("radix join: no host memory for a %llu-byte intermediate", (unsigned long long)bytes);
      return VX_E_NOMEM;
    }
    p = (char *)(((uintptr_t)mem.get() + 4095) & ~(uintptr_t)4095);
    return reg.add(p, bytes);
  }
};

}  // namespace

vx_status radix_join(vx_ctx *ctx, const Column *bk, const Column *bp, const Column *pk, const vx_join_opts &o,
                     vx_join_result *out) {
  const double t0 = now_ms();
  const int bits = o.radix_bits ? o.radix_bits : 24;
  if (bits != 8 && bits != 16 && bits != 24) {
    set_error("vx_join: radix_bits must be 8, 16 or 24");
    return VX_E_INVAL;
  }
  const int npass = bits / 8;
  const uint64_t G = 1ull << bits, G1 = G + 1;
  const uint64_t nb = bk->n_rows, np = pk->n_rows;
  vx_join_result res{};
  res.algorithm = VX_JOIN_RADIX;
  const int S = std::max(2, ctx->cfg.n_slots);
  cudaStream_t s = ctx->s_compute;
  DevBuf accb;
  accb.arena = &ctx->arena;
  accb.p = ctx->arena.alloc(256);
  if (!accb.p) {
    set_error("vx_join: arena exhausted");
    return VX_E_NOMEM;
  }
  RjAcc *acc = accb.as<RjAcc>();
  VX_CUDA_TRY(cudaMemsetAsync(acc, 0, sizeof(RjAcc), s));

  // ---- partition pass chunk size: R tuples per slot (both tables), and
  // chunk-local rows must fit 32 bits
  const uint64_t avail = ctx->arena.largest_free();
  const uint64_t fixed = 4 * G1 + 4 * ((G1 + kRjSeg - 1) / kRjSeg) + 8192;
  if (avail < S * (fixed + (1 << 20))) {
    set_error("vx_join: budget too small for the radix join's staging slots");
    return VX_E_NOMEM;
  }
  uint64_t R = (uint64_t)((double)(avail / S - fixed) / (40.0 + 256.0 * 8 / kRxTile) * 0.9);
  R = std::min<uint64_t>(R / kRxTile * kRxTile, kPipelineRows);
  if (R < kRxTile) {
    set_error("vx_join: budget too small for the radix join");
    return VX_E_NOMEM;
  }
  const uint32_t NA = (uint32_t)((nb + R - 1) / R), NB = (uint32_t)((np + R - 1) / R);

  // ---- host intermediates
  HostBuf ha_keys, ha_pay, hb_keys, hb_rows, ha_bnd, hb_bnd;
  VX_TRY(ha_keys.alloc(8 * std::max<uint64_t>(nb, 1)));
  VX_TRY(ha_pay.alloc(8 * std::max<uint64_t>(nb, 1)));
  VX_TRY(hb_keys.alloc(8 * std::max<uint64_t>(np, 1)));
  VX_TRY(hb_rows.alloc(4 * std::max<uint64_t>(np, 1)));
  VX_TRY(ha_bnd.alloc(4 * G1 * std::max<uint32_t>(NA, 1)));
  VX_TRY(hb_bnd.alloc(4 * G1 * std::max<uint32_t>(NB, 1)));

  // ---- RadixPartitionExKer over both tables
  const double tp = now_ms();
  for (int side = 0; side < 2; ++side) {
    const uint64_t n = side ? np : nb;
    if (!n) continue;
    RjPartitionPass pp;
    pp.ctx = ctx;
    pp.keys = (const uint64_t *)(side ? pk->host : bk->host);
    pp.payload = side ? nullptr : (const uint64_t *)bp->host;
    pp.n = n;
    pp.R = R;
    pp.bits = bits;
    pp.npass = npass;
    pp.S = S;
    pp.mid_keys = (uint64_t *)(side ? hb_keys.p : ha_keys.p);
    pp.mid_pay = (uint64_t *)ha_pay.p;
    pp.mid_rows = (uint32_t *)hb_rows.p;
    pp.mid_bnd = (uint32_t *)(side ? hb_bnd.p : ha_bnd.p);
    ExecStats es;
    VX_TRY(run_pipeline(ctx, pp, &es));
    res.bytes_h2d += es.bytes_h2d;
    res.bytes_d2h += es.bytes_d2h;
    res.kernel_launches += es.kernel_launches * (npass + 12);
    res.ms_kernel += es.ms_kernel;
  }
  res.ms_partition = now_ms() - tp;
  res.ms_build = res.ms_partition;

  // ---- HashJoinExKer data mapping: group ranges whose tuples and boundary
  // slices fit a slot, by binary search over the boundary arrays
  const double tj = now_ms();
  const uint32_t *abnd = (const uint32_t *)ha_bnd.p, *bbnd = (const uint32_t *)hb_bnd.p;
  auto tuples_below = [&](const uint32_t *bnd, uint32_t N, uint64_t g) {
    uint64_t t = 0;
    for (uint32_t c = 0; c < N; ++c) t += bnd[c * G1 + g];
    return t;
  };
  const uint64_t slot_b = (uint64_t)((double)ctx->arena.largest_free() / S * 0.95) / 256 * 256;
  auto layout = [&](RjRange &r) {
    const uint64_t ng1 = r.g1 - r.g0 + 1;
    r.na_tuples = tuples_below(abnd, NA, r.g1) - tuples_below(abnd, NA, r.g0);
    r.nb_tuples = tuples_below(bbnd, NB, r.g1) - tuples_below(bbnd, NB, r.g0);
    auto al = [](uint64_t x) { return (x + 255) & ~255ull; };
    r.akeys = 0;
    r.apay = r.akeys + al(8 * r.na_tuples);
    r.bkeys = r.apay + al(8 * r.na_tuples);
    r.brows = r.bkeys + al(8 * r.nb_tuples);
    r.abnd = r.brows + al(4 * r.nb_tuples);
    r.bbnd = r.abnd + al(4 * NA * ng1);
    r.abase = r.bbnd + al(4 * NB * ng1);
    r.bbase = r.abase + 8 * NA;
    r.heavy = r.abase + al(8 * (NA + NB));
    r.bytes = r.heavy + al(4 * kRjHeavyCap + 256);
  };
  RjJoinPass jp;
  jp.ctx = ctx;
  jp.S = S;
  jp.NA = NA;
  jp.NB = NB;
  jp.G1 = G1;
  jp.RA = R;
  jp.RB = R;
  jp.akeys = (const uint64_t *)ha_keys.p;
  jp.apay = (const uint64_t *)ha_pay.p;
  jp.bkeys = (const uint64_t *)hb_keys.p;
  jp.brows = (const uint32_t *)hb_rows.p;
  jp.abnd_h = abnd;
  jp.bbnd_h = bbnd;
  jp.bits = bits;
  jp.acc = acc;
  jp.slot_b = slot_b;
  if (nb && np) {
    for (uint64_t g0 = 0; g0 < G;) {
      RjRange r{};
      r.g0 = g0;
      uint64_t lo = g0 + 1, hi = G;  // largest g1 in [g0 + 1, G] whose range fits
      r.g1 = lo;
      layout(r);
      if (r.bytes > slot_b) {
        set_error("vx_join: radix group %llu alone (%llu build, %llu probe tuples) exceeds a staging slot",
                  (unsigned long long)g0, (unsigned long long)r.na_tuples, (unsigned long long)r.nb_tuples);
        return VX_E_NOMEM;
      }
      while (lo < hi) {
        const uint64_t mid = lo + (hi - lo + 1) / 2;
        RjRange t = r;
        t.g1 = mid;
        layout(t);
        if (t.bytes <= slot_b) lo = mid; else hi = mid - 1;
      }
      r.g1 = lo;
      layout(r);
      jp.ranges.push_back(r);
      g0 = r.g1;
    }
  }
  res.ranges = (uint32_t)jp.ranges.size();
  HostBuf hbase;
  if (!jp.ranges.empty()) {
    // per range and chunk: where the chunk's segment starts in the range's slot
    VX_TRY(hbase.alloc(8ull * jp.ranges.size() * (NA + NB)));
    uint64_t *base = (uint64_t *)hbase.p;
    for (size_t q = 0; q < jp.ranges.size(); ++q) {
      const RjRange &r = jp.ranges[q];
      uint64_t *b = base + q * (NA + NB);
      uint64_t at = 0;
      for (uint32_t c = 0; c < NA; ++c) {
        b[c] = at;
        at += abnd[c * G1 + r.g1] - abnd[c * G1 + r.g0];
      }
      at = 0;
      for (uint32_t c = 0; c < NB; ++c) {
        b[NA + c] = at;
        at += bbnd[c * G1 + r.g1] - bbnd[c * G1 + r.g0];
      }
    }
    jp.base_h = base;
    if (ctx->cfg.sched == VX_SCHED_IMMEDIATE) {
      jp.ev0.resize(S);
      jp.ev1.resize(S);
      for (int i = 0; i < S; ++i) {
        VX_CUDA_TRY(cudaEventCreate(&jp.ev0[i]));
        VX_CUDA_TRY(cudaEventCreate(&jp.ev1[i]));
      }
    }
    ExecStats es;
    VX_TRY(run_pipeline(ctx, jp, &es));
    res.bytes_h2d += es.bytes_h2d;
    res.kernel_launches += es.kernel_launches;
    res.ms_kernel += jp.ms_join;
    res.ms_probe_kernel = jp.ms_join;
  }
  VX_CUDA_TRY(cudaStreamSynchronize(s));
  res.ms_probe = now_ms() - tj;
  RjAcc h{};
  VX_CUDA_TRY(cudaMemcpy(&h, acc, sizeof h, cudaMemcpyDeviceToHost));
  if (h.err & ERR_DUPKEY) {
    set_error("vx_join: duplicate build key");
    return VX_E_DUPKEY;
  }
  res.count = h.count;
  res.payload_sum = h.psum;
  res.pair_fp = h.fp;
  res.n_partitions = (uint32_t)G;
  res.max_partition = 0;
  res.ms_total = now_ms() - t0;
  *out = res;
  return VX_OK;
}

}  // namespace vx

using namespace vx;

VX_API vx_status vx_radix_cluster(vx_ctx *ctx, const uint64_t *keys, uint64_t n, int32_t bits, uint64_t *out_keys,
                                  uint32_t *out_rows, uint32_t *out_boundary) {
  clear_error();
  VX_TRY(check_ctx(ctx));
  if ((bits != 8 && bits != 16 && bits != 24) || n >= (1ull << 32) || (n && (!keys || !out_keys || !out_rows)) ||
      !out_boundary) {
    set_error("vx_radix_cluster: bad argument (bits 8, 16 or 24; n < 2^32)");
    return VX_E_INVAL;
  }
  std::lock_guard<std::recursive_mutex> g(ctx->mu);
  const uint64_t G1 = (1ull << bits) + 1, m = std::max<uint64_t>(n, 1);
  const uint64_t kb = (8 * m + 255) & ~255ull, vb = (4 * m + 255) & ~255ull, bb = (4 * G1 + 255) & ~255ull;
  const uint64_t cb = (4 * ((G1 + kRjSeg - 1) / kRjSeg) + 255) & ~255ull;
  DevBuf buf;
  buf.arena = &ctx->arena;
  buf.p = ctx->arena.alloc(2 * kb + 2 * vb + radix_temp_bytes(m) + bb + cb);
  if (!buf.p) {
    set_error("vx_radix_cluster: %llu keys do not fit the arena", (unsigned long long)n);
    return VX_E_NOMEM;
  }
  char *p = buf.as<char>();
  RadixBufs b;
  b.keys[0] = (uint64_t *)p;
  b.keys[1] = (uint64_t *)(p + kb);
  b.vals[0] = (uint32_t *)(p + 2 * kb);
  b.vals[1] = (uint32_t *)(p + 2 * kb + vb);
  char *temp = p + 2 * kb + 2 * vb;
  uint32_t *bnd = (uint32_t *)(temp + radix_temp_bytes(m));
  uint32_t *carry = (uint32_t *)((char *)bnd + bb);
  cudaStream_t s = ctx->s_compute;
  const int npass = bits / 8;
  if (n) VX_CUDA_TRY(cudaMemcpyAsync(b.keys[0], keys, 8 * n, cudaMemcpyHostToDevice, s));
  rj_iota_kernel<<<grid_for(ctx, m, 256, 8), 256, 0, s>>>(b.vals[0], n);
  VX_TRY(radix_sort_enqueue(b, n, temp, s, ctx->num_sms, npass, ctx->cfg.lookback_spin_limit));
  const RadixState *st = radix_state_of(temp);
  VX_TRY(find_boundary_enqueue(ctx, b, st, npass, n, bits, bnd, carry, s));
  RadixState h;
  VX_CUDA_TRY(cudaMemcpyAsync(&h, st, offsetof(RadixState, totals), cudaMemcpyDeviceToHost, s));
  VX_CUDA_TRY(cudaStreamSynchronize(s));
  if (h.err) {
    set_error("vx_radix_cluster: a look-back wait gave up");
    return VX_E_TIMEOUT;
  }
  const int c = n ? h.cur[npass] : 0;
  if (n) {
    VX_CUDA_TRY(cudaMemcpyAsync(out_keys, b.keys[c], 8 * n, cudaMemcpyDeviceToHost, s));
    VX_CUDA_TRY(cudaMemcpyAsync(out_rows, b.vals[c], 4 * n, cudaMemcpyDeviceToHost, s));
  }
  VX_CUDA_TRY(cudaMemcpyAsync(out_boundary, bnd, 4 * G1, cudaMemcpyDeviceToHost, s));
  VX_CUDA_TRY(cudaStreamSynchronize(s));
  return VX_OK;
}
