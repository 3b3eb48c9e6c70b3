// Device helpers of the row logic shared by the fused star kernels and the
// operator-at-a-time kernels: predicate ranges, dimension-table lookups and
// fact-column reads (staged slice or mapped host column).
#pragma once
#include <climits>
#include <cstdint>

#include "vx_star.cuh"

namespace vx {

// Every comparison operator as one inclusive range [lo, hi] tested on uint32
// offsets, v - lo <= hi - lo, optionally complemented: NE is the complement of
// [lo, lo], and an empty range (BETWEEN with lo > hi, LT INT_MIN, GT INT_MAX,
// an unknown operator) is the complement of the full range.  Built once per
// predicate, so the per-row test is a subtract and a compare.
struct PredRange {
  uint32_t lo, span;
  bool inv;
};

__device__ __forceinline__ PredRange pred_range(int32_t op, int32_t lo, int32_t hi) {
  int32_t a = lo, b = hi;
  bool inv = false, none = false;
  switch (op) {
    case VX_BETWEEN: none = lo > hi; break;
    case VX_EQ: b = lo; break;
    case VX_NE: b = lo, inv = true; break;
    case VX_LT: none = lo == INT_MIN, a = INT_MIN, b = lo - (lo != INT_MIN); break;
    case VX_LE: a = INT_MIN, b = lo; break;
    case VX_GT: none = lo == INT_MAX, a = lo + (lo != INT_MAX), b = INT_MAX; break;
    case VX_GE: a = lo, b = INT_MAX; break;
    default: none = true;
  }
  if (none) a = INT_MIN, b = INT_MAX, inv = true;
  return PredRange{(uint32_t)a, (uint32_t)b - (uint32_t)a, inv};
}

__device__ __forceinline__ bool pred_in(const PredRange &r, int32_t v) { return ((uint32_t)v - r.lo <= r.span) != r.inv; }

__device__ __forceinline__ bool pred_ok(int32_t v, int32_t op, int32_t lo, int32_t hi) {
  return pred_in(pred_range(op, lo, hi), v);
}

__device__ __forceinline__ uint32_t ht_hash32(int32_t k, uint32_t log2cap) {
  return ((uint32_t)k * 0x9E3779B1u) >> (32u - log2cap);
}

__device__ __forceinline__ bool ht_lookup(const uint64_t *__restrict__ slots, uint32_t log2cap, int32_t key,
                                          uint32_t &val) {
  const uint32_t mask = (1u << log2cap) - 1u;
  uint32_t h = ht_hash32(key, log2cap);
  for (uint32_t n = 0; n <= mask; ++n) {
    const uint64_t s = __ldg(&slots[h]);
    const uint32_t v = (uint32_t)(s >> 32);
    if (v == HT_EMPTY_VAL) return false;
    if ((int32_t)(uint32_t)s == key) {
      val = v;
      return v != HT_FILTERED;
    }
    h = (h + 1u) & mask;
  }
  return false;
}

// value idx of a direct map of vb-byte values (1, 2 or 4), widened to 32
// bits: the two largest values of a narrow width are the markers, which map
// to HT_EMPTY_VAL (no such key) and HT_FILTERED (key filtered out)
__device__ __forceinline__ uint32_t dmap_get(const void *map, uint32_t vb, uint32_t idx) {
  if (vb == 1) {
    const uint32_t v = __ldg(reinterpret_cast<const uint8_t *>(map) + idx);
    return v >= 0xFEu ? v + 0xFFFFFF00u : v;
  }
  if (vb == 2) {
    const uint32_t v = __ldg(reinterpret_cast<const uint16_t *>(map) + idx);
    return v >= 0xFFFEu ? v + 0xFFFF0000u : v;
  }
  return __ldg(reinterpret_cast<const uint32_t *>(map) + idx);
}

// lookup in dimension d of a plan: direct map or hash table
__device__ __forceinline__ bool dim_lookup(const ChunkParams &p, int d, int32_t key, uint32_t &val) {
  if (p.dspan[d]) {
    const uint32_t idx = (uint32_t)(key - p.dmin[d]);
    if (idx >= p.dspan[d]) return false;
    val = dmap_get(p.ht[d], p.dvb[d], idx);
    return val < HT_FILTERED;
  }
  return ht_lookup(p.ht[d], p.ht_log2[d], key, val);
}

__device__ __forceinline__ int32_t load_role(const ChunkParams &p, int r, uint64_t i) {
  const int32_t *s = p.staged[r];
  return s ? __ldg(&s[i]) : p.zc[r][p.row0 + i];
}

}  // namespace vx
