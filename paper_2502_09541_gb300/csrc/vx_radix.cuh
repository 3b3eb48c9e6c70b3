// Stable counting scatter of (uint64 key, uint32 value) pairs by a digit, the
// building block of the range partition (digit = partition id, Section 6.2.1
// clustering with a monotone range function) and of the LSD radix sort of a
// partition (digit = one key byte; Section 6.1 sorts chunks with a radix sort
// over a double buffer).
//
// Range partition = upsweep (per-tile digit histograms) -> row scan (per
// digit, exclusive over tiles) -> totals scan (exclusive over digits: the
// boundary array of Section 6.2.1) -> downsweep (stable scatter).  An LSD sort
// pass is one scatter kernel: the global digit offsets of all eight passes
// come from one histogram read of the keys, and each tile finds the count of
// its digits in the tiles before it by decoupled look-back (tiles take
// tickets in launch order, publish their counts, then their inclusive
// prefixes; every wait is bounded and sets the error word when it gives up).
// Ranking inside a tile is warp-contiguous: warp w owns 512 consecutive pairs
// and processes them in 16 rounds of 32; __match_any_sync groups equal digits
// of a round, so pairs keep their input order (stability).
//
// Double buffer: `cur[pass]` (device) says which of (A, B) holds the input of
// LSD pass `pass`; a pass whose digit is constant over all pairs is skipped on
// the device and leaves cur unchanged — the paper's double-buffer marker used
// as the executor's type code (Section 6.1).
#pragma once
#include <cstdint>

namespace vx {

constexpr int kRxThreads = 256;
constexpr int kRxWarps = kRxThreads / 32;
constexpr int kRxItems = 16;
constexpr int kRxTile = kRxThreads * kRxItems;  // 4096 pairs
constexpr int kRxDigits = 256;
constexpr uint32_t kRxInvalid = 0x100;

struct RadixBufs {
  uint64_t *keys[2];
  uint32_t *vals[2];
};

// per-pass device state: cur[0..8], skip[0..7], an error word (a look-back
// wait that gave up), the polls a look-back makes of one predecessor word
// before giving up, totals[256], base[257]
struct RadixState {
  int32_t cur[12];
  int32_t skip[12];
  uint32_t err, spin_limit;
  uint64_t totals[kRxDigits];
  uint64_t base[kRxDigits + 1];
};

}  // namespace vx
