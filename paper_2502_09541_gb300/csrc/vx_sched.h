// The immediate schedule of the pipelined executor (Section 5.3), written
// against an abstract device so that the same decisions drive the GPU's copy
// and compute streams and, in tests, a simulated copy engine on the CPU.
//
// In cycle n the kernel of chunk n-1 runs while the copy engine loads chunk n
// and saves the output of chunk n-2.  A chunk's loads are issued only when its
// slot is free (the slot's previous chunk has been stored) and fewer than
// max_in_flight chunks are loaded, computing or storing, so every copy can
// start at once (Section 4.3, principle 1).  Chunks retire in order; a chunk's
// stores are issued only once its kernel has completed, which in turn waited
// for its loads, so the device-to-host queue never drains ahead of the
// host-to-device queue (Section 4.3's flow-control policy).  The loop polls
// with a short pause (Section 4.3's retry period); wait_limit_ms bounds the
// time since the last completed step, so an operator that keeps progressing
// never times out however long it runs.
#pragma once
#include <cstdint>
#include <vector>

#include "../../include/vx.h"

namespace vx {

// Dev provides:
//   vx_status load(uint64_t it, int slot)    issue chunk it's loads into slot, then its kernel
//   int kernel_state(int slot)               1 the slot's kernel completed, 0 not yet, < 0 an error status
//   vx_status retire(uint64_t it, int slot)  chunk it's kernel has completed
//   bool has_outputs()
//   vx_status store(uint64_t it, int slot)   issue chunk it's stores
//   int store_state(int slot)                as kernel_state, for the slot's stores
//   vx_status stored(uint64_t it, int slot)  chunk it's stores have completed
//   vx_status timed_out(uint64_t it)         no step completed within the limit (waiting at chunk it)
//   double now_ms()
//   void pause()
template <class Dev>
vx_status immediate_schedule(Dev &d, uint64_t N, int S, uint64_t max_in_flight, double wait_limit_ms) {
  std::vector<int> phase(S, 0);  // 0 free, 1 kernel issued, 2 storing
  if (max_in_flight < 1) max_in_flight = 1;
  double last_progress = d.now_ms();
  uint64_t next_load = 0, next_retire = 0;
  while (next_retire < N) {
    bool progress = false;
    // retire in chunk order
    while (next_retire < next_load) {
      const int s = (int)(next_retire % (uint64_t)S);
      if (phase[s] == 1) {
        const int q = d.kernel_state(s);
        if (q == 0) break;
        if (q < 0) return q;
        vx_status st = d.retire(next_retire, s);
        if (st != VX_OK) return st;
        if (d.has_outputs()) {
          st = d.store(next_retire, s);
          if (st != VX_OK) return st;
          phase[s] = 2;
        } else {
          phase[s] = 0;
          ++next_retire;
        }
        progress = true;
      } else if (phase[s] == 2) {
        const int q = d.store_state(s);
        if (q == 0) break;
        if (q < 0) return q;
        const vx_status st = d.stored(next_retire, s);
        if (st != VX_OK) return st;
        phase[s] = 0;
        ++next_retire;
        progress = true;
      } else {
        break;
      }
    }
    // load the next chunk when its slot is free and the pipeline holds fewer
    // than max_in_flight chunks
    if (next_load < N && next_load - next_retire < (uint64_t)S && next_load - next_retire < max_in_flight) {
      const int s = (int)(next_load % (uint64_t)S);
      if (phase[s] == 0) {
        const vx_status st = d.load(next_load, s);
        if (st != VX_OK) return st;
        phase[s] = 1;
        ++next_load;
        progress = true;
      }
    }
    if (progress) {
      last_progress = d.now_ms();
    } else {
      if (d.now_ms() - last_progress > wait_limit_ms) return d.timed_out(next_retire);
      d.pause();
    }
  }
  return VX_OK;
}

}  // namespace vx
