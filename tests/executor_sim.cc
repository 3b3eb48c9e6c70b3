// The executor's immediate schedule (paper_2502_09541_gb300/csrc/vx_sched.h)
// against a simulated device on the CPU: three in-order streams (host to
// device, compute, device to host) on a simulated clock, seeded random
// durations, and injected faults — a failing copy, a kernel that never
// completes, slow but progressing chunks.  Every decision is checked against
// the executor's rules: a slot is reused only after its previous chunk has
// been stored, a chunk is stored only after its kernel completed, chunks
// retire in order, at most max_in_flight chunks are in the pipeline, and every
// chunk is loaded, run and stored exactly once.
//
//   executor_sim <scenario> <seed>    exit 0 when the scenario's outcome and
//                                     every rule hold, 1 otherwise
#include <algorithm>
#include <cinttypes>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <limits>
#include <random>
#include <string>
#include <vector>

#include "vx_sched.h"

namespace {

constexpr double kNever = std::numeric_limits<double>::infinity();

struct Sim {
  // configuration
  uint64_t N = 64;
  int S = 3;
  uint64_t max_in_flight = 3;
  bool outputs = true;
  double limit_ms = 1.0;
  uint64_t fail_load_at = UINT64_MAX;  // this chunk's loads fail to issue
  uint64_t stuck_kernel_at = UINT64_MAX;
  double kernel_ms_fixed = -1;  // > 0: every kernel takes exactly this long
  std::mt19937_64 rng;

  // simulated device
  double t = 0;
  double h2d_free = 0, comp_free = 0, d2h_free = 0;
  std::vector<double> kernel_end, store_end, slot_free_at;
  std::vector<int64_t> slot_chunk;
  std::vector<int> loaded, ran, stored_n;
  uint64_t retired = 0, in_pipe = 0, peak_in_pipe = 0;
  bool timed_out_flag = false;
  std::string violation;

  void check(bool ok, const char *what, uint64_t it) {
    if (!ok && violation.empty()) {
      char b[256];
      snprintf(b, sizeof b, "%s (chunk %" PRIu64 ", t = %.4f ms)", what, it, t);
      violation = b;
    }
  }
  double dur(double lo, double hi) { return std::uniform_real_distribution<double>(lo, hi)(rng); }

  // ---- the device interface of vx_sched.h
  vx_status load(uint64_t it, int s) {
    check(it < N, "load past the end", it);
    check(t >= slot_free_at[s], "slot reused before its previous chunk was stored", it);
    check(loaded[it] == 0, "chunk loaded twice", it);
    if (it == fail_load_at) return VX_E_CUDA;
    loaded[it] += 1;
    in_pipe += 1;
    peak_in_pipe = std::max(peak_in_pipe, in_pipe);
    const double h_end = std::max(h2d_free, t) + dur(0.05, 0.4);
    h2d_free = h_end;
    const double k_len = kernel_ms_fixed > 0 ? kernel_ms_fixed : dur(0.01, 0.3);
    const double k_end = it == stuck_kernel_at ? kNever : std::max(comp_free, h_end) + k_len;
    comp_free = k_end;
    kernel_end[s] = k_end;
    slot_chunk[s] = (int64_t)it;
    slot_free_at[s] = kNever;  // until the chunk retires
    return VX_OK;
  }
  int kernel_state(int s) { return t >= kernel_end[s] ? 1 : 0; }
  vx_status retire(uint64_t it, int s) {
    check(slot_chunk[s] == (int64_t)it, "retired a chunk from another slot", it);
    check(it == retired, "retired out of order", it);
    check(t >= kernel_end[s], "retired before the kernel completed", it);
    ran[it] += 1;
    if (!outputs) {
      retired += 1;
      in_pipe -= 1;
      slot_free_at[s] = t;
    }
    return VX_OK;
  }
  bool has_outputs() { return outputs; }
  vx_status store(uint64_t it, int s) {
    check(ran[it] == 1, "stored before its kernel retired", it);
    check(t >= kernel_end[s], "stored before the kernel completed", it);
    const double e = std::max(d2h_free, t) + dur(0.05, 0.35);
    d2h_free = e;
    store_end[s] = e;
    return VX_OK;
  }
  int store_state(int s) { return t >= store_end[s] ? 1 : 0; }
  vx_status stored(uint64_t it, int s) {
    check(t >= store_end[s], "store reported before it completed", it);
    check(it == retired, "stored out of order", it);
    stored_n[it] += 1;
    retired += 1;
    in_pipe -= 1;
    slot_free_at[s] = t;
    return VX_OK;
  }
  vx_status timed_out(uint64_t) {
    timed_out_flag = true;
    return VX_E_TIMEOUT;
  }
  double now_ms() { return t; }
  void pause() { t += 0.01; }  // the executor's 10 us back-off

  vx_status run() {
    kernel_end.assign(S, 0);
    store_end.assign(S, 0);
    slot_free_at.assign(S, 0);
    slot_chunk.assign(S, -1);
    loaded.assign(N, 0);
    ran.assign(N, 0);
    stored_n.assign(N, 0);
    return vx::immediate_schedule(*this, N, S, max_in_flight, limit_ms);
  }
  bool all_done_once() const {
    for (uint64_t i = 0; i < N; ++i)
      if (loaded[i] != 1 || ran[i] != 1 || (outputs && stored_n[i] != 1)) return false;
    return true;
  }
};

int finish(const Sim &s, bool ok, const char *scenario) {
  if (!s.violation.empty()) {
    printf("%s: rule broken: %s\n", scenario, s.violation.c_str());
    return 1;
  }
  printf("%s: %s (t = %.3f ms, peak in pipeline %" PRIu64 ")\n", scenario, ok ? "ok" : "FAILED", s.t, s.peak_in_pipe);
  return ok ? 0 : 1;
}

}  // namespace

int main(int argc, char **argv) {
  if (argc < 3) {
    fprintf(stderr, "usage: executor_sim <scenario> <seed>\n");
    return 2;
  }
  const std::string sc = argv[1];
  Sim s;
  s.rng.seed(strtoull(argv[2], nullptr, 10));
  if (sc == "random") {  // random durations, stores on, three slots
    const vx_status st = s.run();
    return finish(s, st == VX_OK && s.all_done_once() && s.peak_in_pipe <= s.max_in_flight, sc.c_str());
  }
  if (sc == "random_deep") {  // more slots than chunks in flight, no outputs
    s.S = 6;
    s.max_in_flight = 4;
    s.outputs = false;
    const vx_status st = s.run();
    return finish(s, st == VX_OK && s.all_done_once() && s.peak_in_pipe <= 4, sc.c_str());
  }
  if (sc == "copy_fails") {  // the error of a failing copy comes back, nothing later is issued
    s.fail_load_at = 17;
    const vx_status st = s.run();
    bool later = false;
    for (uint64_t i = 18; i < s.N; ++i) later |= s.loaded[i] != 0;
    return finish(s, st == VX_E_CUDA && !later, sc.c_str());
  }
  if (sc == "stuck_kernel") {  // a kernel that never completes: VX_E_TIMEOUT after the limit
    s.stuck_kernel_at = 9;
    s.limit_ms = 2.0;
    const vx_status st = s.run();
    return finish(s, st == VX_E_TIMEOUT && s.timed_out_flag && s.retired == 9 && s.t < 60.0, sc.c_str());
  }
  if (sc == "slow_progress") {  // every wait is under the limit: the whole run is far longer, no timeout
    s.limit_ms = 1.5;
    s.kernel_ms_fixed = 0.6;
    const vx_status st = s.run();
    return finish(s, st == VX_OK && s.all_done_once() && s.t > 10 * s.limit_ms, sc.c_str());
  }
  fprintf(stderr, "unknown scenario %s\n", sc.c_str());
  return 2;
}
