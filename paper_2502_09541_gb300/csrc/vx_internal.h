// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>

#include <chrono>
#include <cstdint>
#include <cstring>
#include <functional>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/vx.h"

#define VX_API extern "C" __attribute__((visibility("default")))

namespace vx {

// ------------------------------------------------------------------ errors
void set_error(const char *fmt, ...);
void clear_error();

struct Status {
  vx_status code = VX_OK;
  bool ok() const { return code == VX_OK; }
};

#define VX_CUDA_TRY(expr)                                                               \
  do {                                                                                  \
    cudaError_t e_ = (expr);                                                            \
    if (e_ != cudaSuccess) {                                                            \
      ::vx::set_error("%s failed: %s (%s:%d)", #expr, cudaGetErrorString(e_), __FILE__, \
                      __LINE__);                                                        \
      return VX_E_CUDA;                                                                 \
    }                                                                                   \
  } while (0)

#define VX_TRY(expr)              \
  do {                            \
    vx_status s_ = (expr);        \
    if (s_ != VX_OK) return s_;   \
  } while (0)

// device error word bits (kernels set them, the host turns them into statuses)
enum : uint32_t {
  ERR_DUPKEY = 1u,
  ERR_RANGE = 2u,
  ERR_HT_FULL = 4u,
  ERR_OVERFLOW = 8u,
  ERR_WAIT = 16u,  // a bounded device-side wait gave up
};

// ------------------------------------------------------------------ arena
// First-fit allocator over one device region; 256-byte aligned blocks.
class Arena {
 public:
  void init(char *base, uint64_t bytes);
  // returns nullptr if the request does not fit
  void *alloc(uint64_t bytes);
  void free(void *p);
  uint64_t capacity() const { return bytes_; }
  uint64_t used() const { return used_; }
  uint64_t largest_free() const;
  char *base() const { return base_; }

 private:
  char *base_ = nullptr;
  uint64_t bytes_ = 0, used_ = 0;
  std::map<uint64_t, uint64_t> free_;  // offset -> size
  std::map<uint64_t, uint64_t> live_;  // offset -> size
};

// RAII arena block
struct DevBuf {
  Arena *arena = nullptr;
  void *p = nullptr;
  uint64_t bytes = 0;
  DevBuf() = default;
  DevBuf(const DevBuf &) = delete;
  DevBuf &operator=(const DevBuf &) = delete;
  DevBuf(DevBuf &&o) noexcept { *this = std::move(o); }
  DevBuf &operator=(DevBuf &&o) noexcept {
    release();
    arena = o.arena; p = o.p; bytes = o.bytes;
    o.p = nullptr; o.arena = nullptr; o.bytes = 0;
    return *this;
  }
  ~DevBuf() { release(); }
  void release() {
    if (arena && p) arena->free(p);
    p = nullptr;
  }
  template <class T> T *as() const { return reinterpret_cast<T *>(p); }
};

// ------------------------------------------------------------------ columns
struct Column {
  std::string name;
  int32_t dtype = VX_I32;
  const void *host = nullptr;
  const void *dev = nullptr;  // device-visible address of the host data (mapped)
  uint64_t n_rows = 0;
  uint32_t elem = 4;
  bool we_registered = false;
  bool live = false;
};

inline uint32_t dtype_size(int32_t dt) { return (dt == VX_I64 || dt == VX_U64) ? 8u : 4u; }

// ------------------------------------------------------------------ context
struct ResidentHT;  // cached dimension hash table (serving)
struct GraphEntry;  // captured chunk pipeline of one plan (batching)

}  // namespace vx

struct vx_ctx {
  int device = 0;
  int num_sms = 0;
  cudaStream_t s_compute = nullptr, s_h2d = nullptr, s_d2h = nullptr;
  bool own_compute = false;
  char *arena_base = nullptr;
  uint64_t arena_bytes = 0;
  bool own_arena = false;
  vx::Arena arena;
  std::vector<vx::Column> cols;
  vx_config cfg{};
  std::recursive_mutex mu;
  vx_query_stats last{};
  // small pinned + mapped host block for device->host scalars (counts, error word)
  uint64_t *h_scalars = nullptr;  // host view
  uint64_t *d_scalars = nullptr;  // device view
  static constexpr int kScalars = 4096;
  // resident dimension hash tables, keyed by a signature string
  std::map<std::string, std::shared_ptr<vx::ResidentHT>> resident;
  // captured pipelines (use_graphs), keyed by plan signature; released before
  // the resident tables and the arena
  std::map<std::string, std::shared_ptr<vx::GraphEntry>> graphs;
  // per-chunk statistics logged by plans (features, survivor fraction) and the
  // cardinality regressor fitted on them
  std::vector<float> chunk_log_x, chunk_log_y;
  float reg_w[8] = {0};
  bool reg_trained = false;
  void *serve = nullptr;  // serving engine (vx_serve_start .. vx_serve_stop)
  // set when device work of a call that gave up on a wait did not finish
  // within the drain limit either: the arena blocks that work may still write
  // are never handed out again, and every later call fails
  bool poisoned = false;
  bool host_ptr_ok = false;  // kernels may use host pointers of registered memory as they are
  // per-chunk timeline of the last pipeline run with log_timeline (rows of
  // VX_TIMELINE_COLS floats)
  std::vector<float> timeline;
  // page-locked host intermediates of operator-at-a-time plans, kept between
  // calls and grown on demand
  char *op_host = nullptr;
  uint64_t op_host_bytes = 0;
};

namespace vx {
void serve_shutdown(vx_ctx *ctx);  // stops and frees the serving engine, if any
}

namespace vx {

vx_status check_ctx(vx_ctx *ctx);
const Column *get_col(vx_ctx *ctx, int32_t id, int32_t want_dtype /* -1 any */);
double now_ms();

// ------------------------------------------------------------------ executor
// A host->device or device->host copy of one extent.
struct CopyOp {
  const void *src;
  void *dst;
  uint64_t bytes;
};

// The paper's ExKernel (Section 5.2): a data mapping (size(), inputs(it) as a
// list of host extents copied into the staging slot, outputs(it) as device ->
// host extents known once the kernel of chunk `it` has finished) plus a kernel
// adaptation (kernel(slot, it, stream)) that sees device memory only.
struct ExKernel {
  virtual ~ExKernel() = default;
  virtual uint64_t size() = 0;                 // number of chunks
  virtual uint64_t slot_bytes() = 0;           // bytes of one staging slot
  virtual void inputs(uint64_t it, char *slot, std::vector<CopyOp> &h2d) = 0;
  virtual vx_status kernel(char *slot, uint64_t it, cudaStream_t s) = 0;
  virtual bool has_outputs() { return false; }
  // called once the kernel of chunk `it` has completed (immediate schedule)
  virtual void on_retire(uint64_t it) {}
  // called after kernel(it) has completed on the device
  virtual vx_status outputs(uint64_t it, char *slot, std::vector<CopyOp> &d2h) { return VX_OK; }
  // slots of the ring (0: the context's n_slots) and chunks the immediate
  // schedule keeps in flight at once (loaded, computing or storing)
  virtual int n_slots() { return 0; }
  virtual int max_in_flight() { return 3; }
};

struct ExecStats {
  uint64_t chunks = 0, bytes_h2d = 0, bytes_d2h = 0, kernel_launches = 0;
  double ms_kernel = 0;
};

// Issues host <-> device copies on stream s (bytes += their sizes): the copy
// engine, or for host-to-device copies with sm_blocks > 0 a copy kernel of
// that many blocks reading the pinned host memory (4-byte aligned ops only;
// others go to the copy engine).  Host addresses off a 512-byte boundary are
// split for the copy engine into a short head and an aligned body.
vx_status issue_copies(const std::vector<CopyOp> &ops, cudaMemcpyKind kind, cudaStream_t s, uint64_t *bytes,
                       int sm_blocks);
// the context's choice for host-to-device staging: copy-kernel blocks, or 0
int h2d_sm_blocks(const vx_ctx *ctx);

// Runs all chunks of `k` through a ring of cfg.n_slots staging slots allocated
// from the arena (Section 5.3 pipelined executor).
vx_status run_pipeline(vx_ctx *ctx, ExKernel &k, ExecStats *st);

// Waits, without blocking on the device, until the work already issued on the
// context's three streams has finished, for at most max(wait_timeout_ms,
// kDrainLimitMs).  Returns false (and marks the context poisoned) if it had
// not finished by then.
constexpr double kDrainLimitMs = 10000;
bool drain_streams(vx_ctx *ctx);

// A context over a block of `bytes` from the parent's arena, with its own
// streams and scalar block, sharing the parent's registered columns (the
// parent keeps their registrations): one operator runs in it concurrently
// with the parent's own work.  close_child gives the block back.
vx_status open_child(vx_ctx *parent, uint64_t bytes, vx_ctx **out);
void close_child(vx_ctx *parent, vx_ctx *child);

// Enqueues every chunk of `k` as a stream/event DAG into a caller-owned ring
// while the compute stream is being captured: the copy stream is forked from
// and joined back into the compute stream, nothing is synchronised.
vx_status enqueue_pipeline_for_capture(vx_ctx *ctx, ExKernel &k, char *ring, int n_slots, ExecStats *st);

// Registers caller host memory for the duration of a call unless it is
// already page-locked: copies to or from pageable memory hold the issuing
// thread until the stream's earlier work is done.
struct HostReg {
  void *p = nullptr;
  bool reg = false;
  vx_status add(void *ptr, uint64_t bytes) {
    if (!ptr || !bytes) return VX_OK;
    cudaPointerAttributes at{};
    cudaError_t e = cudaPointerGetAttributes(&at, ptr);
    cudaGetLastError();
    if (e == cudaSuccess && at.type == cudaMemoryTypeHost) return VX_OK;
    e = cudaHostRegister(ptr, bytes, cudaHostRegisterMapped);
    if (e != cudaSuccess) {
      cudaGetLastError();
      set_error("cudaHostRegister(%llu) failed: %s", (unsigned long long)bytes, cudaGetErrorString(e));
      return VX_E_CUDA;
    }
    p = ptr;
    reg = true;
    return VX_OK;
  }
  ~HostReg() {
    if (reg) cudaHostUnregister(p);
  }
};

}  // namespace vx
