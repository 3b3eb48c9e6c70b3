// Parameter blocks and constants of the star-join / filter kernels.
#pragma once
#include <cstdint>
#include <memory>
#include <string>

#include "vx_internal.h"

namespace vx {

// open-addressing slot: (value << 32) | uint32(key); value 0xFFFFFFFF = empty,
// 0xFFFFFFFE = key present but the row fails the dimension predicates
constexpr uint32_t HT_EMPTY_VAL = 0xFFFFFFFFu;
constexpr uint32_t HT_FILTERED = 0xFFFFFFFEu;
constexpr unsigned long long HT_EMPTY = 0xFFFFFFFF00000000ull;

constexpr int kMaxRoles = 12;        // distinct fact columns a plan may reference
constexpr uint32_t kSmemGroups = 4096;  // groups accumulated in shared memory
// Zero-copy threshold for 4-byte columns on one host link: TH = (E / G) *
// (B_zc / B_ce) (Section 6.3, generalised) with a 64-byte link granule and
// equal zero-copy and copy-engine bandwidth.
constexpr double kDefaultZeroCopyTH = 4.0 / 64.0;

constexpr int kFilterThreads = 256;
constexpr int kFilterItems = 8;
constexpr int kFilterTile = kFilterThreads * kFilterItems;

struct DimSpec {
  const int32_t *key = nullptr;
  int32_t key_col = -1;
  uint64_t rows = 0;
  int n_attr = 0;
  const int32_t *attr[4] = {};
  int32_t attr_col[4] = {-1, -1, -1, -1};
  uint32_t stride[4] = {};
  int32_t card[4] = {};
  int n_preds = 0;
  int32_t pred_attr[4] = {}, pred_op[4] = {}, pred_lo[4] = {}, pred_hi[4] = {};
};

// A dimension table on the device: an open-addressing hash table of 8-byte
// slots, or — when the keys are dense (span <= 2 x rows) — a direct map of one
// value per key in [kmin, kmin + span), 1, 2 or 4 bytes wide: the narrowest
// that holds the dimension's largest group-code contribution below its two
// marker values (no such key, key filtered out), so the map of a 2M-row
// dimension takes 2 MB instead of 8 and stays in L2 while chunks stream.
struct BuiltDim {
  DevBuf buf;
  uint32_t log2cap = 0;
  uint64_t rows = 0, passed = 0;
  int32_t kmin = 0;
  uint32_t span = 0;  // > 0: direct map
  uint32_t vbytes = 4;  // direct map: bytes per value (1, 2 or 4)
};

struct ResidentHT {
  BuiltDim dim;
  bool built = false;
};

inline std::string dim_signature(const DimSpec &d) {
  std::string s = "k" + std::to_string(d.key_col) + ":" + std::to_string(d.rows);
  for (int a = 0; a < d.n_attr; ++a)
    s += "|a" + std::to_string(d.attr_col[a]) + "s" + std::to_string(d.stride[a]) + "c" + std::to_string(d.card[a]);
  for (int q = 0; q < d.n_preds; ++q)
    s += "|p" + std::to_string(d.pred_attr[q]) + "o" + std::to_string(d.pred_op[q]) + "l" +
         std::to_string(d.pred_lo[q]) + "h" + std::to_string(d.pred_hi[q]);
  return s;
}

struct DimBuildParams {
  const int32_t *key;
  uint64_t rows;
  int n_attr;
  const int32_t *attr[4];
  uint32_t stride[4];
  int32_t card[4];
  int n_preds;
  int32_t pred_attr[4], pred_op[4], pred_lo[4], pred_hi[4];
  uint64_t *slots;
  uint32_t log2cap;
  uint32_t *err;
  unsigned long long *passed;
  uint32_t *dmap;  // non-null: build the direct map instead of the hash table
  int32_t kmin;
  uint32_t span;
};

struct ChunkParams {
  const int32_t *staged[kMaxRoles];  // role -> column slice in the staging slot (chunk-local rows)
  const int32_t *zc[kMaxRoles];      // role -> mapped host column (global rows), for late roles
  int n_fact_preds;
  int8_t fp_role[VX_MAX_PREDS];
  int32_t fp_op[VX_MAX_PREDS], fp_lo[VX_MAX_PREDS], fp_hi[VX_MAX_PREDS];
  int n_dims;
  int8_t dim_role[VX_MAX_DIMS];
  const uint64_t *ht[VX_MAX_DIMS];  // hash slots, or the uint32 direct map when dspan[d] > 0
  uint32_t ht_log2[VX_MAX_DIMS];
  int32_t dmin[VX_MAX_DIMS];
  uint32_t dspan[VX_MAX_DIMS];
  uint8_t dvb[VX_MAX_DIMS];         // direct map: bytes per value (1, 2 or 4; see dmap_get)
  int n_fgk;
  int8_t fgk_role[VX_MAX_GKEYS];
  int32_t fgk_card[VX_MAX_GKEYS];
  uint32_t fgk_stride[VX_MAX_GKEYS];
  int agg_op;
  int8_t agg_a_role, agg_b_role;
  uint32_t n_groups;
  unsigned long long *g_sum, *g_cnt;
  uint32_t *err;
  uint64_t row0, n;
  unsigned long long *chunk_surv;  // optional per-chunk survivor counts (statistics log)
  uint64_t chunk_idx;
  uint2 *surv_list;                // split mode: (chunk row, group id) of every survivor
  unsigned int *surv_cnt;          // survivors of the chunk (counted past surv_cap)
  unsigned int surv_cap;           // entries surv_list holds; survivors past it are not written
  unsigned int *chunk_ovf;         // optional per-chunk flag: the list overflowed, the chunk was not aggregated
  // vector path: the staged roles the row logic reads (predicates, keys,
  // fact group keys), and where each predicate / key / group key finds its
  // value among them
  int n_rowroles;
  int8_t rowrole[8];
  int8_t fp_slot[VX_MAX_PREDS], dim_slot[VX_MAX_DIMS], fgk_slot[VX_MAX_GKEYS];
  // slot of each aggregate column among them when it is staged in every chunk
  // (loaded with the row logic's columns), else -1 (loaded per survivor)
  int8_t agg_slot[2];
  // shared-scan kernel (serving): row-logic slot k of this query lives in
  // union column ucol[k] of the staged chunk; the query's rows of the chunk
  // are [row_lo, n); scan_kr = its vector width (0: the (query, tile) kernel)
  int8_t ucol[8];
  int8_t scan_kr;
  uint64_t row_lo;
};

constexpr uint32_t kStarTileRows = 2048;  // rows of one block tile (256 threads x 8 rows)
// ---- end of what the fused chunk kernel's device code reads

// work item of the persistent multi-query kernel: rows [tile * kMultiTile,
// (tile + 1) * kMultiTile) of query q's part of the staged chunk
struct MultiItem {
  uint32_t q, tile;
};
constexpr uint32_t kMultiTile = 256 * 8;
// Shared-scan kernel of the serving engine: resident blocks pull 1024-row
// tiles of the staged chunk (n_rows rows, n_cols union columns of col_stride
// bytes from dcols), stage each tile's union columns in shared memory once
// and evaluate every query with scan_kr != 0 against them.
vx_status launch_star_scan(vx_ctx *ctx, const ChunkParams *d_params, uint32_t n_q, const char *dcols,
                           uint64_t col_stride, uint32_t n_cols, uint64_t n_rows, unsigned int *d_next,
                           cudaStream_t s);
vx_status launch_star_multi(vx_ctx *ctx, const ChunkParams *d_params, const MultiItem *d_items, uint32_t n_items,
                            unsigned int *d_next, cudaStream_t s);

// per-chunk features of the cardinality regressor: [1, f_fact, f_all, f_fact * dim_sel]
constexpr int kChunkFeatures = 4;
constexpr int kChunkSampleRows = 256;  // 4 runs of 64 consecutive rows per chunk

struct SampleParams {
  int n_preds;
  const int32_t *col[VX_MAX_PREDS];
  int32_t op[VX_MAX_PREDS], lo[VX_MAX_PREDS], hi[VX_MAX_PREDS];
  uint64_t row_begin, n;
  uint32_t n_samples;
  unsigned long long *out;
};

struct FilterParams {
  int n_preds;
  const int32_t *col[VX_MAX_PREDS];
  int32_t colidx[VX_MAX_PREDS];
  int32_t op[VX_MAX_PREDS], lo[VX_MAX_PREDS], hi[VX_MAX_PREDS];
  uint64_t row0, n;
};

// A plan's whole chunk pipeline captured as one CUDA graph: it owns the
// staging ring and accumulators the graph writes and keeps the dimension
// tables it reads alive.
struct GraphEntry {
  DevBuf ring, acc, err;
  DevBuf ovf;  // per-chunk survivor-list overflow flags of the replay
  cudaGraphExec_t exec = nullptr;
  std::vector<std::shared_ptr<ResidentHT>> tables;
  uint64_t chunks = 0, bytes_h2d = 0, launches = 0;
  // per chunk: events recorded as graph nodes around the fused kernel [a, b)
  // and the late-column gather [b, c) (split chunks only), read after a replay
  std::vector<cudaEvent_t> ev_a, ev_b, ev_c;
  std::vector<uint8_t> split;
  ~GraphEntry() {
    if (exec) cudaGraphExecDestroy(exec);
    for (auto v : {&ev_a, &ev_b, &ev_c})
      for (cudaEvent_t e : *v)
        if (e) cudaEventDestroy(e);
  }
};

vx_status build_dim_table(vx_ctx *ctx, const DimSpec &d, BuiltDim *out, uint32_t *d_err, uint64_t *d_passed);
vx_status check_err_word(vx_ctx *ctx, const uint32_t *d_err);
// A planned star query ready to be executed chunk by chunk by another executor
// (the serving engine): kernel parameters (tables, predicates, roles, late
// columns as zero-copy pointers), zeroed accumulators and the columns to stage.
struct PreparedStar {
  ChunkParams P{};
  DevBuf acc, scratch;
  std::vector<std::shared_ptr<ResidentHT>> tables;
  std::vector<int32_t> role_col;          // role -> column id
  std::vector<const Column *> staged_cols;
  std::vector<int> staged_role;
  uint64_t G = 0, row_begin = 0, n_rows = 0;
  uint32_t late_mask = 0;
  double est = 0;
};

bool evict_unused_resident(vx_ctx *ctx);
// a star plan one operator at a time with host intermediates
vx_status run_star_operators(vx_ctx *ctx, const vx_plan *plan, vx_result *out);

// Plans and runs a star query; with prep != nullptr it only plans (tables
// built, accumulators zeroed) and moves the plan into *prep.
vx_status run_star(vx_ctx *ctx, const vx_plan *plan, vx_result *out, bool use_resident,
                   PreparedStar *prep = nullptr);

}  // namespace vx
