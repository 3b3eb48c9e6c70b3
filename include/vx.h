/*
 * vx.h — C ABI of the GB300 out-of-core query library.
 *
 * The library runs relational operators over columns that live in host memory
 * and are larger than the device budget (Vortex, arXiv 2502.09541).  As in the
 * paper's IO-decoupled programming model (Section 5), every operator is split
 * into (a) a data mapping — which host extents form chunk `it` — and (b) an
 * IO-agnostic kernel that sees only device buffers; a pipelined executor
 * (Section 5.3) streams chunks from pinned host memory into staging slots on
 * a copy-engine stream while the kernel of the previous chunk runs and the
 * output of the chunk before it is saved.  Columns whose estimated selectivity
 * is below the zero-copy threshold are not staged: the kernel reads them from
 * mapped host memory for qualifying rows only (Section 6.3).
 *
 * Conventions
 *   - Every call returns vx_status: VX_OK (0) or a negative VX_E_* code.
 *     vx_last_error() returns a thread-local message for the last failure.
 *   - Handles are opaque.  One context may be used by one thread at a time
 *     (calls take an internal lock; concurrent calls serialise).
 *   - Host memory: the caller owns every host buffer.  Registered columns must
 *     stay alive and unchanged until they are unregistered or the context is
 *     closed.  The library page-locks (cudaHostRegister, mapped) columns that
 *     are not already pinned and unlocks them again on unregister/close.
 *     Output buffers are plain host memory sized by the caller; a call whose
 *     output does not fit returns VX_E_CAPACITY and reports the size needed.
 *   - Device memory: all device memory the library uses comes from one arena
 *     of exactly the budget given to vx_open (or the arena handed to
 *     vx_open_ex).  A request that does not fit returns VX_E_NOMEM.
 *   - Results are exact: integer keys, two's-complement wrapping 64-bit sums,
 *     row ids in ascending order, stable sort order.
 */
#ifndef VX_H
#define VX_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t vx_status;

enum {
  VX_OK = 0,
  VX_E_INVAL = -1,       /* bad argument */
  VX_E_NOMEM = -2,       /* device arena or host allocation exhausted */
  VX_E_CUDA = -3,        /* CUDA runtime error (message in vx_last_error) */
  VX_E_CAPACITY = -4,    /* caller output buffer too small; required size reported */
  VX_E_TIMEOUT = -5,     /* a bounded wait expired */
  VX_E_BUSY = -6,        /* serving queue full */
  VX_E_UNSUPPORTED = -7, /* valid request outside what the library implements */
  VX_E_DUPKEY = -8,      /* duplicate key on the build side of a join */
  VX_E_RANGE = -9        /* a group-key code outside [0, card) */
};

typedef enum { VX_I32 = 0, VX_U32 = 1, VX_I64 = 2, VX_U64 = 3 } vx_dtype;

typedef struct vx_ctx vx_ctx;

/* ---------------------------------------------------------------- config */
enum { VX_SCHED_IMMEDIATE = 0, VX_SCHED_DAG = 1 };
/* Late materialization of a plan's aggregate columns (Section 6.3):
 * AUTO decides once per plan (estimated selectivity below TH -> zero-copy);
 * PER_CHUNK decides per chunk from the per-chunk cardinality regressor's
 * predicted selectivity (or the chunk's sampled selectivity while no
 * regressor is trained). */
enum { VX_LATE_AUTO = 0, VX_LATE_FORCE_EARLY = 1, VX_LATE_FORCE_LATE = 2, VX_LATE_PER_CHUNK = 3 };

typedef struct {
  uint64_t chunk_bytes;     /* staged host bytes per chunk, all staged columns (default 64 MiB) */
  int32_t n_slots;          /* staging slots in the ring, >= 2 (default 3) */
  int32_t sched;            /* VX_SCHED_IMMEDIATE: the host issues a copy only when it can run at
                               once (Section 4.3, principle 1); VX_SCHED_DAG: every copy and kernel
                               is enqueued up front with stream/event dependencies (Section 4.2) */
  int32_t late_mat;         /* default late-materialization policy of vx_run_plan */
  double zc_threshold;      /* selectivity threshold TH of Section 6.3; 0 = default */
  int32_t use_graphs;       /* vx_run_plan: capture the chunk pipeline in a CUDA graph and replay it */
  int32_t block_threads;    /* threads per block of the chunk kernels (default 256) */
  int32_t blocks_per_sm;    /* resident blocks per SM of the chunk kernels (default 4) */
  uint32_t wait_timeout_ms; /* limit of every host-side wait (default 60000) */
  int32_t log_chunk_stats;  /* vx_run_plan logs per-chunk features and survivor fractions (the
                               cardinality regressor's training data); not with use_graphs */
  int32_t log_timeline;     /* the immediate schedule records when every chunk's copies and kernel
                               ran (vx_last_timeline); not with use_graphs */
  int32_t kernel_rows;      /* shape of the fused chunk kernel: 0 = automatic (where the columns
                               allow, one 1024-row tile per block, 4 rows per thread read as
                               16-byte column vectors; else the scalar kernel at 8 rows per
                               thread), 2 = the bulk-copy pipeline (persistent blocks, at most
                               blocks_per_sm per SM, 1024-row tiles of the row-logic columns
                               copied into a ring of shared-memory stages, 4 rows per thread),
                               8 or 16 = the scalar kernel with that many rows per thread and at
                               most blocks_per_sm blocks per SM */
  uint32_t lookback_spin_limit; /* polls a radix sort pass makes of one predecessor tile's published
                               count before it gives up, sets its error word and the call returns
                               VX_E_TIMEOUT (0 = 2^20) */
  int32_t h2d_copy_blocks;  /* host-to-device staging of every executor: 0 = the copy engine
                               (cudaMemcpyAsync); n > 0 = a copy kernel of n blocks of 256 threads
                               on the host-to-device stream, loading the pinned host memory through
                               its device-visible address (where the device allows it, else the
                               copy engine), launched at the device's greatest stream priority (and
                               captured graphs honour it) so that its blocks are not queued behind
                               a chunk kernel's; at most 1024 */
  int32_t reserved;         /* 0 */
} vx_config;

/* ---------------------------------------------------------------- lifetime */

/* Opens a context on the current CUDA device with a device arena of exactly
 * device_budget_bytes (one cudaMalloc).  The budget caps every operator so that
 * data larger than it must stream (Section 5.3: the executor divides device
 * memory into staging buffers and temporary space).  Creates three streams:
 * compute, host-to-device and device-to-host. */
vx_status vx_open(uint64_t device_budget_bytes, vx_ctx **out);

/* As vx_open, but uses a caller-owned device arena [dev_arena, dev_arena+bytes)
 * (e.g. allocated by PyTorch) and, if cuda_stream is non-NULL, that stream as
 * the compute stream.  The arena must stay allocated until vx_close. */
vx_status vx_open_ex(void *dev_arena, uint64_t bytes, void *cuda_stream, vx_ctx **out);

/* Unregisters all columns, frees what the context allocated, destroys its
 * streams.  NULL is accepted. */
vx_status vx_close(vx_ctx *ctx);

/* Thread-local text of the last error ("" if none). */
const char *vx_last_error(void);

vx_status vx_get_config(vx_ctx *ctx, vx_config *out);
vx_status vx_set_config(vx_ctx *ctx, const vx_config *cfg);

/* ---------------------------------------------------------------- columns */

/* Registers a host column of n_rows elements of dtype (the paper's stationary
 * DRAM data, Section 5.2: only a mapping table refers to it).  flags: 0.
 * Returns its id in *col_id. */
vx_status vx_register_host_column(vx_ctx *ctx, const char *name, int32_t dtype, const void *host,
                                  uint64_t n_rows, uint32_t flags, int32_t *col_id);
vx_status vx_unregister_host_column(vx_ctx *ctx, int32_t col_id);

/* ---------------------------------------------------------------- predicates */
enum { VX_BETWEEN = 0, VX_EQ = 1, VX_NE = 2, VX_LT = 3, VX_LE = 4, VX_GT = 5, VX_GE = 6 };

/* Row predicate on an int32 column: BETWEEN is lo <= v <= hi; the others
 * compare v with lo. */
typedef struct {
  int32_t col;
  int32_t op;
  int32_t lo, hi;
} vx_pred;

/* Filter with stream compaction (Section 6.3, selection sigma): writes the
 * ascending global row ids r in [row_begin, row_end) for which every predicate
 * holds into out_rows[0 .. min(count, cap)), and the full count into
 * *out_count.  row_end = 0 means the column length.  out_rows may be NULL (count
 * only).  All predicate columns must be int32 and of equal length.
 * Returns VX_E_CAPACITY if count > cap (the first cap ids are written). */
vx_status vx_filter(vx_ctx *ctx, const vx_pred *preds, int32_t n_preds, uint64_t row_begin,
                    uint64_t row_end, uint64_t *out_rows, uint64_t cap, uint64_t *out_count);

/* Allocation-free filter over device-resident columns.  The paper has no
 * counterpart: this entry point exists for callers that cannot let a library
 * allocate device memory — code running inside another framework's memory
 * manager that owns all device memory and hands out only input and output
 * buffers, and latency-critical paths where a cudaMalloc/cudaFree (which may
 * synchronise the device) is not acceptable.  It needs no context.
 *
 * cols: host array of n_cols device pointers to int32 columns of n_rows
 * elements; preds[q].col indexes cols.  Writes the ascending ids row0 + i of
 * the rows satisfying every predicate to the device buffer out_rows[0 ..
 * min(count, cap)) and the full count to *out_count (host).  stream: the
 * caller's cudaStream_t (NULL = default stream); the call returns after the
 * work on that stream has finished.
 *
 * Scratch lives in a fixed file-scope device array (256 KiB + 256 B, held on
 * every GPU that loads the library until the process exits); it allocates
 * nothing: no cudaMalloc, cudaFree or allocating library routine.  Limits and
 * behaviour:
 *   - n_rows above 67,108,864 (2^26) returns VX_E_INVAL;
 *   - count > cap returns VX_E_CAPACITY after writing the first cap ids;
 *   - the first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress with that device current) and keeps it for the
 *     life of the process, so the device must not be reset (cudaDeviceReset)
 *     between calls;
 *   - every call shares the one array, so calls whose work overlaps on the
 *     GPU (other streams, other host threads) race and give wrong results:
 *     serialise them. */
vx_status vx_filter_device_static(const int32_t *const *cols, int32_t n_cols, const vx_pred *preds,
                                  int32_t n_preds, uint64_t n_rows, uint64_t row0, uint64_t *out_rows,
                                  uint64_t cap, uint64_t *out_count, void *stream);

/* ---------------------------------------------------------------- plans */
enum { VX_AGG_COUNT = 0, VX_AGG_SUM = 1, VX_AGG_MUL = 2, VX_AGG_SUB = 3 };
#define VX_MAX_DIMS 8
#define VX_MAX_PREDS 8
#define VX_MAX_GKEYS 4

/* One dimension of a star plan: the fact column fact_fk_col is joined to
 * key_col (unique int32 keys, an inner join), and the dimension predicates
 * are applied to its attribute columns (Section 7.1: dimensions are filtered
 * and hashed on the device and kept there while fact chunks stream). */
typedef struct {
  int32_t key_col;
  int32_t fact_fk_col;
  int32_t n_attr;
  int32_t attr_col[4];
  int32_t n_preds;
  int32_t pred_attr[4]; /* index into attr_col */
  int32_t pred_op[4], pred_lo[4], pred_hi[4];
} vx_plan_dim;

/* Group key: dim >= 0 -> attribute attr of dimension dim; dim == -1 -> the
 * int32 fact column fact_col.  Codes must lie in [0, card). */
typedef struct {
  int32_t dim;
  int32_t attr;
  int32_t card;
  int32_t fact_col;
} vx_plan_gkey;

/* A star query: filter fact rows, probe the dimensions in the given order,
 * group by the mixed-radix number of the group-key codes (first key most
 * significant) and aggregate agg(a, b) as wrapping int64 sums plus counts. */
typedef struct {
  int32_t n_dims;
  vx_plan_dim dims[VX_MAX_DIMS];
  int32_t n_fact_preds;
  vx_pred fact_preds[VX_MAX_PREDS];
  int32_t n_group_keys;
  vx_plan_gkey group_keys[VX_MAX_GKEYS];
  int32_t agg_op;        /* VX_AGG_* */
  int32_t agg_a, agg_b;  /* int32 fact columns (-1 if unused) */
  int32_t late_mat;      /* VX_LATE_* for the aggregate columns */
  uint64_t row_begin, row_end; /* fact row range; row_end = 0 means all rows */
} vx_plan;

/* Per-call statistics (host-visible). */
typedef struct {
  uint64_t rows;           /* fact rows scanned */
  uint64_t survivors;      /* rows aggregated / emitted */
  uint64_t chunks;
  uint64_t bytes_h2d;      /* bytes moved by the copy engine host->device */
  uint64_t bytes_d2h;      /* bytes moved by the copy engine device->host */
  uint64_t bytes_zero_copy;/* estimated bytes crossing the link for zero-copy reads (64 B granules) */
  uint64_t bytes_logical;  /* referenced column bytes x rows (the host data the query consumes) */
  uint32_t late_mask;      /* bit i set: aggregate column i was read by zero-copy */
  uint32_t overflow_retries;
  double est_selectivity;  /* planner estimate used for the late/early decision */
  double ms_total;         /* wall time of the call */
  double ms_kernel;        /* summed device time of the fused chunk kernels (CUDA events around each
                              launch, as event nodes inside a captured graph) */
  uint64_t kernel_launches;/* kernels launched by the call */
  uint64_t late_chunks;    /* VX_LATE_PER_CHUNK: chunks whose aggregate columns were read by zero-copy */
  double ms_gather;        /* summed device time of the zero-copy gathers of late chunks (CUDA events;
                              0 when not timed: DAG schedule, serving) */
  double ms_features;      /* wall time of the per-chunk feature pass before the pipeline (sampling
                              kernel, copy-back and the per-chunk decisions); 0 when it did not run */
  uint64_t surv_list_bytes;/* device bytes of one staging slot's survivor list (split mode): every
                              row of a chunk, or with VX_LATE_PER_CHUNK the regressor's predicted
                              survivors plus headroom (overflow_retries counts chunks rerun with a
                              full list because their survivors did not fit) */
} vx_query_stats;

/* Result of vx_run_plan / vx_groupby: groups with count > 0 in ascending group
 * id.  The caller provides arrays of capacity cap; *n_out receives the number
 * of non-empty groups (VX_E_CAPACITY if it exceeds cap). */
typedef struct {
  uint64_t cap;
  uint64_t *gid;
  int64_t *sum;
  uint64_t *cnt;
  uint64_t n_out;
  vx_query_stats stats;
} vx_result;

/* Runs a star plan over the registered columns (Sections 5-7: chunked fact
 * stream, resident dimension hash tables, zero-copy late materialization). */
vx_status vx_run_plan(vx_ctx *ctx, const vx_plan *plan, vx_result *out);

/* The same star plan run one operator at a time with host intermediates
 * (Section 6.4: operators extended with the IO decoupling can be chained,
 * with CPU memory holding the intermediate results): a filter over the fact
 * predicates, one probe per dimension in plan order and the aggregate, each
 * a pipelined pass over the fact chunks that loads the previous operator's
 * (row, group code) entries from page-locked host memory and stores its own
 * there, so no intermediate has to fit the device budget.  An operator
 * stages a chunk's fact columns by copy engine when its input holds at least
 * TH of the chunk's rows, else reads them through mapped host memory.  The
 * result equals vx_run_plan's; the intermediates (16 bytes per fact row of
 * the plan's range) are kept by the context between calls. */
vx_status vx_run_plan_operators(vx_ctx *ctx, const vx_plan *plan, vx_result *out);

/* Group-by aggregation over fact columns only (a star plan without
 * dimensions): keys are int32 fact columns with codes in [0, card). */
vx_status vx_groupby(vx_ctx *ctx, const vx_plan_gkey *keys, int32_t n_keys, int32_t agg_op, int32_t agg_a,
                     int32_t agg_b, const vx_pred *preds, int32_t n_preds, vx_result *out);

/* ---------------------------------------------------------------- cardinality regressor */

/* Ridge least squares on the device: w = argmin |X w - y|^2 + lambda |w|^2 for
 * n host rows of d <= 8 fp32 features (row-major X), from the normal equations
 * accumulated in fp64 and solved by Cholesky factorisation.  VX_E_INVAL if the
 * system is singular. */
vx_status vx_regressor_fit(vx_ctx *ctx, const float *X, const float *y, uint64_t n, int32_t d, float lambda,
                           float *w_out);

/* Per-chunk cardinality regressor: fits the statistics that plans logged
 * with log_chunk_stats (per chunk, from 256 sampled rows: features [1, f_fact
 * (fraction passing the fact predicates), f_all (fraction passing every
 * predicate and probe), f_fact x the product over dimensions of the fraction
 * whose key passes that dimension's filter]; target = exact survivor
 * fraction) and keeps
 * the 4 weights in the context; VX_LATE_PER_CHUNK plans then decide late vs
 * early materialization per chunk from the predicted selectivity against TH
 * (Section 6.3 decides from an estimator S_c given before the operator runs)
 * and size each staging slot's survivor list from the largest predicted
 * survivor count of a late chunk (plus a quarter and four standard
 * deviations): a chunk whose survivors do not fit is flagged on the device,
 * left out of the aggregate and rerun with a full list, so results never
 * depend on the prediction. */
vx_status vx_regressor_train(vx_ctx *ctx, float lambda, float *w_out, uint64_t *n_used);

/* Sets the regressor's 4 weights (as vx_regressor_train would leave them). */
vx_status vx_regressor_set(vx_ctx *ctx, const float *w, int32_t d);

/* Copies up to cap logged (features, target) rows; *n = rows logged. */
vx_status vx_chunk_log(vx_ctx *ctx, float *X, float *y, uint64_t cap, uint64_t *n);
/* Clears the log and the trained regressor. */
vx_status vx_chunk_log_clear(vx_ctx *ctx);

/* Autotuner of the executor and the fused kernel's launch shape for one
 * plan: times the plan over its first sample_rows fact rows (best of two
 * timed runs after one warm-up each) for every chunk size in {8, 16, 32, 64,
 * 128, 256} MiB and staging ring depth in {2, 3, 4} that fits the arena, then,
 * at the fastest of those, for every kernel shape in {one tile per block, the
 * bulk-copy pipeline at 4 or 6 blocks per SM, scalar 8 or 16 rows per thread
 * at 4 or 8 blocks per SM}, then host-to-device staging by the copy engine or
 * by a copy kernel of 32 blocks (h2d_copy_blocks, where the device allows
 * it); keeps the fastest in the context's config and returns it.  A candidate within 1 % of the fastest time (a tie on a
 * link-bound plan) wins if its fused-kernel time is lower.  Section 8.1 sweeps
 * Exchange's packet size the same way (fixed per-copy overhead against
 * pipeline depth).  Results do not depend on the configuration, only the time
 * does. */
vx_status vx_autotune(vx_ctx *ctx, const vx_plan *plan, uint64_t sample_rows, vx_config *best);

/* Frees the dimension hash tables that vx_run_plan keeps resident on the
 * device between calls (Section 7.1 keeps filtered dimension tables on the
 * GPU); the next plan rebuilds them from the host columns. */
vx_status vx_drop_resident(vx_ctx *ctx);

/* Statistics of the last completed call on this context. */
vx_status vx_last_stats(vx_ctx *ctx, vx_query_stats *out);

/* Per-chunk timeline of the last pipeline the immediate schedule ran with
 * log_timeline set (the copy / compute overlap of Section 5.3's executor,
 * measured with CUDA events on the copy and compute streams).  Row c of
 * VX_TIMELINE_COLS floats: chunk index, host time the chunk's loads were
 * issued, then start and end of its host-to-device copies, of its kernel and
 * of its device-to-host copies (-1 when it had none); times in ms from the
 * start of the pipeline.  Copies up to cap rows to out (row-major); *n =
 * rows recorded. */
#define VX_TIMELINE_COLS 8
vx_status vx_last_timeline(vx_ctx *ctx, float *out, uint64_t cap, uint64_t *n);

/* ---------------------------------------------------------------- sort */
enum { VX_PART_SAMPLE = 0, VX_PART_LEARNED_PL = 1, VX_PART_LEARNED_MLP = 2 };
/* Sort plans.  PARTITION: range-partition, then sort each partition (pass 1
 * needs splitters: sample or learned).  MERGE: Section 6.1's SortExKernel then
 * MergeExKernel: sort each contiguous chunk into a sorted run, cut the runs
 * into partitions at exact ranks (binary search over the runs, no sample, no
 * imbalance), merge each partition's segments; `partitioner` is not used. */
enum { VX_SORT_PARTITION = 0, VX_SORT_MERGE = 1 };

typedef struct {
  int32_t partitioner;        /* VX_PART_*: how the range partition's splitters are chosen */
  int32_t n_partitions;       /* 0 = smallest count whose expected partition fits a slot; <= 256 */
  uint64_t seed;              /* sample positions */
  uint64_t sample_size;       /* keys sampled for the splitters (0 = 1 Mi) */
  uint32_t mlp_steps;         /* Adam steps of the CDF MLP (0 = 300) */
  uint32_t region_slack_pct;  /* headroom of each partition's host region over its sample
                                 estimate, in percent (0 = 1 % plus four standard deviations of
                                 the sample count); smaller regions only add extents */
  void *host_scratch;         /* optional host memory of >= 12 * n bytes for the partitioned
                                 intermediate (else allocated for the call).  With room for
                                 the partitions' headroom (12 * (n + n / 16) bytes suffice at
                                 1e9 pairs; smaller inputs need a larger share) every partition
                                 gets a contiguous region, which the sort pass loads faster than
                                 the per-chunk pieces of an intermediate of exactly 12 * n
                                 bytes (stats: contiguous_layout) */
  uint64_t host_scratch_bytes;
  uint64_t max_slot_pairs;    /* optional cap on the pairs per staging slot (0 = from the arena) */
  uint64_t *splitters_out;    /* optional: receives the P-1 top-level splitters (PARTITION plan) */
  int32_t plan;               /* VX_SORT_PARTITION (default) or VX_SORT_MERGE */
  int32_t runs_mode;          /* MERGE: 0 = when a sample of adjacent pairs suggests the input is
                                 made of at most 256 ascending runs, find them (one pass over the
                                 keys) and merge them as they are, skipping pass 1; 1 = always
                                 sort the chunks into runs */
} vx_sort_opts;

typedef struct {
  uint32_t n_partitions;
  uint32_t passthrough_partitions; /* single-key partitions copied through unsorted */
  uint32_t overflow_retries;       /* multi-key partitions above the slot, sorted recursively */
  uint32_t contiguous_layout;      /* 1: the intermediate gave every partition its own region */
  uint64_t max_partition, min_partition, slot_pairs;
  double imbalance;                /* largest partition / mean partition */
  double ms_sample, ms_train, ms_partition, ms_sort, ms_total;
  uint64_t bytes_h2d, bytes_d2h, kernel_launches;
  double ms_sort_kernel;           /* device time of the per-partition radix sorts (CUDA events) */
  uint64_t radix_pass_pairs;       /* pairs x executed LSD passes in those sorts (skipped digits excluded) */
  uint64_t out_of_region_pairs;    /* pairs stored past their partition's region (overflow area,
                                      spill buffers) */
  uint64_t spill_buffers;          /* host buffers registered for the call when the overflow area
                                      ran out */
  uint32_t plan;                   /* VX_SORT_* that ran */
  uint32_t n_runs;                 /* MERGE: sorted runs written by pass 1 */
  double ms_merge_kernel;          /* MERGE: device time of the merge rounds (CUDA events) */
  uint64_t merge_pass_pairs;       /* MERGE: pairs x executed merge rounds */
  uint32_t natural_runs;           /* MERGE: 1 = the input's own ascending runs were merged (n_runs
                                      of them; pass 1 skipped, ms_partition is the detection) */
  uint32_t reserved;
} vx_sort_stats;

/* Out-of-core sort of (uint64 key, uint32 row id) pairs held in two registered
 * host columns (Section 6.1 sorts 64-bit integers larger than device memory).
 * The output is the stable sort by key (equal keys keep input order) written
 * to out_keys/out_rowids (n elements each, caller-owned host memory).
 * PARTITION plan: pass 1 range-partitions the input chunk by chunk into a
 * host intermediate with per-chunk boundary arrays (Section 6.2.1); pass 2
 * gathers each partition's extents, radix-sorts it in HBM and stores it at
 * its final offset (Section 5.3 pipeline for both).  Splitters come from a
 * sorted key sample (VX_PART_SAMPLE) or from a learned monotone CDF model: a
 * 1,024-segment piecewise-linear model (VX_PART_LEARNED_PL) or a 1-32-1 MLP
 * trained on the device (VX_PART_LEARNED_MLP).  MERGE plan (opts->plan): pass
 * 1 radix-sorts each contiguous chunk into a sorted run of the intermediate;
 * the runs are cut at exact ranks (vx_exact_splits) into equal partitions;
 * pass 2 loads each partition's run segments and merges them (vx_merge_runs);
 * an input already made of at most 256 ascending runs is merged as it is
 * (opts->runs_mode).
 * Both plans and any splitters give the same output; they decide only where
 * to cut.  The intermediate is opts->host_scratch when it holds 12 n bytes,
 * else allocated for the call. */
vx_status vx_sort(vx_ctx *ctx, int32_t key_col, int32_t rowid_col, uint64_t *out_keys, uint32_t *out_rowids,
                  const vx_sort_opts *opts, vx_sort_stats *stats);

/* In-HBM stable LSD radix sort of n pairs given in host buffers (the
 * per-partition sort of vx_sort, Section 6.1); n must fit the arena. */
vx_status vx_radix_sort_pairs(vx_ctx *ctx, const uint64_t *keys, const uint32_t *vals, uint64_t n,
                              uint64_t *out_keys, uint32_t *out_vals);

/* In-HBM stable range partition of n pairs (Section 6.2.1 clustering with a
 * range function): partition id = number of splitters <= key; writes the
 * pairs grouped by partition in input order and the P+1 boundary array
 * (boundary[p] = first position of partition p, boundary[P] = n; empty
 * partitions repeat the next start, as find_boundary back-fills them). */
vx_status vx_range_partition(vx_ctx *ctx, const uint64_t *keys, const uint32_t *vals, uint64_t n,
                             const uint64_t *splitters, uint32_t n_partitions, uint64_t *out_keys,
                             uint32_t *out_vals, uint64_t *boundary);

/* Splitters for n_partitions (2..128) requested partitions of a registered
 * uint64 column: sample_size keys at positions mix64(seed * 0x9E3779B97F4A7C15
 * + i) mod n (mix64 = SplitMix64 finalizer), sorted on the device, then the
 * chosen partitioner; then heavy-key isolation: a splitter not above the last
 * kept one becomes that one + 1, and a kept value occurring at least m/(2P)
 * times in the sample is followed by value + 1 so it forms its own partition.
 * splitters_out needs room for 2 * (n_partitions - 1) values; *n_out receives
 * the count. */
vx_status vx_sort_splitters(vx_ctx *ctx, int32_t key_col, int32_t partitioner, uint32_t n_partitions,
                            uint64_t sample_size, uint64_t seed, uint64_t *splitters_out, uint32_t *n_out);

/* Exact cut of sorted runs (the data mapping of Section 6.1's MergeExKernel:
 * regroup N sorted chunks into partitions with max(P_i) <= min(P_i+1)).  The
 * runs are n_runs consecutive sorted pieces of `keys` (host memory, run r =
 * [run_off[r], run_off[r+1]), run_off has n_runs + 1 entries starting at 0);
 * for each target rank k = ranks[q] writes out[q * n_runs + r] = how many
 * elements of run r precede the element of rank k in the stable order (by
 * key, then by position in `keys`), so the cut takes exactly k elements and
 * every element left of it orders before every element right of it.  A rank
 * >= the total takes every run whole.  Works on the device: a fence per 4,096
 * keys of every run in HBM, then per rank a binary search over the key value
 * whose counts read the runs through mapped host memory.  n_runs <= 256.
 * Runs that are not sorted give cuts of no meaning but stay within bounds. */
vx_status vx_exact_splits(vx_ctx *ctx, const uint64_t *keys, const uint64_t *run_off, uint32_t n_runs,
                          const uint64_t *ranks, uint32_t n_ranks, uint64_t *out);

/* In-HBM stable merge of n_runs sorted runs of (key, value) pairs given
 * back to back in host buffers (run r = [run_off[r], run_off[r+1])): the
 * per-partition kernel of Section 6.1's MergeExKernel, pairwise merge-path
 * merges in rounds over a double buffer, ties taken from the earlier run.
 * Writes the merged pairs to out_keys/out_vals; the input must fit the arena
 * twice over.  n_runs <= 256. */
vx_status vx_merge_runs(vx_ctx *ctx, const uint64_t *keys, const uint32_t *vals, const uint64_t *run_off,
                        uint32_t n_runs, uint64_t *out_keys, uint32_t *out_vals);

/* ---------------------------------------------------------------- join */
/* Join algorithms.  DIRECT: key-range partitions of the build side, each a
 * hash table in HBM probed by the streamed probe side (no partition is
 * written to host memory).  RADIX: Section 6.2's radix-partitioned join:
 * RadixPartitionExKer clusters every chunk of both tables by the low
 * radix_bits bits of the key and stores the clustered chunks and their
 * boundary arrays (find_boundary, Fig. 9) in host memory; HashJoinExKer then
 * loads ranges of groups, cut by binary search over the boundary arrays, and
 * joins each group in shared memory. */
enum { VX_JOIN_DIRECT = 0, VX_JOIN_RADIX = 1 };

typedef struct {
  int32_t partitioner;  /* VX_PART_*: splitters over the build keys when P > 1 */
  int32_t n_partitions; /* 0 = smallest P whose hash tables fit the budget; <= 256 */
  uint64_t seed;        /* sample positions */
  uint64_t sample_size; /* build keys sampled for the splitters (0 = 1 Mi) */
  double load_factor;   /* hash-table load; 0 = automatic: partitions counted at 0.8, each table then spread over the free budget down to 0.5 */
  int32_t count_pass;   /* 1: size tables from an exact count pass over the build keys (plain
                           form); 0: from the partition sizes the model implies, rebuilding a
                           table that overflows (learned form) */
  int32_t algorithm;    /* VX_JOIN_DIRECT (default) or VX_JOIN_RADIX */
  int32_t radix_bits;   /* RADIX: group bits, 8, 16 or 24 (0 = 24, the paper's 2^24 groups) */
  int32_t reserved;
} vx_join_opts;

typedef struct {
  uint64_t count;       /* matching (probe, build) pairs */
  uint64_t payload_sum; /* sum of matched build payloads, mod 2^64 */
  uint64_t pair_fp;     /* sum over matches of mix64(probe_row ^ rotl(payload, 17)), mod 2^64;
                           mix64 = SplitMix64 finalizer */
  uint32_t n_partitions, overflow_retries;
  uint64_t max_partition, bytes_h2d, kernel_launches;
  double ms_sample, ms_train, ms_build, ms_probe, ms_kernel, ms_total;
  double ms_probe_kernel;  /* device time of the probe kernels alone (CUDA events); every probe key
                              is looked up in exactly one partition */
  uint64_t bytes_d2h;      /* RADIX: clustered chunks and boundary arrays stored to host memory */
  uint32_t algorithm;      /* VX_JOIN_* that ran */
  uint32_t ranges;         /* RADIX: group ranges of the join pass */
  double ms_partition;     /* RADIX: wall time of the partition passes of both tables */
} vx_join_result;

/* Equi-join of a build table (unique 64-bit keys, 64-bit payload) with a
 * probe key column, all in registered host memory and possibly larger than
 * the budget (Section 6.2; A.key == B.key).  DIRECT: the build keys are cut
 * into n_partitions key ranges; for each range an open-addressing table is
 * built in HBM from the streamed build side and the streamed probe side
 * probes it (Section 5.3 executor for every stream).  RADIX (opts->algorithm):
 * the paper's radix-partitioned join (see VX_JOIN_RADIX); its host
 * intermediates (16 B per build row, 12 B per probe row, 4 (2^bits + 1) B per
 * chunk) are allocated for the call.  Returns VX_E_DUPKEY if a build key
 * repeats. */
vx_status vx_join(vx_ctx *ctx, int32_t build_key, int32_t build_payload, int32_t probe_key, const vx_join_opts *opts,
                  vx_join_result *out);

/* The clustering step of Section 6.2.1's RadixPartitionExKer on one chunk of
 * n < 2^32 keys (host buffers, in HBM for the call): a stable sort of
 * (key, chunk-local row) by the low `bits` bits of the key (8, 16 or 24),
 * written to out_keys / out_rows, and find_boundary (Fig. 9) of the
 * clustered groups: out_boundary gets 2^bits + 1 entries, entry g = first
 * position of group g (of the next non-empty group when g is empty), entry
 * 2^bits = n. */
vx_status vx_radix_cluster(vx_ctx *ctx, const uint64_t *keys, uint64_t n, int32_t bits, uint64_t *out_keys,
                           uint32_t *out_rows, uint32_t *out_boundary);

/* ---------------------------------------------------------------- learned CDF model */

/* Monotone CDF MLP with H hidden units (fp32):
 *   y(x) = gamma + sum_j softplus(alpha_j) * sigmoid(softplus(omega_j) * x + beta_j),
 * theta = [omega(H), beta(H), alpha(H), gamma].  Loss L = mean_i (y(x_i) - t_i)^2.
 * Evaluates L and dL/dtheta over m host points with the device forward and
 * backward kernels. */
vx_status vx_mlp_loss_grad(vx_ctx *ctx, const float *theta, int32_t H, const float *x, const float *t, uint64_t m,
                           float *grad_out, float *loss_out);

/* Trains theta in place with `steps` full-batch Adam steps (lr, beta1 0.9,
 * beta2 0.999, eps 1e-8; moments start at zero) on the device; writes the
 * final loss. */
vx_status vx_mlp_train(vx_ctx *ctx, float *theta, int32_t H, const float *x, const float *t, uint64_t m,
                       uint32_t steps, float lr, float *loss_out);

/* ---------------------------------------------------------------- serving */
typedef struct {
  uint64_t chunk_rows;  /* rows per chunk of the shared scan, multiple of 1024 (0 = 1 Mi) */
  uint32_t max_active;  /* queries attached to the scan at once (0 = 32, <= 256) */
  uint32_t n_slots;     /* staging slots (0 = 3) */
} vx_serve_opts;

enum { VX_QUERY_STAR = 0, VX_QUERY_SORT = 1, VX_QUERY_JOIN = 2 };

typedef struct {
  uint64_t submitted, completed, failed, cycles, bytes_h2d, active_peak;
  double p50_ms, p99_ms, mean_ms, max_ms; /* latency from submission to completion, all queries */
  double wall_ms;                         /* since vx_serve_start */
  uint64_t work_rows;                     /* query rows evaluated by the multi-query kernels */
  double ms_kernel;                       /* their device time (CUDA events) */
  double ms_admit;                        /* host time spent admitting (planning) queries */
  double ms_cycle;                        /* host time spent issuing scan cycles */
  double ms_wait;                         /* of which waiting for a staging slot's previous kernel */
  uint64_t completed_kind[3];             /* per VX_QUERY_* */
  double p50_kind_ms[3], p99_kind_ms[3];
} vx_serve_stats;

/* A sort- or join-shaped query for the serving engine (vx_submit_op). */
typedef struct {
  int32_t kind;                 /* VX_QUERY_SORT or VX_QUERY_JOIN */
  int32_t key_col, val_col;     /* sort: uint64 key and uint32 row-id columns; join: build key and payload */
  int32_t probe_col;            /* join: probe key column */
  uint64_t row_begin, row_end;  /* sort: pairs [row_begin, row_end); join: probe rows; row_end 0 = all */
  uint64_t *out_keys;           /* sort: the row_end - row_begin sorted keys, caller-owned until done */
  uint32_t *out_rowids;         /* sort: their row ids */
  uint64_t device_budget;       /* device bytes the query holds while it runs (0 = a quarter of the arena) */
  vx_sort_opts sort;            /* sort: as for vx_sort (host_scratch, if given, must be the query's own) */
  vx_join_opts join;            /* join: as for vx_join (VX_JOIN_DIRECT) */
} vx_op_request;

typedef struct {
  vx_sort_stats sort;     /* sort queries */
  vx_join_result join;    /* join queries: count, payload sum, pair fingerprint (probe rows are global) */
  double ms_total;        /* submission to completion */
  double ms_queued;       /* submission to admission */
} vx_op_result;

/* Starts the serving engine of a context: a thread that runs one shared
 * circular scan over the registered fact columns.  Each cycle stages one chunk
 * (the union of the columns its attached queries read, copied once) and runs
 * one persistent multi-query kernel over it.  Submitted star plans are
 * admitted when their accumulators and dimension tables fit the device budget
 * (tables stay resident and are shared by plans with equal dimension
 * filters) and attach at the current chunk (continuous batching); a query
 * completes once it has seen every chunk of its row range.  Results equal
 * vx_run_plan's.  Sort- and join-shaped queries (vx_submit_op) go to a second
 * thread: each is admitted once its device budget can be carved from the
 * arena (first come, first served) and runs as its own out-of-core operator
 * on its own streams, overlapping the shared scan on the device.  While
 * serving, other calls on the context are serialised with the engine. */
vx_status vx_serve_start(vx_ctx *ctx, const vx_serve_opts *opts);
/* Queues a plan; *ticket identifies it.  Does not block on device work. */
vx_status vx_submit(vx_ctx *ctx, const vx_plan *plan, uint64_t *ticket);
/* Queues a sort- or join-shaped query; *ticket identifies it (vx_wait_op,
 * vx_poll).  The result equals vx_sort's on the range (a stable sort of the
 * pairs [row_begin, row_end)) or vx_join's with the probe rows restricted to
 * the range. */
vx_status vx_submit_op(vx_ctx *ctx, const vx_op_request *req, uint64_t *ticket);
/* Blocks until the query of an op ticket finished or timeout_ms passed
 * (VX_E_TIMEOUT); fills out and returns the query's status. */
vx_status vx_wait_op(vx_ctx *ctx, uint64_t ticket, vx_op_result *out, uint32_t timeout_ms);
/* *done = 1 once the query finished; then fills out (groups, stats with
 * stats.ms_total = latency; for an op ticket only n_out = 0 and
 * stats.ms_total) and returns the query's status. */
vx_status vx_poll(vx_ctx *ctx, uint64_t ticket, vx_result *out, int32_t *done);
/* Blocks until the query finished or timeout_ms passed (VX_E_TIMEOUT). */
vx_status vx_wait(vx_ctx *ctx, uint64_t ticket, vx_result *out, uint32_t timeout_ms);
/* Counters and latency percentiles of completed queries. */
vx_status vx_serve_stats_get(vx_ctx *ctx, vx_serve_stats *out);
/* Stops the engine (pending queries are dropped); vx_close also does this. */
vx_status vx_serve_stop(vx_ctx *ctx);

/* ---------------------------------------------------------------- zero-copy probe */

/* The Section 6.3 micro-benchmark behind TH: for each SEL in sels,
 *   sum over i < n of (pred[i mod npred] mod SEL == 0 ? v[i] : 0)
 * with pred (npred = min(n, 2^24) int32) in device memory and v (n int32) in
 * pinned host memory, timed twice: reading v through mapped host memory
 * (ms_zero_copy[k]) and after double-buffered copy-engine transfers into HBM
 * (ms_copy[k]).  The sums of both reads must agree (checksums[k], optional).
 * Zero-copy wins for SEL above 1/TH. */
vx_status vx_probe_zero_copy(vx_ctx *ctx, uint64_t n, const int32_t *sels, int32_t n_sel, double *ms_zero_copy,
                             double *ms_copy, uint64_t *checksums);

/* Ceiling of the late-materialization gather (Section 6.3's zero-copy reads,
 * sparse): one launch reads n_reads 4-byte values at sorted uniform positions
 * (SplitMix64 of seed) of a window_bytes buffer of pinned, mapped host memory,
 * grid of 4 blocks of 256 threads per SM, one read per thread, the link
 * otherwise idle.  us_first: the first launch (the window's pages touched for
 * the first time); us_warm: the best of three more.  The sum of the values
 * read is checked on the host (checksum, optional).  The paper has no
 * counterpart: it is this library's denominator for the gather kernel.
 * VX_E_INVAL for window_bytes < 4 or above 2^34, or n_reads == 0; VX_E_NOMEM
 * if the indices do not fit the arena. */
vx_status vx_probe_zero_copy_gather(vx_ctx *ctx, uint64_t window_bytes, uint32_t n_reads, uint64_t seed,
                                    double *us_first, double *us_warm, uint64_t *checksum);

/* ---------------------------------------------------------------- link probe */

/* Pinned-copy microbenchmark of the host link (Section 8.1 measures Exchange
 * bandwidth against transfer and packet size): copies `bytes` in chunks of
 * `chunk` bytes host->device, device->host and both at once, using the
 * context's copy streams and arena, and reports GB/s (1e9 B/s). */
vx_status vx_probe_link(vx_ctx *ctx, uint64_t bytes, uint64_t chunk, double *h2d_gbs, double *d2h_gbs,
                        double *bidir_gbs);

/* ---------------------------------------------------------------- random-read probe */

/* Random-access ceiling of HBM, the roofline of a hash probe into a table far
 * larger than L2 (every probe is a random DRAM access; Section 6.2's join
 * probes such tables).  The paper has no counterpart: it is this library's
 * denominator for the join probe kernel.  Reads n_reads 16-byte values, one
 * from each of n_reads pseudo-random 32-byte-aligned buckets of a table of
 * table_bytes (allocated from the arena, zero-filled), eight independent reads
 * in flight per thread, and reports the best of three timed runs in 1e9 reads
 * per second.  VX_E_NOMEM if the table does not fit the arena; VX_E_INVAL for
 * table_bytes < 32 or n_reads == 0. */
vx_status vx_probe_hbm_random(vx_ctx *ctx, uint64_t table_bytes, uint64_t n_reads, double *g_reads_per_s);

/* ---------------------------------------------------------------- streaming probe */

/* What one kernel launch that reads `bytes` of HBM once can reach: the
 * ceiling of a chunk kernel at the same launch size (the fused chunk kernel of
 * Section 7.1 reads each staged chunk once).  The paper has no counterpart.
 * Each of reps + 1 rounds copies `bytes` (rounded down to a multiple of 16)
 * from a pinned host buffer into an arena buffer by copy engine, as the
 * executor stages a chunk, then times one coalesced read of them with CUDA
 * events on the context's compute stream; the first round warms up.  Reports
 * the median in GB/s (1e9 B/s).  VX_E_NOMEM if the bytes do not fit the arena;
 * VX_E_INVAL for bytes < 16, reps < 1 or a null output. */
vx_status vx_probe_stream(vx_ctx *ctx, uint64_t bytes, int32_t reps, double *gbs);

/* The same read with a host-to-device copy in flight: in each round a copy of
 * copy_bytes from pinned host memory into a second arena buffer is issued on
 * the context's host-to-device stream (a 4 MiB lead copy, then the rest), and
 * the read starts on the compute stream once the lead has landed, so it runs
 * while the rest streams in, as a chunk's kernel runs while the executor
 * copies the next chunk.  The paper has no counterpart: it is the in-pipeline
 * ceiling of the fused chunk kernel.  VX_E_NOMEM if bytes + copy_bytes do not
 * fit the arena; VX_E_INVAL for copy_bytes < 16 and as vx_probe_stream. */
vx_status vx_probe_stream_copying(vx_ctx *ctx, uint64_t bytes, int32_t reps, uint64_t copy_bytes, double *gbs);

#ifdef __cplusplus
}
#endif
#endif /* VX_H */
