// Shared declarations of the sort, partition and learned-partitioner code.
#pragma once
#include <cstdint>

#include "vx_internal.h"
#include "vx_radix.cuh"

namespace vx {

constexpr uint32_t kPLSegments = 1024;  // piecewise-linear CDF model segments
constexpr int kMlpHidden = 32;          // width of the monotone CDF MLP
constexpr int kMlpParams = 3 * kMlpHidden + 1;

uint64_t radix_temp_bytes(uint64_t cap);
RadixState *radix_state_of(char *temp);
// spin_limit: polls of one predecessor's look-back word before the pass gives
// up and sets the error word (0 = the default of 2^20)
vx_status radix_sort_enqueue(RadixBufs b, uint64_t n, char *temp, cudaStream_t s, int num_sms, int npass = 8,
                             uint32_t spin_limit = 0);
// after radix_sort_enqueue on s: publishes to a mapped host word the buffer
// holding the result (low byte), the executed passes (next byte) and whether
// a look-back wait gave up (bit 16)
vx_status radix_publish_enqueue(char *temp, uint64_t *host_word, cudaStream_t s, int npass = 8);
vx_status range_partition_enqueue(RadixBufs b, uint64_t n, const uint64_t *spl, uint32_t P, char *temp,
                                  cudaStream_t s);
constexpr uint32_t kMaxRequestedPartitions = 128;  // isolation may add up to P-1 boundaries
constexpr int kMaxSortSlots = 6;                   // staging slots of the partition sort pass, at most
// pairs per partition-pass chunk (a multiple of the radix tile).  A
// partition's pairs sit in one extent per chunk of the intermediate buffer,
// and the sort pass loads them extent by extent: larger chunks make fewer,
// larger copies (combined H2D + D2H throughput falls from 340 GB/s at 64 MB
// copies to 255 GB/s at 2-4 MB).  On 1e9 Zipf pairs the sort phase took
// 97.5 / 95.0 / 94.1 ms with 32M / 48M / 64M and the partition phase 74 ms
// with each.
constexpr uint64_t kPipelineRows = 48ull << 20;
constexpr uint64_t kSplitterBufBytes = 8ull * (512 + kPLSegments + 1 + 8);

// out-of-core sort (partition plan) of n contiguous host pairs; dev_keys is
// the device-visible address of keys
vx_status sort_contiguous(vx_ctx *ctx, const uint64_t *keys, const uint32_t *vals, const uint64_t *dev_keys, uint64_t n,
                          uint64_t *out_keys, uint32_t *out_vals, const vx_sort_opts &o, vx_sort_stats &ss, int depth);
// equi-join of the build columns with probe rows [probe_begin, probe_end)
vx_status join_columns(vx_ctx *ctx, const Column *bk, const Column *bp, const Column *pk, uint64_t probe_begin,
                       uint64_t probe_end, const vx_join_opts *opts, vx_join_result *out);
// the radix-partitioned join of vx_join (VX_JOIN_RADIX)
vx_status radix_join(vx_ctx *ctx, const Column *bk, const Column *bp, const Column *pk, const vx_join_opts &o,
                     vx_join_result *out);

// the merge plan of vx_sort (sorted runs, exact cuts, merged partitions)
vx_status merge_sort_plan(vx_ctx *ctx, const uint64_t *keys, const uint32_t *vals, const uint64_t *dev_keys,
                          uint64_t n, uint64_t *out_keys, uint32_t *out_vals, const vx_sort_opts &o,
                          vx_sort_stats &ss);

vx_status sample_and_sort(vx_ctx *ctx, const uint64_t *dev_keys, uint64_t n, uint64_t &m, uint64_t seed,
                          DevBuf &sorted_out, uint64_t **sorted_ptr);
// splitters for P requested partitions from a sorted device sample with
// partitioner `kind`, then heavy-key isolation; *n_spl receives their count
vx_status splitters_from_sample(vx_ctx *ctx, int32_t kind, const uint64_t *sorted, uint64_t m, uint32_t P,
                                uint64_t *spl_buf, uint32_t mlp_steps, double *ms_train, uint32_t *n_spl);
// trains the monotone CDF MLP on the sorted sample and writes P-1 splitters
vx_status mlp_splitters(vx_ctx *ctx, const uint64_t *sorted, uint64_t m, uint32_t P, uint32_t steps, uint64_t *d_spl,
                        double *ms_train);

}  // namespace vx
