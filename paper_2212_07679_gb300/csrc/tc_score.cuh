// Tensor-core (tcgen05, BF16) band scoring for the query phase.
#pragma once
#include "common.cuh"
#include "query_kernels.cuh"

struct snn_index;

namespace snn {

// Scores every band item of `a` on the tensor cores and appends survivors
// exactly like the FP32 kernels do.  Builds the index's BF16 copy on first
// use (FP16 or BF16 parts).  Returns SNN_ENOTSUP where the tensor-core path
// is not available.
// Rx: largest true distance the FP64 test can accept; e_data: bound on the
// centring error norm of a data row.  Query operands live in `scr`.
// *mma_flops_per_pair receives the tensor-core flops executed per scored
// pair (2 x 16 x k-steps x MMAs per k-step); *split_used the operand split
// (SNN_SPLIT_* of snn.h).
snn_status tc_score_launch(const snn_index *ix, const ScoreArgs &a, cudaStream_t s, double Rx,
                           double e_data, Scratch &scr, int64_t *mma_flops_per_pair, int *split_used);

// FP8 e4m3 variant of tc_score_launch (per-row power-of-two scales, folded
// per-pair error bound).  Available where f8_eligible holds: the streamed
// high-dimensional shape (d + 9 > 64) with norms and radius below 2^20.
bool f8_eligible(const snn_index *ix, double Rx);
snn_status f8_score_launch(const snn_index *ix, const ScoreArgs &a, cudaStream_t s, double Rx,
                           double e_data, Scratch &scr, int64_t *mma_flops_per_pair,
                           int *split_used = nullptr);

// Tensor-core scoring inside a batched query plan.  A group holds the
// out-of-sample query sets of a plan that share one resident-query-tile
// shape (fold column 16: d <= 16, query tiles paired as in the single-index
// scorer; fold column 32 or 48: 16 < d <= 48).  The sets' two FP16 parts
// (each set scaled by its own power of two) are packed once, concatenated
// (set t's rows from its own offset); every run packs the group's queries
// into tiles that never straddle sets (padding rows can never survive), scores
// them in one launch appending to the plan's survivor list, and rewrites
// those survivors as (global query number, row of the set's index).
struct TcBatchGroup;
// sets: plan set numbers of the group, with their indices and descriptors
// (host copies; the query arrays of the descriptors are the plan's).
snn_status tc_batch_create(const snn_index *const *idx, const SetDesc *sd, const int *sets, int nsets,
                           int fold_col, cudaStream_t s, TcBatchGroup **out);
// One run: enqueued on s, no synchronisation.  tile_lo / tile_hi: the plan's
// bands (set-local rows); surv / cap / count: the plan's survivor list; err:
// bit 0 a bounded wait expired, bit 1 a query too large for the FP16 range.
snn_status tc_batch_enqueue(TcBatchGroup *g, const int64_t *tile_lo, const int64_t *tile_hi, uint2 *surv,
                            int64_t cap, unsigned long long *count, int *err, cudaStream_t s);
void tc_batch_release(TcBatchGroup *g, cudaStream_t s);
// The group's sets (plan set numbers) and its query tile rows (256 or 128).
const int *tc_batch_sets(const TcBatchGroup *g, int *nsets);

// Releases the index's packed tensor-core operands (stream-ordered on s) and
// empties its operand cache.  The caller holds the index's lock or owns the
// index exclusively (release, update).
void release_tc_operands(snn_index *ix, cudaStream_t s);

}  // namespace snn
