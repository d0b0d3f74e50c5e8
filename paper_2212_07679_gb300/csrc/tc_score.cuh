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

// Releases the index's packed tensor-core operands (stream-ordered on s) and
// empties its operand cache.  The caller holds the index's lock or owns the
// index exclusively (release, update).
void release_tc_operands(snn_index *ix, cudaStream_t s);

}  // namespace snn
