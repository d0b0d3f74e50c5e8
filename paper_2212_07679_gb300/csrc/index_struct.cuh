// Definition of the opaque index (Algorithm 1 output) shared by the host
// modules of libsnn.
#pragma once
#include <atomic>
#include <mutex>
#include "common.cuh"

// Pool blocks shared by the indices of one batched build: each index holds a
// reference; the blocks are released (stream-ordered) with the last index.
struct snn_shared_blocks {
    std::atomic<int> refs{0};
    void *blocks[16] = {};
    int nblocks = 0;
    cudaStream_t stream = nullptr;
};

// One packed operand set of the tensor-core scorers: part[p] holds part p of
// the split of every centred row (n x k2 16-bit values for part 1, n x k2n
// for parts 2 and 3; FP16 or BF16, or e4m3 bytes), fold the separate block
// of 16 folded BF16 columns per row where the kind has one.
struct snn_tc_operands {
    int kind = 0;                 // SNN_SPLIT_* code (e4m3: + products); 0: free slot
    int k2 = 0, k2n = 0;          // row widths (elements)
    int sigma = 0;                // two FP16 parts: the rows are scaled by 2^sigma
    void *part[3] = {nullptr, nullptr, nullptr};
    uint16_t *fold = nullptr;
    cudaEvent_t ready = nullptr;  // recorded on the packing stream after packing
};
constexpr int kMaxTcOperands = 8;

struct snn_index {
    int64_t n = 0;
    int d = 0, dp = 0;
    int device = 0;
    cudaStream_t stream = nullptr;   // build stream: the index's arrays are
                                     // released in order on it
    double *mu64 = nullptr;
    float *mu32 = nullptr;
    double *v64 = nullptr;
    float *v32 = nullptr;
    float *alpha = nullptr;
    int32_t *order = nullptr;
    float *praw = nullptr;
    float *xc = nullptr;
    float *hx = nullptr;
    float *nrm = nullptr;
    float *dconst = nullptr;      // device: [0] alpha error bound, [1] max norm
    // Packed operands of the tensor-core scorers, one entry per operand kind
    // (split, row widths, scale), built on first use and kept until the
    // index is released or updated; an entry is never replaced while the
    // index lives, so a scorer on any stream may read it once its stream has
    // waited for the entry's `ready` event.
    snn_tc_operands tc_ops[kMaxTcOperands];
    float alpha_err = 0.f;
    float nrm_max = 0.f;
    mutable double surv_hint = 0.0;   // survivors per query seen last time
    snn_shared_blocks *shared = nullptr;   // set: the arrays are slices of shared blocks
    mutable std::mutex mu;
};

namespace snn {
// Releases an index (its own arrays, or its reference to a batched build's
// shared blocks), stream-ordered.
void index_release(snn_index *ix);
}  // namespace snn
