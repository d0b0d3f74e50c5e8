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
    // 16-bit split operands of the tensor-core path (built on first use):
    // tc_part[p] is n x tc_k2 16-bit values, part p of the split of each
    // centred row (FP16 or BF16) plus the folded threshold columns (BF16).
    uint16_t *tc_part[3] = {nullptr, nullptr, nullptr};
    int tc_nsplit = 0;
    int tc_k2 = 0;                // row width of part 1 (columns)
    int tc_k2n = 0;               // row width of parts 2 and 3
    int tc_f16 = 0;               // the parts are FP16 (of x 2^tc_sigma), else BF16
    int tc_sigma = 0;
    // FP8 e4m3 operands (built on first use): f8_part[p] is n x f8_k8 bytes,
    // part p of each row scaled by its power of two; f8_fold is n x 16 bf16,
    // the folded threshold and error-bound columns.  Keyed by the split, the
    // products per k-step and the row width.
    uint8_t *f8_part[3] = {nullptr, nullptr, nullptr};
    uint16_t *f8_fold = nullptr;
    int f8_nsplit = 0;
    int f8_np = 0;
    int f8_k8 = 0;
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
