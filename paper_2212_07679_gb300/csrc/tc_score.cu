// Tensor-core (tcgen05, BF16) band scoring.  Not built yet.
#include "tc_score.cuh"

namespace snn {

snn_status tc_score_launch(const snn_index *, const ScoreArgs &, cudaStream_t) {
    set_error("BF16 tensor-core scoring is not available in this build");
    return SNN_ENOTSUP;
}

}  // namespace snn
