// Cosine and angular radius search through the Euclidean reduction of
// Section 3: for unit vectors u, v the cosine distance 1 - u.v equals
// ||u - v||^2 / 2, and the angle between them is at most alpha exactly when
// ||u - v||^2 <= 2 - 2 cos(alpha).  Rows are normalised here; the search
// itself is the Euclidean one on the unit rows.
#include <cmath>

#include "common.cuh"

namespace snn {
namespace {

// One thread per row: s = sum over ascending k of x_k^2 in FP64, each
// operation rounded to nearest (explicit _rn intrinsics, so no fused
// multiply-add), r = 1 / sqrt(s) (both correctly rounded), u_k = fl32(x_k r);
// a row of zeros stays zero, a NaN or infinity gives NaN in its row.  The
// warp's 32 rows are read column by column, so the cached lines of a load
// serve the next columns; out may equal X (each element is read before it is
// written).
__global__ void k_normalize_rows(const float *X, int64_t n, int d, int64_t ld, float *out,
                                 int64_t ldo) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float *x = X + i * ld;
    double s = 0.0;
    for (int k = 0; k < d; ++k) {
        const double v = (double)x[k];
        s = __dadd_rn(s, __dmul_rn(v, v));
    }
    float *u = out + i * ldo;
    if (s == 0.0) {
        for (int k = 0; k < d; ++k) u[k] = 0.f;
        return;
    }
    const double r = __ddiv_rn(1.0, __dsqrt_rn(s));
    for (int k = 0; k < d; ++k) u[k] = __double2float_rn(__dmul_rn((double)x[k], r));
}

}  // namespace
}  // namespace snn

using namespace snn;

extern "C" {

snn_status snn_normalize_rows(const float *X, int64_t n, int32_t d, int64_t ld, float *out,
                              int64_t ldo, void *stream) {
    NvtxPhase nvtx_("snn normalize rows");
    clear_error();
    if (n < 0 || d < 1 || ld < d || ldo < d || (n > 0 && (!X || !out))) {
        set_error("invalid arguments (n >= 0, d >= 1, ld and ldo >= d, non-NULL arrays)");
        return SNN_EINVAL;
    }
    if (n == 0) return SNN_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    SNN_LAUNCH(k_normalize_rows, unsigned(cdiv(n, int64_t(128))), 128, 0, s)(X, n, d, ld, out, ldo);
    SNN_LAUNCH_CHECK();
    return SNN_OK;
}

double snn_radius_for_cosine_distance(double c) {
    if (!(c >= 0.0 && c <= 2.0)) return NAN;
    return std::sqrt(2.0 * c);
}

double snn_radius_for_cosine_similarity(double t) {
    if (!(t >= -1.0 && t <= 1.0)) return NAN;
    return std::sqrt(2.0 - 2.0 * t);
}

}  // extern "C"
