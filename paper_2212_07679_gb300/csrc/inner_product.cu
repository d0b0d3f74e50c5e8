// Inner-product threshold search (Section 3's maximum-inner-product
// variant).  Section 3 maps p.q to a Euclidean distance with augmented rows
// p~ = [sqrt(xi^2 - ||p||^2), p], q~ = [0, q], xi = max ||p||:
// ||p~ - q~||^2 = xi^2 + ||q||^2 - 2 p.q.  The Euclidean search on the
// augmented rows, with a radius for the largest query norm and a slack for
// the rounding of the augmented coordinate, returns every pair with
// p.q >= tau (and more); the exact decision here keeps those whose FP64 dot
// product (ascending k, no FMA) reaches tau.
#include "inner_product.cuh"

namespace snn {

__global__ void k_row_sq64(const float *__restrict__ X, int64_t n, int d, int64_t ld,
                           double *__restrict__ sq, double *__restrict__ sq_max, int *__restrict__ bad) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    double s = 0.0;
    if (i < n) {
        const float *x = X + i * ld;
        for (int k = 0; k < d; ++k) {
            const double v = (double)x[k];
            s = __dadd_rn(s, __dmul_rn(v, v));
        }
        sq[i] = s;
        if (!isfinite(s)) atomicOr(bad, 1);
    }
    // block maximum of non-negative doubles through their bit patterns
    unsigned long long b = i < n && isfinite(s) ? (unsigned long long)__double_as_longlong(s) : 0ull;
    for (int o = 16; o; o >>= 1) b = max(b, (unsigned long long)__shfl_xor_sync(0xffffffffu, b, o));
    if ((threadIdx.x & 31) == 0) atomicMax(reinterpret_cast<unsigned long long *>(sq_max), b);
}

__global__ void k_augment(const float *__restrict__ X, int64_t n, int d, int64_t ld,
                          const double *__restrict__ sq, const double *__restrict__ xi2, int query,
                          float *__restrict__ out) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float *x = X + i * ld;
    float *o = out + i * int64_t(d + 1);
    // points: sqrt(xi^2 - ||p||^2) (FP64, rounded once to FP32); queries: 0
    o[0] = query ? 0.f : __double2float_rn(sqrt(fmax(0.0, *xi2 - sq[i])));
    for (int k = 0; k < d; ++k) o[k + 1] = x[k];
}

__global__ void k_radii_minmax(const double *__restrict__ R, int64_t m, double *__restrict__ mm,
                               int *__restrict__ bad) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    // min and max of non-negative doubles through their bit patterns
    unsigned long long lo = ~0ull, hi = 0ull;
    if (i < m) {
        const double r = R[i];
        if (!(r >= 0.0) || !isfinite(r)) {
            atomicOr(bad, 1);
        } else {
            lo = hi = (unsigned long long)__double_as_longlong(r);
        }
    }
    for (int o = 16; o; o >>= 1) {
        lo = min(lo, (unsigned long long)__shfl_xor_sync(0xffffffffu, lo, o));
        hi = max(hi, (unsigned long long)__shfl_xor_sync(0xffffffffu, hi, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMin(reinterpret_cast<unsigned long long *>(mm), lo);
        atomicMax(reinterpret_cast<unsigned long long *>(mm + 1), hi);
    }
}

__global__ void k_ip_radii(const double *__restrict__ sqQ, int64_t m, const double *__restrict__ xi2,
                           double tau, double *__restrict__ R) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= m) return;
    // ||p~ - q~||^2 = xi^2 + ||q||^2 - 2 p.q up to the rounding of the
    // augmented coordinate and of the FP64 norms, all far below 2^-20 of
    // xi^2 + ||q||^2
    const double a = *xi2 + sqQ[i];
    const double r2 = (a - 2.0 * tau) + 0x1p-20 * a;
    R[i] = r2 > 0.0 ? sqrt(r2) * (1.0 + 0x1p-40) : 0.0;
}

__global__ void k_csr_rows(const int64_t *__restrict__ offsets, int64_t m, int64_t nnz,
                           int64_t *__restrict__ rows) {
    const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e >= nnz) return;
    // the row r with offsets[r] <= e < offsets[r + 1]
    int64_t lo = 0, hi = m;
    while (hi - lo > 1) {
        const int64_t mid = (lo + hi) >> 1;
        if (offsets[mid] <= e) lo = mid;
        else hi = mid;
    }
    rows[e] = lo;
}

namespace {
__device__ __forceinline__ void two_sum32(float a, float b, float &s, float &t) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    t = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
}  // namespace

// One group of G lanes per candidate (query row, point).  Each lane keeps an
// unevaluated sum H + L of its exact products p_k q_k = ph + pl (two_sum for
// H, plain FP32 sums for L) and an upward-rounded sum A of |ph|; the groups
// combine their lanes the same way.  With B bounding both |H + L - exact| and
// |FP64 sequential - exact| (2^-47 (d+G+3)^2 A + 1.01 (d+2) 2^-53 A + 2^-52 A
// + underflow), the pair is kept when H + L - B >= tau, dropped when
// H + L + B < tau, and its value is fl32 of the bracket when both ends round
// alike; otherwise the FP64 definition decides.
template <int G>
__device__ __forceinline__ void ip_decide_body(const int64_t *__restrict__ rows,
                                                   const int32_t *__restrict__ ids, int64_t nnz,
                                                   const float *__restrict__ P, int64_t ldp,
                                                   const float *__restrict__ Q, int64_t ldq, int d,
                                                   double tau, int64_t *__restrict__ keep,
                                                   float *__restrict__ vals,
                                                   unsigned long long *__restrict__ n_fp64) {
    const int lane = int(threadIdx.x % G);
    const int64_t g0 = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) / G;
    const int64_t gstride = (int64_t(gridDim.x) * blockDim.x) / G;
    const int64_t base_end = (nnz + (32 / G) - 1) / (32 / G) * (32 / G);   // whole warps iterate alike
    for (int64_t e = g0; e < base_end; e += gstride) {
        const bool valid = e < nnz;
        const float *p = P + (valid ? int64_t(ids[e]) * ldp : 0);
        const float *q = Q + (valid ? rows[e] * ldq : 0);
        float H = 0.f, L = 0.f, A = 0.f;
        if (valid)
            for (int k = lane; k < d; k += G) {
                const float a = p[k], b = q[k];
                const float ph = __fmul_rn(a, b);
                const float pl = __fmaf_rn(a, b, -ph);
                float s, t;
                two_sum32(H, ph, s, t);
                H = s;
                L = __fadd_rn(__fadd_rn(L, t), pl);
                A = __fadd_ru(A, fabsf(ph));
            }
        if (G > 1) {
#pragma unroll
            for (int o = G / 2; o; o >>= 1) {
                const float H2 = __shfl_down_sync(0xffffffffu, H, o, G);
                const float L2 = __shfl_down_sync(0xffffffffu, L, o, G);
                const float A2 = __shfl_down_sync(0xffffffffu, A, o, G);
                float s, t;
                two_sum32(H, H2, s, t);
                H = s;
                L = __fadd_rn(__fadd_rn(L, t), L2);
                A = __fadd_ru(A, A2);
            }
        }
        if (!valid || lane != 0) continue;
        bool accept = false, decided = false;
        float value = 0.f;
        if (isfinite(H) && isfinite(L) && isfinite(A)) {
            const double Dd = (double)H + (double)L;
            const double Ad = (double)A * (1.0 + 0x1p-22);
            const double dg = double(d + G + 3);
            const double B = (0x1p-47 * dg * dg + 1.01 * (d + 2) * 0x1p-53 + 0x1p-52) * Ad +
                             2.0 * d * 0x1p-149 + 1e-300;
            const double lo = __dsub_rd(Dd, B), hi = __dadd_ru(Dd, B);
            if (hi < tau) {
                decided = true;
            } else if (lo >= tau) {
                const float flo = __double2float_rn(lo), fhi = __double2float_rn(hi);
                if (flo == fhi) {
                    accept = decided = true;
                    value = flo;
                }
            }
        }
        if (!decided) {
            double s = 0.0;
            for (int k = 0; k < d; ++k) s = __dadd_rn(s, __dmul_rn((double)p[k], (double)q[k]));
            accept = s >= tau;
            value = __double2float_rn(s);
            atomicAdd(n_fp64, 1ull);
        }
        keep[e] = accept ? 1 : 0;
        vals[e] = value;
    }
}

#define SNN_IP_ARGS                                                                           \
    const int64_t *__restrict__ rows, const int32_t *__restrict__ ids, int64_t nnz,              \
        const float *__restrict__ P, int64_t ldp, const float *__restrict__ Q, int64_t ldq, int d, \
        double tau, int64_t *__restrict__ keep, float *__restrict__ vals,                        \
        unsigned long long *__restrict__ n_fp64
#define SNN_IP_PASS rows, ids, nnz, P, ldp, Q, ldq, d, tau, keep, vals, n_fp64
__global__ void __launch_bounds__(256) k_ip_decide_g1(SNN_IP_ARGS) { ip_decide_body<1>(SNN_IP_PASS); }
__global__ void __launch_bounds__(256) k_ip_decide_g8(SNN_IP_ARGS) { ip_decide_body<8>(SNN_IP_PASS); }
__global__ void __launch_bounds__(256) k_ip_decide_g32(SNN_IP_ARGS) { ip_decide_body<32>(SNN_IP_PASS); }
#undef SNN_IP_PASS
#undef SNN_IP_ARGS

__global__ void k_ip_offsets(const int64_t *__restrict__ offsets, int64_t m,
                             const int64_t *__restrict__ pos, int64_t *__restrict__ out_offsets) {
    const int64_t r = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (r > m) return;
    out_offsets[r] = pos[offsets[r]];   // pos[nnz] is the total
}

__global__ void k_ip_compact(const int32_t *__restrict__ ids, const float *__restrict__ vals,
                             const int64_t *__restrict__ keep, const int64_t *__restrict__ pos, int64_t nnz,
                             int32_t *__restrict__ out_ids, float *__restrict__ out_vals) {
    const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e >= nnz || !keep[e]) return;
    out_ids[pos[e]] = ids[e];
    out_vals[pos[e]] = vals[e];
}

}  // namespace snn
