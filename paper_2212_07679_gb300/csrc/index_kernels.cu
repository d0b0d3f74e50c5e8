// Index phase kernels (Algorithm 1, Section 3.1):
//   column means mu (float-float per thread, FP64 across threads, NaN/Inf
//   check) and the FP32 centre c = fl32(mu),
//   centred Gram matrix C = (X - c)^T (X - c) for the first principal
//   direction (Eq. (1): v1 is the dominant right singular vector of X, i.e.
//   the dominant eigenvector of C) on CUDA cores for d <= 64 (larger d: the
//   tensor-core kernels of gram_tc.cu),
//   v1 for d <= 64 by repeated squaring of C / trace(C) in one CTA followed by
//   FP64 power steps and FP64 normalisation,
//   scores alpha_i = x_i^T v1 with a per-point rounding bound,
//   gather of the sorted copies and halved squared norms xbar_i = x_i^T x_i/2.
#include "index_kernels.cuh"

namespace snn {

// ------------------------------------------------------------ mean (K1)
// Block (rb, cb) sums rows [rb*rows, (rb+1)*rows) of columns
// [cb*TX, cb*TX + TX) into part[rb][c] (deterministic fixed order).  Each
// thread keeps a float-float (hi, lo) sum of its rows: TwoSum of hi and the
// element, the error added to lo, then a FastTwoSum renormalisation, so the
// per-thread sum is accurate to a few units of 2^-48 of the sum of |x|; the
// threads' sums are then combined in FP64.  Thread (cx, ry) owns column cx
// and rows ry, ry+TY, ...
__global__ void k_colsum_partial(const float *__restrict__ X, int64_t n, int d, int64_t ld,
                                 int64_t rows, double *__restrict__ part, int *__restrict__ bad) {
    extern __shared__ double sh[];   // [TY][TX]
    const int TX = d < 32 ? d : 32;
    const int TY = blockDim.x / TX;
    const int t = threadIdx.x;
    const int cx = t % TX, ry = t / TX;
    const int c = blockIdx.y * TX + cx;
    const int64_t r0 = int64_t(blockIdx.x) * rows;
    const int64_t r1 = min(n, r0 + rows);
    int badl = 0;
    float hi = 0.f, lo = 0.f;
    if (ry < TY && c < d) {
        for (int64_t r = r0 + ry; r < r1; r += TY) {
            const float x = X[r * ld + c];
            badl |= !isfinite(x);
            const float s = hi + x;                       // TwoSum(hi, x)
            const float bb = s - hi;
            const float e = (hi - (s - bb)) + (x - bb);
            const float l = lo + e;
            hi = s + l;                                   // FastTwoSum(s, l)
            lo = l - (hi - s);
        }
    }
    if (ry < TY) sh[ry * TX + cx] = (double)hi + (double)lo;
    __syncthreads();
    if (t < TX && blockIdx.y * TX + t < d) {
        double acc = 0.0;
        for (int y = 0; y < TY; ++y) acc += sh[y * TX + t];
        part[int64_t(blockIdx.x) * d + blockIdx.y * TX + t] = acc;
    }
    if (badl) atomicOr(bad, 1);
}

// mu = column means (FP64); the index centres every point with the FP32
// vector c = fl32(mu) (any fixed centre leaves distances unchanged,
// Section 3.1), so centring is one exact-input FP32 subtraction per value.
// One warp per column: lane-strided partial sums and a shuffle tree (short
// FP64 dependency chains; fixed order, deterministic).
__global__ void k_mean_final(const double *__restrict__ part, int nb, int d, int64_t n,
                             double *__restrict__ mu64, float *__restrict__ mu32) {
    const int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (c >= d) return;
    double s = 0.0;
    for (int b = lane; b < nb; b += 32) s += part[int64_t(b) * d + c];
    for (int o = 16; o; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) {
        const double m = s / (double)n;
        mu64[c] = m;
        mu32[c] = (float)m;
    }
}

// ------------------------------------------------------------ Gram (K2)
// Small d (d <= TG <= 64): the whole d x d matrix is one TG x TG tile.
// (TG/4)^2 threads each own a 4 x 4 block of C; the block's 256 threads form
// 256 / (TG/4)^2 row groups that take interleaved rows of a staged chunk of
// centred rows x = fl32(p - c).  Row groups are summed in shared memory and
// the block writes its partial C (FP32 sums over its rows) to part[b].
constexpr int kGramStageRows = 64;

template <int TG>
__device__ __forceinline__ void gram_small_rows(const float *__restrict__ X, int d, int64_t ld,
                                                const float *__restrict__ cvec, int64_t r0,
                                                int64_t r1, float *__restrict__ out);

template <int TG>
__device__ __forceinline__ void gram_small(const float *__restrict__ X, int64_t n, int d,
                                           int64_t ld, const float *__restrict__ cvec,
                                           int64_t rows, float *__restrict__ part) {
    const int64_t r0 = int64_t(blockIdx.x) * rows;
    gram_small_rows<TG>(X, d, ld, cvec, r0, min(n, r0 + rows), part + int64_t(blockIdx.x) * d * d);
}

// Rows [r0, r1) of X (centred by cvec) into out = their d x d Gram matrix.
template <int TG>
__device__ __forceinline__ void gram_small_rows(const float *__restrict__ X, int d, int64_t ld,
                                                const float *__restrict__ cvec, int64_t r0,
                                                int64_t r1, float *__restrict__ out) {
    constexpr int TT = TG / 4;                  // threads per tile edge
    constexpr int RG = 256 / (TT * TT);         // row groups
    constexpr int LD = TG + 4;
    __shared__ float S[kGramStageRows][LD];
    __shared__ float red[RG > 1 ? RG : 1][RG > 1 ? TG : 1][RG > 1 ? TG + 1 : 1];
    const int tt = threadIdx.x % (TT * TT), g = threadIdx.x / (TT * TT);
    const int ty = tt / TT, tx = tt % TT;
    float acc[4][4] = {};
    for (int64_t rb = r0; rb < r1; rb += kGramStageRows) {
        const int nr = int(min(int64_t(kGramStageRows), r1 - rb));
        for (int e = threadIdx.x; e < kGramStageRows * TG; e += 256) {
            const int rr = e / TG, cc = e % TG;
            float x = 0.f;
            if (rr < nr && cc < d) x = X[(rb + rr) * ld + cc] - cvec[cc];
            S[rr][cc] = x;
        }
        __syncthreads();
        for (int rr = g; rr < nr; rr += RG) {
            float a[4], b[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                a[u] = S[rr][ty * 4 + u];
                b[u] = S[rr][tx * 4 + u];
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int w = 0; w < 4; ++w) acc[u][w] = fmaf(a[u], b[w], acc[u][w]);
        }
        __syncthreads();
    }
    if constexpr (RG > 1) {
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int w = 0; w < 4; ++w) red[g][ty * 4 + u][tx * 4 + w] = acc[u][w];
        __syncthreads();
        for (int e = threadIdx.x; e < d * d; e += 256) {
            const int i = e / d, j = e % d;
            float v = 0.f;
            for (int q = 0; q < RG; ++q) v += red[q][i][j];
            out[e] = v;
        }
    } else {
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int w = 0; w < 4; ++w) {
                const int i = ty * 4 + u, j = tx * 4 + w;
                if (i < d && j < d) out[int64_t(i) * d + j] = acc[u][w];
            }
    }
}

__global__ void __launch_bounds__(256)
k_gram_small16(const float *X, int64_t n, int d, int64_t ld, const float *cvec, int64_t rows,
               float *part) {
    gram_small<16>(X, n, d, ld, cvec, rows, part);
}
__global__ void __launch_bounds__(256)
k_gram_small32(const float *X, int64_t n, int d, int64_t ld, const float *cvec, int64_t rows,
               float *part) {
    gram_small<32>(X, n, d, ld, cvec, rows, part);
}
__global__ void __launch_bounds__(256)
k_gram_small64(const float *X, int64_t n, int d, int64_t ld, const float *cvec, int64_t rows,
               float *part) {
    gram_small<64>(X, n, d, ld, cvec, rows, part);
}

// C64[i][j] = sum over chunks (FP64), upper triangle mirrored.  One warp per
// entry (lane-strided partial sums, shuffle tree: short FP64 chains).
__global__ void k_gram_reduce(const float *__restrict__ part, int nchunk, int d,
                              double *__restrict__ C) {
    const int64_t e = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (e >= int64_t(d) * d) return;
    const int i = int(e / d), j = int(e % d);
    const int a = min(i, j), b = max(i, j);
    double s = 0.0;
    for (int c = lane; c < nchunk; c += 32) s += (double)part[int64_t(c) * d * d + int64_t(a) * d + b];
    for (int o = 16; o; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) C[e] = s;
}

// ------------------------------------------------- first direction (K3)
// Small d: one CTA.  M = C / trace(C) in FP32 shared memory, squared
// kSquarings times (M <- M*M / trace), so M tends to v1 v1^T; the column with
// the largest diagonal entry seeds power steps v <- C v / ||C v||.
constexpr int kSquarings = 12;
constexpr int kPowerSteps = 4;

__device__ double block_sum_d(double v, double *red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    for (int o = 16; o; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double s = 0.0;
    for (int w = 0; w < nw; ++w) s += red[w];   // fixed order in every thread
    __syncthreads();
    return s;
}

__device__ float block_sum_f(float v, float *red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    for (int o = 16; o; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    float s = 0.f;
    for (int w = 0; w < nw; ++w) s += red[w];
    __syncthreads();
    return s;
}

__device__ __forceinline__ void pc_small_body(const double *__restrict__ C, int d,
                                              double *__restrict__ v64, float *__restrict__ v32);

__global__ void __launch_bounds__(1024)
k_pc_small(const double *__restrict__ C, int d, double *__restrict__ v64, float *__restrict__ v32) {
    pc_small_body(C, d, v64, v32);
}

__device__ __forceinline__ void pc_small_body(const double *__restrict__ C, int d,
                                              double *__restrict__ v64, float *__restrict__ v32) {
    // FP64 is slow on this part: everything but the final normalisation runs
    // in FP32 (v1's accuracy only affects pruning; the FP64 normalisation
    // makes ||v64|| = 1 to FP64 precision, which the score bounds assume)
    extern __shared__ unsigned char smem[];
    double *vd = reinterpret_cast<double *>(smem);         // d
    double *red = vd + d;                                  // 32
    float *redf = reinterpret_cast<float *>(red + 32);     // 32
    float *v = redf + 32;                                  // d
    float *w = v + d;                                      // d
    float *M = w + d;                                      // d*d
    float *T = M + d * d;                                  // d*d (later: C in FP32)
    const int t = threadIdx.x, nt = blockDim.x;
    const int warp = t >> 5, lane = t & 31, nw = nt >> 5;
    const int dd = d * d;

    if (warp == 0) {
        double tr = 0.0;
        for (int i = lane; i < d; i += 32) tr += C[int64_t(i) * d + i];
        for (int o = 16; o; o >>= 1) tr += __shfl_xor_sync(0xffffffffu, tr, o);
        if (lane == 0) red[0] = tr;
    }
    __syncthreads();
    const double tr = red[0];
    const bool degenerate = !(tr > 0.0) || !isfinite(tr);
    if (!degenerate) {
        const float inv_tr = (float)(1.0 / tr);
        for (int e = t; e < dd; e += nt) M[e] = (float)C[e] * inv_tr;
        __syncthreads();
        for (int it = 0; it < kSquarings; ++it) {
            for (int e = t; e < dd; e += nt) {
                const int i = e / d, j = e % d;
                float acc = 0.f;
                for (int k = 0; k < d; ++k) acc = fmaf(M[i * d + k], M[k * d + j], acc);
                T[e] = acc;
            }
            __syncthreads();
            float part = 0.f;
            for (int i = t; i < d; i += nt) part += T[i * d + i];
            const float trT = block_sum_f(part, redf);
            if (!(trT > 0.f) || !isfinite(trT)) break;
            const float inv = 1.f / trT;
            for (int e = t; e < dd; e += nt) M[e] = T[e] * inv;
            __syncthreads();
        }
        // column with the largest diagonal entry
        int jbest = 0;
        float best = -1.f;
        for (int j = 0; j < d; ++j) {
            const float x = M[j * d + j];
            if (x > best) { best = x; jbest = j; }
        }
        for (int i = t; i < d; i += nt) v[i] = M[i * d + jbest];
        // FP32 copy of C for the power steps
        for (int e = t; e < dd; e += nt) T[e] = (float)C[e];
        __syncthreads();
        // power steps v <- C v / ||C v|| (FP32, one warp per row)
        for (int it = 0; it < kPowerSteps; ++it) {
            for (int i = warp; i < d; i += nw) {
                float s = 0.f;
                for (int k = lane; k < d; k += 32) s = fmaf(T[i * d + k], v[k], s);
                for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
                if (lane == 0) w[i] = s;
            }
            __syncthreads();
            float part = 0.f;
            for (int i = t; i < d; i += nt) part += w[i] * w[i];
            const float n2 = block_sum_f(part, redf);
            if (!(n2 > 0.f) || !isfinite(n2)) break;
            const float inv = 1.f / sqrtf(n2);
            for (int i = t; i < d; i += nt) v[i] = w[i] * inv;
            __syncthreads();
        }
    } else {
        for (int i = t; i < d; i += nt) v[i] = (i == 0) ? 1.f : 0.f;
        __syncthreads();
    }
    // FP64 normalisation (one warp)
    if (warp == 0) {
        double n2 = 0.0;
        for (int i = lane; i < d; i += 32) n2 += (double)v[i] * (double)v[i];
        for (int o = 16; o; o >>= 1) n2 += __shfl_xor_sync(0xffffffffu, n2, o);
        const bool ok = n2 > 0.0 && isfinite(n2);
        const double inv = ok ? 1.0 / sqrt(n2) : 1.0;
        for (int i = lane; i < d; i += 32) {
            const double x = ok ? (double)v[i] * inv : (i == 0 ? 1.0 : 0.0);
            vd[i] = x;
        }
        __syncwarp();
        for (int i = lane; i < d; i += 32) {
            v64[i] = vd[i];
            v32[i] = (float)vd[i];
        }
    }
}

// w = C v (FP64), one warp per row.
__global__ void k_matvec64(const double *__restrict__ C, int d, const double *__restrict__ v,
                           double *__restrict__ w) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= d) return;
    double s = 0.0;
    for (int k = lane; k < d; k += 32) s += C[int64_t(warp) * d + k] * v[k];
    for (int o = 16; o; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) w[warp] = s;
}

// v = w / ||w|| (FP64); keeps v when w vanished.  final != 0 also writes v32.
__global__ void k_normalise64(const double *__restrict__ w, int d, double *__restrict__ v,
                              float *__restrict__ v32, int final_) {
    __shared__ double red[32];
    double part = 0.0;
    for (int i = threadIdx.x; i < d; i += blockDim.x) part += w[i] * w[i];
    const double nrm2 = block_sum_d(part, red);
    const bool ok = nrm2 > 0.0 && isfinite(nrm2);
    const double inv = ok ? 1.0 / sqrt(nrm2) : 1.0;
    for (int i = threadIdx.x; i < d; i += blockDim.x) {
        double x = ok ? w[i] * inv : v[i];
        v[i] = x;
        if (final_) v32[i] = (float)x;
    }
}

// ------------------------------------------------------ projection (K4)
// alpha_i = fl32(sum_k x_k v_k) with x_k = fl32(p_ik - c_k) (c = fl32(mu)) and
// FP32 FMA accumulation.  |alpha_hat - alpha| <= (d+4) u32 sum_k |x_k||v_k|
// (1.01): centring u32 |x_k|, v rounding u32 |v_k|, accumulation gamma_d,
// where alpha is the exact (p_i - c) . v1.
// Writes the sort key of alpha and the point id; *eps_max gets the largest
// bound.  One thread per point (d <= 32) or one warp per point.
__global__ void k_project(const float *__restrict__ X, int64_t n, int d, int64_t ld,
                          const float *__restrict__ cvec, const float *__restrict__ v32,
                          uint32_t *__restrict__ keys, uint32_t *__restrict__ vals,
                          float *__restrict__ eps_max, int *__restrict__ bad, int vec) {
    const bool warp_mode = d > 32;
    const int64_t gt = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    const int64_t i = warp_mode ? gt >> 5 : gt;
    const int lane = warp_mode ? int(threadIdx.x & 31) : 0;
    const int step = warp_mode ? 32 : 1;
    const bool live = i < n;   // whole warps leave together in warp mode
    if (warp_mode && !live) return;
    float a = 0.f, b = 0.f;
    int badl = 0;
    if (live) {
        if (vec) {
            // rows of d = 4k floats at 16-byte aligned addresses
            const float4 *row = reinterpret_cast<const float4 *>(X + i * ld);
            const float4 *c4 = reinterpret_cast<const float4 *>(cvec);
            const float4 *w4 = reinterpret_cast<const float4 *>(v32);
            for (int k = lane; k < d / 4; k += step) {
                const float4 p = row[k], c = c4[k], w = w4[k];
                badl |= !isfinite(p.x) | !isfinite(p.y) | !isfinite(p.z) | !isfinite(p.w);
                const float x0 = p.x - c.x, x1 = p.y - c.y, x2 = p.z - c.z, x3 = p.w - c.w;
                a = fmaf(x0, w.x, a);
                a = fmaf(x1, w.y, a);
                a = fmaf(x2, w.z, a);
                a = fmaf(x3, w.w, a);
                b = fmaf(fabsf(x0), fabsf(w.x), b);
                b = fmaf(fabsf(x1), fabsf(w.y), b);
                b = fmaf(fabsf(x2), fabsf(w.z), b);
                b = fmaf(fabsf(x3), fabsf(w.w), b);
            }
        } else {
            for (int k = lane; k < d; k += step) {
                const float p = X[i * ld + k];
                badl |= !isfinite(p);
                const float x = p - cvec[k];
                a = fmaf(x, v32[k], a);
                b = fmaf(fabsf(x), fabsf(v32[k]), b);
            }
        }
    }
    if (warp_mode) {
        for (int o = 16; o; o >>= 1) {
            a += __shfl_down_sync(0xffffffffu, a, o);
            b += __shfl_down_sync(0xffffffffu, b, o);
            badl |= __shfl_down_sync(0xffffffffu, badl, o);
        }
    }
    float eps = 0.f;
    if (live && lane == 0) {
        eps = (float)(d + 4) * kU32 * 1.01f * b + 1e-37f;
        keys[i] = float_to_key(a);
        vals[i] = (uint32_t)i;
    }
    if (!warp_mode) {
        // one atomic per warp for the largest bound and the NaN flag
        for (int o = 16; o; o >>= 1) {
            eps = fmaxf(eps, __shfl_xor_sync(0xffffffffu, eps, o));
            badl |= __shfl_xor_sync(0xffffffffu, badl, o);
        }
        if ((threadIdx.x & 31) == 0) {
            atomic_max_nonneg(eps_max, eps);
            if (badl) atomicOr(bad, 1);
        }
    } else if (lane == 0) {
        atomic_max_nonneg(eps_max, eps);
        if (badl) atomicOr(bad, 1);
    }
}

// ---------------------------------------------------------- gather (K6)
// Sorted position r takes point order[r]: raw row (zero-padded to dp),
// centred FP32 row x = fl32(p - c), score, halved squared norm xbar = fl32(sum x_k^2)/2 and an
// upper bound on ||x||.  Padding entries are zero in both copies.
__global__ void k_gather(const uint32_t *__restrict__ skeys, const uint32_t *__restrict__ order,
                         const float *__restrict__ X, int64_t n, int d, int64_t ld, int dp,
                         const float *__restrict__ cvec, float *__restrict__ alpha,
                         int32_t *__restrict__ order_out, float *__restrict__ praw,
                         float *__restrict__ xc, float *__restrict__ hx,
                         float *__restrict__ nrm, int vec) {
    const bool warp_mode = d > 32;
    const int64_t gt = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    const int64_t r = warp_mode ? gt >> 5 : gt;
    const int lane = warp_mode ? int(threadIdx.x & 31) : 0;
    const int step = warp_mode ? 32 : 1;
    if (r >= n) return;
    const int64_t i = order[r];
    float s = 0.f;
    if (vec) {
        // d = dp = 4k, 16-byte aligned rows
        const float4 *src = reinterpret_cast<const float4 *>(X + i * ld);
        const float4 *c4 = reinterpret_cast<const float4 *>(cvec);
        float4 *pr = reinterpret_cast<float4 *>(praw + r * dp);
        float4 *pc = reinterpret_cast<float4 *>(xc + r * dp);
        for (int k = lane; k < dp / 4; k += step) {
            const float4 p = src[k], c = c4[k];
            const float4 x = make_float4(p.x - c.x, p.y - c.y, p.z - c.z, p.w - c.w);
            pr[k] = p;
            pc[k] = x;
            s = fmaf(x.x, x.x, s);
            s = fmaf(x.y, x.y, s);
            s = fmaf(x.z, x.z, s);
            s = fmaf(x.w, x.w, s);
        }
    } else {
        for (int k = lane; k < dp; k += step) {
            float p = 0.f, x = 0.f;
            if (k < d) {
                p = X[i * ld + k];
                x = p - cvec[k];
            }
            praw[r * dp + k] = p;
            xc[r * dp + k] = x;
            s = fmaf(x, x, s);
        }
    }
    if (warp_mode)
        for (int o = 16; o; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) {
        alpha[r] = key_to_float(skeys[r]);
        order_out[r] = (int32_t)i;
        hx[r] = 0.5f * s;
        // ||x|| <= sqrt(s (1 + gamma_d)) (1 + u): inflate by (d+4)u
        nrm[r] = sqrtf(s) * (1.f + (float)(d + 4) * kU32);
    }
}

// ------------------------------------------------ batched index build
// The same steps as above for many small sets at once: one launch per step,
// each block working on one set (block tables built on the host), the
// scores of all sets sorted together by the composite key (set, score).

// Column sums of rows [r0, r1) of one set, 32 columns per block (float-float
// per thread, FP64 across threads, fixed order).
__global__ void __launch_bounds__(256)
k_colsum_batch(const BSet *__restrict__ sets, const BBlk *__restrict__ blks,
               double *__restrict__ part, int *__restrict__ bad) {
    __shared__ double sh[256];
    const BBlk b = blks[blockIdx.x];
    const BSet &st = sets[b.set];
    const int d = st.d;
    const int TX = d < 32 ? d : 32;
    const int TY = 256 / TX;
    const int t = threadIdx.x;
    const int cx = t % TX, ry = t / TX;
    const int c = b.cb * TX + cx;
    int badl = 0;
    float hi = 0.f, lo = 0.f;
    if (ry < TY && c < d) {
        for (int64_t r = b.r0 + ry; r < b.r1; r += TY) {
            const float x = st.X[r * st.ld + c];
            badl |= !isfinite(x);
            const float s = hi + x;
            const float bb = s - hi;
            const float e = (hi - (s - bb)) + (x - bb);
            const float l = lo + e;
            hi = s + l;
            lo = l - (hi - s);
        }
    }
    if (ry < TY) sh[ry * TX + cx] = (double)hi + (double)lo;
    __syncthreads();
    if (t < TX && b.cb * TX + t < d) {
        double acc = 0.0;
        for (int y = 0; y < TY; ++y) acc += sh[y * TX + t];
        part[st.part_off + int64_t(b.rb) * d + b.cb * TX + t] = acc;
    }
    if (badl) atomicOr(bad, 1);
}

// One block per set: mu = column means (one warp per column), c = fl32(mu).
__global__ void k_mean_final_batch(const BSet *__restrict__ sets, const double *__restrict__ part) {
    const BSet &st = sets[blockIdx.x];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int c = warp; c < st.d; c += nw) {
        double s = 0.0;
        for (int b = lane; b < st.nb; b += 32) s += part[st.part_off + int64_t(b) * st.d + c];
        for (int o = 16; o; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (lane == 0) {
            const double m = s / (double)st.n;
            st.mu64[c] = m;
            st.mu32[c] = (float)m;
        }
    }
}

#define SNN_GRAM_BATCH(TG)                                                                     \
    __global__ void __launch_bounds__(256)                                                     \
    k_gram_batch##TG(const BSet *__restrict__ sets, const BBlk *__restrict__ blks,            \
                     float *__restrict__ gpart) {                                              \
        const BBlk b = blks[blockIdx.x];                                                       \
        const BSet &st = sets[b.set];                                                          \
        gram_small_rows<TG>(st.X, st.d, st.ld, st.mu32, b.r0, b.r1,                            \
                            gpart + st.gpart_off + int64_t(b.rb) * st.d * st.d);               \
    }
SNN_GRAM_BATCH(16)
SNN_GRAM_BATCH(32)
SNN_GRAM_BATCH(64)
#undef SNN_GRAM_BATCH

// One block per set: C = sum of the set's Gram partials (FP64), one warp per
// entry (lane-strided partial sums, shuffle tree).
__global__ void k_gram_reduce_batch(const BSet *__restrict__ sets, const float *__restrict__ gpart,
                                    double *__restrict__ C) {
    const BSet &st = sets[blockIdx.x];
    const int d = st.d, dd = d * d;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int e = warp; e < dd; e += nw) {
        const int i = e / d, j = e % d;
        const int a = min(i, j), b = max(i, j);
        double s = 0.0;
        for (int c = lane; c < st.nb; c += 32)
            s += (double)gpart[st.gpart_off + (int64_t(c) * d + a) * d + b];
        for (int o = 16; o; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (lane == 0) C[st.c_off + e] = s;
    }
}

// One block per set: v1 (the single-CTA squaring of the unbatched build).
__global__ void __launch_bounds__(1024) k_pc_small_batch(const BSet *__restrict__ sets,
                                                         const double *__restrict__ C) {
    const BSet &st = sets[blockIdx.x];
    pc_small_body(C + st.c_off, st.d, st.v64, st.v32);
}

// Scores of rows [r0, r1) of one set, one thread per point: key (set << 32 |
// score key), value = global point index; the largest score bound of the
// block goes to the set's dconst[0].
__global__ void __launch_bounds__(256)
k_project_batch(const BSet *__restrict__ sets, const BBlk *__restrict__ blks,
                uint64_t *__restrict__ keys, uint32_t *__restrict__ vals, int *__restrict__ bad) {
    const BBlk b = blks[blockIdx.x];
    const BSet &st = sets[b.set];
    const int64_t i = b.r0 + threadIdx.x;
    const bool live = i < b.r1;
    float a = 0.f, e = 0.f;
    int badl = 0;
    if (live) {
        for (int k = 0; k < st.d; ++k) {
            const float p = st.X[i * st.ld + k];
            badl |= !isfinite(p);
            const float x = p - st.mu32[k];
            a = fmaf(x, st.v32[k], a);
            e = fmaf(fabsf(x), fabsf(st.v32[k]), e);
        }
        const int64_t g = st.p0 + i;
        keys[g] = (uint64_t(b.set) << 32) | uint64_t(float_to_key(a));
        vals[g] = uint32_t(g);
    }
    float eps = live ? (float)(st.d + 4) * kU32 * 1.01f * e + 1e-37f : 0.f;
    for (int o = 16; o; o >>= 1) {
        eps = fmaxf(eps, __shfl_xor_sync(0xffffffffu, eps, o));
        badl |= __shfl_xor_sync(0xffffffffu, badl, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomic_max_nonneg(st.dconst + 0, eps);
        if (badl) atomicOr(bad, 1);
    }
}

// Sorted position p of the composite order: the set is the key's high word;
// the point lands at its rank inside the set (raw and centred rows, score,
// halved norm, norm bound, original id); the set's largest norm bound goes to
// its dconst[1] (one atomic per group of lanes of the same set).
__global__ void __launch_bounds__(256)
k_gather_batch(const BSet *__restrict__ sets, const uint64_t *__restrict__ skeys,
               const uint32_t *__restrict__ svals, int64_t total) {
    const int64_t p = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    const bool live = p < total;
    const int set = live ? int(skeys[p] >> 32) : -1;
    float nb = 0.f;
    if (live) {
        const BSet &st = sets[set];
        const int64_t r = p - st.p0;
        const int64_t i = int64_t(svals[p]) - st.p0;
        const int d = st.d, dp = st.dp;
        // float4 rows out (dp = 4k); float4 rows in where every input row
        // starts on a 16-byte boundary and d = dp
        const bool vin = d == dp && (st.ld & 3) == 0 && (reinterpret_cast<uintptr_t>(st.X) & 15) == 0;
        const float *xi = st.X + i * st.ld;
        float4 *praw4 = reinterpret_cast<float4 *>(st.praw + r * dp);
        float4 *xc4 = reinterpret_cast<float4 *>(st.xc + r * dp);
        float s = 0.f;
        for (int k4 = 0; k4 < dp / 4; ++k4) {
            float pv[4], x[4];
            if (vin) {
                const float4 v = reinterpret_cast<const float4 *>(xi)[k4];
                pv[0] = v.x, pv[1] = v.y, pv[2] = v.z, pv[3] = v.w;
            } else {
#pragma unroll
                for (int e = 0; e < 4; ++e) pv[e] = 4 * k4 + e < d ? xi[4 * k4 + e] : 0.f;
            }
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int k = 4 * k4 + e;
                x[e] = k < d ? pv[e] - st.mu32[k] : 0.f;
                s = fmaf(x[e], x[e], s);
            }
            praw4[k4] = make_float4(pv[0], pv[1], pv[2], pv[3]);
            xc4[k4] = make_float4(x[0], x[1], x[2], x[3]);
        }
        st.alpha[r] = key_to_float(uint32_t(skeys[p] & 0xffffffffu));
        st.order[r] = int32_t(i);
        st.hx[r] = 0.5f * s;
        nb = sqrtf(s) * (1.f + (float)(d + 4) * kU32);
        st.nrm[r] = nb;
    }
    const unsigned grp = __match_any_sync(0xffffffffu, set);
    const unsigned mx = __reduce_max_sync(grp, __float_as_uint(nb));   // nb >= 0
    if (live && (threadIdx.x & 31) == __ffs(grp) - 1) atomic_max_nonneg(sets[set].dconst + 1, __uint_as_float(mx));
}

}  // namespace snn
