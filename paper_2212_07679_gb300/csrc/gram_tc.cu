// Tensor-core Gram matrix and first principal direction of the index phase
// for d > 64 (Algorithm 1; Eq. (1): v1 is the dominant right singular vector
// of the centred data, i.e. the dominant eigenvector of C = sum_r x_r x_r^T).
//
// C is a contraction over the n data rows.  The centred rows x = fl32(p - c)
// are written transposed (feature-major, rows contiguous) as BF16 parts,
// x = x1 (+ x2), so that both MMA operands are K-major tiles of 128 features
// x 64 rows that TMA stages with the 128-byte swizzle.  One CTA computes one
// 128 x 128 tile of the upper triangle of C over a range of k-blocks (split
// K), accumulating x1.x1 (+ x1.x2 + x2.x1) in TMEM (FP32); the partial tiles
// are summed in FP64.  v1 then comes from repeated squaring of C / trace(C)
// on the same kernels (M symmetric, so M^2 is the Gram matrix of M's rows),
// the column of the last power with the largest diagonal, and FP64 power
// steps on C.  Only the pruning power depends on the accuracy of v1; any unit
// vector keeps the search exact.
//
// Warp roles (128 threads): warp 0 lane 0 issues the TMA loads, warp 1 owns
// TMEM and lane 0 issues the MMAs, then all four warps drain the accumulator
// (warp w reads TMEM lanes 32w..32w+31).  Every mbarrier wait is bounded.
#include <cuda_bf16.h>

#include "index_kernels.cuh"
#include "tc_common.cuh"

namespace snn {

namespace {

constexpr int kGM = 128;    // tile edge: MMA M and N (features)
constexpr int kGKB = 64;    // contraction rows per k-block (128-byte BF16 rows)
constexpr int kPT = 64;     // transpose tile of the packing kernel
constexpr int kSquarings = 12;
constexpr int kPowerSteps = 4;

// out_p[i * n64 + r] (i < dpad features, r < n64 rows) = part p of the BF16
// split of x = fl32(X[r][i] - c[i]) (c NULL: x = X[r][i]), or, with a
// diagonal array `diag` of the square matrix X, of x = fl32(X[r][i] /
// trace(X)).  Zero where r >= n or i >= d.  Grid (n64 / 64, dpad / 64).
template <typename T, int NSPLIT>
__global__ void __launch_bounds__(256)
k_gram_pack(const T *__restrict__ X, int64_t n, int d, int64_t ld, const float *__restrict__ cvec,
            const T *__restrict__ diag, uint16_t *__restrict__ o0, uint16_t *__restrict__ o1,
            int64_t n64) {
    __shared__ __align__(16) uint16_t sh[NSPLIT][kPT][kPT + 8];   // [feature][row]
    __shared__ T s_inv;
    const int64_t r0 = int64_t(blockIdx.x) * kPT;
    const int i0 = blockIdx.y * kPT;
    const bool trace_norm = diag != nullptr;
    if (trace_norm) {
        if (threadIdx.x < 32) {
            T tr = T(0);
            for (int i = threadIdx.x; i < d; i += 32) tr += diag[i];
            for (int o = 16; o; o >>= 1) tr += __shfl_xor_sync(0xffffffffu, tr, o);
            if (threadIdx.x == 0) s_inv = (tr > T(0) && isfinite(tr)) ? T(1) / tr : T(1);
        }
        __syncthreads();
    }
    const int cc = threadIdx.x & 63;
#pragma unroll 4
    for (int k = 0; k < kPT / 4; ++k) {
        const int rr = (threadIdx.x >> 6) + 4 * k;
        const int64_t r = r0 + rr;
        const int i = i0 + cc;
        float x = 0.f;
        if (r < n && i < d) {
            const T v = X[r * ld + i];
            if (trace_norm)
                x = (float)(v * s_inv);
            else
                x = cvec ? (float)v - cvec[i] : (float)v;
        }
        const __nv_bfloat16 h = __float2bfloat16_rn(x);
        sh[0][cc][rr] = __bfloat16_as_ushort(h);
        if (NSPLIT == 2) {
            const __nv_bfloat16 l = __float2bfloat16_rn(x - __bfloat162float(h));
            sh[NSPLIT - 1][cc][rr] = __bfloat16_as_ushort(l);
        }
    }
    __syncthreads();
    const int fi = threadIdx.x >> 2, seg = threadIdx.x & 3;
    const int64_t off = int64_t(i0 + fi) * n64 + r0 + seg * 16;
#pragma unroll
    for (int p = 0; p < NSPLIT; ++p) {
        uint16_t *o = p == 0 ? o0 : o1;
        const uint4 *src = reinterpret_cast<const uint4 *>(&sh[p][fi][seg * 16]);
        uint4 *dst = reinterpret_cast<uint4 *>(o + off);
        dst[0] = src[0];
        dst[1] = src[1];
    }
}

struct GramArgs {
    int nb;          // 128-feature blocks
    int ntiles;      // upper-triangle tiles nb (nb + 1) / 2
    int nkb;         // 64-row k-blocks in total
    int kb_per;      // k-blocks per split
    int d;
    float *part;     // [split][d][d] FP32 partial tiles (upper triangle used)
    float *Cf;       // DIRECT: the full symmetric result (FP32) ...
    float *diagf;    // ... and its diagonal
    int *err;
};

template <int NSPLIT>
struct GramShape {
    static constexpr int kTile = kGM * kGKB * 2;              // 16 KB
    static constexpr int kStageBytes = 2 * NSPLIT * kTile;    // A and B parts
    static constexpr int kStages = NSPLIT == 2 ? 3 : 6;       // 192 KB of stages
    static constexpr int kNP = NSPLIT == 2 ? 3 : 1;           // MMAs per k-step
    static constexpr size_t kSmem = size_t(kStages) * kStageBytes + 1024 + 256;
};

// Bounded wait that ignores the abort flag (used before TMEM is released,
// so that no MMA is still in flight).
__device__ __forceinline__ void mbar_wait_final(uint32_t bar, uint32_t parity, int *err) {
    const long long t0 = clock64();
    while (!mbar_try(bar, parity)) {
        if (clock64() - t0 > kTcTimeoutCycles) {
            atomicOr(err, 1);
            return;
        }
    }
}

// DIRECT (one split): the epilogue writes C[i][j], its mirror C[j][i] and the
// diagonal itself; otherwise FP32 partial tiles for k_gram_reduce2.
template <int NSPLIT, bool DIRECT>
__global__ void __launch_bounds__(128, 1)
k_gram_tc(const __grid_constant__ CUtensorMap m0, const __grid_constant__ CUtensorMap m1,
          GramArgs a) {
    using Sh = GramShape<NSPLIT>;
    constexpr int S = Sh::kStages;
    constexpr int NP = Sh::kNP;
    constexpr uint32_t kIdesc = idesc_bf16<kGM, kGM>();
    constexpr int kPa[3] = {0, 0, 1};
    constexpr int kPb[3] = {0, 1, 0};

    extern __shared__ unsigned char smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    unsigned char *gbase = smem_raw + (base - raw);
    auto a_tile = [&](int s, int p) { return base + uint32_t(s * Sh::kStageBytes + p * Sh::kTile); };
    auto b_tile = [&](int s, int p) {
        return base + uint32_t(s * Sh::kStageBytes + (NSPLIT + p) * Sh::kTile);
    };
    const uint32_t bar0 = base + uint32_t(S * Sh::kStageBytes);
    auto full_bar = [&](int s) { return bar0 + 8u * s; };
    auto empty_bar = [&](int s) { return bar0 + 8u * (S + s); };
    const uint32_t done_bar = bar0 + 8u * (2 * S);
    unsigned char *gmisc = gbase + (bar0 - base) + 8 * (2 * S + 1);
    volatile uint32_t *s_tmem = reinterpret_cast<volatile uint32_t *>(gmisc);
    volatile int *s_abort = reinterpret_cast<volatile int *>(gmisc + 4);
    volatile int *s_consumed = reinterpret_cast<volatile int *>(gmisc + 8);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const CUtensorMap *maps[2] = {&m0, &m1};

    // block -> (split, tile); tiles of one split are adjacent so that the
    // CTAs running together read the same rows
    const int split = blockIdx.x / a.ntiles;
    int t = blockIdx.x % a.ntiles, bi = 0;
    while (t >= a.nb - bi) {
        t -= a.nb - bi;
        ++bi;
    }
    const int bj = bi + t;
    const int kb0 = split * a.kb_per;
    const int nk = min(a.nkb, kb0 + a.kb_per) - kb0;

    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(full_bar(s), 1);
            mbar_init(empty_bar(s), 1);
        }
        mbar_init(done_bar, 1);
        *s_abort = 0;
        *s_consumed = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32((const void *)s_tmem)),
                     "n"(kGM)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tmem_fence_before();
    __syncthreads();
    tmem_fence_after();
    const uint32_t tmem = *s_tmem;

    int issued = 0;
    if (warp == 0 && lane == 0) {
        // ------------------------------------------------ TMA producer
        for (int it = 0; it < nk && !*s_abort; ++it) {
            const int s = it % S;
            const uint32_t round = uint32_t(it / S);
            if (!mbar_wait(empty_bar(s), (round & 1u) ^ 1u, s_abort, a.err)) break;
            mbar_expect_tx(full_bar(s), uint32_t(Sh::kStageBytes));
            const int kx = (kb0 + it) * kGKB;
            for (int p = 0; p < NSPLIT; ++p) {
                tma_load_2d(a_tile(s, p), maps[p], kx, bi * kGM, full_bar(s));
                tma_load_2d(b_tile(s, p), maps[p], kx, bj * kGM, full_bar(s));
            }
            issued = it + 1;
        }
    } else if (warp == 1 && lane == 0) {
        // ------------------------------------------------- MMA issuer
        for (int it = 0; it < nk; ++it) {
            const int s = it % S;
            if (!mbar_wait(full_bar(s), uint32_t(it / S) & 1u, s_abort, a.err)) break;
            tmem_fence_after();
#pragma unroll
            for (int ks = 0; ks < kGKB / 16; ++ks)
#pragma unroll
                for (int pr = 0; pr < NP; ++pr) {
                    const uint64_t ad = smem_desc<128>(a_tile(s, kPa[pr]) + 32u * ks);
                    const uint64_t bd = smem_desc<128>(b_tile(s, kPb[pr]) + 32u * ks);
                    mma_bf16(tmem, ad, bd, kIdesc, (it | ks | pr) != 0 ? 1u : 0u);
                }
            mma_commit(empty_bar(s));
            *s_consumed = it + 1;
        }
        // completes when every MMA issued above has completed
        mma_commit(done_bar);
        mbar_wait_final(done_bar, 0u, a.err);
    }
    __syncwarp();
    // ---------------------------------------------------- epilogue
    // warp-uniform, so that the collective TMEM loads below run in whole warps
    const bool ok = __all_sync(0xffffffffu, mbar_wait(done_bar, 0u, s_abort, a.err) && !*s_abort);
    tmem_fence_after();
    if (ok) {
        const int i = bi * kGM + warp * 32 + lane;
#pragma unroll 1
        for (int h = 0; h < kGM / 64; ++h) {
            uint32_t r[64];
            tmem_ld64(tmem + (uint32_t(warp * 32) << 16) + uint32_t(h * 64), r);
            if (i < a.d) {
                const int j0 = bj * kGM + h * 64;
                if (DIRECT) {
                    float *row = a.Cf + int64_t(i) * a.d;
#pragma unroll
                    for (int c = 0; c < 64; ++c) {
                        const int j = j0 + c;
                        if (j < a.d) {
                            const float v = __uint_as_float(r[c]);
                            row[j] = v;
                            if (bi != bj) a.Cf[int64_t(j) * a.d + i] = v;
                            if (j == i) a.diagf[i] = v;
                        }
                    }
                } else {
                    float *row = a.part + (int64_t(split) * a.d + i) * a.d;
#pragma unroll
                    for (int c = 0; c < 64; ++c)
                        if (j0 + c < a.d) row[j0 + c] = __uint_as_float(r[c]);
                }
            }
        }
    }
    __syncthreads();
    // drain TMA copies still in flight (only after an abort)
    if (warp == 0 && lane == 0)
        for (int it = *s_consumed; it < issued; ++it)
            mbar_wait_final(full_bar(it % S), uint32_t(it / S) & 1u, a.err);
    tmem_fence_before();
    __syncthreads();
    tmem_fence_after();
    if (warp == 1)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "n"(kGM)
                     : "memory");
}

// C[i][j] = sum over splits of the partial tiles (FP64), the upper triangle
// mirrored; diag[i] = C[i][i].
__global__ void k_gram_reduce2(const float *__restrict__ part, int nsplit, int d,
                               double *__restrict__ C, double *__restrict__ diag) {
    const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e >= int64_t(d) * d) return;
    const int i = int(e / d), j = int(e % d);
    const int a = min(i, j), b = max(i, j);
    double s = 0.0;
    for (int c = 0; c < nsplit; ++c) s += (double)part[(int64_t(c) * d + a) * d + b];
    C[e] = s;
    if (i == j) diag[i] = s;
}

// v = row (= column) jbest of the symmetric T, jbest = the largest diagonal
// entry (smallest index among equals); e1 when no diagonal entry is positive
// (C = 0: all points equal).  One block.
__global__ void __launch_bounds__(1024)
k_pick_column64(const float *__restrict__ T, const float *__restrict__ diag, int d,
                double *__restrict__ v) {
    __shared__ double sb[32];
    __shared__ int sj[32];
    double best = 0.0;
    int jb = 0x7fffffff;
    for (int j = threadIdx.x; j < d; j += blockDim.x) {
        const double x = (double)diag[j];
        if (x > best) {
            best = x;
            jb = j;
        }
    }
    for (int o = 16; o; o >>= 1) {
        const double b2 = __shfl_xor_sync(0xffffffffu, best, o);
        const int j2 = __shfl_xor_sync(0xffffffffu, jb, o);
        if (b2 > best || (b2 == best && j2 < jb)) {
            best = b2;
            jb = j2;
        }
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    if (lane == 0) {
        sb[warp] = best;
        sj[warp] = jb;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < nw; ++w)
            if (sb[w] > sb[0] || (sb[w] == sb[0] && sj[w] < sj[0])) {
                sb[0] = sb[w];
                sj[0] = sj[w];
            }
    }
    __syncthreads();
    const bool degenerate = !(sb[0] > 0.0) || !isfinite(sb[0]);
    const int jbest = sj[0];
    for (int i = threadIdx.x; i < d; i += blockDim.x)
        v[i] = degenerate ? (i == 0 ? 1.0 : 0.0) : (double)T[int64_t(jbest) * d + i];
}

// w = C v / ||v|| (FP64; v = 0 gives w = 0), one warp per row.  Every block
// computes ||v|| itself in the same fixed order.
__global__ void __launch_bounds__(256)
k_power64(const double *__restrict__ C, int d, const double *__restrict__ v,
          double *__restrict__ w) {
    __shared__ double red[8];
    double p = 0.0;
    for (int k = threadIdx.x; k < d; k += blockDim.x) p += v[k] * v[k];
    for (int o = 16; o; o >>= 1) p += __shfl_xor_sync(0xffffffffu, p, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = p;
    __syncthreads();
    double nrm2 = 0.0;
    for (int q = 0; q < 8; ++q) nrm2 += red[q];
    const double inv = (nrm2 > 0.0 && isfinite(nrm2)) ? 1.0 / sqrt(nrm2) : 1.0;
    const int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (row >= d) return;
    double s = 0.0;
    for (int k = lane; k < d; k += 32) s += C[int64_t(row) * d + k] * v[k];
    for (int o = 16; o; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) w[row] = s * inv;
}

// C (d x d, FP64, full) and diag = the Gram matrix of the columns held
// transposed in the BF16 parts p0 (p1) of dpad x n64 elements.  DIRECT: one
// split, written by the tensor-core kernel itself; otherwise split K with
// FP32 partials summed in FP64.
template <int NSPLIT, bool DIRECT>
snn_status gram_gemm(const uint16_t *p0, const uint16_t *p1, int d, int dpad, int64_t n64,
                     double *C, double *diag, float *Cf, float *diagf, int *err, cudaStream_t s,
                     Scratch &scr) {
    using Sh = GramShape<NSPLIT>;
    CUtensorMap maps[2];
    SNN_TRY(make_map(&maps[0], p0, dpad, n64, kGKB, kGM));
    SNN_TRY(make_map(&maps[1], NSPLIT == 2 ? p1 : p0, dpad, n64, kGKB, kGM));
    GramArgs a;
    a.nb = dpad / kGM;
    a.ntiles = a.nb * (a.nb + 1) / 2;
    a.nkb = int(n64 / kGKB);
    int nsplitk = 1;
    if (!DIRECT) {
        const int sms = device_sm_count();
        nsplitk = std::max(1, std::min(sms / a.ntiles, a.nkb / 2));
    }
    a.kb_per = int(cdiv(a.nkb, nsplitk));
    nsplitk = int(cdiv(a.nkb, a.kb_per));   // every split holds at least one k-block
    a.d = d;
    a.err = err;
    a.Cf = Cf;
    a.diagf = diagf;
    a.part = nullptr;
    if (!DIRECT) SNN_TRY(scr.alloc(&a.part, size_t(nsplitk) * d * d));
    auto kern = k_gram_tc<NSPLIT, DIRECT>;
    SNN_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(Sh::kSmem)));
    SNN_LAUNCH(kern, unsigned(a.ntiles * nsplitk), 128, Sh::kSmem, s)(maps[0], maps[1], a);
    SNN_LAUNCH_CHECK();
    if (!DIRECT) {
        SNN_LAUNCH(k_gram_reduce2, unsigned(cdiv(int64_t(d) * d, 256)), 256, 0, s)(a.part, nsplitk,
                                                                                  d, C, diag);
        SNN_LAUNCH_CHECK();
    }
    return SNN_OK;
}

}  // namespace

snn_status gram_tc(const float *X, int64_t n, int d, int64_t ld, const float *cvec, double *C,
                   double *diag, int *err, cudaStream_t s, Scratch &scr) {
    const int dpad = int(cdiv(d, kGM) * kGM);
    const int64_t n64 = cdiv(n, kGKB) * kGKB;
    uint16_t *p0, *p1;
    SNN_TRY(scr.alloc(&p0, size_t(dpad) * n64));
    SNN_TRY(scr.alloc(&p1, size_t(dpad) * n64));
    auto pack = k_gram_pack<float, 2>;
    SNN_LAUNCH(pack, dim3(unsigned(n64 / kPT), unsigned(dpad / kPT)), 256, 0, s)(
        X, n, d, ld, cvec, nullptr, p0, p1, n64);
    SNN_LAUNCH_CHECK();
    return gram_gemm<2, false>(p0, p1, d, dpad, n64, C, diag, nullptr, nullptr, err, s, scr);
}

snn_status first_direction_tc(const double *C, const double *diagC, int d, double *v64,
                              float *v32, int *err, cudaStream_t s, Scratch &scr) {
    const int dpad = int(cdiv(d, kGM) * kGM);
    const int64_t n64 = cdiv(d, kGKB) * kGKB;
    uint16_t *p0;
    float *T, *diag;
    double *w0, *w1;
    SNN_TRY(scr.alloc(&p0, size_t(dpad) * n64));
    SNN_TRY(scr.alloc(&T, size_t(d) * d));
    SNN_TRY(scr.alloc(&diag, d));
    SNN_TRY(scr.alloc(&w0, d));
    SNN_TRY(scr.alloc(&w1, d));
    const dim3 pgrid(unsigned(n64 / kPT), unsigned(dpad / kPT));
    // M0 = C / trace(C); M_{k+1} = M_k^2 / trace(M_k^2), one BF16 part and
    // FP32 powers (only the pruning power depends on the accuracy of v1)
    auto pack64 = k_gram_pack<double, 1>;
    auto pack32 = k_gram_pack<float, 1>;
    SNN_LAUNCH(pack64, pgrid, 256, 0, s)(C, d, d, d, nullptr, diagC, p0, nullptr, n64);
    SNN_LAUNCH_CHECK();
    for (int it = 0; it < kSquarings; ++it) {
        SNN_TRY((gram_gemm<1, true>(p0, nullptr, d, dpad, n64, nullptr, nullptr, T, diag, err, s,
                                    scr)));
        if (it + 1 < kSquarings) {
            SNN_LAUNCH(pack32, pgrid, 256, 0, s)(T, d, d, d, nullptr, diag, p0, nullptr, n64);
            SNN_LAUNCH_CHECK();
        }
    }
    SNN_LAUNCH(k_pick_column64, 1, 1024, 0, s)(T, diag, d, v64);
    SNN_LAUNCH_CHECK();
    // FP64 power steps on C (normalised on the fly), then FP64 normalisation
    // into v64 (kept as is when C v vanished: C = 0)
    const double *src = v64;
    double *dst = w0;
    for (int it = 0; it < kPowerSteps; ++it) {
        SNN_LAUNCH(k_power64, unsigned(cdiv(int64_t(d) * 32, 256)), 256, 0, s)(C, d, src, dst);
        SNN_LAUNCH_CHECK();
        src = dst;
        dst = dst == w0 ? w1 : w0;
    }
    SNN_LAUNCH(k_normalise64, 1, 1024, 0, s)(src, d, v64, v32, 1);
    SNN_LAUNCH_CHECK();
    return SNN_OK;
}

}  // namespace snn
