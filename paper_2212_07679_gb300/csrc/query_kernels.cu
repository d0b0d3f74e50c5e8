// Query-phase kernels (Algorithm 2, Section 3.2; Section 4).
//
// Queries are sorted by score and cut into tiles of kBQ; a tile scores the
// union of its queries' candidate ranges (a contiguous band of the sorted
// data, Eq. (2) and Section 4's gemm over the union of J) in chunks of kBR
// rows.  The FP32 score is the left side of Eq. (4), xbar_j - x_j^T x_q, from
// centred FP32 rows; a pair is rejected only when a rigorous bound proves
// ||p_j - q|| > R for the FP64 definition; every other pair ("survivor") is
// decided by the FP64 direct form Eq. (3) in k_recheck, which also yields the
// reported squared distance.
#include "query_kernels.cuh"

namespace snn {

// Per sorted query i, the part of the rejection threshold (halved units) that
// does not depend on the band chunk:
//   thrA_i >= (Rx + e_data + e_i)^2 / 2 - ||y_i||^2 / 2,
// where Rx bounds the largest true distance the FP64 test can accept,
// e_data / e_i bound the centring error norms of a data row / this query, and
// hy_i = fl32(||y_i||^2)/2 underestimates ||y_i||^2/2 by at most gamma_d.
__global__ void k_query_consts(const float *__restrict__ hy, const float *__restrict__ qn,
                               int64_t m, int d, double Rx, double e_data,
                               float *__restrict__ thrA, const double *__restrict__ Rq) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= m) return;
    const double ei = 1.0001 * (double)kU32 * (double)qn[i];
    const double r = (Rq ? radius_slack(Rq[i], d) : Rx) + e_data + ei;
    const double hy_low = (double)hy[i] * (1.0 - 1.05 * (d + 2) * (double)kU32);
    const double a = 0.5 * r * r - hy_low;
    thrA[i] = __double2float_ru(a + 4.0 * kU64 * (fabs(a) + 0.5 * r * r + (double)hy[i]));
}

// Binary searches over the sorted FP32 scores with FP64 thresholds, in FP32:
// for a float a, a < x <=> a < ru(x) and a <= x <=> a <= rd(x), with ru / rd
// the float roundings of x upward / downward (one conversion per search).
__device__ __forceinline__ int64_t lower_bound_ge(const float *__restrict__ a, int64_t n, double x) {
    const float xf = __double2float_ru(x);
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (a[mid] < xf) lo = mid + 1; else hi = mid;
    }
    return lo;
}
__device__ __forceinline__ int64_t upper_bound_gt(const float *__restrict__ a, int64_t n, double x) {
    const float xf = __double2float_rd(x);
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (a[mid] <= xf) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// Candidate band of tile t: every data row whose score is within W of the
// score of some query of the tile (the candidate range of Algorithm 2 for all of them at once).
// W = Wbase + eps_d + eps_q covers |alpha_j - alpha_q| <= ||v1|| ||p_j - q||
// (Eq. (2)) for every pair the FP64 test can accept, plus the rounding bounds
// of both computed scores.
__global__ void k_tile_band(const float *__restrict__ qalpha, int64_t m,
                            const float *__restrict__ alpha, int64_t n, double Wbase,
                            const float *__restrict__ eps_d, const float *__restrict__ eps_q,
                            int64_t *__restrict__ tile_lo, int64_t *__restrict__ tile_hi,
                            int64_t *__restrict__ items, int ntiles, int sym,
                            unsigned long long *__restrict__ band_pairs, const double *__restrict__ Rq,
                            int d) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ntiles) return;
    const double eps = (double)*eps_d + (double)*eps_q;
    const double W = Wbase + eps;
    const int64_t q0 = int64_t(t) * kBQ;
    const int64_t q1 = min(m, q0 + kBQ) - 1;
    const double a0 = (double)qalpha[q0], a1 = (double)qalpha[q1];
    double lo_x = (a0 - W) - 4.0 * kU64 * (fabs(a0) + W);
    double hi_x = (a1 + W) + 4.0 * kU64 * (fabs(a1) + W);
    if (Rq) {
        // the union of the tile's windows, each with its own radius
        lo_x = 1e308;
        hi_x = -1e308;
        for (int64_t q = q0; q <= q1; ++q) {
            const double a = (double)qalpha[q], Wq = window_base(Rq[q], d) + eps;
            lo_x = fmin(lo_x, (a - Wq) - 4.0 * kU64 * (fabs(a) + Wq));
            hi_x = fmax(hi_x, (a + Wq) + 4.0 * kU64 * (fabs(a) + Wq));
        }
    }
    // symmetric self-join: a tile scores only rows at or after its own first
    // query, each unordered pair once (the mirror is emitted on acceptance)
    const int64_t lo = sym ? q0 : lower_bound_ge(alpha, n, lo_x);
    const int64_t hi = max(lo, upper_bound_gt(alpha, n, hi_x));
    tile_lo[t] = lo;
    tile_hi[t] = hi;
    const int64_t chunks = cdiv(hi - lo, kBR);
    items[t] = cdiv(chunks, kChunksPerItem);
    if (band_pairs) atomicAdd(band_pairs, (unsigned long long)((hi - lo) * (q1 - q0 + 1)));
}

// item_tile[i] = the tile whose band chunk group i is (one thread per tile).
__global__ void k_item_tiles(const int64_t *__restrict__ item_off, int ntiles,
                             int32_t *__restrict__ item_tile) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ntiles) return;
    for (int64_t i = item_off[t]; i < item_off[t + 1]; ++i) item_tile[i] = t;
}

// Per-query candidate range sizes |J_q| (statistics only).
__global__ void k_query_windows(const float *__restrict__ qalpha, int64_t m,
                                const float *__restrict__ alpha, int64_t n, double Wbase,
                                const float *__restrict__ eps_d, const float *__restrict__ eps_q,
                                unsigned long long *__restrict__ cand, const double *__restrict__ Rq, int d) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    unsigned long long c = 0;
    if (i < m) {
        const double W = (Rq ? window_base(Rq[i], d) : Wbase) + (double)*eps_d + (double)*eps_q;
        const double a = (double)qalpha[i];
        const double slack = 4.0 * kU64 * (fabs(a) + W);
        const int64_t lo = lower_bound_ge(alpha, n, a - W - slack);
        const int64_t hi = upper_bound_gt(alpha, n, a + W + slack);
        c = hi > lo ? (unsigned long long)(hi - lo) : 0ull;
    }
    for (int o = 16; o; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(cand, c);
}

__global__ void k_query_radii(const double *__restrict__ R, const int32_t *__restrict__ qorder, int64_t m,
                              int d, double *__restrict__ Rs, double *__restrict__ R2s,
                              DecideConsts *__restrict__ dcs) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= m) return;
    const double r = R[qorder[i]];
    Rs[i] = r;
    R2s[i] = __dmul_rn(r, r);
    dcs[i] = decide_consts(d, __dmul_rn(r, r));
}

// ------------------------------------------------------------ FP32 score
// 256 threads; thread (tx, ty) owns queries {ty*4+u, 64+ty*4+u} and rows
// {tx*4+w, 64+tx*4+w}, u, w < 4.  acc starts at -xbar_j and accumulates
// x_j . y_i with FMA, so acc = -(xbar_j - x_j^T y_i) (Eq. (4) left side).
// Rounding: |(-acc) - (||x||^2/2 - x.y)| <= c1 (xbar_j + ||x_j|| ||y_i||).
// A pair survives iff -acc <= thrA_i + c1 (max xbar + max||x|| ||y_i||) over
// the chunk, i.e. unless the bound proves S > R^2.
constexpr int kKC = 16;
constexpr int kScoreThreads = 256;

template <bool kSingle>
__device__ __forceinline__ void score_item(const ScoreJob &jb, float c1, uint2 *__restrict__ surv,
                                           int64_t cap, unsigned long long *__restrict__ count) {
    __shared__ __align__(16) float Qs[kKC][kBQ + 4];
    __shared__ __align__(16) float Xs[kKC][kBR + 4];
    __shared__ float s_thrA[kBQ], s_qn[kBQ];
    __shared__ float s_hx[kBR];
    __shared__ unsigned s_hxmax, s_nmax;

    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    const int lane = tid & 31;
    const int dp = jb.dp;
    const int64_t q0 = jb.q0;
    const int64_t band_lo = jb.band_lo, band_hi = jb.band_hi;

    __syncthreads();
    if (tid < kBQ) {
        const int64_t q = q0 + tid;
        s_thrA[tid] = q < jb.m ? jb.thrA[q] : -3.0e38f;   // never survives
        s_qn[tid] = q < jb.m ? jb.qnrm[q] : 0.f;
    }
    if (kSingle) {
        // whole query rows fit one k-chunk: stage them once per item
        for (int e = tid; e < kBQ * (dp / 4); e += kScoreThreads) {
            const int r = e / (dp / 4), k4 = e % (dp / 4);
            const int64_t q = q0 + r;
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (q < jb.m) v = *reinterpret_cast<const float4 *>(jb.qxc + q * dp + k4 * 4);
            Qs[k4 * 4 + 0][r] = v.x;
            Qs[k4 * 4 + 1][r] = v.y;
            Qs[k4 * 4 + 2][r] = v.z;
            Qs[k4 * 4 + 3][r] = v.w;
        }
    }
    for (int64_t c = jb.c_first; c < jb.c_end; ++c) {
        const int64_t j0 = band_lo + c * kBR;
        __syncthreads();
        if (tid == 0) { s_hxmax = 0u; s_nmax = 0u; }
        __syncthreads();
        if (tid < kBR) {
            const int64_t j = j0 + tid;
            float h = 0.f, nr = 0.f;
            if (j < band_hi) { h = jb.xhx[j]; nr = jb.xnrm[j]; }
            s_hx[tid] = h;
            // block max of non-negative floats through their bit patterns
            unsigned hb = __float_as_uint(h), nb = __float_as_uint(nr);
            for (int o = 16; o; o >>= 1) {
                hb = max(hb, __shfl_xor_sync(0xffffffffu, hb, o));
                nb = max(nb, __shfl_xor_sync(0xffffffffu, nb, o));
            }
            if (lane == 0) { atomicMax(&s_hxmax, hb); atomicMax(&s_nmax, nb); }
        }
        __syncthreads();
        float acc[8][8];
#pragma unroll
        for (int w = 0; w < 8; ++w) {
            const float h = -s_hx[(w < 4 ? 0 : 64) + tx * 4 + (w & 3)];
#pragma unroll
            for (int u = 0; u < 8; ++u) acc[u][w] = h;
        }
        for (int k0 = 0; k0 < dp; k0 += kKC) {
            const int kc = min(kKC, dp - k0);
            __syncthreads();
            if (!kSingle) {
                for (int e = tid; e < kBQ * (kc / 4); e += kScoreThreads) {
                    const int r = e / (kc / 4), k4 = e % (kc / 4);
                    const int64_t q = q0 + r;
                    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                    if (q < jb.m) v = *reinterpret_cast<const float4 *>(jb.qxc + q * dp + k0 + k4 * 4);
                    Qs[k4 * 4 + 0][r] = v.x;
                    Qs[k4 * 4 + 1][r] = v.y;
                    Qs[k4 * 4 + 2][r] = v.z;
                    Qs[k4 * 4 + 3][r] = v.w;
                }
            }
            for (int e = tid; e < kBR * (kc / 4); e += kScoreThreads) {
                const int r = e / (kc / 4), k4 = e % (kc / 4);
                const int64_t j = j0 + r;
                float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                if (j < band_hi) v = *reinterpret_cast<const float4 *>(jb.xxc + j * dp + k0 + k4 * 4);
                Xs[k4 * 4 + 0][r] = v.x;
                Xs[k4 * 4 + 1][r] = v.y;
                Xs[k4 * 4 + 2][r] = v.z;
                Xs[k4 * 4 + 3][r] = v.w;
            }
            __syncthreads();
#pragma unroll 4
            for (int kk = 0; kk < kc; ++kk) {
                const float4 qa = *reinterpret_cast<const float4 *>(&Qs[kk][ty * 4]);
                const float4 qb = *reinterpret_cast<const float4 *>(&Qs[kk][64 + ty * 4]);
                const float4 xa = *reinterpret_cast<const float4 *>(&Xs[kk][tx * 4]);
                const float4 xb = *reinterpret_cast<const float4 *>(&Xs[kk][64 + tx * 4]);
                const float qv[8] = {qa.x, qa.y, qa.z, qa.w, qb.x, qb.y, qb.z, qb.w};
                const float xv[8] = {xa.x, xa.y, xa.z, xa.w, xb.x, xb.y, xb.z, xb.w};
#pragma unroll
                for (int u = 0; u < 8; ++u)
#pragma unroll
                    for (int w = 0; w < 8; ++w) acc[u][w] = fmaf(qv[u], xv[w], acc[u][w]);
            }
        }
        // epilogue: survivors
        const float hxmax = __uint_as_float(s_hxmax), nmax = __uint_as_float(s_nmax);
        unsigned long long mask = 0ull;
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int qi = (u < 4 ? 0 : 64) + ty * 4 + (u & 3);
            float b = c1 * fmaf(nmax, s_qn[qi], hxmax);
            b = b * 1.0000010f;
            float thr = s_thrA[qi] + b;
            thr = thr + fabsf(thr) * 1e-6f + 1e-30f;
            const float neg = -thr;
#pragma unroll
            for (int w = 0; w < 8; ++w) {
                const int rj = (w < 4 ? 0 : 64) + tx * 4 + (w & 3);
                const int64_t jj = j0 + rj;
                const bool ok = (acc[u][w] >= neg) && (jj < band_hi) &&
                                (!jb.sym || jj >= q0 + qi);
                mask |= (unsigned long long)ok << (u * 8 + w);
            }
        }
        const int cnt = __popcll(mask);
        if (__any_sync(0xffffffffu, cnt != 0)) {
            int incl = cnt;
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            const int wtotal = __shfl_sync(0xffffffffu, incl, 31);
            unsigned long long base = 0;
            if (lane == 31) base = atomicAdd(count, (unsigned long long)wtotal);
            base = __shfl_sync(0xffffffffu, base, 31);
            unsigned long long pos = base + (unsigned long long)(incl - cnt);
            while (mask) {
                const int b = __ffsll((long long)mask) - 1;
                mask &= mask - 1;
                const int u = b >> 3, w = b & 7;
                const int qi = (u < 4 ? 0 : 64) + ty * 4 + (u & 3);
                const int rj = (w < 4 ? 0 : 64) + tx * 4 + (w & 3);
                if (pos < (unsigned long long)cap)
                    surv[pos] = make_uint2((unsigned)(jb.q_out + q0 + qi), (unsigned)(j0 + rj));
                ++pos;
            }
        }
    }
}

// One work item of a single query set.
__device__ __forceinline__ ScoreJob single_job(const ScoreArgs &a, int64_t item) {
    const int tile = a.item_tile[item];
    ScoreJob jb;
    jb.m = a.q.m;
    jb.qxc = a.q.xc;
    jb.qnrm = a.q.nrm;
    jb.thrA = a.thrA;
    jb.xxc = a.x.xc;
    jb.xhx = a.x.hx;
    jb.xnrm = a.x.nrm;
    jb.dp = a.x.dp;
    jb.sym = a.sym;
    jb.q0 = int64_t(tile) * kBQ;
    jb.band_lo = a.tile_lo[tile];
    jb.band_hi = a.tile_hi[tile];
    jb.c_first = (item - a.item_off[tile]) * kChunksPerItem;
    jb.c_end = min(cdiv(jb.band_hi - jb.band_lo, kBR), jb.c_first + kChunksPerItem);
    jb.q_out = 0;
    return jb;
}

template <bool kSingle>
__device__ __forceinline__ void score_loop(const ScoreArgs &a) {
    __shared__ long long s_item;
    const int64_t total_items = a.item_off[a.ntiles];
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_item = (long long)atomicAdd(a.work, 1ull);
        __syncthreads();
        const int64_t item = s_item;
        if (item >= total_items) break;
        score_item<kSingle>(single_job(a, item), a.c1, a.surv, a.cap, a.count);
    }
}

__global__ void __launch_bounds__(kScoreThreads, 2) k_score_fp32_single(ScoreArgs a) {
    score_loop<true>(a);
}
__global__ void __launch_bounds__(kScoreThreads, 2) k_score_fp32_multi(ScoreArgs a) {
    score_loop<false>(a);
}

// Many query sets in one persistent launch: every work item names a global
// tile, the tile names its set, and the set descriptor gives that set's
// arrays, row stride and radius-dependent thresholds.  Survivors carry the
// global query number (the set's first global query + local sorted query).
__global__ void __launch_bounds__(kScoreThreads, 2) k_score_fp32_batch(BatchScoreArgs a) {
    __shared__ long long s_item;
    const int64_t total_items = a.item_off[a.ntiles];
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_item = (long long)atomicAdd(a.work, 1ull);
        __syncthreads();
        const int64_t item = s_item;
        if (item >= total_items) break;
        const int tile = a.item_tile[item];
        const SetDesc &sd = a.sets[a.tile_set[tile]];
        ScoreJob jb;
        jb.m = sd.m;
        jb.qxc = sd.q_xc;
        jb.qnrm = sd.q_nrm;
        jb.thrA = a.thrA + sd.q_glob;
        jb.xxc = sd.x_xc;
        jb.xhx = sd.x_hx;
        jb.xnrm = sd.x_nrm;
        jb.dp = sd.dp;
        jb.sym = sd.sym;
        jb.q0 = int64_t(tile - sd.tile0) * kBQ;
        jb.band_lo = a.tile_lo[tile];
        jb.band_hi = a.tile_hi[tile];
        jb.c_first = (item - a.item_off[tile]) * a.cpi;
        jb.c_end = min(cdiv(jb.band_hi - jb.band_lo, kBR), jb.c_first + a.cpi);
        jb.q_out = sd.q_glob;
        if (jb.dp <= kKC)
            score_item<true>(jb, sd.c1, a.surv, a.cap, a.count);
        else
            score_item<false>(jb, sd.c1, a.surv, a.cap, a.count);
    }
}

// ------------------------------------------------------- exact decision
// Each survivor is decided as the FP64 definition Eq. (3) would decide it
// (oracle order: t = p_k - q_k, S = S + t*t, ascending k, no FMA).
//
// Tier 1 evaluates the same sum in compensated FP32 ("double-float"):
// TwoSum gives p_k - q_k = s + e exactly, FMA gives s^2 = ph + pl exactly,
// c = fl(pl + 2 s e) carries the rest (error <= 4u^2 ph with e^2 dropped),
// and (H, L) accumulates with TwoSum / FastTwoSum renormalisation (error
// <= 7u^2 per step relative to the running sum).  So
//   |H + L - S_true| <= (7d + 5) u^2 S,   u = 2^-24,
// and the FP64 oracle sits within gamma_{d+2} S of S_true (the paper's bound
// for the direct form, Section 4).  When R^2 and the nearest float rounding
// boundary of S are both farther than the sum of the two bounds, the FP32
// result decides membership and gives (float)S exactly; otherwise (ties,
// near-ties, overflow or underflow) tier 2 runs the FP64 loop itself.
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    const float bp = __fsub_rn(s, a);
    const float ap = __fsub_rn(s, bp);
    e = __fadd_rn(__fsub_rn(a, ap), __fsub_rn(b, bp));
}

__device__ __forceinline__ double dist2_fp64(const float4 *pp, const float4 *pq, int d, int dp) {
    double S = 0.0;
    for (int k4 = 0; k4 < dp / 4; ++k4) {
        const float4 a = pp[k4], b = pq[k4];
        const float av[4] = {a.x, a.y, a.z, a.w};
        const float bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            if (k4 * 4 + c < d) {
                const double t = __dsub_rn((double)av[c], (double)bv[c]);
                S = __dadd_rn(S, __dmul_rn(t, t));
            }
        }
    }
    return S;
}

// Survivor s of min(*count, cap) (grid-stride: the count is read on the
// device); rec_pos[cap + s] holds the slot in the mirrored row.  NQ bounds
// the float4 columns of a row (dp / 4): every load of both rows is issued
// before the arithmetic.
template <bool kSym, int NQ>
__device__ __forceinline__ void decide_one_survivor(
         int64_t s, const uint2 *__restrict__ surv, int64_t cap, const float *__restrict__ qraw,
         const float *__restrict__ praw, int d, int dp, double R2, const DecideConsts &dc0,
         const double *__restrict__ R2q, const DecideConsts *__restrict__ dcq,
         float *__restrict__ rec_d2, int32_t *__restrict__ rec_pos, int32_t *__restrict__ counts,
         unsigned long long *__restrict__ n_fp64) {
    // the survivor list and the records are read / written once: streaming
    // accesses, so that they do not evict the data rows from L2
    const uint2 e = __ldcs(surv + s);
    if (kSym && e.x == e.y) {
        // a point and itself: S = 0 <= fl64(R*R), dist2 0, one entry
        __stcs(rec_d2 + s, 0.f);
        __stcs(rec_pos + s, atomicAdd(&counts[e.x], 1));
        __stcs(rec_pos + cap + s, -1);
        return;
    }
    const DecideConsts dc = dcq ? dcq[e.x] : dc0;
    const double R2e = R2q ? R2q[e.x] : R2;
    const float4 *pq = reinterpret_cast<const float4 *>(qraw + int64_t(e.x) * dp);
    const float4 *pp = reinterpret_cast<const float4 *>(praw + int64_t(e.y) * dp);
    float4 ra[NQ], rb[NQ];
#pragma unroll
    for (int k4 = 0; k4 < NQ; ++k4) {
        const bool in = k4 < dp / 4;
        ra[k4] = in ? pp[k4] : make_float4(0.f, 0.f, 0.f, 0.f);
        rb[k4] = in ? pq[k4] : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    float H = 0.f, L = 0.f;
#pragma unroll
    for (int k4 = 0; k4 < NQ; ++k4) {
        const float4 a = ra[k4], b = rb[k4];
        const float av[4] = {a.x, a.y, a.z, a.w};
        const float bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            // padding columns (k >= d) are zero in both rows: such a step
            // leaves (H, L) exactly unchanged
            float sd, ed;
            two_sum(av[c], -bv[c], sd, ed);
            const float ph = __fmul_rn(sd, sd);
            const float pl = __fmaf_rn(sd, sd, -ph);
            const float cc = __fmaf_rn(__fadd_rn(sd, sd), ed, pl);
            float s1, t1;
            two_sum(H, ph, s1, t1);
            const float t3 = __fadd_rn(__fadd_rn(t1, L), cc);
            H = __fadd_rn(s1, t3);
            L = __fsub_rn(t3, __fsub_rn(H, s1));
        }
    }
    // H below 2^-100 goes to the FP64 loop (an underflow, or two equal
    // points other than a point and itself)
    float d2 = 0.f;
    int v = decide_df(H, L, true, dc, &d2);
    if (v == 2) {
        const double S = dist2_fp64(pp, pq, d, dp);
        v = S <= R2e ? 1 : 0;
        d2 = (float)S;
        atomicAdd(n_fp64, 1ull);
    }
    const bool accept = v == 1;
    // record: dist2 and the slot of the pair within its row of sorted
    // positions (from the counting atomic, so the scatter needs no atomics);
    // -1 = not a neighbour.  A symmetric self-join pair also takes a slot in
    // the mirrored row.  Neighbouring survivors share rows (one query tile),
    // so the atomics stay within a few cache lines.
    int32_t p0 = -1, p1 = -1;
    if (accept) {
        p0 = atomicAdd(&counts[e.x], 1);
        if (kSym && e.x != e.y) p1 = atomicAdd(&counts[e.y], 1);
    }
    __stcs(rec_d2 + s, d2);
    __stcs(rec_pos + s, p0);
    if (kSym) __stcs(rec_pos + cap + s, p1);
}

template <bool kSym, int NQ>
__device__ __forceinline__ void decide_body(
         const uint2 *__restrict__ surv, const unsigned long long *__restrict__ count, int64_t cap,
         const float *__restrict__ qraw, const float *__restrict__ praw, int d, int dp, double R2,
         const DecideConsts &dc, const double *__restrict__ R2q, const DecideConsts *__restrict__ dcq,
         float *__restrict__ rec_d2, int32_t *__restrict__ rec_pos, int32_t *__restrict__ counts,
         unsigned long long *__restrict__ n_fp64) {
    const int64_t nsurv = min((int64_t)*count, cap);
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t s = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; s < nsurv; s += stride)
        decide_one_survivor<kSym, NQ>(s, surv, cap, qraw, praw, d, dp, R2, dc, R2q, dcq, rec_d2, rec_pos,
                                      counts, n_fp64);
}

// The same decision with G lanes per survivor for long rows: lane l
// accumulates (H, L) over the float4 columns l, l+G, ... (coalesced loads),
// and the G partial double-floats are combined towards lane 0 with the same
// double-float step (TwoSum of the high parts, the low parts added, FastTwoSum
// renormalisation).  Every term passes through at most d/G + log2(G) + 1 <= d
// such steps of error <= 7u^2 relative to the (nonnegative) sum they feed, so
// the tier-1 bound (7d + 5) u^2 S above still holds.  The FP64 fallback runs
// the oracle's ascending loop on lane 0.
template <bool kSym, int G>
__device__ __forceinline__ void decide_group_body(
         const uint2 *__restrict__ surv, const unsigned long long *__restrict__ count, int64_t cap,
         const float *__restrict__ qraw, const float *__restrict__ praw, int d, int dp, double R2,
         const DecideConsts &dc0, const double *__restrict__ R2q, const DecideConsts *__restrict__ dcq,
         float *__restrict__ rec_d2, int32_t *__restrict__ rec_pos, int32_t *__restrict__ counts,
         unsigned long long *__restrict__ n_fp64) {
    constexpr int GPW = 32 / G;   // groups per warp
    const int64_t nsurv = min((int64_t)*count, cap);
    const int lane = int(threadIdx.x % G);
    // tier 0: a plain FP32 sum S0 of the squared (rounded) differences, each
    // lane over at most h0 terms, then log2(G) additions; every term and sum
    // is rounded at most h0 + log2(G) + 2 times, so S0 <= S (1 + u)^(h0 +
    // log2 G + 2) for the exact sum S (underflow only lowers S0).  A pair
    // with S0 above R^2 (1 + 1.01 (h + 3) u) + 2^-40 R^2 has S above R^2 by
    // more than the FP64 definition's own rounding: not a neighbour.
    const int h0 = 4 * int((dp / 4 + G - 1) / G) + (G == 32 ? 5 : 3) + 2;
    const double f0 = 1.0 + 1.01 * (h0 + 3) * 0x1p-24 + 0x1p-40;
    const float thr_uniform = fmaxf(__double2float_ru(R2 * f0), 0x1p-100f);
    const int64_t gw = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int64_t wstride = (int64_t(gridDim.x) * blockDim.x) >> 5;
    // the loop condition is the same for the whole warp; groups past the end
    // still join the shuffles
    for (int64_t base = gw * GPW; base < nsurv; base += wstride * GPW) {
        const int64_t s = base + int((threadIdx.x & 31) / G);
        const bool valid = s < nsurv;
        const uint2 e = valid ? surv[s] : make_uint2(0u, 0u);
        // a point and itself (S = 0, always a neighbour) skips the arithmetic
        const bool self = kSym && valid && e.x == e.y;
        const float4 *pq = reinterpret_cast<const float4 *>(qraw + int64_t(e.x) * dp);
        const float4 *pp = reinterpret_cast<const float4 *>(praw + int64_t(e.y) * dp);
        float S0 = 0.f;
        for (int k4 = lane; valid && !self && k4 < dp / 4; k4 += G) {
            const float4 a = pp[k4], b = pq[k4];
            float t = __fsub_rn(a.x, b.x);
            S0 = __fmaf_rn(t, t, S0);
            t = __fsub_rn(a.y, b.y);
            S0 = __fmaf_rn(t, t, S0);
            t = __fsub_rn(a.z, b.z);
            S0 = __fmaf_rn(t, t, S0);
            t = __fsub_rn(a.w, b.w);
            S0 = __fmaf_rn(t, t, S0);
        }
#pragma unroll
        for (int o = G / 2; o; o >>= 1) S0 = __fadd_rn(S0, __shfl_xor_sync(0xffffffffu, S0, o, G));
        const float thr0 =
            R2q ? (valid ? fmaxf(__double2float_ru(R2q[e.x] * f0), 0x1p-100f) : 0.f) : thr_uniform;
        // clearly outside: the compensated evaluation is skipped (the group
        // still takes part in the warp's shuffles below)
        const bool rej = valid && S0 > thr0;
        float H = 0.f, L = 0.f;
        for (int k4 = lane; valid && !rej && !self && k4 < dp / 4; k4 += G) {
            const float4 a = pp[k4], b = pq[k4];
            const float av[4] = {a.x, a.y, a.z, a.w};
            const float bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                // padding columns (k >= d) are zero in both rows: such a step
                // leaves (H, L) exactly unchanged
                float sd, ed;
                two_sum(av[c], -bv[c], sd, ed);
                const float ph = __fmul_rn(sd, sd);
                const float pl = __fmaf_rn(sd, sd, -ph);
                const float cc = __fmaf_rn(__fadd_rn(sd, sd), ed, pl);
                float s1, t1;
                two_sum(H, ph, s1, t1);
                const float t3 = __fadd_rn(__fadd_rn(t1, L), cc);
                H = __fadd_rn(s1, t3);
                L = __fsub_rn(t3, __fsub_rn(H, s1));
            }
        }
#pragma unroll
        for (int o = G / 2; o; o >>= 1) {
            const float H2 = __shfl_down_sync(0xffffffffu, H, o, G);
            const float L2 = __shfl_down_sync(0xffffffffu, L, o, G);
            float s1, t1;
            two_sum(H, H2, s1, t1);
            const float t3 = __fadd_rn(__fadd_rn(t1, L), L2);
            H = __fadd_rn(s1, t3);
            L = __fsub_rn(t3, __fsub_rn(H, s1));
        }
        if (lane != 0 || !valid) continue;
        if (self) {
            rec_d2[s] = 0.f;
            rec_pos[s] = atomicAdd(&counts[e.x], 1);
            rec_pos[cap + s] = -1;
            continue;
        }
        if (rej) {
            rec_d2[s] = 0.f;
            rec_pos[s] = -1;
            if (kSym) rec_pos[cap + s] = -1;
            continue;
        }
        const DecideConsts dc = dcq ? dcq[e.x] : dc0;
        const double R2e = R2q ? R2q[e.x] : R2;
        // H below 2^-100 goes to the FP64 loop (an underflow, or two equal
        // points other than a point and itself)
        float d2 = 0.f;
        int v = decide_df(H, L, true, dc, &d2);
        if (v == 2) {
            const double S = dist2_fp64(pp, pq, d, dp);
            v = S <= R2e ? 1 : 0;
            d2 = (float)S;
            atomicAdd(n_fp64, 1ull);
        }
        const bool accept = v == 1;
        int32_t p0 = -1, p1 = -1;
        if (accept) {
            p0 = atomicAdd(&counts[e.x], 1);
            if (kSym && e.x != e.y) p1 = atomicAdd(&counts[e.y], 1);
        }
        rec_d2[s] = d2;
        rec_pos[s] = p0;
        if (kSym) rec_pos[cap + s] = p1;
    }
}

#define SNN_DECIDE_ARGS                                                                      \
    const uint2 *__restrict__ surv, const unsigned long long *__restrict__ count, int64_t cap, \
        const float *__restrict__ qraw, const float *__restrict__ praw, int d, int dp,         \
        double R2, DecideConsts dc, const double *__restrict__ R2q,                            \
        const DecideConsts *__restrict__ dcq, float *__restrict__ rec_d2,                      \
        int32_t *__restrict__ rec_pos, int32_t *__restrict__ counts,                           \
        unsigned long long *__restrict__ n_fp64
#define SNN_DECIDE_PASS surv, count, cap, qraw, praw, d, dp, R2, dc, R2q, dcq, rec_d2, rec_pos, counts, \
                        n_fp64
// one lane per survivor: rows of up to 16 floats (4 float4 columns) or 32
__global__ void __launch_bounds__(256) k_decide_sym(SNN_DECIDE_ARGS) {
    decide_body<true, 4>(SNN_DECIDE_PASS);
}
__global__ void __launch_bounds__(256) k_decide_one(SNN_DECIDE_ARGS) {
    decide_body<false, 4>(SNN_DECIDE_PASS);
}
__global__ void __launch_bounds__(256) k_decide_sym_w(SNN_DECIDE_ARGS) {
    decide_body<true, 8>(SNN_DECIDE_PASS);
}
__global__ void __launch_bounds__(256) k_decide_one_w(SNN_DECIDE_ARGS) {
    decide_body<false, 8>(SNN_DECIDE_PASS);
}
__global__ void __launch_bounds__(256) k_decide_sym_g8(SNN_DECIDE_ARGS) {
    decide_group_body<true, 8>(SNN_DECIDE_PASS);
}
__global__ void __launch_bounds__(256) k_decide_one_g8(SNN_DECIDE_ARGS) {
    decide_group_body<false, 8>(SNN_DECIDE_PASS);
}
__global__ void __launch_bounds__(256) k_decide_sym_g32(SNN_DECIDE_ARGS) {
    decide_group_body<true, 32>(SNN_DECIDE_PASS);
}
__global__ void __launch_bounds__(256) k_decide_one_g32(SNN_DECIDE_ARGS) {
    decide_group_body<false, 32>(SNN_DECIDE_PASS);
}
#undef SNN_DECIDE_PASS
#undef SNN_DECIDE_ARGS

__global__ void k_counts_to_i64(const int32_t *__restrict__ counts, int64_t m,
                                int64_t *__restrict__ out) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i < m) out[i] = counts[i];
}

__global__ void k_counts_by_id(const int32_t *__restrict__ counts, const int32_t *__restrict__ order,
                               int64_t m, int64_t *__restrict__ out, const int64_t *__restrict__ soff,
                               uint2 *__restrict__ rinfo) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= m) return;
    const int32_t id = order[i];
    if (out) out[id] = counts[i];
    if (rinfo) rinfo[i] = make_uint2(uint32_t(soff[i]), uint32_t(id));
}

// Writes each accepted pair at its row slot (and the mirrored pair of a
// symmetric self-join) as one packed entry (column id << 32 | dist2 bits) of
// the staging array, whose rows are sorted query positions: the rows of a
// query tile and of its band are neighbours there, so the stores of one
// stretch of survivors fall into a window of the array that stays in L2.
// rinfo[x] = (staging offset of row x, query id qorder[x]); column ids are
// the point ids porder[y] (mirrored: qorder[x]).  In a symmetric self-join
// the points are the queries (porder = qorder), so rinfo[y] gives both the
// mirrored row's offset and porder[y]: two random 8-byte loads per survivor.
__global__ void k_scatter(const uint2 *__restrict__ surv, const int32_t *__restrict__ rec_pos,
                          const float *__restrict__ rec_d2, int64_t nsurv, int64_t rstride, int sym,
                          const uint2 *__restrict__ rinfo, const int32_t *__restrict__ porder,
                          uint64_t *__restrict__ tmp) {
    // four survivors per thread, every load independent of the others (the
    // chain is rec arrays -> row offset and column id -> store)
    constexpr int U = 4;
    const int64_t base = (int64_t(blockIdx.x) * blockDim.x) * U + threadIdx.x;
    int32_t p0[U], p1[U];
    uint2 rc[U];
    uint32_t vb[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
        const int64_t s = base + int64_t(u) * blockDim.x;
        const bool in = s < nsurv;
        p0[u] = in ? __ldcs(rec_pos + s) : -1;
        p1[u] = (in && sym) ? __ldcs(rec_pos + rstride + s) : -1;
        rc[u] = in ? __ldcs(surv + s) : make_uint2(0u, 0u);
        vb[u] = in ? __float_as_uint(__ldcs(rec_d2 + s)) : 0u;
    }
    uint2 ix[U], iy[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
        ix[u] = p0[u] >= 0 ? rinfo[rc[u].x] : make_uint2(0u, 0u);
        if (sym) iy[u] = p0[u] >= 0 ? rinfo[rc[u].y] : make_uint2(0u, 0u);
        else iy[u] = make_uint2(0u, p0[u] >= 0 ? uint32_t(porder[rc[u].y]) : 0u);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
        if (p0[u] >= 0) tmp[int64_t(ix[u].x) + p0[u]] = (uint64_t(iy[u].y) << 32) | vb[u];
        if (p1[u] >= 0) tmp[int64_t(iy[u].x) + p1[u]] = (uint64_t(ix[u].y) << 32) | vb[u];
    }
}

// The same placement for rows that stay in sorted positions (the internal
// neighbourhoods of DBSCAN, a symmetric self-join): column ids only (rinfo[y]
// = (offset of row y, point id); mirrored entries take the id of x), rows
// unsorted.
__global__ void k_scatter_pos(const uint2 *__restrict__ surv, const int32_t *__restrict__ rec_pos,
                              int64_t nsurv, int64_t rstride, const uint2 *__restrict__ rinfo,
                              int32_t *__restrict__ cols) {
    constexpr int U = 4;
    const int64_t base = (int64_t(blockIdx.x) * blockDim.x) * U + threadIdx.x;
    int32_t p0[U], p1[U];
    uint2 rc[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
        const int64_t s = base + int64_t(u) * blockDim.x;
        const bool in = s < nsurv;
        p0[u] = in ? __ldcs(rec_pos + s) : -1;
        p1[u] = in ? __ldcs(rec_pos + rstride + s) : -1;
        rc[u] = in ? __ldcs(surv + s) : make_uint2(0u, 0u);
    }
    uint2 ix[U], iy[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
        ix[u] = p0[u] >= 0 ? rinfo[rc[u].x] : make_uint2(0u, 0u);
        iy[u] = p0[u] >= 0 ? rinfo[rc[u].y] : make_uint2(0u, 0u);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
        if (p0[u] >= 0) cols[int64_t(ix[u].x) + p0[u]] = int32_t(iy[u].y);
        if (p1[u] >= 0) cols[int64_t(iy[u].x) + p1[u]] = int32_t(ix[u].y);
    }
}

// ------------------------------------------- per-row sort by column id
// Rows by length: [7] <= 8 and [8] <= 16 (fine classes only; else in [0]),
// [0] <= 32, [6] <= 64, [1] <= 128, [5] <= 256, [2] <= 512 (warp sorts),
// [3] <= 4096 (one block each), [4] longer (radix sort).  Each list entry is
// the row's descriptor (staging offset | length << 48, output offset), so a
// sort reads its row without further lookups; lists holds one array of m
// entries per class, class c in slot seg_slot(c).
__global__ void k_seg_classify(SegMap mp, int64_t m, int fine, ulonglong2 *__restrict__ lists,
                               int32_t *__restrict__ big_list, int64_t *__restrict__ big_len,
                               unsigned *__restrict__ counters) {
    const int64_t r = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    int64_t o = 0, len = 0;
    if (r < m) {
        o = mp.src[r];
        len = mp.src[r + 1] - o;
    }
    // class of the row (counter index; -1: empty), and its list slot
    int c = -1;
    if (len > 0) {
        if (len <= kSegSmall) c = fine && len <= 8 ? 7 : (fine && len <= 16 ? 8 : 0);
        else if (len <= 2 * kSegSmall) c = 6;
        else if (len <= 4 * kSegSmall) c = 1;
        else if (len <= 8 * kSegSmall) c = 5;
        else if (len <= 16 * kSegSmall) c = 2;
        else if (len <= kSegMid) c = 3;
        else c = 4;
    }
    // one atomic per class present in the warp: lanes of a class take
    // consecutive positions after the leader's reservation
    const unsigned peers = __match_any_sync(0xffffffffu, c);
    const int leader = __ffs(peers) - 1;
    const int lane = threadIdx.x & 31;
    unsigned base = 0;
    if (c >= 0 && lane == leader) base = atomicAdd(&counters[c], unsigned(__popc(peers)));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (c < 0) return;
    const unsigned pos = base + __popc(peers & lanemask_lt());
    if (c == 4) {
        big_list[pos] = (int32_t)r;
        big_len[pos] = len;
    } else {
        const int64_t od = mp.dst[mp.rmap ? mp.rmap[r] : r];
        lists[int64_t(seg_slot(c)) * m + pos] =
            make_ulonglong2(uint64_t(o) | (uint64_t(len) << 48), uint64_t(od));
    }
}

// S lanes per row of <= S*E packed entries (id << 32 | dist2 bits; ids are
// unique in a row, so ordering the packed values orders the ids); S < 32
// (rows of <= 8 or <= 16 entries, E = 1) puts 32/S rows in one warp.  Bitonic
// network over the blocked layout: lane l of the row's group holds entries
// l*E .. l*E+E-1, so the steps with distance < E are compare-exchanges inside
// a lane and only the steps with distance >= E cross lanes (inside the
// group); every step is branch-free.  When every id of the call is below
// 2^(32 - log2(S*E)) the network runs on 32-bit keys (id << log2(S*E) |
// position in the row), which halves the shuffles and replaces each 64-bit
// compare-and-select by a min and a max; the distances are then fetched by
// position after the sort.  The 32-bit keys are loaded striped (lane l takes
// entries l, l + 32, ...: the network sorts whatever order it is given) and
// the sorted keys pass through shared memory back to the striped layout, so
// that every load and store of a row is a run of consecutive words.
__device__ __forceinline__ uint64_t shfl_xor_u64(uint64_t v, int m) {
    const uint32_t lo = __shfl_xor_sync(0xffffffffu, uint32_t(v), m);
    const uint32_t hi = __shfl_xor_sync(0xffffffffu, uint32_t(v >> 32), m);
    return (uint64_t(hi) << 32) | lo;
}

template <int E, int S, typename T>
__device__ __forceinline__ void bitonic_warp(T (&v)[E], int lane) {
    constexpr int N = S * E;
    const int sl = lane & (S - 1);   // lane within the row's group
#pragma unroll
    for (int k = 2; k <= N; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            if (j >= E) {
                const int lj = j / E;
                const bool lower = (sl & lj) == 0;
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    T p;
                    if constexpr (sizeof(T) == 8) p = shfl_xor_u64(v[e], lj);
                    else p = __shfl_xor_sync(0xffffffffu, v[e], lj);
                    const bool asc = ((sl * E + e) & k) == 0;
                    const bool keep_min = lower == asc;
                    if constexpr (sizeof(T) == 8) {
                        const bool pl = p < v[e];
                        v[e] = (keep_min == pl) ? p : v[e];
                    } else {
                        const T lo = min(p, v[e]), hi = max(p, v[e]);
                        v[e] = keep_min ? lo : hi;
                    }
                }
            } else {
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    const int pe = e ^ j;
                    if (pe > e) {
                        const bool asc = ((sl * E + e) & k) == 0;
                        const T a = v[e], b = v[pe];
                        if constexpr (sizeof(T) == 8) {
                            const bool sw = (a > b) == asc;
                            v[e] = sw ? b : a;
                            v[pe] = sw ? a : b;
                        } else {
                            const T lo = min(a, b), hi = max(a, b);
                            v[e] = asc ? lo : hi;
                            v[pe] = asc ? hi : lo;
                        }
                    }
                }
            }
        }
    }
}

constexpr int kSegWarps = 8;   // warps per block of the per-row sorts

__host__ __device__ constexpr int ilog2c(int x) { return x <= 1 ? 0 : 1 + ilog2c(x >> 1); }

template <int E, int S>
__device__ __forceinline__ void seg_sort_warp(const ulonglong2 *__restrict__ list, unsigned total,
                                              const uint64_t *__restrict__ tmp, int32_t *__restrict__ idx,
                                              float *__restrict__ d2, uint32_t id_bound) {
    static_assert(S == 32 || E == 1, "groups of fewer than 32 lanes sort one entry per lane");
    constexpr int N = S * E;
    constexpr int LB = ilog2c(N);
    static_assert((1 << LB) == N, "position bits");
    constexpr int RW = 32 / S;   // rows per warp
    // transpose buffer: position p of a warp's sorted row at p + p / 32 (one
    // padding word per 32, so that both the blocked writes and the striped
    // reads hit 32 distinct banks)
    constexpr int kTr = E > 1 ? N + N / 32 : 1;
    __shared__ uint32_t s_tr[kSegWarps * kTr];
    const bool k32 = id_bound <= (1u << (32 - LB));
    // 32-bit words of the packed entries: [2i] = dist2 bits, [2i+1] = id
    const uint32_t *__restrict__ w32 = reinterpret_cast<const uint32_t *>(tmp);
    const int lane = threadIdx.x & 31;
    const int sl = lane & (S - 1);
    uint32_t *tr = s_tr + (threadIdx.x >> 5) * kTr;
    const int64_t nw = int64_t(gridDim.x) * (blockDim.x >> 5);
    // the loop runs alike on the whole warp (the shuffles need every lane);
    // a group past the last row holds no entries
    for (int64_t wb = (int64_t(blockIdx.x) * (blockDim.x >> 5) + (threadIdx.x >> 5)) * RW; wb < total;
         wb += nw * RW) {
        const int64_t w = wb + lane / S;
        const ulonglong2 rd = w < total ? list[w] : make_ulonglong2(0ull, 0ull);
        const int64_t o = int64_t(rd.x & ((1ull << 48) - 1ull));
        const int len = int(rd.x >> 48);
        const int64_t od = int64_t(rd.y);
        if (k32) {
            uint32_t v[E];
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const int i = e * S + sl;
                v[e] = i < len ? (w32[2 * (o + i) + 1] << LB) | uint32_t(i) : 0xffffffffu;
            }
            bitonic_warp<E, S>(v, lane);
            // sorted: the group's lane l holds positions l * E .. l * E + E - 1
            if constexpr (E > 1) {
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    const int p = lane * E + e;
                    tr[p + (p >> 5)] = v[e];
                }
                __syncwarp();
#pragma unroll
                for (int e = 0; e < E; ++e) v[e] = tr[e * 33 + lane];
                __syncwarp();
            }
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const int i = e * S + sl;
                if (i < len) {
                    const uint32_t src = v[e] & uint32_t(N - 1);
                    idx[od + i] = int32_t(v[e] >> LB);
                    d2[od + i] = __uint_as_float(w32[2 * (o + src)]);
                }
            }
        } else {
            uint64_t v[E];
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const int i = sl * E + e;
                v[e] = i < len ? tmp[o + i] : ~uint64_t(0);
            }
            bitonic_warp<E, S>(v, lane);
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const int i = sl * E + e;
                if (i < len) {
                    idx[od + i] = int32_t(uint32_t(v[e] >> 32));
                    d2[od + i] = __uint_as_float(uint32_t(v[e]));
                }
            }
        }
    }
}

#define SNN_SEG_ARGS                                                                        \
    const ulonglong2 *__restrict__ list, const unsigned *__restrict__ count,                \
        const uint64_t *__restrict__ tmp, int32_t *idx, float *d2, uint32_t id_bound
// blocks of kSegWarps warps (256 threads)
__global__ void __launch_bounds__(256) k_seg_sort_s8(SNN_SEG_ARGS) {
    seg_sort_warp<1, 8>(list, *count, tmp, idx, d2, id_bound);
}
__global__ void __launch_bounds__(256) k_seg_sort_s16(SNN_SEG_ARGS) {
    seg_sort_warp<1, 16>(list, *count, tmp, idx, d2, id_bound);
}
__global__ void __launch_bounds__(256) k_seg_sort_w1(SNN_SEG_ARGS) {
    seg_sort_warp<1, 32>(list, *count, tmp, idx, d2, id_bound);
}
__global__ void __launch_bounds__(256) k_seg_sort_w2(SNN_SEG_ARGS) {
    seg_sort_warp<2, 32>(list, *count, tmp, idx, d2, id_bound);
}
__global__ void __launch_bounds__(256) k_seg_sort_w4(SNN_SEG_ARGS) {
    seg_sort_warp<4, 32>(list, *count, tmp, idx, d2, id_bound);
}
__global__ void __launch_bounds__(256) k_seg_sort_w8(SNN_SEG_ARGS) {
    seg_sort_warp<8, 32>(list, *count, tmp, idx, d2, id_bound);
}
__global__ void __launch_bounds__(256) k_seg_sort_w16(SNN_SEG_ARGS) {
    seg_sort_warp<16, 32>(list, *count, tmp, idx, d2, id_bound);
}

// One block per row of <= 4096 entries: bitonic sort in shared memory, of
// 32-bit keys (id << 12 | position) when every id is below 2^20, else of the
// packed 64-bit entries.
template <typename T>
__device__ __forceinline__ void block_bitonic(T *sk, int N) {
    for (int k = 2; k <= N; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < N; i += blockDim.x) {
                const int ixj = i ^ j;
                if (ixj > i) {
                    const bool asc = (i & k) == 0;
                    const T a = sk[i], b = sk[ixj];
                    const bool sw = (a > b) == asc;
                    sk[i] = sw ? b : a;
                    sk[ixj] = sw ? a : b;
                }
            }
            __syncthreads();
        }
    }
}

__global__ void __launch_bounds__(256) k_seg_sort_mid(SNN_SEG_ARGS) {
    __shared__ uint64_t sk[kSegMid];
    uint32_t *sk32 = reinterpret_cast<uint32_t *>(sk);
    const uint32_t *__restrict__ w32 = reinterpret_cast<const uint32_t *>(tmp);
    const bool k32 = id_bound <= (1u << 20);
    const unsigned total = *count;
    for (unsigned w = blockIdx.x; w < total; w += gridDim.x) {
        const ulonglong2 rd = list[w];
        const int64_t o = int64_t(rd.x & ((1ull << 48) - 1ull));
        const int len = int(rd.x >> 48);
        const int64_t od = int64_t(rd.y);
        int N = 64;
        while (N < len) N <<= 1;
        __syncthreads();
        if (k32) {
            for (int i = threadIdx.x; i < N; i += blockDim.x)
                sk32[i] = i < len ? (w32[2 * (o + i) + 1] << 12) | uint32_t(i) : 0xffffffffu;
            __syncthreads();
            block_bitonic(sk32, N);
            for (int i = threadIdx.x; i < len; i += blockDim.x) {
                const uint32_t v = sk32[i];
                idx[od + i] = int32_t(v >> 12);
                d2[od + i] = __uint_as_float(w32[2 * (o + (v & 4095u))]);
            }
        } else {
            for (int i = threadIdx.x; i < N; i += blockDim.x) sk[i] = i < len ? tmp[o + i] : ~uint64_t(0);
            __syncthreads();
            block_bitonic(sk, N);
            for (int i = threadIdx.x; i < len; i += blockDim.x) {
                idx[od + i] = int32_t(uint32_t(sk[i] >> 32));
                d2[od + i] = __uint_as_float(uint32_t(sk[i]));
            }
        }
    }
}
#undef SNN_SEG_ARGS

snn_status seg_sort_launch(const ulonglong2 *lists, const unsigned *cls, int64_t m, const uint64_t *tmp,
                           int32_t *idx, float *d2, uint32_t id_bound, cudaStream_t s) {
    const int64_t mm = m > 0 ? m : 1;
    auto wgrid = [&](int rpw) {
        return unsigned(std::min<int64_t>(cdiv(cdiv(mm, rpw) * 32, 256), 16384));
    };
    auto lst = [&](int c) { return lists + int64_t(seg_slot(c)) * m; };
    SNN_LAUNCH(k_seg_sort_s8, wgrid(4), 256, 0, s)(lst(7), cls + 7, tmp, idx, d2, id_bound);
    SNN_LAUNCH(k_seg_sort_s16, wgrid(2), 256, 0, s)(lst(8), cls + 8, tmp, idx, d2, id_bound);
    SNN_LAUNCH(k_seg_sort_w1, wgrid(1), 256, 0, s)(lst(0), cls, tmp, idx, d2, id_bound);
    SNN_LAUNCH(k_seg_sort_w2, wgrid(1), 256, 0, s)(lst(6), cls + 6, tmp, idx, d2, id_bound);
    SNN_LAUNCH(k_seg_sort_w4, wgrid(1), 256, 0, s)(lst(1), cls + 1, tmp, idx, d2, id_bound);
    SNN_LAUNCH(k_seg_sort_w8, wgrid(1), 256, 0, s)(lst(5), cls + 5, tmp, idx, d2, id_bound);
    SNN_LAUNCH(k_seg_sort_w16, wgrid(1), 256, 0, s)(lst(2), cls + 2, tmp, idx, d2, id_bound);
    SNN_LAUNCH(k_seg_sort_mid, unsigned(std::min<int64_t>(mm, 4096)), 256, 0, s)(lst(3), cls + 3, tmp, idx, d2,
                                                                             id_bound);
    SNN_LAUNCH_CHECK();
    return SNN_OK;
}

// Long rows: keys (big-row rank << 32 | column), values = source position.
__global__ void k_seg_big_gather(const int32_t *__restrict__ big_list, int nbig, SegMap mp,
                                 const int64_t *__restrict__ toff, const uint64_t *__restrict__ tmp,
                                 uint64_t *__restrict__ keys, uint32_t *__restrict__ vals,
                                 float *__restrict__ gd2) {
    const int b = blockIdx.x;
    if (b >= nbig) return;
    const int32_t r = big_list[b];
    const int64_t o = mp.src[r], len = mp.src[r + 1] - o, t0 = toff[b];
    for (int64_t i = threadIdx.x; i < len; i += blockDim.x) {
        const uint64_t v = tmp[o + i];
        keys[t0 + i] = (uint64_t(b) << 32) | (v >> 32);
        vals[t0 + i] = uint32_t(t0 + i);
        gd2[t0 + i] = __uint_as_float(uint32_t(v));
    }
}

__global__ void k_seg_big_scatter(const uint64_t *__restrict__ keys, const uint32_t *__restrict__ vals,
                                  int64_t total, const int32_t *__restrict__ big_list, SegMap mp,
                                  const int64_t *__restrict__ toff, const float *__restrict__ gd2,
                                  int32_t *__restrict__ idx, float *__restrict__ d2) {
    const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (t >= total) return;
    const uint64_t k = keys[t];
    const int b = int(k >> 32);
    const int32_t r = big_list[b];
    const int64_t pos = mp.dst[mp.rmap ? mp.rmap[r] : r] + (t - toff[b]);
    idx[pos] = int32_t(uint32_t(k & 0xffffffffu));
    d2[pos] = gd2[vals[t]];
}

}  // namespace snn
