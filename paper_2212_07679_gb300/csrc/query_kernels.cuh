// Query-phase kernels (Algorithm 2, Section 3.2; Section 4).
#pragma once
#include "common.cuh"

namespace snn {

// Query tile (queries sorted by score) and band chunk (sorted data rows).
constexpr int kBQ = 128;
constexpr int kBR = 128;
constexpr int kChunksPerItem = 16;  // band chunks scored by one work item

// Sorted query set: either the index's own points (self-join) or
// out-of-sample queries projected, sorted and gathered like the data.
struct QuerySet {
    int64_t m;
    const float *alpha;    // m, sorted scores
    const int32_t *order;  // m, original query row of each sorted position
    const float *raw;      // m x dp raw rows
    const float *xc;       // m x dp centred rows
    const float *hx;       // m, halved squared norms (FP32)
    const float *nrm;      // m, upper bounds on norms
};

struct DataSet {
    int64_t n;
    int d, dp;
    const float *alpha;
    const int32_t *order;
    const float *raw;
    const float *xc;
    const float *hx;
    const float *nrm;
};

struct ScoreArgs {
    QuerySet q;
    DataSet x;
    const float *thrA;          // m: per-query constant part of the threshold
    const int64_t *tile_lo;     // ntiles
    const int64_t *tile_hi;
    const int64_t *item_off;    // ntiles + 1, exclusive scan of items per tile
    const int32_t *item_tile;   // tile of each work item
    int ntiles;
    int sym;                    // symmetric self-join: only pairs with row >= query
    float c1;                   // rounding constant of the FP32 score
    uint2 *surv;                // survivor pairs (sorted query pos, sorted row)
    int64_t cap;
    unsigned long long *count;  // survivors found (may exceed cap)
    unsigned long long *work;   // work-item counter
    int *err;                   // device error flag (bounded waits that gave up)
    const double *Rq = nullptr; // per-query radii (sorted query order), or null
    double q_nrm_max = 0.0;     // largest centred query norm bound (tensor-core scaling)
    cudaEvent_t ev_kernel[2] = {nullptr, nullptr};   // host: recorded around the scoring launch
};

// One work item of the FP32 scorer: a 128-query tile against band chunks
// [c_first, c_end) of its band; survivors are reported with query number
// q_out + local sorted query.
struct ScoreJob {
    int64_t m;
    const float *qxc, *qnrm, *thrA;
    const float *xxc, *xhx, *xnrm;
    int dp, sym;
    int64_t q0, band_lo, band_hi, c_first, c_end, q_out;
};

// Per-set descriptor of a batched query (device memory).
// Constants of the FP32 tier-1 decision (see decide_df).
struct DecideConsts {
    float r2h, r2l, rel, rel2, tiny;
};

struct SetDesc {
    int64_t m, n;               // queries, data points
    int d, dp, sym;             // dims, row stride, symmetric self-join
    float c1;                   // FP32 score rounding constant of this d
    int64_t q_glob;             // first global query number of the set
    int64_t tile0;              // first global tile of the set
    double R2, Wbase;           // fl64(R*R), band half-width base
    DecideConsts dc;            // decision constants for R2
    const float *q_alpha, *q_raw, *q_xc, *q_hx, *q_nrm;
    const int32_t *q_order;
    const float *x_alpha, *x_raw, *x_xc, *x_hx, *x_nrm;
    const int32_t *x_order;
    const float *eps_d, *eps_q; // device scalars: score rounding bounds
    double Rx, e_data;          // radius slack and centring error bound
    int tc;                     // scored by a tensor-core group (no FP32 items)
};

struct BatchScoreArgs {
    const SetDesc *sets;
    const int32_t *tile_set;    // set of each global tile
    const float *thrA;          // per global query
    const int64_t *tile_lo, *tile_hi, *item_off;
    const int32_t *item_tile;
    int ntiles;
    int cpi;                    // band chunks per work item
    uint2 *surv;
    int64_t cap;
    unsigned long long *count, *work;
};

__global__ void k_score_fp32_batch(BatchScoreArgs a);
__global__ void k_item_tiles(const int64_t *item_off, int ntiles, int32_t *item_tile);
// Largest true distance the FP64 test with radius R can accept (the FP64
// rounding of S, R*R and the comparison).
__host__ __device__ inline double radius_slack(double R, int d) { return R * (1.0 + (d + 8) * 0x1p-52); }
// Window half-width base for a radius: |alpha_j - alpha_q| <= ||v|| D + eps_j + eps_q.
__host__ __device__ inline double window_base(double R, int d) {
    return radius_slack(R, d) * (1.0 + (d + 4) * 0x1p-52) * (1.0 + 0x1p-30);
}

// Per-query radii (sorted query order): Rq non-null replaces the scalar
// radius arguments of the kernels below with Rq[i] for query i.
__global__ void k_query_consts(const float *hy, const float *qn, int64_t m, int d, double Rx,
                               double e_data, float *thrA, const double *Rq);
__global__ void k_tile_band(const float *qalpha, int64_t m, const float *alpha, int64_t n,
                            double Wbase, const float *eps_d, const float *eps_q,
                            int64_t *tile_lo, int64_t *tile_hi, int64_t *items, int ntiles,
                            int sym, unsigned long long *band_pairs, const double *Rq, int d);
__global__ void k_query_windows(const float *qalpha, int64_t m, const float *alpha, int64_t n,
                                double Wbase, const float *eps_d, const float *eps_q,
                                unsigned long long *cand, const double *Rq, int d);
// Per-query radii in sorted query order (Rs[i] = R[qorder[i]]), fl64(R*R)
// and the decision constants of each.
__global__ void k_query_radii(const double *R, const int32_t *qorder, int64_t m, int d, double *Rs,
                              double *R2s, DecideConsts *dcs);
__global__ void k_score_fp32_single(ScoreArgs a);
__global__ void k_score_fp32_multi(ScoreArgs a);
// Tier-1 membership and dist2 from the compensated FP32 value H + L of S
// (|H + L - S_true| <= (7d + 5) u^2 S, and the FP64 oracle within
// gamma_{d+2} S of S_true) with FP32 arithmetic only (FP64 is slow on this
// part).  R^2 = fl64(R*R) is held as the float pair (r2h, r2l) with
// |R^2 - r2h - r2l| <= 2^-48 R^2.  D = fl(fl(H - r2h) + fl(L - r2l)) is within
// 2^-46 max(H, r2h) of H + L - R^2 (H - r2h is exact when the two are within a
// factor of two; otherwise |D| is far beyond the tolerance and only its sign
// matters).  Returns 1 (accept, *d2 = (float)S), 0 (reject) or 2 (take the
// FP64 loop: near-ties, values near a float rounding boundary, overflow,
// underflow).  nz: some coordinate differs (H = 0 with nz may be an
// underflow); a caller that does not track it passes true, and then every H
// below 2^-100, equal points included, takes the FP64 loop.


// (computed on the host and passed to the kernels: FP64 is slow on this part)
__host__ __device__ inline DecideConsts decide_consts(int d, double R2) {
    DecideConsts c;
    c.r2h = (float)R2;
    c.r2l = (float)(R2 - (double)c.r2h);
    c.rel = (float)(((7.0 * d + 6.0) * 0x1p-48 + (d + 3.0) * 0x1p-53) * 1.02);
    c.rel2 = 0x1p-45f;
    c.tiny = (float)(d * 0x1p-140);
    return c;
}

__device__ __forceinline__ int decide_df(float H, float L, bool nz, const DecideConsts &c,
                                         float *d2) {
    if (!(H < 0x1p100f) || !(H >= 0.f)) return 2;      // overflow / NaN
    if (H < 0x1p-100f && nz) return 2;                 // possible underflow
    // three round-to-nearest operations (relative error below 2^-22 in all),
    // then a 2^-20 margin: T is never below its exact value
    const float T = fmaf(c.rel, H, fmaf(c.rel2, fmaxf(H, c.r2h), c.tiny)) * (1.f + 0x1p-20f);
    const float D = __fadd_rn(__fsub_rn(H, c.r2h), __fsub_rn(L, c.r2l));
    if (D > T) return 0;
    if (!(D < -T)) return 2;
    if (H > 0.f) {
        // (float)S = H unless S lies within T of a rounding boundary of H
        const float up = __uint_as_float(__float_as_uint(H) + 1u);
        const float dn = __uint_as_float(__float_as_uint(H) - 1u);
        const float half_up = 0.5f * __fsub_rn(up, H), half_dn = 0.5f * __fsub_rn(H, dn);
        const float room = L >= 0.f ? __fsub_rn(half_up, L) : __fadd_rn(half_dn, L);
        if (!(room > fmaf(0x1p-22f, half_up, T))) return 2;
    }
    *d2 = H;
    return 1;
}

// Exact decision of survivors; _sym emits both orientations of a self-join
// pair, _one emits the (query, point) orientation only; _g8 / _g32 use 8 or
// 32 lanes per survivor (long rows).  R2q / dcq non-null: per-query fl64(R*R)
// and decision constants (sorted query order) instead of R2 / dc.  The survivor count is read on the
// device (min(*count, cap)).  Rows and columns are sorted positions: counts[x]
// counts the neighbours of query position x (and of point position y for the
// mirrored pairs of a self-join); rec_pos[s] is the pair's slot in its row,
// rec_pos[cap + s] the mirrored slot, -1 for a pair that is not a neighbour.
#define SNN_DECIDE_DECL(name)                                                                \
    __global__ void name(const uint2 *surv, const unsigned long long *count, int64_t cap,    \
                         const float *qraw, const float *praw, int d, int dp, double R2,     \
                         DecideConsts dc, const double *R2q, const DecideConsts *dcq,        \
                         float *rec_d2, int32_t *rec_pos, int32_t *counts,                   \
                         unsigned long long *n_fp64)
SNN_DECIDE_DECL(k_decide_sym);
SNN_DECIDE_DECL(k_decide_one);
SNN_DECIDE_DECL(k_decide_sym_w);
SNN_DECIDE_DECL(k_decide_one_w);
SNN_DECIDE_DECL(k_decide_sym_g8);
SNN_DECIDE_DECL(k_decide_one_g8);
SNN_DECIDE_DECL(k_decide_sym_g32);
SNN_DECIDE_DECL(k_decide_one_g32);
#undef SNN_DECIDE_DECL
__global__ void k_counts_to_i64(const int32_t *counts, int64_t m, int64_t *out);
// out[order[i]] = counts[i] (out not null): per-position counts to per-id counts; with
// rinfo set also rinfo[i] = (soff[i], order[i]) (offsets below 2^31)
__global__ void k_counts_by_id(const int32_t *counts, const int32_t *order, int64_t m, int64_t *out,
                               const int64_t *soff, uint2 *rinfo);
__global__ void k_scatter(const uint2 *surv, const int32_t *rec_pos, const float *rec_d2,
                          int64_t nsurv, int64_t rstride, int sym, const uint2 *rinfo,
                          const int32_t *porder, uint64_t *tmp);

__global__ void k_scatter_pos(const uint2 *surv, const int32_t *rec_pos, int64_t nsurv, int64_t rstride,
                              const uint2 *rinfo, int32_t *cols);

// Segmented sort of CSR rows by column id; id_bound is an exclusive upper
// bound on the ids (it selects 32-bit sort keys where they fit).
constexpr int kSegSmall = 32;
constexpr int kSegMid = 4096;
// Row placement of the per-row sort: row r is read from the staging array at
// src[r] .. src[r + 1] and written to the output at dst[rmap ? rmap[r] : r].
struct SegMap {
    const int64_t *src;
    const int64_t *dst;
    const int32_t *rmap;
};
// Length classes (counter index c): 0 <= 32 entries (fine: 17-32), 6 <= 64,
// 1 <= 128, 5 <= 256, 2 <= 512, 3 <= 4096, 4 longer, and with fine set
// 7 <= 8 and 8 <= 16.  List slot of class c (class 4 has none: big_list).
__host__ __device__ constexpr int seg_slot(int c) { return c < 4 ? c : c - 1; }
constexpr int kSegSlotsCoarse = 6;   // list slots without the fine classes
constexpr int kSegSlotsFine = 8;
constexpr int kSegClasses = 9;       // counters
// Classifies row r < m by length: appends its descriptor (src offset |
// length << 48, output offset) to its class list (slot seg_slot(c), m
// entries each), or for rows longer than kSegMid its index and length to
// big_list / big_len.  counters[c] counts the rows of class c (zeroed first).
__global__ void k_seg_classify(SegMap mp, int64_t m, int fine, ulonglong2 *lists, int32_t *big_list,
                               int64_t *big_len, unsigned *counters);
#define SNN_SEG_DECL(name)                                                                   \
    __global__ void name(const ulonglong2 *list, const unsigned *count, const uint64_t *tmp, \
                         int32_t *idx, float *d2, uint32_t id_bound)
// launched with 256 threads per block
SNN_SEG_DECL(k_seg_sort_s8);
SNN_SEG_DECL(k_seg_sort_s16);
SNN_SEG_DECL(k_seg_sort_w1);
SNN_SEG_DECL(k_seg_sort_w2);
SNN_SEG_DECL(k_seg_sort_w4);
SNN_SEG_DECL(k_seg_sort_w8);
SNN_SEG_DECL(k_seg_sort_w16);
SNN_SEG_DECL(k_seg_sort_mid);
#undef SNN_SEG_DECL
// Every per-row sort of lists classified with the fine classes (m entries per
// list slot), grids sized for m rows per class: the class counts are read on
// the device, so the launches are the same whatever the row lengths.
snn_status seg_sort_launch(const ulonglong2 *lists, const unsigned *cls, int64_t m, const uint64_t *tmp,
                           int32_t *idx, float *d2, uint32_t id_bound, cudaStream_t s);
__global__ void k_seg_big_gather(const int32_t *big_list, int nbig, SegMap mp, const int64_t *toff,
                                 const uint64_t *tmp, uint64_t *keys, uint32_t *vals, float *gd2);
__global__ void k_seg_big_scatter(const uint64_t *keys, const uint32_t *vals, int64_t total,
                                  const int32_t *big_list, SegMap mp, const int64_t *toff,
                                  const float *gd2, int32_t *idx, float *d2);

}  // namespace snn
