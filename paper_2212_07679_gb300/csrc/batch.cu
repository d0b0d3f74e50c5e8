// Many independent (index, queries, radius) problems of uneven n, d and m in
// one call.  All sets share one pipeline: a composite-key sort of every
// out-of-sample query by (set, score), one band computation over the global
// list of query tiles, ONE persistent scoring launch driven by a device work
// counter over (set, tile, band chunk) items, one exact-decision pass, one
// CSR build whose per-set slices are the per-set results.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include <cstdio>
#include <mutex>
#include <string>

#include "index_struct.cuh"
#include "query_kernels.cuh"
#include "tc_score.cuh"

namespace snn {

snn_status register_block(void *block, void *const *ptrs, int count, cudaStream_t s);

namespace {

__device__ __forceinline__ int find_set(const int64_t *__restrict__ off, int nsets, int64_t g) {
    int lo = 0, hi = nsets;   // last s with off[s] <= g
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (off[mid] <= g) lo = mid; else hi = mid;
    }
    return lo;
}

struct OosDesc {
    const float *Q;        // caller's queries
    int64_t ldq;
    const float *cvec;     // the index's FP32 centre c = fl32(mu)
    const float *v32;
    int d, dp;
    int set;               // batch set number
    int64_t elem_off;      // offset of this set's rows in the concatenated arrays (floats)
};

// Projection of every out-of-sample query: key = (set rank << 32) | score key.
__global__ void k_b_project(const OosDesc *__restrict__ od, const int64_t *__restrict__ ooff,
                            int noos, int64_t total, uint64_t *__restrict__ keys,
                            uint32_t *__restrict__ vals, float *__restrict__ eps,
                            int *__restrict__ bad) {
    const int64_t g = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (g >= total) return;
    const int r = find_set(ooff, noos, g);
    const OosDesc &o = od[r];
    const float *q = o.Q + (g - ooff[r]) * o.ldq;
    float a = 0.f, b = 0.f;
    int badl = 0;
    for (int k = 0; k < o.d; ++k) {
        const float p = q[k];
        badl |= !isfinite(p);
        const float x = p - o.cvec[k];
        a = fmaf(x, o.v32[k], a);
        b = fmaf(fabsf(x), fabsf(o.v32[k]), b);
    }
    keys[g] = (uint64_t(r) << 32) | uint64_t(float_to_key(a));
    vals[g] = uint32_t(g);
    atomic_max_nonneg(&eps[r], (float)(o.d + 4) * kU32 * 1.01f * b + 1e-37f);
    if (badl) atomicOr(bad, 1);
}

// Sorted position p (within the set's contiguous range) takes query vals[p].
__global__ void k_b_gather(const OosDesc *__restrict__ od, const int64_t *__restrict__ ooff,
                           int noos, int64_t total, const uint64_t *__restrict__ keys,
                           const uint32_t *__restrict__ vals, float *__restrict__ q_alpha,
                           int32_t *__restrict__ q_order, float *__restrict__ q_raw,
                           float *__restrict__ q_xc, float *__restrict__ q_hx,
                           float *__restrict__ q_nrm) {
    const int64_t p = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (p >= total) return;
    const int r = int(keys[p] >> 32);
    const OosDesc &o = od[r];
    const int64_t g = vals[p];
    const int64_t local_row = g - ooff[r];
    const int64_t local_pos = p - ooff[r];
    const float *q = o.Q + local_row * o.ldq;
    float *raw = q_raw + o.elem_off + local_pos * o.dp;
    float *xc = q_xc + o.elem_off + local_pos * o.dp;
    float s = 0.f;
    for (int k = 0; k < o.dp; ++k) {
        float pv = 0.f, x = 0.f;
        if (k < o.d) {
            pv = q[k];
            x = pv - o.cvec[k];
        }
        raw[k] = pv;
        xc[k] = x;
        s = fmaf(x, x, s);
    }
    q_alpha[p] = key_to_float(uint32_t(keys[p] & 0xffffffffu));
    q_order[p] = int32_t(local_row);
    q_hx[p] = 0.5f * s;
    q_nrm[p] = sqrtf(s) * (1.f + (float)(o.d + 4) * kU32);
}

__global__ void k_b_qset(const int64_t *__restrict__ qglob, int nsets, int64_t total,
                         int32_t *__restrict__ qset) {
    const int64_t g = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (g < total) qset[g] = find_set(qglob, nsets, g);
}

__global__ void k_b_tileset(const int64_t *__restrict__ tile0, int nsets, int64_t ntiles,
                            int32_t *__restrict__ tile_set) {
    const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (t < ntiles) tile_set[t] = find_set(tile0, nsets, t);
}

// Threshold constant of every global query (as k_query_consts, per set).
__global__ void k_b_consts(const SetDesc *__restrict__ sets, const int32_t *__restrict__ qset,
                           int64_t total, float *__restrict__ thrA) {
    const int64_t g = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (g >= total) return;
    const SetDesc &sd = sets[qset[g]];
    const int64_t i = g - sd.q_glob;
    const double ei = 1.0001 * (double)kU32 * (double)sd.q_nrm[i];
    const double r = sd.Rx + sd.e_data + ei;
    const double hy = (double)sd.q_hx[i];
    const double hy_low = hy * (1.0 - 1.05 * (sd.d + 2) * (double)kU32);
    const double a = 0.5 * r * r - hy_low;
    thrA[g] = __double2float_ru(a + 4.0 * kU64 * (fabs(a) + 0.5 * r * r + hy));
}

// (FP32 searches: for a float a, a < x <=> a < ru(x), a <= x <=> a <= rd(x))
__device__ __forceinline__ int64_t lb_ge(const float *__restrict__ a, int64_t n, double x) {
    const float xf = __double2float_ru(x);
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (a[mid] < xf) lo = mid + 1; else hi = mid;
    }
    return lo;
}
__device__ __forceinline__ int64_t ub_gt(const float *__restrict__ a, int64_t n, double x) {
    const float xf = __double2float_rd(x);
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (a[mid] <= xf) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// Band of every global tile (as k_tile_band, in the tile's own set).
__global__ void k_b_band(const SetDesc *__restrict__ sets, const int32_t *__restrict__ tile_set,
                         int64_t ntiles, int64_t *__restrict__ tile_lo, int64_t *__restrict__ tile_hi,
                         int64_t *__restrict__ items, int cpi) {
    const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (t >= ntiles) return;
    const SetDesc &sd = sets[tile_set[t]];
    const int64_t q0 = (t - sd.tile0) * kBQ;
    const int64_t q1 = min(sd.m, q0 + kBQ) - 1;
    const double W = sd.Wbase + (double)*sd.eps_d + (double)*sd.eps_q;
    const double a0 = (double)sd.q_alpha[q0], a1 = (double)sd.q_alpha[q1];
    const double lo_x = (a0 - W) - 4.0 * kU64 * (fabs(a0) + W);
    const double hi_x = (a1 + W) + 4.0 * kU64 * (fabs(a1) + W);
    const int64_t lo = sd.sym ? q0 : lb_ge(sd.x_alpha, sd.n, lo_x);
    const int64_t hi = max(lo, ub_gt(sd.x_alpha, sd.n, hi_x));
    tile_lo[t] = lo;
    tile_hi[t] = hi;
    // sets of a tensor-core group are scored by that group's launch
    items[t] = sd.tc ? 0 : cdiv(cdiv(hi - lo, kBR), int64_t(cpi));
}

__device__ __forceinline__ void two_sum_b(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    const float bp = __fsub_rn(s, a);
    const float ap = __fsub_rn(s, bp);
    e = __fadd_rn(__fsub_rn(a, ap), __fsub_rn(b, bp));
}

// Exact decision of every survivor (same arithmetic as k_decide_*), with the
// set looked up from the global query number.  rec_pos[s] / rec_pos[N + s]:
// slot of the pair in its (global) row / in the mirrored row, or -1.
__device__ __forceinline__ void b_decide_one(int64_t s, int64_t cap, const uint2 *__restrict__ surv,
                                             const SetDesc *__restrict__ sets,
                                             const int32_t *__restrict__ qset,
                                             float *__restrict__ rec_d2,
                                             int32_t *__restrict__ rec_pos,
                                             int32_t *__restrict__ counts);

// Survivors min(*count, cap), grid-stride (the count is read on the device);
// rec_pos[cap + s] is the mirrored slot.
__global__ void __launch_bounds__(256)
k_b_decide(const uint2 *__restrict__ surv, const unsigned long long *__restrict__ count, int64_t cap,
           const SetDesc *__restrict__ sets, const int32_t *__restrict__ qset,
           float *__restrict__ rec_d2, int32_t *__restrict__ rec_pos, int32_t *__restrict__ counts) {
    const int64_t nsurv = min((int64_t)*count, cap);
    for (int64_t s = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; s < nsurv;
         s += int64_t(gridDim.x) * blockDim.x)
        b_decide_one(s, cap, surv, sets, qset, rec_d2, rec_pos, counts);
}

__device__ __forceinline__ void b_decide_one(int64_t s, int64_t cap, const uint2 *__restrict__ surv,
                                             const SetDesc *__restrict__ sets,
                                             const int32_t *__restrict__ qset,
                                             float *__restrict__ rec_d2,
                                             int32_t *__restrict__ rec_pos,
                                             int32_t *__restrict__ counts) {
    const uint2 e = surv[s];
    const SetDesc &sd = sets[qset[e.x]];
    const int64_t ql = int64_t(e.x) - sd.q_glob;
    const int d = sd.d, dp = sd.dp;
    const float4 *pq = reinterpret_cast<const float4 *>(sd.q_raw + ql * dp);
    const float4 *pp = reinterpret_cast<const float4 *>(sd.x_raw + int64_t(e.y) * dp);
    float H = 0.f, L = 0.f;
    bool nz = false;
    for (int k4 = 0; k4 < dp / 4; ++k4) {
        const float4 a = pp[k4], b = pq[k4];
        const float av[4] = {a.x, a.y, a.z, a.w};
        const float bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            // padding columns (k >= d) are zero in both rows: such a step
            // leaves (H, L) exactly unchanged
            float sd_, ed;
            two_sum_b(av[c], -bv[c], sd_, ed);
            nz |= sd_ != 0.f;
            const float ph = __fmul_rn(sd_, sd_);
            const float pl = __fmaf_rn(sd_, sd_, -ph);
            const float cc = __fmaf_rn(__fadd_rn(sd_, sd_), ed, pl);
            float s1, t1;
            two_sum_b(H, ph, s1, t1);
            const float t3 = __fadd_rn(__fadd_rn(t1, L), cc);
            H = __fadd_rn(s1, t3);
            L = __fsub_rn(t3, __fsub_rn(H, s1));
        }
    }
    const double R2 = sd.R2;
    const DecideConsts &dc = sd.dc;
    float d2 = 0.f;
    int v = decide_df(H, L, nz, dc, &d2);
    if (v == 2) {
        double S = 0.0;
        for (int k = 0; k < d; ++k) {
            const double t = __dsub_rn((double)sd.x_raw[int64_t(e.y) * dp + k],
                                       (double)sd.q_raw[ql * dp + k]);
            S = __dadd_rn(S, __dmul_rn(t, t));
        }
        v = S <= R2 ? 1 : 0;
        d2 = (float)S;
    }
    const bool accept = v == 1;
    int32_t p0 = -1, p1 = -1;
    if (accept) {
        const int64_t row = sd.q_glob + sd.q_order[ql];
        p0 = atomicAdd(&counts[row], 1);
        if (sd.sym && int64_t(e.y) != ql) p1 = atomicAdd(&counts[sd.q_glob + sd.x_order[e.y]], 1);
    }
    rec_d2[s] = d2;
    rec_pos[s] = p0;
    rec_pos[cap + s] = p1;
}

__device__ __forceinline__ void b_scatter_one(int64_t s, int64_t cap, const uint2 *__restrict__ surv,
                                              const SetDesc *__restrict__ sets,
                                              const int32_t *__restrict__ qset,
                                              const float *__restrict__ rec_d2,
                                              const int32_t *__restrict__ rec_pos,
                                              const int64_t *__restrict__ offsets,
                                              uint64_t *__restrict__ tmp);

// Survivors min(*count, cap), grid-stride; nothing when *skip (a plan whose
// capacities were exceeded) is set.
__global__ void k_b_scatter(const uint2 *__restrict__ surv, const unsigned long long *__restrict__ count,
                            int64_t cap, const SetDesc *__restrict__ sets,
                            const int32_t *__restrict__ qset, const float *__restrict__ rec_d2,
                            const int32_t *__restrict__ rec_pos, const int64_t *__restrict__ offsets,
                            uint64_t *__restrict__ tmp, const int *__restrict__ skip) {
    if (skip && *skip) return;
    const int64_t nsurv = min((int64_t)*count, cap);
    for (int64_t s = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; s < nsurv;
         s += int64_t(gridDim.x) * blockDim.x)
        b_scatter_one(s, cap, surv, sets, qset, rec_d2, rec_pos, offsets, tmp);
}

__device__ __forceinline__ void b_scatter_one(int64_t s, int64_t cap, const uint2 *__restrict__ surv,
                                              const SetDesc *__restrict__ sets,
                                              const int32_t *__restrict__ qset,
                                              const float *__restrict__ rec_d2,
                                              const int32_t *__restrict__ rec_pos,
                                              const int64_t *__restrict__ offsets,
                                              uint64_t *__restrict__ tmp) {
    const int32_t p0 = rec_pos[s];
    if (p0 < 0) return;
    const uint2 e = surv[s];
    const SetDesc &sd = sets[qset[e.x]];
    const int64_t ql = int64_t(e.x) - sd.q_glob;
    const int32_t qrow = sd.q_order[ql], col = sd.x_order[e.y];
    const uint64_t vb = __float_as_uint(rec_d2[s]);
    tmp[offsets[sd.q_glob + qrow] + p0] = (uint64_t(uint32_t(col)) << 32) | vb;
    const int32_t p1 = rec_pos[cap + s];
    if (p1 >= 0) tmp[offsets[sd.q_glob + col] + p1] = (uint64_t(uint32_t(qrow)) << 32) | vb;
}

// Per-set offsets, rebased to start at 0, into the output block: entry
// g - qglob[s] of set s for every global query g, then each set's end entry.
__global__ void k_b_offsets(const int64_t *__restrict__ goff, const int64_t *__restrict__ qglob,
                            int nsets, int64_t total, int64_t *__restrict__ out_off,
                            const int64_t *__restrict__ out_off_pos) {
    const int64_t g = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (g >= total) return;
    const int s = find_set(qglob, nsets, g);
    out_off[out_off_pos[s] + (g - qglob[s])] = goff[g] - goff[qglob[s]];
}

__global__ void k_b_offsets_end(const int64_t *__restrict__ goff, const int64_t *__restrict__ qglob,
                                int nsets, int64_t *__restrict__ out_off,
                                const int64_t *__restrict__ out_off_pos) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nsets) return;
    out_off[out_off_pos[s] + (qglob[s + 1] - qglob[s])] = goff[qglob[s + 1]] - goff[qglob[s]];
}

}  // namespace

// Host side of snn_query_radius_batch.
// Exclusive bound on the point ids in any set's rows (selects the per-row
// sort's key width).
static uint32_t ids_bound(const std::vector<SetDesc> &sd) {
    int64_t n = 0;
    for (const SetDesc &d : sd) n = std::max<int64_t>(n, d.n);
    return uint32_t(n);
}

snn_status batch_query(int32_t nsets, const snn_index *const *idx, const float *const *Q,
                       const int64_t *m_in, const int64_t *ldq_in, const double *R_in,
                       cudaStream_t s, snn_csr *out) {
    NvtxPhase nvtx_("snn batched query");
    for (int32_t t = 0; t < nsets; ++t) std::memset(&out[t], 0, sizeof(out[t]));
    if (nsets == 0) return SNN_OK;
    // ------------------------------------------------------- host plan
    std::vector<SetDesc> sd(nsets);
    std::vector<int64_t> qglob(nsets + 1, 0), tile0(nsets + 1, 0);
    std::vector<OosDesc> od;
    std::vector<int64_t> ooff(1, 0);
    std::vector<int> oos_of(nsets, -1);
    int64_t oos_elems = 0;
    for (int32_t t = 0; t < nsets; ++t) {
        const snn_index *ix = idx[t];
        if (!ix) { set_error("set %d: index is NULL", t); return SNN_EINVAL; }
        if (!(R_in[t] >= 0.0) || !std::isfinite(R_in[t])) {
            set_error("set %d: R must be finite and >= 0", t);
            return SNN_EINVAL;
        }
        const bool self = Q[t] == nullptr;
        const int64_t m = self ? ix->n : m_in[t];
        if (!self && (m < 0 || m >= (int64_t(1) << 31))) {
            set_error("set %d: m must be in [0, 2^31)", t);
            return SNN_EINVAL;
        }
        if (!self && m > 0 && ldq_in[t] < ix->d) { set_error("set %d: ldq must be >= d", t); return SNN_EINVAL; }
        SetDesc &d = sd[t];
        std::memset(&d, 0, sizeof(d));
        d.m = m;
        d.n = ix->n;
        d.d = ix->d;
        d.dp = ix->dp;
        d.sym = self ? 1 : 0;
        d.c1 = (float)((2.0 * ix->d + 4.0) * (double)kU32 * 1.05);
        d.q_glob = qglob[t];
        d.tile0 = tile0[t];
        d.R2 = R_in[t] * R_in[t];
        d.dc = decide_consts(d.d, d.R2);
        d.Rx = R_in[t] * (1.0 + (ix->d + 8) * 0x1p-52);
        d.Wbase = d.Rx * (1.0 + (ix->d + 4) * 0x1p-52) * (1.0 + 0x1p-30);
        d.e_data = 1.0001 * (double)kU32 * (double)ix->nrm_max;
        d.x_alpha = ix->alpha;
        d.x_raw = ix->praw;
        d.x_xc = ix->xc;
        d.x_hx = ix->hx;
        d.x_nrm = ix->nrm;
        d.x_order = ix->order;
        d.eps_d = ix->dconst;
        if (self) {
            d.q_alpha = ix->alpha;
            d.q_raw = ix->praw;
            d.q_xc = ix->xc;
            d.q_hx = ix->hx;
            d.q_nrm = ix->nrm;
            d.q_order = ix->order;
            d.eps_q = ix->dconst;
        } else if (m > 0) {
            OosDesc o;
            o.Q = Q[t];
            o.ldq = ldq_in[t];
            o.cvec = ix->mu32;
            o.v32 = ix->v32;
            o.d = ix->d;
            o.dp = ix->dp;
            o.set = t;
            o.elem_off = oos_elems;
            oos_of[t] = int(od.size());
            od.push_back(o);
            ooff.push_back(ooff.back() + m);
            oos_elems += m * ix->dp;
        }
        qglob[t + 1] = qglob[t] + m;
        tile0[t + 1] = tile0[t] + cdiv(m, kBQ);
    }
    const int64_t M = qglob[nsets];
    const int64_t ntiles = tile0[nsets];
    const int noos = int(od.size());
    const int64_t Moos = ooff.back();

    Scratch scr(s);
    std::vector<void *> to_free;
    // ------------------------------------------- out-of-sample query prep
    float *q_alpha = nullptr, *q_raw = nullptr, *q_xc = nullptr, *q_hx = nullptr, *q_nrm = nullptr;
    int32_t *q_order = nullptr;
    float *oeps = nullptr;
    int *bad = nullptr;
    SNN_TRY(scr.alloc(&bad, 1));
    SNN_CUDA(cudaMemsetAsync(bad, 0, sizeof(int), s));
    if (noos > 0) {
        OosDesc *d_od;
        int64_t *d_ooff;
        uint64_t *keys, *keys_alt;
        uint32_t *vals, *vals_alt;
        SNN_TRY(scr.alloc(&d_od, noos));
        SNN_TRY(scr.alloc(&d_ooff, noos + 1));
        SNN_TRY(scr.alloc(&oeps, noos));
        SNN_TRY(scr.alloc(&keys, Moos));
        SNN_TRY(scr.alloc(&keys_alt, Moos));
        SNN_TRY(scr.alloc(&vals, Moos));
        SNN_TRY(scr.alloc(&vals_alt, Moos));
        SNN_TRY(scr.alloc(&q_alpha, Moos));
        SNN_TRY(scr.alloc(&q_order, Moos));
        SNN_TRY(scr.alloc(&q_hx, Moos));
        SNN_TRY(scr.alloc(&q_nrm, Moos));
        SNN_TRY(scr.alloc(&q_raw, oos_elems));
        SNN_TRY(scr.alloc(&q_xc, oos_elems));
        SNN_CUDA(cudaMemcpyAsync(d_od, od.data(), noos * sizeof(OosDesc), cudaMemcpyHostToDevice, s));
        SNN_CUDA(cudaMemcpyAsync(d_ooff, ooff.data(), (noos + 1) * sizeof(int64_t),
                                 cudaMemcpyHostToDevice, s));
        SNN_CUDA(cudaMemsetAsync(oeps, 0, noos * sizeof(float), s));
        SNN_LAUNCH(k_b_project, unsigned(cdiv(Moos, 256)), 256, 0, s)(d_od, d_ooff, noos, Moos, keys,
                                                                      vals, oeps, bad);
        SNN_LAUNCH_CHECK();
        int bits = 32;
        while ((int64_t(1) << (bits - 32)) < noos) ++bits;
        SNN_TRY(radix_sort_pairs<uint64_t>(keys, vals, keys_alt, vals_alt, Moos, bits, s));
        SNN_LAUNCH(k_b_gather, unsigned(cdiv(Moos, 256)), 256, 0, s)(
            d_od, d_ooff, noos, Moos, keys, vals, q_alpha, q_order, q_raw, q_xc, q_hx, q_nrm);
        SNN_LAUNCH_CHECK();
        // NaN/Inf and norm range of the queries, checked before any scoring
        float *qnmax;
        SNN_TRY(scr.alloc(&qnmax, 1));
        SNN_CUDA(cudaMemsetAsync(qnmax, 0, sizeof(float), s));
        SNN_LAUNCH(k_max_nonneg, std::min<unsigned>(unsigned(cdiv(Moos, 256)), 1024u), 256, 0, s)(
            q_nrm, Moos, qnmax);
        SNN_LAUNCH_CHECK();
        float hq = 0.f;
        int hb = 0;
        SNN_CUDA(cudaMemcpyAsync(&hq, qnmax, sizeof(float), cudaMemcpyDeviceToHost, s));
        SNN_CUDA(cudaMemcpyAsync(&hb, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
        SNN_CUDA(cudaStreamSynchronize(s));
        if (hb) { set_error("a query set contains NaN or Inf"); return SNN_EINVAL; }
        if (!(hq <= kMaxCentredNorm)) {
            set_error("a centred query norm of %g exceeds %g", (double)hq, kMaxCentredNorm);
            return SNN_ENOTSUP;
        }
        for (int32_t t = 0; t < nsets; ++t) {
            const int r = oos_of[t];
            if (r < 0) continue;
            SetDesc &d = sd[t];
            d.q_alpha = q_alpha + ooff[r];
            d.q_order = q_order + ooff[r];
            d.q_hx = q_hx + ooff[r];
            d.q_nrm = q_nrm + ooff[r];
            d.q_raw = q_raw + od[r].elem_off;
            d.q_xc = q_xc + od[r].elem_off;
            d.eps_q = oeps + r;
        }
    }
    // sets with m == 0 and no self-join keep NULL query arrays; they own no tiles
    SetDesc *d_sets;
    int64_t *d_qglob, *d_tile0;
    SNN_TRY(scr.alloc(&d_sets, nsets));
    SNN_TRY(scr.alloc(&d_qglob, nsets + 1));
    SNN_TRY(scr.alloc(&d_tile0, nsets + 1));
    SNN_CUDA(cudaMemcpyAsync(d_sets, sd.data(), nsets * sizeof(SetDesc), cudaMemcpyHostToDevice, s));
    SNN_CUDA(cudaMemcpyAsync(d_qglob, qglob.data(), (nsets + 1) * sizeof(int64_t),
                             cudaMemcpyHostToDevice, s));
    SNN_CUDA(cudaMemcpyAsync(d_tile0, tile0.data(), (nsets + 1) * sizeof(int64_t),
                             cudaMemcpyHostToDevice, s));

    // ------------------------------------------------ thresholds, bands
    int32_t *qset, *tile_set;
    float *thrA;
    int64_t *tile_lo, *tile_hi, *items, *item_off;
    unsigned long long *ctr;
    SNN_TRY(scr.alloc(&qset, M));
    SNN_TRY(scr.alloc(&thrA, M));
    SNN_TRY(scr.alloc(&tile_set, ntiles));
    SNN_TRY(scr.alloc(&tile_lo, ntiles));
    SNN_TRY(scr.alloc(&tile_hi, ntiles));
    SNN_TRY(scr.alloc(&items, ntiles));
    SNN_TRY(scr.alloc(&item_off, ntiles + 1));
    SNN_TRY(scr.alloc(&ctr, 4));
    SNN_CUDA(cudaMemsetAsync(ctr, 0, 4 * sizeof(unsigned long long), s));
    if (M > 0) {
        SNN_LAUNCH(k_b_qset, unsigned(cdiv(M, 256)), 256, 0, s)(d_qglob, nsets, M, qset);
        SNN_LAUNCH(k_b_consts, unsigned(cdiv(M, 256)), 256, 0, s)(d_sets, qset, M, thrA);
        SNN_LAUNCH(k_b_tileset, unsigned(cdiv(ntiles, 256)), 256, 0, s)(d_tile0, nsets, ntiles,
                                                                         tile_set);
        SNN_LAUNCH(k_b_band, unsigned(cdiv(ntiles, 128)), 128, 0, s)(d_sets, tile_set, ntiles,
                                                                     tile_lo, tile_hi, items,
                                                                     kChunksPerItem);
        SNN_LAUNCH_CHECK();
    }
    SNN_TRY(scan_exclusive<int64_t>(items, item_off, ntiles, s));
    int64_t max_items = 0;
    for (int32_t t = 0; t < nsets; ++t)
        max_items += cdiv(sd[t].m, kBQ) * (cdiv(sd[t].n, int64_t(kBR) * kChunksPerItem) + 1);
    int32_t *item_tile;
    SNN_TRY(scr.alloc(&item_tile, std::max<int64_t>(max_items, 1)));
    if (ntiles > 0) {
        SNN_LAUNCH(k_item_tiles, unsigned(cdiv(ntiles, 128)), 128, 0, s)(item_off, int(ntiles),
                                                                          item_tile);
        SNN_LAUNCH_CHECK();
    }

    // ------------------------------------- one persistent scoring launch
    int64_t cap = std::max<int64_t>(int64_t(1) << 20, 64 * M + 4096);
    uint2 *surv = nullptr;
    SNN_TRY(scr.alloc(&surv, cap));
    BatchScoreArgs ba;
    ba.sets = d_sets;
    ba.tile_set = tile_set;
    ba.thrA = thrA;
    ba.tile_lo = tile_lo;
    ba.tile_hi = tile_hi;
    ba.item_off = item_off;
    ba.item_tile = item_tile;
    ba.ntiles = int(ntiles);
    ba.cpi = kChunksPerItem;
    ba.count = ctr;
    ba.work = ctr + 1;
    unsigned long long hctr[2] = {0, 0};
    int hbad = 0;
    for (int attempt = 0; attempt < 2; ++attempt) {
        ba.surv = surv;
        ba.cap = cap;
        if (ntiles > 0) {
            SNN_LAUNCH(k_score_fp32_batch, device_sm_count() * 2, 256, 0, s)(ba);
            SNN_LAUNCH_CHECK();
        }
        SNN_CUDA(cudaMemcpyAsync(hctr, ctr, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
        SNN_CUDA(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
        SNN_CUDA(cudaStreamSynchronize(s));
        if (hbad) { set_error("a query set contains NaN or Inf"); return SNN_EINVAL; }
        if ((int64_t)hctr[0] <= cap) break;
        if (attempt == 1) { set_error("survivor buffer overflow after retry"); return SNN_EOVERFLOW; }
        cap = (int64_t)hctr[0] + 1024;
        SNN_TRY(scr.alloc(&surv, cap));
        SNN_CUDA(cudaMemsetAsync(ctr, 0, 2 * sizeof(unsigned long long), s));
    }
    const int64_t nsurv = (int64_t)hctr[0];

    // ------------------------------------------------- exact decision
    float *rec_d2;
    int32_t *rec_pos, *counts;
    int64_t *counts64, *goff;
    SNN_TRY(scr.alloc(&rec_d2, std::max<int64_t>(nsurv, 1)));
    SNN_TRY(scr.alloc(&rec_pos, 2 * std::max<int64_t>(nsurv, 1)));
    SNN_TRY(scr.alloc(&counts, M));
    SNN_TRY(scr.alloc(&counts64, M));
    SNN_TRY(scr.alloc(&goff, M + 1));
    SNN_CUDA(cudaMemsetAsync(counts, 0, std::max<int64_t>(M, 1) * sizeof(int32_t), s));
    if (nsurv > 0) {
        SNN_LAUNCH(k_b_decide, unsigned(cdiv(nsurv, 256)), 256, 0, s)(surv, ctr, nsurv, d_sets, qset,
                                                                      rec_d2, rec_pos, counts);
        SNN_LAUNCH_CHECK();
    }
    if (M > 0) {
        SNN_LAUNCH(k_counts_to_i64, unsigned(cdiv(M, 256)), 256, 0, s)(counts, M, counts64);
        SNN_LAUNCH_CHECK();
    }
    SNN_TRY(scan_exclusive<int64_t>(counts64, goff, M, s));
    int64_t nnz = 0;
    SNN_CUDA(cudaMemcpyAsync(&nnz, goff + M, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    SNN_CUDA(cudaStreamSynchronize(s));
    if (nnz >= (int64_t(1) << 31)) {
        set_error("%lld neighbour pairs exceed this build's limit of 2^31-1", (long long)nnz);
        return SNN_ENOTSUP;
    }
    // nnz of every set
    std::vector<int64_t> hgoff_set(nsets + 1);
    {
        int64_t *tmp;
        SNN_TRY(scr.alloc(&tmp, nsets + 1));
        for (int32_t t = 0; t <= nsets; ++t)
            SNN_CUDA(cudaMemcpyAsync(tmp + t, goff + qglob[t], sizeof(int64_t),
                                     cudaMemcpyDeviceToDevice, s));
        SNN_CUDA(cudaMemcpyAsync(hgoff_set.data(), tmp, (nsets + 1) * sizeof(int64_t),
                                 cudaMemcpyDeviceToHost, s));
        SNN_CUDA(cudaStreamSynchronize(s));
    }

    // ---------------------------- one output block, per-set slices of it
    std::vector<int64_t> off_pos(nsets);
    int64_t off_words = 0;
    for (int32_t t = 0; t < nsets; ++t) {
        off_pos[t] = off_words;
        off_words += (sd[t].m + 1 + 31) & ~int64_t(31);   // 256-byte aligned slices
    }
    const size_t idx_bytes = ((size_t(nnz) * 4 + 255) & ~size_t(255));
    const size_t bytes = size_t(off_words) * 8 + 2 * std::max<size_t>(idx_bytes, 256);
    char *block = nullptr;
    {
        cudaError_t e = cudaMallocAsync(reinterpret_cast<void **>(&block), bytes, s);
        if (e != cudaSuccess) {
            cudaGetLastError();
            set_error("output allocation of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
            return SNN_ENOMEM;
        }
    }
    int64_t *out_off = reinterpret_cast<int64_t *>(block);
    int32_t *gidx = reinterpret_cast<int32_t *>(block + size_t(off_words) * 8);
    float *gd2 = reinterpret_cast<float *>(block + size_t(off_words) * 8 + std::max<size_t>(idx_bytes, 256));
    int64_t *d_offpos;
    snn_status st = scr.alloc(&d_offpos, nsets);
    auto fail = [&](snn_status code) {
        cudaFreeAsync(block, s);
        return code;
    };
    if (st != SNN_OK) return fail(st);
    if (cudaMemcpyAsync(d_offpos, off_pos.data(), nsets * sizeof(int64_t), cudaMemcpyHostToDevice, s) !=
        cudaSuccess) {
        set_error("offset table upload failed");
        return fail(SNN_ECUDA);
    }
    if (M > 0)
        SNN_LAUNCH(k_b_offsets, unsigned(cdiv(M, 256)), 256, 0, s)(goff, d_qglob, nsets, M, out_off,
                                                                   d_offpos);
    SNN_LAUNCH(k_b_offsets_end, unsigned(cdiv(nsets, 128)), 128, 0, s)(goff, d_qglob, nsets, out_off,
                                                                       d_offpos);
    if (nsurv > 0 && nnz > 0) {
        uint64_t *tmp;
        if ((st = scr.alloc(&tmp, nnz)) != SNN_OK) return fail(st);
        SNN_LAUNCH(k_b_scatter, unsigned(cdiv(nsurv, 256)), 256, 0, s)(
            surv, ctr, nsurv, d_sets, qset, rec_d2, rec_pos, goff, tmp, nullptr);
        // per-row ascending ids over the global CSR (rows of every set)
        ulonglong2 *lists;
        int32_t *big_list;
        int64_t *big_len, *toff;
        unsigned *cls;
        st = scr.alloc(&lists, int64_t(kSegSlotsFine) * M);
        if (st == SNN_OK) st = scr.alloc(&big_list, M);
        if (st == SNN_OK) st = scr.alloc(&big_len, M);
        if (st == SNN_OK) st = scr.alloc(&toff, M + 1);
        if (st == SNN_OK) st = scr.alloc(&cls, kSegClasses);
        if (st != SNN_OK) return fail(st);
        cudaMemsetAsync(cls, 0, kSegClasses * sizeof(unsigned), s);
        const SegMap gm{goff, goff, nullptr};
        SNN_LAUNCH(k_seg_classify, unsigned(cdiv(M, 256)), 256, 0, s)(gm, M, 1, lists, big_list, big_len,
                                                                      cls);
        seg_sort_launch(lists, cls, M, tmp, gidx, gd2, ids_bound(sd), s);
        unsigned hcls[kSegClasses];
        if (cudaMemcpyAsync(hcls, cls, sizeof(hcls), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess) {
            set_error("batched CSR build failed: %s", cudaGetErrorString(cudaGetLastError()));
            return fail(SNN_ECUDA);
        }
        const int nbig = int(hcls[4]);
        if (nbig > 0) {
            // rows longer than 4096 entries: radix sort of (row rank, id)
            if ((st = scan_exclusive<int64_t>(big_len, toff, nbig, s)) != SNN_OK) return fail(st);
            int64_t tot = 0;
            cudaMemcpyAsync(&tot, toff + nbig, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
            cudaStreamSynchronize(s);
            uint64_t *bk, *bka;
            uint32_t *bv, *bva;
            float *bd2;
            st = scr.alloc(&bk, tot);
            if (st == SNN_OK) st = scr.alloc(&bka, tot);
            if (st == SNN_OK) st = scr.alloc(&bv, tot);
            if (st == SNN_OK) st = scr.alloc(&bva, tot);
            if (st == SNN_OK) st = scr.alloc(&bd2, tot);
            if (st != SNN_OK) return fail(st);
            SNN_LAUNCH(k_seg_big_gather, nbig, 256, 0, s)(big_list, nbig, gm, toff, tmp, bk, bv, bd2);
            int bits = 32;
            while ((int64_t(1) << (bits - 32)) < nbig) ++bits;
            if ((st = radix_sort_pairs<uint64_t>(bk, bv, bka, bva, tot, bits, s)) != SNN_OK)
                return fail(st);
            SNN_LAUNCH(k_seg_big_scatter, unsigned(cdiv(tot, 256)), 256, 0, s)(
                bk, bv, tot, big_list, gm, toff, bd2, gidx, gd2);
        }
    }
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) {
        set_error("batched CSR build failed");
        return fail(SNN_ECUDA);
    }
    // hand out the slices; the block is freed when every slice was freed
    std::vector<void *> ptrs;
    for (int32_t t = 0; t < nsets; ++t) {
        const int64_t nz = hgoff_set[t + 1] - hgoff_set[t];
        out[t].m = sd[t].m;
        out[t].nnz = nz;
        out[t].offsets = out_off + off_pos[t];
        out[t].indices = nz > 0 ? gidx + hgoff_set[t] : nullptr;
        out[t].dist2 = nz > 0 ? gd2 + hgoff_set[t] : nullptr;
        ptrs.push_back(out[t].offsets);
        if (nz > 0) {
            ptrs.push_back(out[t].indices);
            ptrs.push_back(out[t].dist2);
        }
    }
    st = register_block(block, ptrs.data(), int(ptrs.size()), s);
    if (st != SNN_OK) {
        for (int32_t t = 0; t < nsets; ++t) std::memset(&out[t], 0, sizeof(out[t]));
        return fail(st);
    }
    return SNN_OK;
}

// ---------------------------------------------------------- batch plan
// A batched query with every size fixed in advance (queries per set, the
// survivor and neighbour capacities), so that one run is a pure sequence of
// stream-ordered device work: no host synchronisation, no host-dependent
// sizes.  It can be captured into a CUDA graph and replayed with new query
// values written into the plan's query buffers.  Capacities that turn out too
// small, NaN/Inf queries and rows longer than 4096 neighbours are reported in
// a device status word that snn_batch_plan_result reads.

// Status of a run, decided on the device after the row classification: when
// a capacity is exceeded (or a row needs the long-row radix path) the CSR
// build is skipped (the scatter checks *skip, the sorts see empty classes).
struct PlanStatus {
    unsigned long long surv;   // survivors counted
    long long nnz;             // neighbour entries counted
    int bad;                   // NaN/Inf in a query set
    int big;                   // rows longer than 4096 entries
    int skip;                  // the CSR build was skipped
    float qnorm;               // largest centred query norm
    int tcerr;                 // tensor-core groups: 1 a bounded wait expired, 2 a query beyond FP16
};

__global__ void k_plan_guard(const unsigned long long *__restrict__ ctr,
                             const int64_t *__restrict__ nnz, unsigned *__restrict__ cls,
                             const int *__restrict__ bad, const float *__restrict__ qnmax,
                             const int *__restrict__ tcerr, int64_t surv_cap, int64_t nnz_cap,
                             PlanStatus *__restrict__ st) {
    const unsigned long long sv = ctr[0];
    const long long nz = *nnz;
    const int big = cls[4] > 0;
    const int skip = sv > (unsigned long long)surv_cap || nz > nnz_cap || big || *bad ||
                     !(*qnmax <= (float)kMaxCentredNorm) || *tcerr;
    st->surv = sv;
    st->nnz = nz;
    st->bad = *bad;
    st->big = big;
    st->skip = skip;
    st->qnorm = *qnmax;
    st->tcerr = *tcerr;
    if (skip)
        for (int k = 0; k < kSegClasses; ++k) cls[k] = 0;
}

// set_nnz[t] = first global neighbour entry of set t (t <= nsets).
__global__ void k_plan_set_nnz(const int64_t *__restrict__ goff, const int64_t *__restrict__ qglob,
                               int nsets, int64_t *__restrict__ set_nnz) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t <= nsets) set_nnz[t] = goff[qglob[t]];
}

}  // namespace snn

struct snn_batch_plan {
    int32_t nsets = 0;
    int device = 0;
    snn_precision prec = SNN_PREC_FP32;
    std::vector<snn::SetDesc> sd;
    std::vector<snn::OosDesc> od;
    std::vector<int64_t> qglob, tile0, ooff, off_pos, qbuf_off;
    std::vector<int> oos_of;
    int64_t M = 0, ntiles = 0, Moos = 0, oos_elems = 0, off_words = 0, max_items = 0;
    int noos = 0;
    int64_t surv_cap = 0, nnz_cap = 0;
    int cpi = snn::kChunksPerItem;   // tuned: band chunks per scoring item
    int ctas_per_sm = 2;             // tuned: persistent scoring grid
    // tensor-core groups (16-bit precision): out-of-sample sets of d <= 48 by
    // fold column; tc_mask bit k: group k scores its sets (else they go to
    // the FP32 scorer)
    std::vector<snn::TcBatchGroup *> tc_groups;
    unsigned tc_mask = 0;
    int *tc_err = nullptr;
    int tuned_from_cache = 0;
    std::vector<void *> blocks;      // pool blocks owned by the plan
    // device arrays
    float *qbuf = nullptr;
    snn::OosDesc *d_od = nullptr;
    int64_t *d_ooff = nullptr;
    float *oeps = nullptr, *q_alpha = nullptr, *q_raw = nullptr, *q_xc = nullptr, *q_hx = nullptr,
          *q_nrm = nullptr, *qnmax = nullptr, *thrA = nullptr, *rec_d2 = nullptr, *gd2 = nullptr;
    int32_t *q_order = nullptr, *qset = nullptr, *tile_set = nullptr, *item_tile = nullptr,
            *rec_pos = nullptr, *counts = nullptr, *big_list = nullptr, *gidx = nullptr;
    ulonglong2 *lists = nullptr;
    uint64_t *keys = nullptr, *keys_alt = nullptr, *tmp = nullptr;
    uint32_t *vals = nullptr, *vals_alt = nullptr;
    int *bad = nullptr;
    snn::SetDesc *d_sets = nullptr;
    int64_t *d_qglob = nullptr, *d_tile0 = nullptr, *tile_lo = nullptr, *tile_hi = nullptr,
            *items = nullptr, *item_off = nullptr, *counts64 = nullptr, *goff = nullptr,
            *big_len = nullptr, *toff = nullptr, *out_off = nullptr, *d_offpos = nullptr,
            *set_nnz = nullptr;
    unsigned long long *ctr = nullptr;
    uint2 *surv = nullptr;
    unsigned *cls = nullptr;
    snn::PlanStatus *status = nullptr;
    // graph of one run
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    unsigned long long graph_launches = 0;   // kernels in the graph
};

namespace snn {

void note_launches(unsigned long long k);
unsigned long long launch_count_now();

namespace {

template <typename T>
snn_status plan_alloc(snn_batch_plan *p, T **ptr, int64_t count, cudaStream_t s) {
    void *q = nullptr;
    const size_t bytes = (std::max<size_t>(size_t(count) * sizeof(T), 16) + 255) & ~size_t(255);
    if (cudaMallocAsync(&q, bytes, s) != cudaSuccess) {
        cudaGetLastError();
        set_error("plan allocation of %zu bytes failed", bytes);
        return SNN_ENOMEM;
    }
    p->blocks.push_back(q);
    *ptr = static_cast<T *>(q);
    return SNN_OK;
}

// One run, enqueued on s: no synchronisation, every size from the plan.
snn_status plan_enqueue(snn_batch_plan *p, cudaStream_t s) {
    NvtxPhase nvtx_("snn batch plan run");
    const int nsets = p->nsets;
    const int64_t M = p->M, ntiles = p->ntiles, Moos = p->Moos;
    SNN_CUDA(cudaMemsetAsync(p->bad, 0, sizeof(int), s));
    SNN_CUDA(cudaMemsetAsync(p->qnmax, 0, sizeof(float), s));
    SNN_CUDA(cudaMemsetAsync(p->tc_err, 0, sizeof(int), s));
    if (p->noos > 0) {
        SNN_CUDA(cudaMemsetAsync(p->oeps, 0, p->noos * sizeof(float), s));
        SNN_LAUNCH(k_b_project, unsigned(cdiv(Moos, 256)), 256, 0, s)(p->d_od, p->d_ooff, p->noos, Moos,
                                                                      p->keys, p->vals, p->oeps, p->bad);
        SNN_LAUNCH_CHECK();
        int bits = 32;
        while ((int64_t(1) << (bits - 32)) < p->noos) ++bits;
        // (a bounded wait of the sort that gives up sets bit 0 of tc_err)
        SNN_TRY(radix_sort_pairs<uint64_t>(p->keys, p->vals, p->keys_alt, p->vals_alt, Moos, bits, s, p->tc_err));
        SNN_LAUNCH(k_b_gather, unsigned(cdiv(Moos, 256)), 256, 0, s)(
            p->d_od, p->d_ooff, p->noos, Moos, p->keys, p->vals, p->q_alpha, p->q_order, p->q_raw,
            p->q_xc, p->q_hx, p->q_nrm);
        SNN_LAUNCH(k_max_nonneg, std::min<unsigned>(unsigned(cdiv(Moos, 256)), 1024u), 256, 0, s)(
            p->q_nrm, Moos, p->qnmax);
        SNN_LAUNCH_CHECK();
    }
    SNN_CUDA(cudaMemsetAsync(p->ctr, 0, 4 * sizeof(unsigned long long), s));
    if (M > 0) {
        SNN_LAUNCH(k_b_qset, unsigned(cdiv(M, 256)), 256, 0, s)(p->d_qglob, nsets, M, p->qset);
        SNN_LAUNCH(k_b_consts, unsigned(cdiv(M, 256)), 256, 0, s)(p->d_sets, p->qset, M, p->thrA);
        SNN_LAUNCH(k_b_tileset, unsigned(cdiv(ntiles, 256)), 256, 0, s)(p->d_tile0, nsets, ntiles,
                                                                         p->tile_set);
        SNN_LAUNCH(k_b_band, unsigned(cdiv(ntiles, 128)), 128, 0, s)(p->d_sets, p->tile_set, ntiles,
                                                                     p->tile_lo, p->tile_hi, p->items,
                                                                     p->cpi);
        SNN_LAUNCH_CHECK();
        SNN_TRY(scan_exclusive<int64_t>(p->items, p->item_off, ntiles, s));
        SNN_LAUNCH(k_item_tiles, unsigned(cdiv(ntiles, 128)), 128, 0, s)(p->item_off, int(ntiles),
                                                                          p->item_tile);
        BatchScoreArgs ba;
        ba.sets = p->d_sets;
        ba.tile_set = p->tile_set;
        ba.thrA = p->thrA;
        ba.tile_lo = p->tile_lo;
        ba.tile_hi = p->tile_hi;
        ba.item_off = p->item_off;
        ba.item_tile = p->item_tile;
        ba.ntiles = int(ntiles);
        ba.cpi = p->cpi;
        ba.surv = p->surv;
        ba.cap = p->surv_cap;
        ba.count = p->ctr;
        ba.work = p->ctr + 1;
        SNN_LAUNCH(k_score_fp32_batch, device_sm_count() * p->ctas_per_sm, 256, 0, s)(ba);
        SNN_LAUNCH_CHECK();
        // tensor-core groups append their survivors after the FP32 scorer's
        for (size_t k = 0; k < p->tc_groups.size(); ++k)
            if (p->tc_mask & (1u << k))
                SNN_TRY(tc_batch_enqueue(p->tc_groups[k], p->tile_lo, p->tile_hi, p->surv, p->surv_cap, p->ctr,
                                         p->tc_err, s));
    }
    SNN_CUDA(cudaMemsetAsync(p->counts, 0, std::max<int64_t>(M, 1) * sizeof(int32_t), s));
    SNN_LAUNCH(k_b_decide, unsigned(4 * device_sm_count()), 256, 0, s)(
        p->surv, p->ctr, p->surv_cap, p->d_sets, p->qset, p->rec_d2, p->rec_pos, p->counts);
    if (M > 0)
        SNN_LAUNCH(k_counts_to_i64, unsigned(cdiv(M, 256)), 256, 0, s)(p->counts, M, p->counts64);
    SNN_LAUNCH_CHECK();
    SNN_TRY(scan_exclusive<int64_t>(p->counts64, p->goff, M, s));
    SNN_CUDA(cudaMemsetAsync(p->cls, 0, kSegClasses * sizeof(unsigned), s));
    const SegMap gm{p->goff, p->goff, nullptr};
    if (M > 0) {
        SNN_CUDA(cudaMemsetAsync(p->big_len, 0, M * sizeof(int64_t), s));
        SNN_LAUNCH(k_seg_classify, unsigned(cdiv(M, 256)), 256, 0, s)(gm, M, 1, p->lists, p->big_list,
                                                                      p->big_len, p->cls);
    }
    SNN_LAUNCH(k_plan_guard, 1, 1, 0, s)(p->ctr, p->goff + M, p->cls, p->bad, p->qnmax, p->tc_err,
                                         p->surv_cap, p->nnz_cap, p->status);
    SNN_LAUNCH(k_b_scatter, unsigned(4 * device_sm_count()), 256, 0, s)(
        p->surv, p->ctr, p->surv_cap, p->d_sets, p->qset, p->rec_d2, p->rec_pos, p->goff, p->tmp,
        &p->status->skip);
    SNN_LAUNCH_CHECK();
    seg_sort_launch(p->lists, p->cls, M, p->tmp, p->gidx, p->gd2, ids_bound(p->sd), s);
    if (M > 0)
        SNN_LAUNCH(k_b_offsets, unsigned(cdiv(M, 256)), 256, 0, s)(p->goff, p->d_qglob, nsets, M,
                                                                   p->out_off, p->d_offpos);
    SNN_LAUNCH(k_b_offsets_end, unsigned(cdiv(nsets, 128)), 128, 0, s)(p->goff, p->d_qglob, nsets,
                                                                       p->out_off, p->d_offpos);
    SNN_LAUNCH(k_plan_set_nnz, unsigned(cdiv(nsets + 1, 128)), 128, 0, s)(p->goff, p->d_qglob, nsets,
                                                                          p->set_nnz);
    SNN_LAUNCH_CHECK();
    return SNN_OK;
}

}  // namespace

void plan_release(snn_batch_plan *p, cudaStream_t s) {
    if (!p) return;
    for (TcBatchGroup *g : p->tc_groups) tc_batch_release(g, s);
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->graph) cudaGraphDestroy(p->graph);
    for (void *b : p->blocks) cudaFreeAsync(b, s);
    delete p;
}

snn_status plan_create(int32_t nsets, const snn_index *const *idx, const int64_t *m_in,
                       const double *R_in, snn_precision prec, int64_t surv_cap, int64_t nnz_cap,
                       cudaStream_t s, snn_batch_plan **out) {
    *out = nullptr;
    snn_batch_plan *p = new (std::nothrow) snn_batch_plan();
    if (!p) {
        set_error("host allocation failed");
        return SNN_ENOMEM;
    }
    auto fail = [&](snn_status st) {
        cudaStreamSynchronize(s);
        plan_release(p, s);
        return st;
    };
    cudaGetDevice(&p->device);
    p->nsets = nsets;
    p->prec = prec;
    p->sd.resize(nsets);
    p->qglob.assign(nsets + 1, 0);
    p->tile0.assign(nsets + 1, 0);
    p->ooff.assign(1, 0);
    p->oos_of.assign(nsets, -1);
    p->qbuf_off.assign(nsets, -1);
    int64_t qelems = 0;
    for (int32_t t = 0; t < nsets; ++t) {
        const snn_index *ix = idx[t];
        if (!ix) { set_error("set %d: index is NULL", t); return fail(SNN_EINVAL); }
        if (!(R_in[t] >= 0.0) || !std::isfinite(R_in[t])) {
            set_error("set %d: R must be finite and >= 0", t);
            return fail(SNN_EINVAL);
        }
        const bool self = m_in[t] < 0;
        const int64_t m = self ? ix->n : m_in[t];
        if (m >= (int64_t(1) << 31)) { set_error("set %d: m must be < 2^31", t); return fail(SNN_EINVAL); }
        SetDesc &d = p->sd[t];
        std::memset(&d, 0, sizeof(d));
        d.m = m;
        d.n = ix->n;
        d.d = ix->d;
        d.dp = ix->dp;
        d.sym = self ? 1 : 0;
        d.c1 = (float)((2.0 * ix->d + 4.0) * (double)kU32 * 1.05);
        d.q_glob = p->qglob[t];
        d.tile0 = p->tile0[t];
        d.R2 = R_in[t] * R_in[t];
        d.dc = decide_consts(d.d, d.R2);
        d.Rx = R_in[t] * (1.0 + (ix->d + 8) * 0x1p-52);
        d.Wbase = d.Rx * (1.0 + (ix->d + 4) * 0x1p-52) * (1.0 + 0x1p-30);
        d.e_data = 1.0001 * (double)kU32 * (double)ix->nrm_max;
        d.x_alpha = ix->alpha;
        d.x_raw = ix->praw;
        d.x_xc = ix->xc;
        d.x_hx = ix->hx;
        d.x_nrm = ix->nrm;
        d.x_order = ix->order;
        d.eps_d = ix->dconst;
        if (self) {
            d.q_alpha = ix->alpha;
            d.q_raw = ix->praw;
            d.q_xc = ix->xc;
            d.q_hx = ix->hx;
            d.q_nrm = ix->nrm;
            d.q_order = ix->order;
            d.eps_q = ix->dconst;
        } else if (m > 0) {
            OosDesc o;
            o.Q = nullptr;   // set below (query buffer)
            o.ldq = ix->d;
            o.cvec = ix->mu32;
            o.v32 = ix->v32;
            o.d = ix->d;
            o.dp = ix->dp;
            o.set = t;
            o.elem_off = p->oos_elems;
            p->oos_of[t] = int(p->od.size());
            p->qbuf_off[t] = qelems;
            qelems += (m * ix->d + 63) & ~int64_t(63);
            p->od.push_back(o);
            p->ooff.push_back(p->ooff.back() + m);
            p->oos_elems += m * ix->dp;
        }
        p->qglob[t + 1] = p->qglob[t] + m;
        p->tile0[t + 1] = p->tile0[t] + cdiv(m, kBQ);
    }
    p->M = p->qglob[nsets];
    p->ntiles = p->tile0[nsets];
    p->noos = int(p->od.size());
    p->Moos = p->ooff.back();
    const int64_t M = p->M;
    p->surv_cap = std::max<int64_t>(surv_cap, 1024);
    p->nnz_cap = std::max<int64_t>(nnz_cap, 1024);
    // worst-case item count of the smallest granularity the tuner may pick
    for (int32_t t = 0; t < nsets; ++t)
        p->max_items += cdiv(p->sd[t].m, kBQ) * (cdiv(p->sd[t].n, int64_t(kBR) * 4) + 1);
    // per-set output offsets: 256-byte aligned slices
    p->off_pos.resize(nsets);
    for (int32_t t = 0; t < nsets; ++t) {
        p->off_pos[t] = p->off_words;
        p->off_words += (p->sd[t].m + 1 + 31) & ~int64_t(31);
    }
    // ---------------------------------------------------- device memory
#define PTRY(expr)                               \
    do {                                         \
        snn_status _st = (expr);                 \
        if (_st != SNN_OK) return fail(_st);     \
    } while (0)
    PTRY(plan_alloc(p, &p->qbuf, qelems, s));
    PTRY(plan_alloc(p, &p->bad, 1, s));
    PTRY(plan_alloc(p, &p->qnmax, 1, s));
    if (p->noos > 0) {
        for (int32_t t = 0; t < nsets; ++t)
            if (p->oos_of[t] >= 0) p->od[p->oos_of[t]].Q = p->qbuf + p->qbuf_off[t];
        PTRY(plan_alloc(p, &p->d_od, p->noos, s));
        PTRY(plan_alloc(p, &p->d_ooff, p->noos + 1, s));
        PTRY(plan_alloc(p, &p->oeps, p->noos, s));
        PTRY(plan_alloc(p, &p->keys, p->Moos, s));
        PTRY(plan_alloc(p, &p->keys_alt, p->Moos, s));
        PTRY(plan_alloc(p, &p->vals, p->Moos, s));
        PTRY(plan_alloc(p, &p->vals_alt, p->Moos, s));
        PTRY(plan_alloc(p, &p->q_alpha, p->Moos, s));
        PTRY(plan_alloc(p, &p->q_order, p->Moos, s));
        PTRY(plan_alloc(p, &p->q_hx, p->Moos, s));
        PTRY(plan_alloc(p, &p->q_nrm, p->Moos, s));
        PTRY(plan_alloc(p, &p->q_raw, p->oos_elems, s));
        PTRY(plan_alloc(p, &p->q_xc, p->oos_elems, s));
        for (int32_t t = 0; t < nsets; ++t) {
            const int r = p->oos_of[t];
            if (r < 0) continue;
            SetDesc &d = p->sd[t];
            d.q_alpha = p->q_alpha + p->ooff[r];
            d.q_order = p->q_order + p->ooff[r];
            d.q_hx = p->q_hx + p->ooff[r];
            d.q_nrm = p->q_nrm + p->ooff[r];
            d.q_raw = p->q_raw + p->od[r].elem_off;
            d.q_xc = p->q_xc + p->od[r].elem_off;
            d.eps_q = p->oeps + r;
        }
    }
    PTRY(plan_alloc(p, &p->d_sets, nsets, s));
    PTRY(plan_alloc(p, &p->d_qglob, nsets + 1, s));
    PTRY(plan_alloc(p, &p->d_tile0, nsets + 1, s));
    PTRY(plan_alloc(p, &p->qset, M, s));
    PTRY(plan_alloc(p, &p->thrA, M, s));
    PTRY(plan_alloc(p, &p->tile_set, p->ntiles, s));
    PTRY(plan_alloc(p, &p->tile_lo, p->ntiles, s));
    PTRY(plan_alloc(p, &p->tile_hi, p->ntiles, s));
    PTRY(plan_alloc(p, &p->items, p->ntiles, s));
    PTRY(plan_alloc(p, &p->item_off, p->ntiles + 1, s));
    PTRY(plan_alloc(p, &p->item_tile, std::max<int64_t>(p->max_items, 1), s));
    PTRY(plan_alloc(p, &p->ctr, 4, s));
    PTRY(plan_alloc(p, &p->surv, p->surv_cap, s));
    PTRY(plan_alloc(p, &p->rec_d2, p->surv_cap, s));
    PTRY(plan_alloc(p, &p->rec_pos, 2 * p->surv_cap, s));
    PTRY(plan_alloc(p, &p->counts, M, s));
    PTRY(plan_alloc(p, &p->counts64, M, s));
    PTRY(plan_alloc(p, &p->goff, M + 1, s));
    PTRY(plan_alloc(p, &p->lists, int64_t(kSegSlotsFine) * std::max<int64_t>(M, 1), s));
    PTRY(plan_alloc(p, &p->big_list, M, s));
    PTRY(plan_alloc(p, &p->big_len, M, s));
    PTRY(plan_alloc(p, &p->toff, M + 1, s));
    PTRY(plan_alloc(p, &p->cls, kSegClasses, s));
    PTRY(plan_alloc(p, &p->tmp, p->nnz_cap, s));
    PTRY(plan_alloc(p, &p->out_off, p->off_words, s));
    PTRY(plan_alloc(p, &p->gidx, p->nnz_cap, s));
    PTRY(plan_alloc(p, &p->gd2, p->nnz_cap, s));
    PTRY(plan_alloc(p, &p->d_offpos, nsets, s));
    PTRY(plan_alloc(p, &p->set_nnz, nsets + 1, s));
    PTRY(plan_alloc(p, &p->status, 1, s));
    PTRY(plan_alloc(p, &p->tc_err, 1, s));
    if (prec != SNN_PREC_FP32) {
        // tensor-core groups: out-of-sample sets of d <= 48 by fold column
        // (d rounded up to 16), two FP16 parts of each set's scaled rows
        std::vector<int> grp[3];
        for (int32_t t = 0; t < nsets; ++t) {
            const SetDesc &d = p->sd[t];
            if (d.sym || d.m <= 0 || d.d > 48) continue;
            grp[d.d <= 16 ? 0 : (d.d <= 32 ? 1 : 2)].push_back(t);
        }
        for (int k = 0; k < 3; ++k) {
            if (grp[k].empty()) continue;
            TcBatchGroup *g = nullptr;
            PTRY(tc_batch_create(idx, p->sd.data(), grp[k].data(), int(grp[k].size()), 16 * (k + 1), s, &g));
            p->tc_mask |= 1u << p->tc_groups.size();
            p->tc_groups.push_back(g);
            for (int t : grp[k]) p->sd[t].tc = 1;
        }
    }
#undef PTRY
    if ((p->noos > 0 &&
         (cudaMemcpyAsync(p->d_od, p->od.data(), p->noos * sizeof(OosDesc), cudaMemcpyHostToDevice,
                          s) != cudaSuccess ||
          cudaMemcpyAsync(p->d_ooff, p->ooff.data(), (p->noos + 1) * sizeof(int64_t),
                          cudaMemcpyHostToDevice, s) != cudaSuccess)) ||
        cudaMemcpyAsync(p->d_sets, p->sd.data(), nsets * sizeof(SetDesc), cudaMemcpyHostToDevice, s) !=
            cudaSuccess ||
        cudaMemcpyAsync(p->d_qglob, p->qglob.data(), (nsets + 1) * sizeof(int64_t),
                        cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(p->d_tile0, p->tile0.data(), (nsets + 1) * sizeof(int64_t),
                        cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(p->d_offpos, p->off_pos.data(), nsets * sizeof(int64_t),
                        cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemsetAsync(p->qbuf, 0, std::max<int64_t>(qelems, 1) * sizeof(float), s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        set_error("plan setup failed: %s", cudaGetErrorString(cudaGetLastError()));
        return fail(SNN_ECUDA);
    }
    *out = p;
    return SNN_OK;
}

// All out-of-sample sets' query rows in one launch: element e of the
// concatenated m_t x d_t blocks (prefix eoff) goes to the plan buffer.
struct QCopyJob {
    const float *src;
    float *dst;
    int64_t ld;
    int d;
};
__global__ void k_plan_copy_queries(const QCopyJob *__restrict__ jobs, const int64_t *__restrict__ eoff, int njobs) {
    const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e >= eoff[njobs]) return;
    int lo = 0, hi = njobs - 1;   // last job with eoff <= e
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (eoff[mid] <= e) lo = mid; else hi = mid - 1;
    }
    const QCopyJob &J = jobs[lo];
    const int64_t k = e - eoff[lo], r = k / J.d, c = k - r * J.d;
    J.dst[k] = J.src[r * J.ld + c];
}

snn_status plan_set_queries(snn_batch_plan *p, const float *const *Q, const int64_t *ldq, cudaStream_t s) {
    std::vector<QCopyJob> jobs;
    std::vector<int64_t> eoff(1, 0);
    for (int32_t t = 0; t < p->nsets; ++t) {
        if (p->qbuf_off[t] < 0 || p->sd[t].m == 0) continue;
        const int d = p->sd[t].d;
        if (!Q[t] || ldq[t] < d) {
            set_error("set %d: queries NULL or ldq < d", t);
            return SNN_EINVAL;
        }
        jobs.push_back(QCopyJob{Q[t], p->qbuf + p->qbuf_off[t], ldq[t], d});
        eoff.push_back(eoff.back() + p->sd[t].m * d);
    }
    const int nj = int(jobs.size());
    if (nj == 0) return SNN_OK;
    Scratch scr(s);
    QCopyJob *dj;
    int64_t *de;
    SNN_TRY(scr.alloc(&dj, nj));
    SNN_TRY(scr.alloc(&de, nj + 1));
    // (copies from pageable host memory have read their source on return)
    SNN_CUDA(cudaMemcpyAsync(dj, jobs.data(), nj * sizeof(QCopyJob), cudaMemcpyHostToDevice, s));
    SNN_CUDA(cudaMemcpyAsync(de, eoff.data(), (nj + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s));
    SNN_LAUNCH(k_plan_copy_queries, unsigned(cdiv(eoff.back(), 256)), 256, 0, s)(dj, de, nj);
    SNN_LAUNCH_CHECK();
    return SNN_OK;
}

float *plan_queries(snn_batch_plan *p, int32_t t) {
    if (!p || t < 0 || t >= p->nsets || p->qbuf_off[t] < 0) return nullptr;
    return p->qbuf + p->qbuf_off[t];
}

snn_status plan_run(snn_batch_plan *p, cudaStream_t s) { return plan_enqueue(p, s); }

// Captures one run into a CUDA graph on first use, then launches the graph.
snn_status plan_launch_graph(snn_batch_plan *p, cudaStream_t s) {
    if (!p->exec) {
        cudaStream_t cs;
        SNN_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        const unsigned long long l0 = launch_count_now();
        snn_status st = SNN_OK;
        if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
            set_error("stream capture could not start");
            st = SNN_ECUDA;
        } else {
            st = plan_enqueue(p, cs);
            cudaGraph_t g = nullptr;
            const cudaError_t e = cudaStreamEndCapture(cs, &g);
            if (st == SNN_OK && e != cudaSuccess) {
                set_error("stream capture failed: %s", cudaGetErrorString(e));
                st = SNN_ECUDA;
            }
            if (st == SNN_OK && cudaGraphInstantiate(&p->exec, g, 0) != cudaSuccess) {
                set_error("graph instantiation failed");
                st = SNN_ECUDA;
            }
            p->graph = g;
        }
        cudaStreamDestroy(cs);
        // the captured launches are counted when the graph runs, not here
        p->graph_launches = launch_count_now() - l0;
        note_launches(0ull - p->graph_launches);
        if (st != SNN_OK) return st;
    }
    SNN_CUDA(cudaGraphLaunch(p->exec, s));
    note_launches(p->graph_launches);
    return SNN_OK;
}

// Synchronises s, reads the status and hands out per-set views.
snn_status plan_result(snn_batch_plan *p, cudaStream_t s, snn_csr *out, int64_t *need_surv,
                       int64_t *need_nnz) {
    PlanStatus hs;
    std::vector<int64_t> hn(p->nsets + 1);
    if (cudaMemcpyAsync(&hs, p->status, sizeof(hs), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(hn.data(), p->set_nnz, (p->nsets + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost,
                        s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        set_error("plan result read failed: %s", cudaGetErrorString(cudaGetLastError()));
        return SNN_ECUDA;
    }
    if (need_surv) *need_surv = (int64_t)hs.surv;
    if (need_nnz) *need_nnz = hs.nnz;
    if (hs.bad) { set_error("a query set contains NaN or Inf"); return SNN_EINVAL; }
    if (hs.tcerr & 1) {
        set_error("a bounded wait gave up (tensor-core scoring or the query sort)");
        return SNN_ETIMEOUT;
    }
    if (hs.tcerr & 2) {
        set_error("a query of a tensor-core set is too large for its set's FP16 scaling; create the plan "
                  "with FP32 precision for such queries");
        return SNN_ENOTSUP;
    }
    if (!(hs.qnorm <= (float)kMaxCentredNorm)) {
        set_error("a centred query norm of %g exceeds %g", (double)hs.qnorm, kMaxCentredNorm);
        return SNN_ENOTSUP;
    }
    if ((int64_t)hs.surv > p->surv_cap || hs.nnz > p->nnz_cap) {
        set_error("plan capacities exceeded: %llu survivors (capacity %lld), %lld neighbours "
                  "(capacity %lld)", hs.surv, (long long)p->surv_cap, hs.nnz, (long long)p->nnz_cap);
        return SNN_EOVERFLOW;
    }
    if (hs.big) {
        set_error("a row holds more than 4096 neighbours (use snn_query_radius_batch)");
        return SNN_ENOTSUP;
    }
    for (int32_t t = 0; t < p->nsets; ++t) {
        const int64_t nz = hn[t + 1] - hn[t];
        out[t].m = p->sd[t].m;
        out[t].nnz = nz;
        out[t].offsets = p->out_off + p->off_pos[t];
        out[t].indices = nz > 0 ? p->gidx + hn[t] : nullptr;
        out[t].dist2 = nz > 0 ? p->gd2 + hn[t] : nullptr;
    }
    return SNN_OK;
}

// Scoring choice of every tensor-core group (bit k of mask: group k scores
// its sets on the tensor cores, else the FP32 scorer takes them): the set
// descriptors' flags, copied to the device.
static snn_status plan_apply_mask(snn_batch_plan *p, unsigned mask, cudaStream_t s) {
    for (size_t k = 0; k < p->tc_groups.size(); ++k) {
        int n = 0;
        const int *sets = tc_batch_sets(p->tc_groups[k], &n);
        for (int i = 0; i < n; ++i) p->sd[sets[i]].tc = (mask >> k) & 1u;
    }
    p->tc_mask = mask;
    SNN_CUDA(cudaMemcpyAsync(p->d_sets, p->sd.data(), p->nsets * sizeof(SetDesc), cudaMemcpyHostToDevice, s));
    return SNN_OK;
}

static void plan_drop_graph(snn_batch_plan *p) {
    if (p->exec) {
        cudaGraphExecDestroy(p->exec);
        p->exec = nullptr;
    }
    if (p->graph) {
        cudaGraphDestroy(p->graph);
        p->graph = nullptr;
    }
}

// Tuning cache key of a plan: log2 buckets of the rows and queries of each
// tensor-core group (by fold column) and of the FP32-scored sets.
static std::string plan_key(const snn_batch_plan *p) {
    int64_t rows[4] = {0, 0, 0, 0}, qs[4] = {0, 0, 0, 0};
    for (int32_t t = 0; t < p->nsets; ++t) {
        const SetDesc &d = p->sd[t];
        const int b = (d.sym || d.d > 48) ? 3 : (d.d <= 16 ? 0 : (d.d <= 32 ? 1 : 2));
        rows[b] += d.n;
        qs[b] += d.m;
    }
    auto lg = [](int64_t v) { return v > 0 ? 64 - __builtin_clzll(uint64_t(v)) : 0; };
    char buf[160];
    snprintf(buf, sizeof(buf), "d16:%d/%d,d32:%d/%d,d48:%d/%d,fp32:%d/%d,prec:%d", lg(rows[0]), lg(qs[0]),
             lg(rows[1]), lg(qs[1]), lg(rows[2]), lg(qs[2]), lg(rows[3]), lg(qs[3]), int(p->prec));
    return buf;
}

// The tuning cache (SNN_TUNE_CACHE): JSON Lines, one object per plan key
// with the chosen "cpi", "ctas_per_sm", "tc_mask" and the measured "ms".
static std::mutex g_tune_mu;

static bool tune_cache_lookup(const std::string &key, int *cpi, int *ctas, unsigned *mask) {
    const char *path = getenv("SNN_TUNE_CACHE");
    if (!path || !*path) return false;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    FILE *f = fopen(path, "r");
    if (!f) return false;
    char line[512];
    bool hit = false;
    const std::string want = "{\"key\": \"" + key + "\",";
    while (fgets(line, sizeof(line), f)) {
        if (strncmp(line, want.c_str(), want.size()) != 0) continue;
        int c = 0, t = 0;
        unsigned m = 0;
        if (sscanf(line + want.size(), " \"cpi\": %d, \"ctas_per_sm\": %d, \"tc_mask\": %u", &c, &t, &m) == 3 &&
            (c == 4 || c == 8 || c == 16 || c == 32) && (t == 1 || t == 2)) {
            *cpi = c;
            *ctas = t;
            *mask = m;
            hit = true;
        }
    }
    fclose(f);
    return hit;
}

static void tune_cache_store(const std::string &key, int cpi, int ctas, unsigned mask, float ms) {
    const char *path = getenv("SNN_TUNE_CACHE");
    if (!path || !*path) return;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    std::vector<std::string> keep;
    const std::string want = "{\"key\": \"" + key + "\",";
    if (FILE *f = fopen(path, "r")) {
        char line[512];
        while (fgets(line, sizeof(line), f))
            if (strncmp(line, want.c_str(), want.size()) != 0) keep.push_back(line);
        fclose(f);
    }
    const std::string tmp = std::string(path) + ".tmp";
    FILE *f = fopen(tmp.c_str(), "w");
    if (!f) return;
    for (const std::string &l : keep) fputs(l.c_str(), f);
    fprintf(f, "{\"key\": \"%s\", \"cpi\": %d, \"ctas_per_sm\": %d, \"tc_mask\": %u, \"ms\": %.4f}\n", key.c_str(), cpi,
            ctas, mask, double(ms));
    fclose(f);
    rename(tmp.c_str(), path);
}

// Autotuner: the median of three timed runs (after one warm-up run) on the
// plan's current query values for each candidate, keeping the fastest:
// first the scoring of every tensor-core group (its sets on the tensor cores
// or on the FP32 scorer, every combination), then, with that choice, the
// FP32 scorer's work granularity (band chunks per item: 4, 8, 16, 32) and grid
// (1 or 2 CTAs per SM).  With SNN_TUNE_CACHE naming a file, a plan whose key
// (row and query buckets per group) is in it takes the stored choice without
// timing, and a tuned choice is stored.  Any captured graph is dropped.
snn_status plan_tune(snn_batch_plan *p, cudaStream_t s, int *best_cpi, int *best_ctas,
                     float *best_ms) {
    const std::string key = plan_key(p);
    const unsigned full = (1u << p->tc_groups.size()) - 1u;
    int cc = 0, ct = 0;
    unsigned cm = 0;
    plan_drop_graph(p);
    p->tuned_from_cache = 0;
    if (tune_cache_lookup(key, &cc, &ct, &cm) && (cm & ~full) == 0) {
        p->cpi = cc;
        p->ctas_per_sm = ct;
        SNN_TRY(plan_apply_mask(p, cm, s));
        p->tuned_from_cache = 1;
        if (best_cpi) *best_cpi = cc;
        if (best_ctas) *best_ctas = ct;
        if (best_ms) *best_ms = 0.f;
        return SNN_OK;
    }
    cudaEvent_t e0, e1;
    SNN_CUDA(cudaEventCreate(&e0));
    SNN_CUDA(cudaEventCreate(&e1));
    snn_status st = SNN_OK;
    auto time_run = [&](float *out) {
        float t[3];
        for (int rep = 0; rep < 4 && st == SNN_OK; ++rep) {   // the first run warms up
            cudaEventRecord(e0, s);
            st = plan_enqueue(p, s);
            cudaEventRecord(e1, s);
            if (cudaEventSynchronize(e1) != cudaSuccess) st = SNN_ECUDA;
            if (rep > 0) cudaEventElapsedTime(&t[rep - 1], e0, e1);
        }
        std::sort(t, t + 3);
        *out = t[1];
    };
    float best = 1e30f;
    unsigned bm = p->tc_mask;
    for (unsigned m = 0; m <= full && st == SNN_OK; ++m) {
        if ((st = plan_apply_mask(p, m, s)) != SNN_OK) break;
        float ms = 0.f;
        time_run(&ms);
        if (st == SNN_OK && ms < best) {
            best = ms;
            bm = m;
        }
    }
    if (st == SNN_OK) st = plan_apply_mask(p, bm, s);
    const int cpis[4] = {4, 8, 16, 32};
    const int ctas[2] = {1, 2};
    int bc = p->cpi, bt = p->ctas_per_sm;
    best = 1e30f;
    for (int a = 0; a < 4 && st == SNN_OK; ++a)
        for (int b = 0; b < 2 && st == SNN_OK; ++b) {
            p->cpi = cpis[a];
            p->ctas_per_sm = ctas[b];
            float ms = 0.f;
            time_run(&ms);
            if (st == SNN_OK && ms < best) {
                best = ms;
                bc = cpis[a];
                bt = ctas[b];
            }
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    p->cpi = bc;
    p->ctas_per_sm = bt;
    if (st == SNN_OK) tune_cache_store(key, bc, bt, bm, best);
    if (best_cpi) *best_cpi = bc;
    if (best_ctas) *best_ctas = bt;
    if (best_ms) *best_ms = best;
    return st;
}

snn_status plan_config(const snn_batch_plan *p, int *cpi, int *ctas, int *ngroups, unsigned *mask,
                       int *from_cache) {
    if (cpi) *cpi = p->cpi;
    if (ctas) *ctas = p->ctas_per_sm;
    if (ngroups) *ngroups = int(p->tc_groups.size());
    if (mask) *mask = p->tc_mask;
    if (from_cache) *from_cache = p->tuned_from_cache;
    return SNN_OK;
}

}  // namespace snn
