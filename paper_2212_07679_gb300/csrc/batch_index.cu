// Batched index build (Algorithm 1 for many small sets at once): one launch
// per step over every set (block tables built here), the scores of all sets
// sorted together by the composite key (set, score), one synchronisation.
// The indices' arrays are slices of shared pool blocks, released with the
// last index of the batch.
#include <algorithm>
#include <vector>

#include "index_kernels.cuh"
#include "index_struct.cuh"

namespace snn {

void ensure_pool();

namespace {

int64_t align_up(int64_t x, int64_t a) { return (x + a - 1) / a * a; }

}  // namespace

snn_status index_build_batch(int32_t nsets, const float *const *X, const int64_t *n,
                             const int32_t *d, const int64_t *ld, cudaStream_t s,
                             snn_index **out) {
    NvtxPhase nvtx_("snn batched index build");
    ensure_pool();
    for (int32_t t = 0; t < nsets; ++t) out[t] = nullptr;
    if (nsets == 0) return SNN_OK;
    // ------------------------------------------------------- layout
    std::vector<BSet> st(nsets);
    int64_t N = 0, part = 0, gpart = 0, coff = 0, dsum = 0, nsum = 0, esum = 0;
    std::vector<int64_t> voff(nsets), noff(nsets), eoff(nsets);
    for (int32_t t = 0; t < nsets; ++t) {
        if (!X[t] || n[t] < 1 || d[t] < 1 || d[t] > kPcSmallMaxD || ld[t] < d[t]) {
            set_error("set %d: need X, n >= 1, 1 <= d <= %d and ld >= d", t, kPcSmallMaxD);
            return SNN_EINVAL;
        }
        BSet &b = st[t];
        b.X = X[t];
        b.n = n[t];
        b.ld = ld[t];
        b.d = d[t];
        b.dp = (d[t] + 3) & ~3;
        b.p0 = N;
        b.nb = int(std::min<int64_t>(64, std::max<int64_t>(1, cdiv(n[t], 2048))));
        b.part_off = part;
        b.gpart_off = gpart;
        b.c_off = coff;
        b.vec = 0;
        N += n[t];
        part += int64_t(b.nb) * b.d;
        gpart += int64_t(b.nb) * b.d * b.d;
        coff += int64_t(b.d) * b.d;
        voff[t] = dsum;
        dsum += align_up(b.d, 32);
        noff[t] = nsum;
        nsum += align_up(b.n, 64);
        eoff[t] = esum;
        esum += align_up(b.n * b.dp, 64);
    }
    if (N >= (int64_t(1) << 31)) {
        set_error("a batch holds at most 2^31 - 1 points");
        return SNN_EINVAL;
    }
    // ------------------------------------------------ shared blocks
    snn_shared_blocks *sb = new (std::nothrow) snn_shared_blocks();
    if (!sb) {
        set_error("host allocation failed");
        return SNN_ENOMEM;
    }
    sb->stream = s;
    auto block = [&](size_t bytes) -> void * {
        void *p = nullptr;
        if (cudaMallocAsync(&p, std::max<size_t>(bytes, 256), s) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        sb->blocks[sb->nblocks++] = p;
        return p;
    };
    auto fail_blocks = [&](snn_status code) {
        for (int i = 0; i < sb->nblocks; ++i) cudaFreeAsync(sb->blocks[i], s);
        delete sb;
        return code;
    };
    double *mu64 = static_cast<double *>(block(dsum * 8));
    double *v64 = static_cast<double *>(block(dsum * 8));
    float *mu32 = static_cast<float *>(block(dsum * 4));
    float *v32 = static_cast<float *>(block(dsum * 4));
    float *alpha = static_cast<float *>(block(nsum * 4));
    int32_t *order = static_cast<int32_t *>(block(nsum * 4));
    float *hx = static_cast<float *>(block(nsum * 4));
    float *nrm = static_cast<float *>(block(nsum * 4));
    float *praw = static_cast<float *>(block(esum * 4));
    float *xc = static_cast<float *>(block(esum * 4));
    float *dconst = static_cast<float *>(block(size_t(nsets) * 4 * 4));
    if (!mu64 || !v64 || !mu32 || !v32 || !alpha || !order || !hx || !nrm || !praw || !xc ||
        !dconst) {
        set_error("batched index allocation failed");
        return fail_blocks(SNN_ENOMEM);
    }
    for (int32_t t = 0; t < nsets; ++t) {
        BSet &b = st[t];
        b.mu64 = mu64 + voff[t];
        b.v64 = v64 + voff[t];
        b.mu32 = mu32 + voff[t];
        b.v32 = v32 + voff[t];
        b.alpha = alpha + noff[t];
        b.order = order + noff[t];
        b.hx = hx + noff[t];
        b.nrm = nrm + noff[t];
        b.praw = praw + eoff[t];
        b.xc = xc + eoff[t];
        b.dconst = dconst + 4 * t;
    }
    // ------------------------------------------------- block tables
    std::vector<BBlk> bcol, bg16, bg32, bg64, bproj;
    int maxd = 0;
    for (int32_t t = 0; t < nsets; ++t) {
        const BSet &b = st[t];
        maxd = std::max(maxd, b.d);
        const int64_t rows = cdiv(b.n, b.nb);
        for (int rb = 0; rb < b.nb; ++rb) {
            const int64_t r0 = rb * rows, r1 = std::min(b.n, r0 + rows);
            for (int cb = 0; cb < int(cdiv(b.d, 32)); ++cb) bcol.push_back(BBlk{t, rb, cb, r0, r1});
            auto &g = b.d <= 16 ? bg16 : (b.d <= 32 ? bg32 : bg64);
            g.push_back(BBlk{t, rb, 0, r0, r1});
        }
        for (int64_t r0 = 0; r0 < b.n; r0 += 256)
            bproj.push_back(BBlk{t, 0, 0, r0, std::min(b.n, r0 + 256)});
    }
    snn_status stt = SNN_OK;
    {
        Scratch scr(s);
        BSet *dsets;
        BBlk *dcol, *dg16, *dg32, *dg64, *dproj;
        double *dpart, *dC;
        float *dgpart;
        uint64_t *keys, *keys_alt;
        uint32_t *vals, *vals_alt;
        int *bad;
#define BTRY(expr)                             \
    do {                                       \
        if ((stt = (expr)) != SNN_OK) break;   \
    } while (0)
        do {
            BTRY(scr.alloc(&dsets, nsets));
            BTRY(scr.alloc(&dcol, bcol.size()));
            BTRY(scr.alloc(&dg16, std::max<size_t>(bg16.size(), 1)));
            BTRY(scr.alloc(&dg32, std::max<size_t>(bg32.size(), 1)));
            BTRY(scr.alloc(&dg64, std::max<size_t>(bg64.size(), 1)));
            BTRY(scr.alloc(&dproj, bproj.size()));
            BTRY(scr.alloc(&dpart, part));
            BTRY(scr.alloc(&dgpart, gpart));
            BTRY(scr.alloc(&dC, coff));
            BTRY(scr.alloc(&keys, N));
            BTRY(scr.alloc(&keys_alt, N));
            BTRY(scr.alloc(&vals, N));
            BTRY(scr.alloc(&vals_alt, N));
            BTRY(scr.alloc(&bad, 2));   // [0] NaN/Inf, [1] a bounded wait of the sort expired
            auto up = [&](void *dst, const void *src, size_t bytes) {
                return bytes == 0 ? cudaSuccess
                                  : cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s);
            };
            if (up(dsets, st.data(), nsets * sizeof(BSet)) != cudaSuccess ||
                up(dcol, bcol.data(), bcol.size() * sizeof(BBlk)) != cudaSuccess ||
                up(dg16, bg16.data(), bg16.size() * sizeof(BBlk)) != cudaSuccess ||
                up(dg32, bg32.data(), bg32.size() * sizeof(BBlk)) != cudaSuccess ||
                up(dg64, bg64.data(), bg64.size() * sizeof(BBlk)) != cudaSuccess ||
                up(dproj, bproj.data(), bproj.size() * sizeof(BBlk)) != cudaSuccess ||
                cudaMemsetAsync(bad, 0, 2 * sizeof(int), s) != cudaSuccess ||
                cudaMemsetAsync(dconst, 0, size_t(nsets) * 16, s) != cudaSuccess) {
                set_error("batched index build: table upload failed");
                stt = SNN_ECUDA;
                break;
            }
            // K1 means, K2 Gram, K3 first direction, K4 scores
            SNN_LAUNCH(k_colsum_batch, unsigned(bcol.size()), 256, 0, s)(dsets, dcol, dpart, bad);
            SNN_LAUNCH(k_mean_final_batch, unsigned(nsets), 256, 0, s)(dsets, dpart);
            if (!bg16.empty()) SNN_LAUNCH(k_gram_batch16, unsigned(bg16.size()), 256, 0, s)(dsets, dg16, dgpart);
            if (!bg32.empty()) SNN_LAUNCH(k_gram_batch32, unsigned(bg32.size()), 256, 0, s)(dsets, dg32, dgpart);
            if (!bg64.empty()) SNN_LAUNCH(k_gram_batch64, unsigned(bg64.size()), 256, 0, s)(dsets, dg64, dgpart);
            SNN_LAUNCH(k_gram_reduce_batch, unsigned(nsets), 256, 0, s)(dsets, dgpart, dC);
            const size_t smem = (maxd + 32) * sizeof(double) + (32 + 2 * maxd) * sizeof(float) +
                                2 * size_t(maxd) * maxd * sizeof(float);
            SNN_LAUNCH(k_pc_small_batch, unsigned(nsets), 1024, smem, s)(dsets, dC);
            SNN_LAUNCH(k_project_batch, unsigned(bproj.size()), 256, 0, s)(dsets, dproj, keys, vals, bad);
            if (cudaGetLastError() != cudaSuccess) {
                set_error("batched index build: launch failed");
                stt = SNN_ECUDA;
                break;
            }
            // K5 one sort of all sets by (set, score); K6 gather
            int bits = 32;
            while ((int64_t(1) << (bits - 32)) < nsets) ++bits;
            BTRY(radix_sort_pairs<uint64_t>(keys, vals, keys_alt, vals_alt, N, bits, s, bad + 1));
            SNN_LAUNCH(k_gather_batch, unsigned(cdiv(N, 256)), 256, 0, s)(dsets, keys, vals, N);
            if (cudaGetLastError() != cudaSuccess) {
                set_error("batched index build: gather launch failed");
                stt = SNN_ECUDA;
                break;
            }
        } while (0);
#undef BTRY
        std::vector<float> hc(size_t(nsets) * 4);
        int hbad[2] = {0, 0};
        if (stt == SNN_OK) {
            if (cudaMemcpyAsync(hc.data(), dconst, hc.size() * 4, cudaMemcpyDeviceToHost, s) !=
                    cudaSuccess ||
                cudaMemcpyAsync(hbad, bad, sizeof(hbad), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                cudaStreamSynchronize(s) != cudaSuccess) {
                set_error("batched index build failed: %s", cudaGetErrorString(cudaGetLastError()));
                stt = SNN_ECUDA;
            } else if (hbad[0]) {
                set_error("a set contains NaN or Inf");
                stt = SNN_EINVAL;
            } else if (hbad[1]) {
                set_error("batched index build: a bounded wait of the score sort expired");
                stt = SNN_ETIMEOUT;
            }
        }
        for (int32_t t = 0; stt == SNN_OK && t < nsets; ++t)
            if (!(hc[4 * t + 1] <= kMaxCentredNorm)) {
                set_error("set %d: a centred point norm of %g exceeds %g", t, (double)hc[4 * t + 1],
                          kMaxCentredNorm);
                stt = SNN_ENOTSUP;
            }
        if (stt != SNN_OK) {
            cudaStreamSynchronize(s);
            return fail_blocks(stt);
        }
        int dev = 0;
        cudaGetDevice(&dev);
        for (int32_t t = 0; t < nsets; ++t) {
            snn_index *ix = new (std::nothrow) snn_index();
            if (!ix) {
                for (int32_t u = 0; u < t; ++u) {
                    index_release(out[u]);
                    out[u] = nullptr;
                }
                set_error("host allocation failed");
                if (t == 0) return fail_blocks(SNN_ENOMEM);
                return SNN_ENOMEM;
            }
            const BSet &b = st[t];
            ix->n = b.n;
            ix->d = b.d;
            ix->dp = b.dp;
            ix->device = dev;
            ix->stream = s;
            ix->mu64 = b.mu64;
            ix->mu32 = b.mu32;
            ix->v64 = b.v64;
            ix->v32 = b.v32;
            ix->alpha = b.alpha;
            ix->order = b.order;
            ix->praw = b.praw;
            ix->xc = b.xc;
            ix->hx = b.hx;
            ix->nrm = b.nrm;
            ix->dconst = b.dconst;
            ix->alpha_err = hc[4 * t + 0];
            ix->nrm_max = hc[4 * t + 1];
            ix->shared = sb;
            sb->refs.fetch_add(1);
            out[t] = ix;
        }
    }
    return SNN_OK;
}

}  // namespace snn
