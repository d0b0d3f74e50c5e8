// Tensor-core band scoring on sm_103a: TMA-staged BF16 operands, tcgen05.mma
// into TMEM (FP32 accumulation), sign test in the epilogue.
//
// The left side of Eq. (4), x_j^T x_j/2 - x_j^T x_q, is scored for a tile of
// 128 queries (sorted by score) against 128-row chunks of the union band
// (Section 4: one gemm over the union of the candidate ranges).  Every
// centred FP32 row is split into BF16 parts, x = x1 + x2 (+ x3), and the
// products x1.y1 + x1.y2 + x2.y1 (+ x1.y3 + x2.y2 + x3.y1) are accumulated
// in FP32.  The rejection threshold is folded into the contraction as
// rank-one columns, so the accumulator itself is
//     acc_ij = x_j.y_i - (1 - c) xbar_j + c ||y_i|| ||x_j|| + A_i,
// where A_i bounds (R + slack)^2/2 - ||y_i||^2/2 and c bounds every rounding
// (split, FP32 accumulation, norms) relative to xbar_j + ||x_j|| ||y_i||.
// A pair the FP64 definition could accept has acc_ij > 0, so a pair is
// rejected exactly when the sign bit of acc_ij is set; all other pairs go to
// the exact decision like the FP32 path's survivors.
//
// The FP8 variant splits each row, scaled by a power of two of its own, into
// e4m3 parts (tcgen05.mma kind::f8f6f4, K = 32 per instruction) and folds the
// threshold together with a per-pair bound on every dropped term (built from
// the measured norms of the parts and of the exact residual) into one final
// BF16 k-step of the same accumulator.
//
// Warp roles: warp 0 issues TMA loads, warp 1 owns TMEM and issues the MMAs,
// the remaining 8 (or 16, with two query tiles per item) warps drain the
// accumulators.  Stages are guarded by mbarriers; every wait is bounded and a
// timeout sets an error flag.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "index_struct.cuh"
#include "tc_common.cuh"
#include "tc_score.cuh"

namespace snn {

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                  const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                  const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn get_encode() {
    static EncodeTiledFn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    }
    return fn;
}

snn_status make_map(CUtensorMap *map, const uint16_t *ptr, int64_t rows, int64_t K2, int bk,
                    int box_rows) {
    EncodeTiledFn enc = get_encode();
    if (!enc) {
        set_error("cuTensorMapEncodeTiled is unavailable");
        return SNN_ENOTSUP;
    }
    cuuint64_t dims[2] = {cuuint64_t(K2), cuuint64_t(rows)};
    cuuint64_t strides[1] = {cuuint64_t(K2) * 2};
    cuuint32_t box[2] = {cuuint32_t(bk), cuuint32_t(box_rows)};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<uint16_t *>(ptr), dims,
                     strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                     bk == 64 ? CU_TENSOR_MAP_SWIZZLE_128B
                              : (bk == 32 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_32B),
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        set_error("cuTensorMapEncodeTiled failed (%d)", int(r));
        return SNN_ECUDA;
    }
    return SNN_OK;
}

namespace {

constexpr int kTM = 128;            // queries per tile (MMA M)
// epilogue: per TMEM lane quadrant and query sub-tile, two warps (half the
// columns each) for chunks of 128 or more rows, one warp below; producer and
// MMA warps in front
__host__ __device__ constexpr int tc_halves(int bn) { return bn >= 128 ? 2 : 1; }
__host__ __device__ constexpr int tc_epi_warps(int mt, int bn) { return 4 * mt * tc_halves(bn); }
// warps: 0 TMA producer, 1 MMA issuer (and 2, a second issuer taking
// alternate chunks, for the shapes with a resident query tile), then the
// epilogue warps
__host__ __device__ constexpr int tc_first_epi(bool ares) { return ares ? 3 : 2; }
__host__ __device__ constexpr int tc_threads(int mt, int bn, bool ares) {
    return 32 * tc_first_epi(ares) + 32 * tc_epi_warps(mt, bn);
}
// accumulator buffers in a CTA's share of the 512 TMEM columns (cps CTAs per
// SM): four when they fit (the MMAs of three chunks then cover the hand-back
// latency of the fourth), else two
__host__ __device__ constexpr int tc_nbuf(int mt, int bn, int cps) {
    return 4 * mt * bn <= 512 / cps ? 4 : (2 * mt * bn <= 512 / cps ? 2 : 1);
}
constexpr int kExtra = 9;           // folded columns
// dynamic shared memory per CTA (minus base alignment and barriers) for 1
// or 2 resident CTAs per SM
__host__ __device__ constexpr int smem_budget(int cps, int align) {
    return (cps == 1 ? 232448 : 115712) - align - 512;
}

// Shape of one kernel instance: NSPLIT BF16 parts, BK columns per k-block
// for part 1 (64: 128-byte rows, 128B swizzle; 32: 64-byte rows, 64B swizzle),
// NW columns for parts 2 and 3 (NW < BK when all data columns fit NW: those
// parts carry no folded columns, so their tiles are narrower), BN band rows
// per chunk (MMA N), ARES: the query tile stays in shared memory for a whole
// work item (only when one k-block holds all columns), in two slots so that
// the next item's tile loads while the current one is in use; CPS resident
// CTAs per SM; MT query tiles of 128 per work item (each band chunk is loaded
// once and multiplied with all MT tiles, M = 128 per MMA).
// F8NP > 0: FP8 e4m3 data k-blocks of 2 BK bytes per row (BK = NW = 16 or
// 32: one or two K = 32 steps of F8NP products each), then one 32-byte BF16
// k-block of folded columns in part 1's slots.
// NSPLIT = 1: one FP16 part, one MMA per 16-column k step, then the same
// separate block of folded BF16 columns (streamed shape only).
template <int NSPLIT, int BK, int BN, bool ARES, int CPS = 1, int NW = BK, int MT = 1, int F8NP = 0>
struct TcShape {
    static constexpr int kAlign = BK == 64 ? 1024 : 512;
    static constexpr int kSmemBudget = smem_budget(CPS, kAlign);
    static constexpr int kTA0 = MT * kTM * BK * 2;      // A part 1 tile
    static constexpr int kTA1 = MT * kTM * NW * 2;      // A parts 2, 3
    static constexpr int kTB0 = BN * BK * 2;            // B part 1 tile
    static constexpr int kTB1 = BN * NW * 2;            // B parts 2, 3
    static constexpr int kASlot = kTA0 + (NSPLIT - 1) * kTA1;
    static constexpr int kBStage = kTB0 + (NSPLIT - 1) * kTB1;
    static constexpr int kAResBytes = ARES ? 2 * kASlot : 0;
    static constexpr int kStageBytes = ARES ? kBStage : kASlot + kBStage;
    // per-epilogue-warp staging of survivors (flushed in batches: one
    // global atomic per batch instead of one per 32-column group)
    static constexpr int kStgEntries = 128;
    static constexpr int kStgBytes = tc_epi_warps(MT, BN) * kStgEntries * 8;
    static constexpr int kStagesRaw = (kSmemBudget - kAResBytes - kStgBytes) / kStageBytes;
    static constexpr int kStages = kStagesRaw > 12 ? 12 : kStagesRaw;
    static constexpr int kNP = F8NP ? F8NP : (NSPLIT == 1 ? 1 : (NSPLIT == 2 ? 3 : 6));   // MMAs per k-step
    // the folded columns come in a k-block of their own (32 bytes per row)
    static constexpr bool kFoldBlock = F8NP != 0 || NSPLIT == 1;
    static constexpr int kKSteps = BK / 16;             // k-steps per k-block
    static constexpr int kRowBytes = BK * 2;
    static constexpr int kRowBytesN = NW * 2;
    static constexpr uint32_t kTmemCols = tc_nbuf(MT, BN, CPS) * MT * BN;
    static constexpr int kEpiWarps = tc_epi_warps(MT, BN);
    static constexpr int kThreads = tc_threads(MT, BN, ARES);
    // two MMA issuers: a parity wait is only sound when the stage is at most
    // one round behind the load it waits for, and an issuer waiting for the
    // first k-block of its chunk has consumed the k-blocks up to its previous
    // chunk, so the ring must hold more stages than a chunk has k-blocks: true
    // for the resident-query-tile shapes (one k-block per chunk)
    static constexpr bool kDual = ARES;
    static constexpr int kFirstEpi = tc_first_epi(ARES);
    static constexpr int kNBuf = tc_nbuf(MT, BN, CPS);
    static constexpr size_t kSmem =
        size_t(kAResBytes) + size_t(kStages) * kStageBytes + kAlign + 512 + kStgBytes;
    static_assert(kStagesRaw >= 2, "shape does not fit shared memory");
    static_assert(ARES || NW == BK, "narrow parts need a resident query tile");
    static_assert(MT == 1 || ARES || NSPLIT == 1,
                  "several streamed query tiles per item: one FP16 part only");
    static_assert(kTmemCols * CPS <= 512, "accumulators exceed TMEM");
    static_assert(!ARES || kNBuf % 2 == 0, "two MMA issuers own alternate accumulator buffers");
    static_assert(!ARES || kStagesRaw >= 2, "two issuers need two stages");
    static_assert(NW == 16 || NW == 32 || NW == 64, "unsupported part width");
    static_assert(!F8NP || ((BK == 16 || BK == 32) && NW == BK && !ARES && MT == 1), "FP8 shape");
    static_assert(!F8NP || (NSPLIT == 2 && (F8NP == 3 || F8NP == 4)) || (NSPLIT == 3 && F8NP == 6),
                  "FP8 products");
    static_assert(NSPLIT != 1 || (!F8NP && !ARES && (MT == 1 || MT == 2) && NW == BK && BK == 32),
                  "one FP16 part: streamed shape with 32-column k-blocks");
};

__host__ __device__ constexpr int tc_npairs(int nsplit) { return nsplit == 2 ? 3 : 6; }

struct TcArgs {
    int64_t m;
    int64_t n;
    int ksteps;                 // 16-wide k steps that hold data or folded columns
    int ksteps_data;            // k steps that hold data columns (the rest: folded only)
    int nkb;                    // k blocks loaded per chunk
    const int64_t *tile_lo;
    const int64_t *tile_hi;
    const int64_t *item_off;
    const int32_t *item_tile;
    int ntiles;
    int sym;
    uint2 *surv;
    int64_t cap;
    unsigned long long *count;
    int *err;
    int stall;                  // test fault: the producer issues no loads
    int f16;                    // data k steps hold FP16 parts (folded ones BF16)
    int scan_rank;              // streamed shapes: branch-free survivor extraction
};

struct ItemInfo {
    int64_t q0, band_lo, band_hi, c_first, c_end;   // chunks of kBR rows
};

// tiles here are groups of MT consecutive 128-query tiles
template <int MT>
__device__ __forceinline__ ItemInfo item_info(const TcArgs &a, int64_t item) {
    const int lo = a.item_tile[item];
    ItemInfo f;
    f.q0 = int64_t(lo) * kTM * MT;
    f.band_lo = a.tile_lo[lo];
    f.band_hi = a.tile_hi[lo];
    f.c_first = (item - a.item_off[lo]) * kChunksPerItem;
    f.c_end = min(cdiv(f.band_hi - f.band_lo, kBR), f.c_first + kChunksPerItem);
    return f;
}

template <int NSPLIT, int BK, int BN, bool ARES, int CPS, int NW, int MT, int F8NP>
__global__ void __launch_bounds__(tc_threads(MT, BN, ARES), CPS)
k_score_tc(const __grid_constant__ CUtensorMap qa0, const __grid_constant__ CUtensorMap qa1,
           const __grid_constant__ CUtensorMap qa2, const __grid_constant__ CUtensorMap xb0,
           const __grid_constant__ CUtensorMap xb1, const __grid_constant__ CUtensorMap xb2,
           const __grid_constant__ CUtensorMap qf, const __grid_constant__ CUtensorMap xf,
           TcArgs a) {
    using Sh = TcShape<NSPLIT, BK, BN, ARES, CPS, NW, MT, F8NP>;
    constexpr int S = Sh::kStages;
    constexpr int NP = Sh::kNP;
    constexpr int NB = Sh::kNBuf;                // accumulator buffers
    constexpr uint32_t kIdesc = idesc_bf16<kTM, BN>();
    // FP16 data parts: both operands of a data k step are FP16 and both of a
    // folded k step BF16 (the folded columns start on a k step boundary)
    constexpr uint32_t kIdescF16 = idesc_f16<kTM, BN>();
    // (A part, B part) products kept by the split: all with pa + pb <= NSPLIT-1
    constexpr int kPa[6] = {0, 0, 1, 0, 1, 2};
    constexpr int kPb[6] = {0, 1, 0, 2, 1, 0};
    // FP8: the same list, except that four products keep (1,1) as the fourth
    constexpr int kPa8[6] = {0, 0, 1, F8NP == 4 ? 1 : 0, 1, 2};
    constexpr int kPb8[6] = {0, 1, 0, F8NP == 4 ? 1 : 2, 1, 0};
    constexpr uint32_t kIdesc8 = idesc_e4m3<kTM, BN>();

    extern __shared__ unsigned char smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + uint32_t(Sh::kAlign - 1)) & ~uint32_t(Sh::kAlign - 1);
    unsigned char *gbase = smem_raw + (base - raw);
    // resident A parts first (ARES), then the stages
    const uint32_t stage0 = base + uint32_t(Sh::kAResBytes);
    // ARES: s is the A slot (item parity); otherwise the stage
    auto a_tile = [&](int s, int p) -> uint32_t {
        const uint32_t po = p == 0 ? 0u : uint32_t(Sh::kTA0 + (p - 1) * Sh::kTA1);
        if (ARES) return base + uint32_t(s * Sh::kASlot) + po;
        return stage0 + uint32_t(s * Sh::kStageBytes) + po;
    };
    auto b_tile = [&](int s, int p) -> uint32_t {
        const uint32_t po = p == 0 ? 0u : uint32_t(Sh::kTB0 + (p - 1) * Sh::kTB1);
        return stage0 + uint32_t(s * Sh::kStageBytes + (ARES ? 0 : Sh::kASlot)) + po;
    };
    const uint32_t bar0 = stage0 + uint32_t(S * Sh::kStageBytes);
    auto full_bar = [&](int s) { return bar0 + 8u * s; };
    auto empty_bar = [&](int s) { return bar0 + 8u * (S + s); };
    auto tfull_bar = [&](int b) { return bar0 + 8u * (2 * S + b); };
    auto tempty_bar = [&](int b) { return bar0 + 8u * (2 * S + NB + b); };
    const uint32_t done_bar = bar0 + 8u * (2 * S + 2 * NB);
    auto afull_bar = [&](int k) { return bar0 + 8u * (2 * S + 2 * NB + 1 + k); };
    auto aempty_bar = [&](int k) { return bar0 + 8u * (2 * S + 2 * NB + 3 + k); };
    unsigned char *gmisc = gbase + (bar0 - base) + 8 * (2 * S + 2 * NB + 5);
    static_assert(8 * (2 * S + 2 * NB + 5) + 16 <= 512, "barrier area");
    volatile uint32_t *s_tmem = reinterpret_cast<volatile uint32_t *>(gmisc);
    volatile int *s_abort = reinterpret_cast<volatile int *>(gmisc + 4);
    // survivor staging: kStgEntries per epilogue warp, after the barriers
    uint2 *s_stg = reinterpret_cast<uint2 *>(gbase + (bar0 - base) + 512);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const CUtensorMap *qa[3] = {&qa0, &qa1, &qa2};
    // Two MMA issuers (kDual, one per warp) take alternate chunks, each into
    // its own accumulator buffers (NB is even), so one thread's barrier waits
    // and commits overlap the other's MMAs; both walk the whole work list to
    // keep the stage and buffer counters.
    constexpr bool dual = Sh::kDual;
    const CUtensorMap *xb[3] = {&xb0, &xb1, &xb2};

    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(full_bar(s), 1);
            mbar_init(empty_bar(s), 1);
        }
        for (int b = 0; b < NB; ++b) {
            mbar_init(tfull_bar(b), 1);
            mbar_init(tempty_bar(b), Sh::kEpiWarps);   // one arrival per epilogue warp
        }
        for (int k = 0; k < 2; ++k) {
            mbar_init(afull_bar(k), 1);
            mbar_init(aempty_bar(k), dual ? 2 : 1);   // one commit per MMA issuer
        }
        mbar_init(done_bar, dual ? 2 : 1);
        *s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) {
        // NB accumulator sets of MT x BN FP32 columns
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32((const void *)s_tmem)),
                     "n"(Sh::kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tmem_fence_before();
    __syncthreads();
    tmem_fence_after();
    const uint32_t tmem = *s_tmem;
    const int64_t total = a.item_off[a.ntiles];

    int issued = 0, a_issued = 0;
    if (warp == 0) {
        // ------------------------------------------------ TMA producer
        // (a test fault withholds every load, so the consumers' bounded waits
        // expire and the call reports SNN_ETIMEOUT)
        if (lane == 0 && !a.stall) {
            int it = 0, itm = 0;
            for (int64_t item = blockIdx.x; item < total && !*s_abort; item += gridDim.x, ++itm) {
                const ItemInfo f = item_info<MT>(a, item);
                if (ARES) {
                    // the query tile of this item, once, into slot itm & 1
                    const int k = itm & 1;
                    const uint32_t use = uint32_t(itm >> 1);
                    if (!mbar_wait(aempty_bar(k), (use & 1u) ^ 1u, s_abort, a.err)) break;
                    mbar_expect_tx(afull_bar(k), uint32_t(Sh::kASlot));
                    for (int p = 0; p < NSPLIT; ++p)
                        tma_load_2d(a_tile(k, p), qa[p], 0, int(f.q0), afull_bar(k));
                    a_issued = itm + 1;
                }
                for (int64_t jr = f.c_first * kBR; jr < f.c_end * kBR && !*s_abort; jr += BN) {
                    const int64_t j0 = f.band_lo + jr;
                    for (int kb = 0; kb < a.nkb; ++kb, ++it) {
                        const int s = it % S;
                        const uint32_t round = uint32_t(it / S);
                        if (!mbar_wait(empty_bar(s), (round & 1u) ^ 1u, s_abort, a.err)) break;
                        if (Sh::kFoldBlock && kb == a.nkb - 1) {
                            // folded BF16 columns, 32 bytes per row, in part 1's slots
                            mbar_expect_tx(full_bar(s), uint32_t((kTM * MT + BN) * 32));
                            tma_load_2d(a_tile(s, 0), &qf, 0, int(f.q0), full_bar(s));
                            tma_load_2d(b_tile(s, 0), &xf, 0, int(j0), full_bar(s));
                        } else {
                            mbar_expect_tx(full_bar(s), uint32_t(Sh::kStageBytes));
                            for (int p = 0; p < NSPLIT; ++p) {
                                const int kx = kb * (p == 0 ? BK : NW);
                                if (!ARES) tma_load_2d(a_tile(s, p), qa[p], kx, int(f.q0), full_bar(s));
                                tma_load_2d(b_tile(s, p), xb[p], kx, int(j0), full_bar(s));
                            }
                        }
                        issued = it + 1;
                    }
                }
            }
        }
    } else if (warp >= 1 && warp < Sh::kFirstEpi) {
        // ------------------------------------------------- MMA issuer(s)
        const int me = warp - 1;
        if (lane == 0) {
            int it = 0, chunk = 0, itm = 0;
            bool ok = true;
            for (int64_t item = blockIdx.x; item < total && ok; item += gridDim.x, ++itm) {
                const ItemInfo f = item_info<MT>(a, item);
                const int aslot = itm & 1;
                if (ARES) {
                    if (!(ok = mbar_wait(afull_bar(aslot), uint32_t(itm >> 1) & 1u, s_abort, a.err)))
                        break;
                    tmem_fence_after();
                }
                for (int64_t jr = f.c_first * kBR; jr < f.c_end * kBR && ok; jr += BN, ++chunk) {
                    if (dual && (chunk & 1) != me) {
                        it += a.nkb;
                        continue;
                    }
                    const int b = chunk % NB;
                    const uint32_t use = uint32_t(chunk / NB);
                    if (!(ok = mbar_wait(tempty_bar(b), (use & 1u) ^ 1u, s_abort, a.err))) break;
                    tmem_fence_after();
                    const uint32_t dt0 = tmem + uint32_t(b * MT * BN);
                    for (int kb = 0; kb < a.nkb; ++kb, ++it) {
                        const int s = it % S;
                        const uint32_t round = uint32_t(it / S);
                        if (!(ok = mbar_wait(full_bar(s), round & 1u, s_abort, a.err))) break;
                        tmem_fence_after();
                        if constexpr (NSPLIT == 1) {
                            // query tile h of the item: 128 rows further into the A tile,
                            // its own accumulator columns
                            if (kb == a.nkb - 1) {
                                // the folded columns: one BF16 K = 16 step
#pragma unroll
                                for (int h = 0; h < MT; ++h)
                                    mma_bf16(dt0 + uint32_t(h * BN),
                                             smem_desc<32>(a_tile(s, 0) + uint32_t(h * kTM * 32)),
                                             smem_desc<32>(b_tile(s, 0)), kIdesc, 1u);
                            } else {
#pragma unroll
                                for (int ks = 0; ks < Sh::kKSteps; ++ks) {
                                    // FP16 data k steps; the last block may hold one
                                    const int kg = kb * Sh::kKSteps + ks;
                                    if (kg >= a.ksteps_data) break;
                                    const uint64_t bd = smem_desc<Sh::kRowBytes>(b_tile(s, 0) + 32u * ks);
#pragma unroll
                                    for (int h = 0; h < MT; ++h) {
                                        const uint32_t aa =
                                            a_tile(s, 0) + uint32_t(h * kTM * Sh::kRowBytes) + 32u * ks;
                                        mma_bf16(dt0 + uint32_t(h * BN), smem_desc<Sh::kRowBytes>(aa), bd,
                                                 kIdescF16, kg != 0 ? 1u : 0u);
                                    }
                                }
                            }
                        } else if constexpr (F8NP != 0) {
                            static_assert(Sh::kRowBytesN == Sh::kRowBytes, "FP8 parts share one width");
                            if (kb == a.nkb - 1) {
                                // the folded columns: one BF16 K = 16 step
                                mma_bf16(dt0, smem_desc<32>(a_tile(s, 0)), smem_desc<32>(b_tile(s, 0)),
                                         kIdesc, 1u);
                            } else {
#pragma unroll
                                for (int ks = 0; ks < Sh::kKSteps; ++ks) {
                                    // 32-byte k steps; the last block may hold one
                                    const int kg = kb * Sh::kKSteps + ks;
                                    if (kg >= a.ksteps_data) break;
#pragma unroll
                                    for (int pr = 0; pr < F8NP; ++pr)
                                        mma_e4m3(dt0, smem_desc<Sh::kRowBytes>(a_tile(s, kPa8[pr]) + 32u * ks),
                                                 smem_desc<Sh::kRowBytes>(b_tile(s, kPb8[pr]) + 32u * ks),
                                                 kIdesc8, (kg | pr) != 0 ? 1u : 0u);
                                }
                            }
                        } else {
#pragma unroll
                            for (int ks = 0; ks < Sh::kKSteps; ++ks) {
                                const int kg = kb * Sh::kKSteps + ks;
                                if (kg >= a.ksteps) break;
                                // the folded columns live in part 0 only: a k step
                                // without data columns needs the (0,0) product alone
                                const int np = kg < a.ksteps_data ? NP : 1;
                                const uint32_t idk = (a.f16 && kg < a.ksteps_data) ? kIdescF16 : kIdesc;
#pragma unroll
                                for (int pr = 0; pr < NP; ++pr) {
                                    if (pr >= np) break;
                                    const uint32_t bb = b_tile(s, kPb[pr]) + 32u * ks;
                                    const uint64_t bd = kPb[pr] == 0 ? smem_desc<Sh::kRowBytes>(bb)
                                                                     : smem_desc<Sh::kRowBytesN>(bb);
#pragma unroll
                                    for (int h = 0; h < MT; ++h) {
                                        // query sub-tile h: 128 rows further into the A tile
                                        const uint32_t arow = kPa[pr] == 0 ? Sh::kRowBytes : Sh::kRowBytesN;
                                        const uint32_t aa = a_tile(ARES ? aslot : s, kPa[pr]) +
                                                            uint32_t(h * kTM) * arow + 32u * ks;
                                        const uint64_t ad = kPa[pr] == 0 ? smem_desc<Sh::kRowBytes>(aa)
                                                                         : smem_desc<Sh::kRowBytesN>(aa);
                                        mma_bf16(dt0 + uint32_t(h * BN), ad, bd, idk,
                                                 (kb | ks | pr) != 0 ? 1u : 0u);
                                    }
                                }
                            }
                        }
                        mma_commit(empty_bar(s));
                    }
                    if (ok) mma_commit(tfull_bar(b));
                }
                if (ARES && ok) mma_commit(aempty_bar(aslot));   // this slot may be refilled
            }
            // every MMA issued by this thread has completed before TMEM is freed
            mma_commit(done_bar);
            mbar_wait(done_bar, 0u, s_abort, a.err);
        }
    } else {
        // ---------------------------------------------------- epilogue
        const int ew = warp - Sh::kFirstEpi;       // 0 .. kEpiWarps-1
        const int quad = warp & 3;                 // TMEM lanes 32*quad .. +31
        const int sub = ew >> 2;
        constexpr int kHalves = tc_halves(BN);
        const int half = sub % kHalves;            // which half of the columns
        const int ht = sub / kHalves;              // which query sub-tile
        const int qi = ht * kTM + quad * 32 + lane;   // query row within the item's tiles
        constexpr int kGroups = BN / 32 / kHalves; // 32-column groups per warp
        constexpr int kStg = Sh::kStgEntries;
        uint2 *stg = s_stg + ew * kStg;
        int scount = 0;                            // staged entries (warp-uniform)
        // moves the staged survivors to the global list: one atomic, then
        // coalesced 8-byte stores
        auto flush = [&]() {
            if (scount == 0) return;
            __syncwarp();
            unsigned long long base = 0;
            if (lane == 0) base = atomicAdd(a.count, (unsigned long long)scount);
            base = __shfl_sync(0xffffffffu, base, 0);
            for (int k = lane; k < scount; k += 32)
                if (base + k < (unsigned long long)a.cap) a.surv[base + k] = stg[k];
            __syncwarp();
            scount = 0;
        };
        int chunk = 0;
        bool ok = true;
        for (int64_t item = blockIdx.x; item < total && ok; item += gridDim.x) {
            const ItemInfo f = item_info<MT>(a, item);
            const int64_t q = f.q0 + qi;
            for (int64_t jr = f.c_first * kBR; jr < f.c_end * kBR && ok; jr += BN, ++chunk) {
                const int64_t j0 = f.band_lo + jr;
                const int b = chunk % NB;
                const uint32_t use = uint32_t(chunk / NB);
                ok = mbar_wait(tfull_bar(b), use & 1u, s_abort, a.err);
                if (!__all_sync(0xffffffffu, ok)) { ok = false; break; }
                tmem_fence_after();
                const uint32_t tbase =
                    tmem + (uint32_t(quad * 32) << 16) + uint32_t(b * MT * BN + ht * BN);
                // chunks away from the band end and from the queries' own rows
                // need no per-column validity checks
                const bool edge = (j0 + BN > f.band_hi) || (a.sym && j0 < f.q0 + int64_t(MT) * kTM);
                const bool qvalid = q < a.m;
#pragma unroll 1
                for (int g2 = 0; g2 < kGroups; g2 += 2) {
                    uint32_t rr[64];
                    float mx[4];
                    const int cb0 = half * kGroups + g2;
                    tmem_ld64_max4(tbase + uint32_t(cb0 * 32), rr, mx);
                    if (kGroups == 2) {
                        // this warp's only load of the chunk is complete: hand
                        // the accumulator back before the survivor processing
                        tmem_fence_before();
                        __syncwarp();
                        if (lane == 0) mbar_arrive(tempty_bar(b));
                    }
                    if (ARES || !a.scan_rank) {
                        // chunks of few k-blocks (the resident-query-tile low-d
                        // shapes and short streamed rows): the epilogue's ALU work
                        // bounds the chunk rate, so only the 16-column groups that
                        // may hold a survivor are scanned, and survivors are
                        // ranked by ballot rounds (one round per survivor of the
                        // lane with most)
                        // a 16-column group whose accumulators are all negative
                        // holds no survivor (an acceptable pair's accumulator is
                        // strictly positive); only groups where some lane of the
                        // warp may hold one are scanned
                        bool anyg[4];
#pragma unroll
                        for (int g = 0; g < 4; ++g) anyg[g] = !(mx[g] < 0.f);
                        if (!__any_sync(0xffffffffu, anyg[0] || anyg[1] || anyg[2] || anyg[3])) continue;
                        // bit i of the mask = column cb0 * 32 + i is a survivor:
                        // (mask << 1) | sign per column, highest column first, one
                        // funnel shift each
                        uint32_t neg[2] = {0xffffffffu, 0xffffffffu};
#pragma unroll
                        for (int g = 0; g < 4; ++g) {
                            if (!__any_sync(0xffffffffu, anyg[g])) continue;
                            uint32_t ng = 0;
#pragma unroll
                            for (int i = 15; i >= 0; --i) ng = __funnelshift_l(rr[16 * g + i], ng, 1);
                            const int sh = 16 * (g & 1);
                            neg[g >> 1] = (neg[g >> 1] & ~(0xffffu << sh)) | (ng << sh);
                        }
                        uint64_t mask = qvalid ? ~((uint64_t(neg[1]) << 32) | neg[0]) : 0ull;
                        if (edge) {
                            // validity near the band end and on the diagonal of a
                            // symmetric self-join (rows >= query only)
                            const int64_t jb = j0 + cb0 * 32;
                            const int64_t lim = f.band_hi - jb;
                            if (lim <= 0) mask = 0;
                            else if (lim < 64) mask &= (1ull << lim) - 1ull;
                            if (a.sym) {
                                const int64_t first = q - jb;
                                if (first >= 64) mask = 0;
                                else if (first > 0) mask &= ~((1ull << first) - 1ull);
                            }
                        }
                        // one survivor per lane per round: a ballot ranks them in
                        // the warp's staging buffer
                        const unsigned lt = lanemask_lt();
                        const uint32_t jcol = unsigned(j0 + cb0 * 32);
                        while (__any_sync(0xffffffffu, mask != 0)) {
                            const bool has = mask != 0;
                            const unsigned bal = __ballot_sync(0xffffffffu, has);
                            const int nb = __popc(bal);
                            if (scount + nb > kStg) flush();
                            if (has) {
                                const int i = __ffsll((long long)mask) - 1;
                                mask &= mask - 1;
                                stg[scount + __popc(bal & lt)] = make_uint2(unsigned(q), jcol + unsigned(i));
                            }
                            scount += nb;
                        }
                    } else {
                        // chunks of many k-blocks (MMA-bound): branch-free sign
                        // masks and one prefix sum for the ranks (shorter
                        // dependency chains)
                        // no survivor among the warp's 64 x 32 pairs unless some
                        // 16-column maximum is non-negative (an acceptable pair's
                        // accumulator is strictly positive)
                        const bool anyl = !(mx[0] < 0.f) || !(mx[1] < 0.f) || !(mx[2] < 0.f) || !(mx[3] < 0.f);
                        if (!__any_sync(0xffffffffu, anyl)) continue;
                        // bit i of the mask = column cb0 * 32 + i is a survivor: the
                        // sign bits of the 64 accumulators, gathered by four
                        // independent funnel-shift chains (highest column first)
                        uint32_t ng[4] = {0u, 0u, 0u, 0u};
#pragma unroll
                        for (int i = 15; i >= 0; --i) {
#pragma unroll
                            for (int g = 0; g < 4; ++g) ng[g] = __funnelshift_l(rr[16 * g + i], ng[g], 1);
                        }
                        const uint32_t neg0 = ng[0] | (ng[1] << 16), neg1 = ng[2] | (ng[3] << 16);
                        uint64_t mask = qvalid ? ~((uint64_t(neg1) << 32) | neg0) : 0ull;
                        if (edge) {
                            // validity near the band end and on the diagonal of a
                            // symmetric self-join (rows >= query only)
                            const int64_t jb = j0 + cb0 * 32;
                            const int64_t lim = f.band_hi - jb;
                            if (lim <= 0) mask = 0;
                            else if (lim < 64) mask &= (1ull << lim) - 1ull;
                            if (a.sym) {
                                const int64_t first = q - jb;
                                if (first >= 64) mask = 0;
                                else if (first > 0) mask &= ~((1ull << first) - 1ull);
                            }
                        }
                        // the lanes' survivors in lane order: an exclusive prefix
                        // sum of the per-lane counts places each lane's run
                        const int cnt = __popcll(mask);
                        int incl = cnt;
#pragma unroll
                        for (int o = 1; o < 32; o <<= 1) {
                            const int t = __shfl_up_sync(0xffffffffu, incl, o);
                            if (lane >= o) incl += t;
                        }
                        const int total = __shfl_sync(0xffffffffu, incl, 31);
                        if (total == 0) continue;
                        const uint32_t jcol = unsigned(j0 + cb0 * 32);
                        if (scount + total > kStg) flush();
                        if (total <= kStg) {
                            int pos = scount + incl - cnt;
                            while (mask != 0) {
                                const int i = __ffsll((long long)mask) - 1;
                                mask &= mask - 1;
                                stg[pos++] = make_uint2(unsigned(q), jcol + unsigned(i));
                            }
                            scount += total;
                        } else {
                            // more than the staging buffer holds: straight to the
                            // global list
                            unsigned long long base = 0;
                            if (lane == 0) base = atomicAdd(a.count, (unsigned long long)total);
                            base = __shfl_sync(0xffffffffu, base, 0) + unsigned(incl - cnt);
                            while (mask != 0) {
                                const int i = __ffsll((long long)mask) - 1;
                                mask &= mask - 1;
                                if (base < (unsigned long long)a.cap)
                                    a.surv[base] = make_uint2(unsigned(q), jcol + unsigned(i));
                                ++base;
                            }
                        }
                    }
                }
                if (kGroups != 2) {
                    // the warp's TMEM loads are complete (waited per thread):
                    // one arrival for the whole warp
                    tmem_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(tempty_bar(b));
                }
            }
        }
        flush();
    }
    __syncthreads();
    // every copy this CTA issued lands before its shared memory is released
    // (after an abort some were never consumed): a load into a stage is issued
    // only after the previous load into that stage was consumed, so waiting
    // for the last load of each stage (the last S) and of each query-tile
    // slot (the last two) covers all of them
    if (warp == 0 && lane == 0) {
        for (int it = issued > S ? issued - S : 0; it < issued; ++it)
            mbar_wait_drain(full_bar(it % S), uint32_t(it / S) & 1u, a.err);
        for (int itm = a_issued > 2 ? a_issued - 2 : 0; itm < a_issued; ++itm)
            mbar_wait_drain(afull_bar(itm & 1), uint32_t(itm >> 1) & 1u, a.err);
    }
    tmem_fence_before();
    __syncthreads();
    tmem_fence_after();
    if (warp == 1)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "n"(Sh::kTmemCols)
                     : "memory");
}

// Work list of the tensor-core scorer over tiles of MT x 128 queries.
struct TileSet {
    const int64_t *lo, *hi, *item_off;
    const int32_t *item_tile;
    int ntiles;
};

// Band of a group of mt consecutive 128-query tiles: the union of their bands.
__global__ void k_group_band(const int64_t *__restrict__ tile_lo, const int64_t *__restrict__ tile_hi,
                             int ntiles, int mt, int64_t *__restrict__ lo2, int64_t *__restrict__ hi2,
                             int64_t *__restrict__ items2, int ngroups) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= ngroups) return;
    const int t0 = g * mt, t1 = min(ntiles, t0 + mt);
    int64_t lo = tile_lo[t0], hi = tile_hi[t0];
    for (int t = t0 + 1; t < t1; ++t) {
        lo = min(lo, tile_lo[t]);
        hi = max(hi, tile_hi[t]);
    }
    lo2[g] = lo;
    hi2[g] = hi;
    items2[g] = cdiv(cdiv(hi - lo, kBR), kChunksPerItem);
}

// ------------------------------------------------ operand packing
__device__ __forceinline__ uint16_t bf16_bits(__nv_bfloat16 v) {
    return __bfloat16_as_ushort(v);
}

// Three BF16 parts of a value w given in FP64: w is rounded once to FP32
// (error <= 2^-24 |w|), then split exactly in FP32 (each remainder is exact,
// the last part leaves <= 2^-24 |w|): |w - w1 - w2 - w3| <= 2^-23 |w|.
__device__ __forceinline__ void split3(double w, uint16_t (&o)[3]) {
    float r = (float)w;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const __nv_bfloat16 b = __float2bfloat16_rn(r);
        o[i] = bf16_bits(b);
        r = r - __bfloat162float(b);
    }
}

// How k_tc_pack writes a row: FP16 parts of x 2^sigma (f16 = 1, two parts)
// or BF16 parts of x; the folded columns from fold_col, scaled by fs1 =
// 2^sigma (norms) and fs2 = 2^(2 sigma) (squares).
struct TcPackMode {
    int f16;
    int fold_col;
    float xscale;
    double fs1, fs2;
};

__device__ __forceinline__ uint16_t half_bits(float v) {
    const __half h = __float2half_rn(v);   // v is already an FP16 value
    return *reinterpret_cast<const uint16_t *>(&h);
}

// Rows of an operand: split parts of the centred row, then the folded
// columns (data side: -(1-c) xbar_j split, ||x_j|| rounded up three times,
// ones; query side: ones, c ||y_i|| split, A'_i split).  One warp per 32
// rows: the data columns as a flat run of (row, 4-column quad) items over
// the lanes, eight loads in flight per lane before the conversions (float4
// loads, 8-byte stores, coalesced in both arrays), then the folded columns
// with one lane per row (their few FP64 operations then run on full warps).
// The 32 rows r0 .. r0 + 31 of one warp.
template <int NSPLIT>
__device__ __forceinline__ void tc_pack_warp(int64_t r0, int lane, const float *__restrict__ xc, int dp,
                                             const float *__restrict__ hx, const float *__restrict__ nrm,
                                             const double *__restrict__ Aq, int64_t rows, int d, int K2,
                                             int K2n, double c, int query_side, uint16_t *__restrict__ p0,
                                             uint16_t *__restrict__ p1, uint16_t *__restrict__ p2,
                                             const TcPackMode &pm) {
    const int nr = int(min(int64_t(32), rows - r0));
    // quads over the folded columns are written as zeros here and
    // overwritten below (after __syncwarp)
    const int nq = K2 / 4;                 // quads per packed row
    const int total = nr * nq;
    constexpr int U = 4;
    for (int base = 0; base < total; base += 32 * U) {
        float4 xv[U];
#pragma unroll
        for (int t = 0; t < U; ++t) {
            const int it = base + t * 32 + lane;
            const int rr = it / nq, k0 = (it - rr * nq) * 4;
            xv[t] = (it < total && k0 < dp)
                        ? reinterpret_cast<const float4 *>(xc + (r0 + rr) * dp)[k0 / 4]
                        : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int t = 0; t < U; ++t) {
            const int it = base + t * 32 + lane;
            if (it >= total) break;
            const int rr = it / nq, k0 = (it - rr * nq) * 4;
            const int64_t r = r0 + rr;
            const float xs[4] = {xv[t].x, xv[t].y, xv[t].z, xv[t].w};
            uint16_t v0[4], v1[4], v2[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                v0[e] = v1[e] = v2[e] = 0;
                if (k0 + e < d) {
                    if (NSPLIT == 2 && pm.f16) {
                        // FP16 parts of x 2^sigma (exact scaling, |x 2^sigma| < 2^14);
                        // parts below the FP16 normal range are set to zero, so no
                        // subnormal ever reaches the tensor core
                        const float x = xs[e] * pm.xscale;
                        float hf = __half2float(__float2half_rn(x));
                        if (fabsf(hf) < 0x1p-14f) hf = 0.f;
                        const float xr1 = x - hf;                             // exact
                        float lf = __half2float(__float2half_rn(xr1));
                        if (fabsf(lf) < 0x1p-14f) lf = 0.f;
                        v0[e] = half_bits(hf);
                        v1[e] = half_bits(lf);
                    } else {
                        const float x = xs[e];
                        const __nv_bfloat16 h = __float2bfloat16_rn(x);
                        const float xr1 = x - __bfloat162float(h);               // exact
                        const __nv_bfloat16 l = __float2bfloat16_rn(xr1);
                        v0[e] = bf16_bits(h);
                        v1[e] = bf16_bits(l);
                        if (NSPLIT == 3) v2[e] = bf16_bits(__float2bfloat16_rn(xr1 - __bfloat162float(l)));
                    }
                }
            }
            auto pack4 = [](const uint16_t *v) {
                return make_uint2(uint32_t(v[0]) | (uint32_t(v[1]) << 16),
                                  uint32_t(v[2]) | (uint32_t(v[3]) << 16));
            };
            *reinterpret_cast<uint2 *>(p0 + r * K2 + k0) = pack4(v0);
            // parts 2 and 3 hold data columns only (zero elsewhere), rows of
            // K2n columns
            if (k0 < K2n) {
                if (NSPLIT >= 2) *reinterpret_cast<uint2 *>(p1 + r * K2n + k0) = pack4(v1);
                if (NSPLIT >= 3) *reinterpret_cast<uint2 *>(p2 + r * K2n + k0) = pack4(v2);
            }
        }
    }
    __syncwarp();
    if (lane < nr) {
        // folded columns (BF16) from column fold_col, in the scaled units
        // (x 2^sigma, squares x 2^(2 sigma); both 1 without FP16 parts)
        const int64_t r = r0 + lane;
        uint16_t *f = p0 + r * K2 + pm.fold_col;
        uint16_t sp[3];
        const uint16_t one = bf16_bits(__float2bfloat16_rn(1.0f));
        if (!query_side) {
            split3(-(1.0 - c) * (double)hx[r] * pm.fs2, sp);
            const uint16_t nb = bf16_bits(__float2bfloat16_ru(float((double)nrm[r] * pm.fs1)));
            for (int t = 0; t < 3; ++t) {
                f[t] = sp[t];
                f[3 + t] = nb;
                f[6 + t] = one;
            }
        } else {
            uint16_t sa[3];
            split3(c * (double)nrm[r] * pm.fs1, sp);
            split3(Aq[r] * pm.fs2, sa);
            for (int t = 0; t < 3; ++t) {
                f[t] = one;
                f[3 + t] = sp[t];
                f[6 + t] = sa[t];
            }
        }
    }
}

template <int NSPLIT>
__global__ void __launch_bounds__(256, 4) k_tc_pack(const float *__restrict__ xc, int dp, const float *__restrict__ hx,
                          const float *__restrict__ nrm, const double *__restrict__ Aq,
                          int64_t rows, int d, int K2, int K2n, double c, int query_side,
                          uint16_t *__restrict__ p0, uint16_t *__restrict__ p1,
                          uint16_t *__restrict__ p2, TcPackMode pm) {
    const int64_t r0 = ((int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5) * 32;
    if (r0 >= rows) return;   // whole warps leave together
    tc_pack_warp<NSPLIT>(r0, threadIdx.x & 31, xc, dp, hx, nrm, Aq, rows, d, K2, K2n, c, query_side, p0, p1, p2,
                         pm);
}

// Data rows of every set of a batch group in one launch (two FP16 parts):
// job t owns the warps warp0[t] .. warp0[t + 1] - 1, 32 rows each.
struct TcPackJob {
    const float *xc, *hx, *nrm;
    uint16_t *p0, *p1;
    int64_t rows;
    int d, dp;
    double c;
    TcPackMode pm;
};
__global__ void __launch_bounds__(256, 2) k_tc_pack_jobs(const TcPackJob *__restrict__ jobs,
                                                         const int64_t *__restrict__ warp0, int njobs, int K2,
                                                         int K2n) {
    const int64_t w = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    if (w >= warp0[njobs]) return;
    int lo = 0, hi = njobs - 1;   // last job with warp0 <= w
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (warp0[mid] <= w) lo = mid; else hi = mid - 1;
    }
    const TcPackJob &J = jobs[lo];
    tc_pack_warp<2>((w - warp0[lo]) * 32, threadIdx.x & 31, J.xc, J.dp, J.hx, J.nrm, nullptr, J.rows, J.d, K2, K2n,
                    J.c, 0, J.p0, J.p1, nullptr, J.pm);
}

// ------------------------------------------------ FP8 operand packing
// Two FP32 values rounded to e4m3 (RN, saturating to +-448): hi in bits 8-15,
// lo in bits 0-7; and two e4m3 bytes back to FP32 (exact, through f16).
__device__ __forceinline__ uint32_t e4m3x2(float hi, float lo) {
    unsigned short r;
    asm("cvt.rn.satfinite.e4m3x2.f32 %0, %1, %2;" : "=h"(r) : "f"(hi), "f"(lo));
    return r;
}
__device__ __forceinline__ void e4m3x2_values(uint32_t b2, float &hi, float &lo) {
    uint32_t h2;
    asm("cvt.rn.f16x2.e4m3x2 %0, %1;" : "=r"(h2) : "h"((unsigned short)b2));
    const __half2 hh = *reinterpret_cast<const __half2 *>(&h2);
    lo = __low2float(hh);
    hi = __high2float(hh);
}

__device__ __forceinline__ float warp_sum_ru(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = __fadd_ru(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

__device__ __forceinline__ uint16_t bf16_up(double v) {
    return bf16_bits(__float2bfloat16_ru(__double2float_ru(v)));
}

// The 16 folded BF16 columns of a row scaled by sc = 2^s (every bound entry
// rounded up; the query side's inflated by 1 + 2 kacc):
//   data:  -(1-ch) lead 2^s (split in 3, lead = halved norm) | 2^s x3 | nsum |
//          ||x'|| | ||e_x|| | b9 | b10 | zeros
//   query: 2^s x3 | lead 2^s (split in 3, lead = A'_i) | kacc nsum | ||e_y|| |
//          ||y'|| + ||e_y|| | b9 | b10 | zeros
// (nsum = sum of the parts' norms, e the exact residual of the split, b9 and
// b10 the norms that bound dropped products, zero where none are dropped).
// Their products are the rank-one terms of the bound on x'.y' minus the kept
// products, plus kacc Nx Ny for the accumulation.
__device__ __forceinline__ void write_fold16(uint16_t *__restrict__ out, int query_side, float sc,
                                             double lead, double ch, double kacc, float nsum, float nx,
                                             float ne, double b9, double b10) {
    uint16_t f[16];
#pragma unroll
    for (int t = 0; t < 16; ++t) f[t] = 0;
    const uint16_t one = bf16_bits(__float2bfloat16_rn(sc));   // exact power of two
    uint16_t sp3[3];
    if (!query_side) {
        split3(-(1.0 - ch) * lead * (double)sc, sp3);
        for (int t = 0; t < 3; ++t) {
            f[t] = sp3[t];
            f[3 + t] = one;
        }
        f[6] = bf16_up(nsum);
        f[7] = bf16_up(nx);
        f[8] = bf16_up(ne);
        f[9] = bf16_up(b9);
        f[10] = bf16_up(b10);
    } else {
        const double infl = 1.0 + 2.0 * kacc;
        split3(lead * (double)sc, sp3);
        for (int t = 0; t < 3; ++t) {
            f[t] = one;
            f[3 + t] = sp3[t];
        }
        f[6] = bf16_up(kacc * (double)nsum * infl);
        f[7] = bf16_up((double)ne * infl);
        f[8] = bf16_up(((double)nx + (double)ne) * infl);
        f[9] = bf16_up(b9 * infl);
        f[10] = bf16_up(b10 * infl);
    }
    uint4 *fo = reinterpret_cast<uint4 *>(out);
    const uint32_t *fw = reinterpret_cast<const uint32_t *>(f);
    fo[0] = make_uint4(fw[0], fw[1], fw[2], fw[3]);
    fo[1] = make_uint4(fw[4], fw[5], fw[6], fw[7]);
}

// FP8 rows, one warp per row.  The centred FP32 row x is scaled by 2^s, s
// chosen from its largest |x_k| so that the scaled row x' peaks in
// [128, 256) (clamped to [-23, 24]), and split x' = x_1 + ... + x_P + e with
// e4m3 parts (each the rounding of the remainder, which stays exact in
// FP32).  The norms of x', of the parts and of the residual e are summed with
// upward rounding, so the bounds built from them hold whatever the
// conversion's rounding.  16 folded BF16 columns follow (scaled units):
//   data:  -(1-ch) hx 2^s (split in 3) | 2^s x3 | Nx | ||x'|| | ||e_x|| |
//          ||x_2|| (3 products) or ||x_2||, ||x_3|| (3 parts) | zeros
//   query: 2^s x3 | A'_i 2^s (split in 3) | kacc Ny | ||e_y|| |
//          ||y'|| + ||e_y|| | ||y_2|| or ||y_3||, ||y_2|| + ||y_3|| | zeros
// (Nx = sum of the parts' norms; the query side's bound entries are inflated
// by 1 + 2 kacc.)  Their products are the rank-one terms of the bound on
// x'.y' minus the kept products, plus kacc Nx Ny for the accumulation.
template <int NSPLIT, int NP>
__global__ void k_f8_pack(const float *__restrict__ xc, int dp, const float *__restrict__ hx,
                          const double *__restrict__ Aq, int64_t rows, int d, int K8, double ch,
                          double kacc, int query_side, uint8_t *__restrict__ p0,
                          uint8_t *__restrict__ p1, uint8_t *__restrict__ p2,
                          uint16_t *__restrict__ fold) {
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t(gridDim.x) * blockDim.x) >> 5;
    constexpr int U = 8;                   // quads per lane in flight (1,024 columns a warp)
    const bool one_chunk = K8 <= 128 * U;  // the row stays in registers between the passes
    for (int64_t r = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; r < rows; r += nwarps) {
        const float4 *xr = reinterpret_cast<const float4 *>(xc + r * dp);
        float4 xv[U];
        auto load = [&](int kc) {
#pragma unroll
            for (int t = 0; t < U; ++t) {
                const int k0 = kc + (lane + 32 * t) * 4;
                xv[t] = k0 < d ? xr[k0 / 4] : make_float4(0.f, 0.f, 0.f, 0.f);
            }
        };
        float mx = 0.f;
        for (int kc = 0; kc < d; kc += 128 * U) {
            load(kc);
#pragma unroll
            for (int t = 0; t < U; ++t) {
                const int k0 = kc + (lane + 32 * t) * 4;
                const float xs[4] = {xv[t].x, xv[t].y, xv[t].z, xv[t].w};
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    if (k0 + e < d) mx = fmaxf(mx, fabsf(xs[e]));
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        int sg = 0;
        if (mx > 0.f) {
            int ex;
            frexpf(mx, &ex);                   // mx in [2^(ex-1), 2^ex)
            sg = min(24, max(-23, 8 - ex));
        }
        const float sc = __uint_as_float(uint32_t(127 + sg) << 23);   // 2^sg
        float sx = 0.f, se = 0.f, sp[3] = {0.f, 0.f, 0.f};
        for (int kc = 0; kc < K8; kc += 128 * U) {
            if (!one_chunk) load(kc);
#pragma unroll
            for (int t = 0; t < U; ++t) {
                const int k0 = kc + (lane + 32 * t) * 4;
                if (k0 >= K8) break;
                const float xs[4] = {xv[t].x, xv[t].y, xv[t].z, xv[t].w};
                uint32_t w[3] = {0u, 0u, 0u};
#pragma unroll
                for (int e = 0; e < 4; e += 2) {
                    // elements e (low byte) and e + 1 (high byte) together
                    const float x0 = k0 + e < d ? xs[e] * sc : 0.f;
                    const float x1 = k0 + e + 1 < d ? xs[e + 1] * sc : 0.f;
                    sx = __fmaf_ru(x0, x0, sx);
                    sx = __fmaf_ru(x1, x1, sx);
                    float r0 = x0, r1 = x1;
#pragma unroll
                    for (int p = 0; p < NSPLIT; ++p) {
                        const uint32_t b2 = e4m3x2(r1, r0);
                        float v1, v0;
                        e4m3x2_values(b2, v1, v0);
                        r0 -= v0;                      // exact (v within a factor 2 of r, or 0)
                        r1 -= v1;
                        sp[p] = __fmaf_ru(v0, v0, sp[p]);
                        sp[p] = __fmaf_ru(v1, v1, sp[p]);
                        w[p] |= b2 << (8 * e);
                    }
                    se = __fmaf_ru(r0, r0, se);
                    se = __fmaf_ru(r1, r1, se);
                }
                *reinterpret_cast<uint32_t *>(p0 + r * K8 + k0) = w[0];
                *reinterpret_cast<uint32_t *>(p1 + r * K8 + k0) = w[1];
                if (NSPLIT == 3) *reinterpret_cast<uint32_t *>(p2 + r * K8 + k0) = w[2];
            }
        }
        sx = warp_sum_ru(sx);
        se = warp_sum_ru(se);
#pragma unroll
        for (int p = 0; p < NSPLIT; ++p) sp[p] = warp_sum_ru(sp[p]);
        if (lane == 0) {
            const float nx = __fsqrt_ru(sx);
            // + 2^-100 covers scaling underflow of tiny elements (s < 0)
            const float ne = __fadd_ru(__fsqrt_ru(se), 0x1p-100f);
            float np[3] = {0.f, 0.f, 0.f}, nsum = 0.f;
#pragma unroll
            for (int p = 0; p < NSPLIT; ++p) {
                np[p] = __fsqrt_ru(sp[p]);
                nsum = __fadd_ru(nsum, np[p]);
            }
            // the dropped products' norms: x_2.y_2 (three products), or
            // x_2.y_3 + x_3.y_2 + x_3.y_3 (three parts)
            double b9 = 0.0, b10 = 0.0;
            if (!query_side) {
                if (NP == 3 || NP == 6) b9 = np[1];
                if (NP == 6) b10 = np[2];
            } else {
                if (NP == 3) b9 = np[1];
                if (NP == 6) {
                    b9 = np[2];
                    b10 = (double)np[1] + (double)np[2];
                }
            }
            write_fold16(fold + r * 16, query_side, sc, query_side ? Aq[r] : (double)hx[r], ch, kacc, nsum,
                         nx, ne, b9, b10);
        }
    }
}

// One FP16 part per row (the single-part 16-bit scorer), one warp per row.
// The centred FP32 row x is scaled by 2^s, s from its largest |x_k| so that
// the scaled row x' peaks in [2^14, 2^15) (clamped to [-23, 24]), and
// rounded once to FP16: x' = x_1 + e, with x_1 set to zero where it would
// fall below the FP16 normal range (or above its largest finite value) and
// the residual e exact in FP32 (Sterbenz).  The norms of x', x_1 and e are
// summed with upward rounding; the 16 folded BF16 columns (write_fold16: one
// part, no dropped products) bound x'.y' - x_1.y_1 = x'.e_y + e_x.y' - e_x.e_y
// and the accumulation per pair.  Rows of K2 FP16 values (zero beyond d).
__global__ void k_h1_pack(const float *__restrict__ xc, int dp, const float *__restrict__ hx,
                          const double *__restrict__ Aq, int64_t rows, int d, int K2, double ch,
                          double kacc, int query_side, uint16_t *__restrict__ p0,
                          uint16_t *__restrict__ fold) {
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t(gridDim.x) * blockDim.x) >> 5;
    constexpr int U = 8;                   // quads per lane in flight (1,024 columns a warp)
    const bool one_chunk = K2 <= 128 * U;  // the row stays in registers between the passes
    for (int64_t r = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; r < rows; r += nwarps) {
        const float4 *xr = reinterpret_cast<const float4 *>(xc + r * dp);
        float4 xv[U];
        auto load = [&](int kc) {
#pragma unroll
            for (int t = 0; t < U; ++t) {
                const int k0 = kc + (lane + 32 * t) * 4;
                xv[t] = k0 < d ? xr[k0 / 4] : make_float4(0.f, 0.f, 0.f, 0.f);
            }
        };
        float mx = 0.f;
        for (int kc = 0; kc < d; kc += 128 * U) {
            load(kc);
#pragma unroll
            for (int t = 0; t < U; ++t) {
                const int k0 = kc + (lane + 32 * t) * 4;
                const float xs[4] = {xv[t].x, xv[t].y, xv[t].z, xv[t].w};
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    if (k0 + e < d) mx = fmaxf(mx, fabsf(xs[e]));
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        int sg = 0;
        if (mx > 0.f) {
            int ex;
            frexpf(mx, &ex);                   // mx in [2^(ex-1), 2^ex)
            sg = min(24, max(-23, 15 - ex));
        }
        const float sc = __uint_as_float(uint32_t(127 + sg) << 23);   // 2^sg
        float sx = 0.f, se = 0.f, s1 = 0.f;
        for (int kc = 0; kc < K2; kc += 128 * U) {
            if (!one_chunk) load(kc);
#pragma unroll
            for (int t = 0; t < U; ++t) {
                const int k0 = kc + (lane + 32 * t) * 4;
                if (k0 >= K2) break;
                const float xs[4] = {xv[t].x, xv[t].y, xv[t].z, xv[t].w};
                uint16_t hb[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const float x = k0 + e < d ? xs[e] * sc : 0.f;
                    const __half h = __float2half_rn(x);
                    float hf = __half2float(h);
                    const bool keep = fabsf(hf) >= 0x1p-14f && fabsf(hf) <= 65504.f;
                    hf = keep ? hf : 0.f;
                    const float rr = x - hf;   // exact: hf is 0 or within a factor 2 of x
                    sx = __fmaf_ru(x, x, sx);
                    s1 = __fmaf_ru(hf, hf, s1);
                    se = __fmaf_ru(rr, rr, se);
                    hb[e] = keep ? *reinterpret_cast<const uint16_t *>(&h) : uint16_t(0);
                }
                *reinterpret_cast<uint2 *>(p0 + r * K2 + k0) =
                    make_uint2(uint32_t(hb[0]) | (uint32_t(hb[1]) << 16), uint32_t(hb[2]) | (uint32_t(hb[3]) << 16));
            }
        }
        sx = warp_sum_ru(sx);
        se = warp_sum_ru(se);
        s1 = warp_sum_ru(s1);
        if (lane == 0) {
            const float nx = __fsqrt_ru(sx);
            const float ne = __fadd_ru(__fsqrt_ru(se), 0x1p-100f);
            const float n1 = __fsqrt_ru(s1);
            write_fold16(fold + r * 16, query_side, sc, query_side ? Aq[r] : (double)hx[r], ch, kacc, n1,
                         nx, ne, 0.0, 0.0);
        }
    }
}

// 1 / (1 - delta) rounded up and 1 / (1 + delta) rounded down: multiplying by
// them (product rounded up) bounds A / (1 -+ delta) from above for A >= 0 and
// A < 0 alike, without an FP64 division per query.
struct DeltaInv {
    double inv_m, inv_p;
};
inline DeltaInv delta_inv(double delta) {
    return DeltaInv{std::nextafter(1.0 / (1.0 - delta), INFINITY), std::nextafter(1.0 / (1.0 + delta), 0.0)};
}

// A'_i >= (Rx + e_data + e_i)^2/2 - ||y_i||^2/2, inflated so that its split
// representation and the accumulation rounding (delta) keep the sign test
// conservative, plus a margin that makes an acceptable pair's acc positive.
__global__ void k_tc_query_consts(const float *__restrict__ hy, const float *__restrict__ qn,
                                  int64_t m, int d, double Rx, double e_data, DeltaInv di,
                                  double margin, double *__restrict__ Aq, const double *__restrict__ Rq,
                                  double abs_n, double abs_q) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= m) return;
    const double ei = 1.0001 * (double)kU32 * (double)qn[i];
    const double r = (Rq ? radius_slack(Rq[i], d) : Rx) + e_data + ei;
    const double hy_low = (double)hy[i] * (1.0 - 1.05 * (d + 2) * (double)kU32);
    // abs_n + abs_q ||y||: the absolute part of the FP16 split bound (0 for
    // BF16 parts)
    double A = 0.5 * r * r - hy_low + (abs_n + abs_q * (double)qn[i]);
    A += 4.0 * kU64 * (fabs(A) + 0.5 * r * r + (double)hy[i]);
    A = A >= 0.0 ? __dmul_ru(A, di.inv_m) : __dmul_ru(A, di.inv_p);
    A += 0x1p-22 * fabs(A) + margin;
    Aq[i] = A;
}

// Rounding constant c of the folded test for a split and a dimension.
double tc_constant(int nsplit, int d, double *u_k_out, bool f16) {
    const int ksteps_data = int(cdiv(d, 16));
    // FP16 parts: the folded columns take a k step of their own
    const int ksteps = f16 ? ksteps_data + 1 : int(cdiv(d + kExtra, 16));
    const int ninstr = tc_npairs(nsplit) * ksteps_data + (ksteps - ksteps_data);
    // FP32 accumulation: each MMA instruction is charged 2^-22 of (|C_in| +
    // sum of its |products|), i.e. (ninstr + 1) 2^-22 of all |products|
    const double u_k = 0x1p-22 * (ninstr + 1);
    // dropped split terms, relative to sum |x_k y_k|: BF16 parts 3.1 2^-16
    // (two) or 4.2 2^-24 (three); two FP16 parts 3.01 2^-22 (x2.y2 + a.e_y +
    // e_x.y', each part within half an FP16 ulp), plus an absolute part for
    // the parts set to zero below the FP16 normal range (in the constants A)
    const double quant = f16 ? 3.01 * 0x1p-22 : (nsplit == 2 ? 3.1 * 0x1p-16 : 4.2 * 0x1p-24);
    const double c_mn = (quant + 1.01 * u_k) / (1.0 - 0x1p-23 - u_k);
    const double c_hx = 0x1p-23 + 1.05 * (d + 2) * 0x1p-24 + u_k;
    if (u_k_out) *u_k_out = u_k;
    return 1.02 * (c_mn > c_hx ? c_mn : c_hx);
}

// Work list, survivor output and error flag of a scoring launch.
TcArgs tc_args(const snn_index *ix, const ScoreArgs &sa, const TileSet &ts) {
    TcArgs a;
    a.m = sa.q.m;
    a.n = ix->n;
    a.ksteps = 0;
    a.ksteps_data = 0;
    a.nkb = 0;
    a.tile_lo = ts.lo;
    a.tile_hi = ts.hi;
    a.item_off = ts.item_off;
    a.item_tile = ts.item_tile;
    a.ntiles = ts.ntiles;
    a.sym = sa.sym;
    a.surv = sa.surv;
    a.cap = sa.cap;
    a.count = sa.count;
    a.err = sa.err;
    a.stall = take_fault(SNN_FAULT_STALL_TC_PRODUCER) ? 1 : 0;
    a.f16 = 0;
    a.scan_rank = 0;
    return a;
}

// maps: query parts 1-3, data parts 1-3, query folded, data folded
template <int NSPLIT, int BK, int BN, bool ARES, int CPS, int NW, int MT, int F8NP>
snn_status run_tc(const CUtensorMap (&maps)[8], const TcArgs &a, const ScoreArgs &sa, cudaStream_t s) {
    using Sh = TcShape<NSPLIT, BK, BN, ARES, CPS, NW, MT, F8NP>;
    auto kern = k_score_tc<NSPLIT, BK, BN, ARES, CPS, NW, MT, F8NP>;
    SNN_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(Sh::kSmem)));
    if (sa.ev_kernel[0]) cudaEventRecord(sa.ev_kernel[0], s);
    SNN_LAUNCH(kern, device_sm_count() * CPS, Sh::kThreads, Sh::kSmem, s)(
        maps[0], maps[1], maps[2], maps[3], maps[4], maps[5], maps[6], maps[7], a);
    SNN_LAUNCH_CHECK();
    if (sa.ev_kernel[1]) cudaEventRecord(sa.ev_kernel[1], s);
    return SNN_OK;
}

template <int NSPLIT, int BK, int BN, bool ARES, int CPS, int NW, int MT>
snn_status launch_tc(const snn_index *ix, const snn_tc_operands &op, const ScoreArgs &sa,
                     const uint16_t *const *qp, int K2, int K2n, const TileSet &ts, cudaStream_t s,
                     int f16) {
    CUtensorMap maps[8];
    for (int p = 0; p < 3; ++p) {
        const int pp = p < NSPLIT ? p : 0;
        const int k2 = pp == 0 ? K2 : K2n, box = pp == 0 ? BK : NW;
        SNN_TRY(make_map(&maps[p], qp[pp], sa.q.m, k2, box, kTM * MT));
        SNN_TRY(make_map(&maps[3 + p], static_cast<const uint16_t *>(op.part[pp]), ix->n, k2, box, BN));
    }
    maps[6] = maps[0];   // no folded block of its own
    maps[7] = maps[3];
    TcArgs a = tc_args(ix, sa, ts);
    a.ksteps_data = int(cdiv(ix->d, 16));
    a.ksteps = f16 ? a.ksteps_data + 1 : int(cdiv(ix->d + kExtra, 16));
    a.nkb = K2 / BK;
    a.f16 = f16;
    return run_tc<NSPLIT, BK, BN, ARES, CPS, NW, MT, 0>(maps, a, sa, s);
}

// FP8 shape: 128 queries x 256 band rows, k-blocks of 2 BK bytes per row (BK
// 16-bit pairs; one or two e4m3 K = 32 steps of F8NP products each; a block
// that reaches past the row is zero-filled by the copy), then the folded BF16
// block.  64-byte blocks halve the copy's row requests per MMA, which is what
// bounds the two-part variants with 32-byte blocks.
template <int NSPLIT, int F8NP, int BK>
snn_status launch_f8(const snn_index *ix, const snn_tc_operands &op, const ScoreArgs &sa,
                     uint8_t *const *qp, const uint16_t *qfold, int K8, const TileSet &ts, cudaStream_t s) {
    CUtensorMap maps[8];
    for (int p = 0; p < 3; ++p) {
        const int pp = p < NSPLIT ? p : 0;
        // e4m3 rows as 16-bit pairs: K8 / 2 elements, boxes of BK pairs
        SNN_TRY(make_map(&maps[p], reinterpret_cast<const uint16_t *>(qp[pp]), sa.q.m, K8 / 2, BK, kTM));
        SNN_TRY(make_map(&maps[3 + p], static_cast<const uint16_t *>(op.part[pp]), ix->n, K8 / 2, BK, 256));
    }
    SNN_TRY(make_map(&maps[6], qfold, sa.q.m, 16, 16, kTM));
    SNN_TRY(make_map(&maps[7], op.fold, ix->n, 16, 16, 256));
    TcArgs a = tc_args(ix, sa, ts);
    a.ksteps_data = K8 / 32;
    a.nkb = int(cdiv(K8, 2 * BK)) + 1;
    return run_tc<NSPLIT, BK, 256, false, 1, BK, 1, F8NP>(maps, a, sa, s);
}

// The operands of `kind` (row widths k2, k2n, scale sigma) from the index's
// cache, packed on stream s by `pack` (which receives the new entry with its
// arrays allocated) when the cache has none.  s then waits for the entry's
// ready event, so an entry packed on another stream is complete before the
// scorer reads it.  Entries are never replaced while the index lives.
template <class Pack>
snn_status cached_operands(snn_index *ix, int kind, int k2, int k2n, int sigma, const size_t (&bytes)[4],
                           cudaStream_t s, Pack &&pack, const snn_tc_operands **out) {
    std::lock_guard<std::mutex> lk(ix->mu);
    snn_tc_operands *hit = nullptr, *slot = nullptr;
    for (auto &e : ix->tc_ops) {
        if (e.kind == kind && e.k2 == k2 && e.k2n == k2n && e.sigma == sigma) {
            hit = &e;
            break;
        }
        if (!e.kind && !slot) slot = &e;
    }
    if (!hit) {
        if (!slot) {
            set_error("tensor-core operand cache of the index is full");
            return SNN_ENOTSUP;
        }
        snn_tc_operands e;
        e.kind = kind;
        e.k2 = k2;
        e.k2n = k2n;
        e.sigma = sigma;
        cudaError_t err = cudaSuccess;
        for (int p = 0; p < 3 && err == cudaSuccess; ++p)
            if (bytes[p]) err = cudaMallocAsync(&e.part[p], bytes[p], s);
        if (err == cudaSuccess && bytes[3])
            err = cudaMallocAsync(reinterpret_cast<void **>(&e.fold), bytes[3], s);
        if (err == cudaSuccess) err = cudaEventCreateWithFlags(&e.ready, cudaEventDisableTiming);
        snn_status st = SNN_OK;
        if (err != cudaSuccess) {
            cudaGetLastError();
            set_error("tensor-core operand allocation failed: %s", cudaGetErrorString(err));
            st = SNN_ENOMEM;
        } else {
            st = pack(e);
            if (st == SNN_OK && cudaEventRecord(e.ready, s) != cudaSuccess) {
                set_error("cudaEventRecord failed");
                st = SNN_ECUDA;
            }
        }
        if (st != SNN_OK) {
            for (void *p : e.part)
                if (p) cudaFreeAsync(p, s);
            if (e.fold) cudaFreeAsync(e.fold, s);
            if (e.ready) cudaEventDestroy(e.ready);
            return st;
        }
        *slot = e;
        hit = slot;
    }
    SNN_CUDA(cudaStreamWaitEvent(s, hit->ready, 0));
    *out = hit;
    return SNN_OK;
}

}  // namespace

void release_tc_operands(snn_index *ix, cudaStream_t s) {
    for (auto &e : ix->tc_ops) {
        for (void *p : e.part)
            if (p) cudaFreeAsync(p, s);
        if (e.fold) cudaFreeAsync(e.fold, s);
        if (e.ready) cudaEventDestroy(e.ready);
        e = snn_tc_operands();
    }
}

bool f8_eligible(const snn_index *ix, double Rx) {
    return ix->d + kExtra > 64 && double(ix->nrm_max) <= 0x1p20 && Rx <= 0x1p20;
}

snn_status f8_score_launch(const snn_index *ixc, const ScoreArgs &sa, cudaStream_t s, double Rx,
                           double e_data, Scratch &scr, int64_t *mma_flops_per_pair, int *split_used) {
    snn_index *ix = const_cast<snn_index *>(ixc);
    const int d = ix->d;
    // products per k-step: the cheapest split whose bound stays a small
    // fraction of R^2.  Two parts leave about 2.5e-3 (three products) or
    // 1.8e-3 (four, x_2.y_2 kept) of ||x|| ||y|| unresolved, three parts
    // about 1e-4; twice that for the largest norms should stay within 1.5 %
    // of R^2, which keeps the extra exact decisions small (normalised rows:
    // three products; the 784-dim images, norms 3.5x R: six).
    // SNN_FP8_PRODUCTS = 3, 4 or 6 overrides.
    const double N2 = double(ix->nrm_max) * double(ix->nrm_max), R2r = Rx * Rx;
    int np = N2 <= 3.0 * R2r ? 3 : (N2 <= 4.2 * R2r ? 4 : 6);
    if (const char *e = getenv("SNN_FP8_PRODUCTS")) {
        const int v = atoi(e);
        if (v == 3 || v == 4 || v == 6) np = v;
    }
    const int nsplit = np == 6 ? 3 : 2;
    if (split_used) *split_used = SNN_SPLIT_E4M3 + np;
    const int K8 = int(cdiv(d, 32) * 32);
    const int ksteps = K8 / 32;
    // accumulation: every instruction (e4m3 or the folded BF16 step) is
    // charged 2^-20 of its input accumulator plus its products
    const int ninstr = ksteps * np + 1;
    const double kacc = 0x1p-20 * (ninstr + 1);
    // halved norm: its FP32 evaluation, its 3-part split, the accumulation
    const double ch = 1.02 * (0x1p-23 + 1.05 * (d + 2) * 0x1p-24 + kacc);
    const int pack_threads = 256;
    auto pack_grid = [&](int64_t rows) {
        return unsigned(std::min<int64_t>(cdiv(rows, pack_threads / 32), int64_t(16) * device_sm_count()));
    };
    auto packer = np == 3 ? k_f8_pack<2, 3> : (np == 4 ? k_f8_pack<2, 4> : k_f8_pack<3, 6>);
    const size_t pb = size_t(ix->n) * K8;
    const size_t bytes[4] = {pb, pb, nsplit == 3 ? pb : 0, size_t(ix->n) * 16 * sizeof(uint16_t)};
    const snn_tc_operands *op = nullptr;
    SNN_TRY(cached_operands(ix, SNN_SPLIT_E4M3 + np, K8, K8, 0, bytes, s,
                            [&](snn_tc_operands &e) -> snn_status {
                                SNN_LAUNCH(packer, pack_grid(ix->n), pack_threads, 0, s)(
                                    ix->xc, ix->dp, ix->hx, nullptr, ix->n, d, K8, ch, kacc, 0,
                                    static_cast<uint8_t *>(e.part[0]), static_cast<uint8_t *>(e.part[1]),
                                    static_cast<uint8_t *>(e.part[2]), e.fold);
                                SNN_LAUNCH_CHECK();
                                return SNN_OK;
                            },
                            &op));
    if (mma_flops_per_pair) *mma_flops_per_pair = int64_t(2) * 32 * np * ksteps + 2 * 16;
    const int64_t m = sa.q.m;
    double *Aq;
    uint8_t *qp[3] = {nullptr, nullptr, nullptr};
    uint16_t *qfold;
    SNN_TRY(scr.alloc(&Aq, m));
    for (int p = 0; p < nsplit; ++p) SNN_TRY(scr.alloc(&qp[p], size_t(m) * K8));
    SNN_TRY(scr.alloc(&qfold, size_t(m) * 16));
    // a margin of 2^-60 keeps A'_i 2^(s_x + s_y) a normal FP32 number
    SNN_LAUNCH(k_tc_query_consts, unsigned(cdiv(m, 256)), 256, 0, s)(
        sa.q.hx, sa.q.nrm, m, d, Rx, e_data, delta_inv(0x1p-23 + kacc), 0x1p-60, Aq, sa.Rq, 0.0, 0.0);
    SNN_LAUNCH_CHECK();
    SNN_LAUNCH(packer, pack_grid(m), pack_threads, 0, s)(sa.q.xc, ix->dp, nullptr, Aq, m, d, K8, ch,
                                                        kacc, 1, qp[0], qp[1], qp[2], qfold);
    SNN_LAUNCH_CHECK();
    TileSet ts1{sa.tile_lo, sa.tile_hi, sa.item_off, sa.item_tile, sa.ntiles};
    // 64-byte k-blocks: four stages of 48 KB (two parts) or three of 72 KB
    if (np == 3) return launch_f8<2, 3, 32>(ix, *op, sa, qp, qfold, K8, ts1, s);
    if (np == 4) return launch_f8<2, 4, 32>(ix, *op, sa, qp, qfold, K8, ts1, s);
    return launch_f8<3, 6, 32>(ix, *op, sa, qp, qfold, K8, ts1, s);
}

namespace {

// One FP16 part per row (per-row power-of-two scales) with the per-pair
// residual bound folded into a separate BF16 k-block: one MMA per 16-column
// k step.  Streamed shape: 128 queries x 256 band rows, 32-column k-blocks.
snn_status h1_score_launch(snn_index *ix, const ScoreArgs &sa, cudaStream_t s, double Rx, double e_data,
                           Scratch &scr, int64_t *mma_flops_per_pair) {
    const int d = ix->d;
    const int K2 = int(cdiv(d, 16) * 16);
    const int ksteps = K2 / 16;
    // accumulation: every instruction (the FP16 steps and the folded BF16
    // step) is charged 2^-22 of its input accumulator plus its products
    const double kacc = 0x1p-22 * (ksteps + 2);
    // halved norm: its FP32 evaluation, its 3-part split, the accumulation
    const double ch = 1.02 * (0x1p-23 + 1.05 * (d + 2) * 0x1p-24 + kacc);
    const int pack_threads = 256;
    auto pack_grid = [&](int64_t rows) {
        return unsigned(std::min<int64_t>(cdiv(rows, pack_threads / 32), int64_t(16) * device_sm_count()));
    };
    const size_t bytes[4] = {size_t(ix->n) * K2 * sizeof(uint16_t), 0, 0, size_t(ix->n) * 16 * sizeof(uint16_t)};
    const snn_tc_operands *op = nullptr;
    SNN_TRY(cached_operands(ix, SNN_SPLIT_FP16X1, K2, 0, 0, bytes, s,
                            [&](snn_tc_operands &e) -> snn_status {
                                SNN_LAUNCH(k_h1_pack, pack_grid(ix->n), pack_threads, 0, s)(
                                    ix->xc, ix->dp, ix->hx, nullptr, ix->n, d, K2, ch, kacc, 0,
                                    static_cast<uint16_t *>(e.part[0]), e.fold);
                                SNN_LAUNCH_CHECK();
                                return SNN_OK;
                            },
                            &op));
    if (mma_flops_per_pair) *mma_flops_per_pair = int64_t(2) * 16 * (ksteps + 1);
    const int64_t m = sa.q.m;
    double *Aq;
    uint16_t *qp, *qfold;
    SNN_TRY(scr.alloc(&Aq, m));
    SNN_TRY(scr.alloc(&qp, size_t(m) * K2));
    SNN_TRY(scr.alloc(&qfold, size_t(m) * 16));
    // a margin of 2^-60 keeps A'_i 2^(s_x + s_y) a normal FP32 number
    SNN_LAUNCH(k_tc_query_consts, unsigned(cdiv(m, 256)), 256, 0, s)(
        sa.q.hx, sa.q.nrm, m, d, Rx, e_data, delta_inv(0x1p-23 + kacc), 0x1p-60, Aq, sa.Rq, 0.0, 0.0);
    SNN_LAUNCH_CHECK();
    SNN_LAUNCH(k_h1_pack, pack_grid(m), pack_threads, 0, s)(sa.q.xc, ix->dp, nullptr, Aq, m, d, K2, ch, kacc,
                                                           1, qp, qfold);
    SNN_LAUNCH_CHECK();
    // two query tiles per work item by default: each band k-block feeds four
    // 128 x 256 MMAs (32 KB per k-block instead of 24 KB for two), the
    // accumulators fill TMEM in one buffer (a chunk of ~26 k-blocks makes the
    // hand-off a small fraction of its MMAs); SNN_H1_TILES=1 keeps one tile
    const char *et = getenv("SNN_H1_TILES");
    const int MTq = (et && et[0] == '1') ? 1 : 2;
    CUtensorMap maps[8];
    SNN_TRY(make_map(&maps[0], qp, m, K2, 32, kTM * MTq));
    SNN_TRY(make_map(&maps[3], static_cast<const uint16_t *>(op->part[0]), ix->n, K2, 32, 256));
    maps[1] = maps[2] = maps[0];
    maps[4] = maps[5] = maps[3];
    SNN_TRY(make_map(&maps[6], qfold, m, 16, 16, kTM * MTq));
    SNN_TRY(make_map(&maps[7], op->fold, ix->n, 16, 16, 256));
    TileSet ts{sa.tile_lo, sa.tile_hi, sa.item_off, sa.item_tile, sa.ntiles};
    if (MTq == 2) {
        const int ng = int(cdiv(sa.ntiles, 2));
        int64_t *lo2, *hi2, *items2, *off2;
        int32_t *it2;
        SNN_TRY(scr.alloc(&lo2, ng));
        SNN_TRY(scr.alloc(&hi2, ng));
        SNN_TRY(scr.alloc(&items2, ng));
        SNN_TRY(scr.alloc(&off2, ng + 1));
        SNN_LAUNCH(k_group_band, unsigned(cdiv(ng, 128)), 128, 0, s)(sa.tile_lo, sa.tile_hi, sa.ntiles, 2, lo2,
                                                                     hi2, items2, ng);
        SNN_LAUNCH_CHECK();
        SNN_TRY(scan_exclusive<int64_t>(items2, off2, ng, s));
        const int64_t max_items = int64_t(ng) * (cdiv(ix->n, int64_t(kBR) * kChunksPerItem) + 1);
        SNN_TRY(scr.alloc(&it2, max_items));
        SNN_LAUNCH(k_item_tiles, unsigned(cdiv(ng, 128)), 128, 0, s)(off2, ng, it2);
        SNN_LAUNCH_CHECK();
        ts = TileSet{lo2, hi2, off2, it2, ng};
    }
    TcArgs a = tc_args(ix, sa, ts);
    a.ksteps_data = ksteps;
    a.nkb = int(cdiv(K2, 32)) + 1;
    // with 12 or more k-blocks per chunk the MMAs, not the epilogue, set the
    // chunk rate (measured: 784 columns faster, 100 columns slower with it)
    a.scan_rank = a.nkb >= 12 ? 1 : 0;
    return MTq == 2 ? run_tc<1, 32, 256, false, 1, 32, 2, 0>(maps, a, sa, s)
                    : run_tc<1, 32, 256, false, 1, 32, 1, 0>(maps, a, sa, s);
}

}  // namespace

snn_status tc_score_launch(const snn_index *ixc, const ScoreArgs &sa, cudaStream_t s,
                           double Rx, double e_data, Scratch &scr, int64_t *mma_flops_per_pair,
                           int *split_used) {
    snn_index *ix = const_cast<snn_index *>(ixc);
    const int d = ix->d;
    const double Nd = (double)ix->nrm_max, Nq = sa.q_nrm_max;
    // operands, chosen by how tight their bound is against R^2 for the
    // largest norms:
    // * one FP16 part per row (per-row scales, the per-pair bound built from
    //   the exact residual norms): one MMA per k step.  Streamed shape only
    //   (d + 9 > 64) and norms below 2^20.  Its residual is typically about
    //   2^-12 of the row norm, so the bound is about 4 2^-12 ||x|| ||y||;
    // * two BF16 parts where their bound stays a small fraction of R^2/2
    //   (high d, moderate norms);
    // * else two FP16 parts of the rows scaled by 2^sigma, which need the
    //   MMAs of two BF16 parts and bound the dropped terms as tightly as three
    //   BF16 parts do.
    // SNN_TC_SPLIT = fp16x1, bf16x2, bf16x3 or fp16x2 overrides (fp16x1 only
    // where its shape and ranges allow it).
    const bool h1_ok = d + kExtra > 64 && Nd <= 0x1p20 && Nq <= 0x1p20 && Rx <= 0x1p20;
    bool h1 = h1_ok && 4.0 * 0x1p-12 * Nd * Nq <= 0.02 * Rx * Rx;
    const double c2 = tc_constant(2, d, nullptr, false);
    bool f16 = !(c2 * 1.5 * Nd * Nd <= 0.02 * 0.5 * Rx * Rx);
    int nsplit = 2;
    if (const char *e = getenv("SNN_TC_SPLIT")) {
        if (!strcmp(e, "bf16x2")) f16 = false, h1 = false;
        else if (!strcmp(e, "bf16x3")) f16 = false, nsplit = 3, h1 = false;
        else if (!strcmp(e, "fp16x2")) f16 = true, h1 = false;
        else if (!strcmp(e, "fp16x1")) h1 = h1_ok;
    }
    if (h1) {
        if (split_used) *split_used = SNN_SPLIT_FP16X1;
        return h1_score_launch(ix, sa, s, Rx, e_data, scr, mma_flops_per_pair);
    }
    // sigma, from the index alone: the largest centred data norm, scaled,
    // lies in [2^13, 2^14), so every scaled data coordinate is an FP16
    // number.  Query coordinates are at most the query norms; where those,
    // scaled, could leave the FP16 range this call takes BF16 parts.
    int sigma = 0;
    if (Nd > 0.0) sigma = std::min(120, std::max(-120, 13 - std::ilogb(Nd)));
    if (f16 && !(std::ldexp(Nq, sigma) <= 60000.0)) f16 = false;
    if (!f16) sigma = 0;
    const double fs1 = std::ldexp(1.0, sigma), fs2 = std::ldexp(1.0, 2 * sigma);
    double u_k = 0.0;
    const double c = tc_constant(nsplit, d, &u_k, f16);
    // absolute part of the FP16 bound, in unscaled units: 1.001 2^-14 sqrt(d)
    // (||x'|| + ||y'||) + 2 d 2^-28 in scaled units (parts below 2^-14 are zero)
    const double abs_q = f16 ? 1.001 * std::sqrt(double(d)) * std::ldexp(1.0, -14 - sigma) : 0.0;
    const double abs_n = f16 ? abs_q * Nd + 2.0 * d * std::ldexp(1.0, -28 - 2 * sigma) : 0.0;
    // shape: one 32- or 64-column k-block holds everything for low d (query
    // tile resident for a whole item); 64-column k-blocks streamed otherwise.
    // With FP16 parts the folded columns start on a k step boundary.
    const int kind = f16 ? SNN_SPLIT_FP16X2 : (nsplit == 3 ? SNN_SPLIT_BF16X3 : SNN_SPLIT_BF16X2);
    if (split_used) *split_used = kind;
    const int fold_col = f16 ? int(cdiv(d, 16) * 16) : d;
    const int kp = fold_col + kExtra;
    const int bk = kp <= 32 ? 32 : 64;
    const int K2 = int(cdiv(kp, bk) * bk);
    // parts 2 and 3 carry no folded columns: with every data column inside
    // the first 16, their rows are 16 columns wide (low-d shape only)
    const int K2n = (kp <= 32 && d <= 16) ? 16 : K2;
    const TcPackMode pm{f16 ? 1 : 0, fold_col, float(fs1), fs1, fs2};
    const size_t bytes[4] = {size_t(ix->n) * K2 * sizeof(uint16_t), size_t(ix->n) * K2n * sizeof(uint16_t),
                             nsplit == 3 ? size_t(ix->n) * K2n * sizeof(uint16_t) : 0, 0};
    const snn_tc_operands *op = nullptr;
    SNN_TRY(cached_operands(ix, kind, K2, K2n, sigma, bytes, s,
                            [&](snn_tc_operands &e) -> snn_status {
                                auto packer = nsplit == 2 ? k_tc_pack<2> : k_tc_pack<3>;
                                SNN_LAUNCH(packer, unsigned(cdiv(cdiv(ix->n, 32) * 32, 256)), 256, 0, s)(
                                    ix->xc, ix->dp, ix->hx, ix->nrm, nullptr, ix->n, d, K2, K2n, c, 0,
                                    static_cast<uint16_t *>(e.part[0]), static_cast<uint16_t *>(e.part[1]),
                                    static_cast<uint16_t *>(e.part[2]), pm);
                                SNN_LAUNCH_CHECK();
                                return SNN_OK;
                            },
                            &op));
    if (mma_flops_per_pair) {
        const int64_t ks_data = cdiv(d, 16), ks_all = f16 ? ks_data + 1 : cdiv(d + kExtra, 16);
        *mma_flops_per_pair = int64_t(2) * 16 * (ks_data * tc_npairs(nsplit) + (ks_all - ks_data));
    }
    // query operands (per call): same split, query-side folded columns
    const int64_t m = sa.q.m;
    double *Aq;
    uint16_t *qp[3] = {nullptr, nullptr, nullptr};
    SNN_TRY(scr.alloc(&Aq, m));
    for (int p = 0; p < nsplit; ++p) SNN_TRY(scr.alloc(&qp[p], size_t(m) * (p == 0 ? K2 : K2n)));
    SNN_LAUNCH(k_tc_query_consts, unsigned(cdiv(m, 256)), 256, 0, s)(
        sa.q.hx, sa.q.nrm, m, d, Rx, e_data, delta_inv(0x1p-23 + u_k), 0x1p-100, Aq, sa.Rq, abs_n, abs_q);
    SNN_LAUNCH_CHECK();
    auto packer = nsplit == 2 ? k_tc_pack<2> : k_tc_pack<3>;
    SNN_LAUNCH(packer, unsigned(cdiv(cdiv(m, 32) * 32, 256)), 256, 0, s)(sa.q.xc, ix->dp, sa.q.hx,
                                                                       sa.q.nrm, Aq,
                                                            m, d, K2, K2n, c, 1, qp[0], qp[1], qp[2], pm);
    SNN_LAUNCH_CHECK();
    const int F = f16 ? 1 : 0;
    TileSet ts1{sa.tile_lo, sa.tile_hi, sa.item_off, sa.item_tile, sa.ntiles};
    if (kp <= 32 && K2n == 16) {
        // low d: the band traffic per pair dominates, so every band chunk is
        // multiplied with two query tiles (256 queries) sharing its load
        constexpr int MT = 2;
        const int ng = int(cdiv(sa.ntiles, MT));
        int64_t *lo2, *hi2, *items2, *off2;
        int32_t *it2;
        SNN_TRY(scr.alloc(&lo2, ng));
        SNN_TRY(scr.alloc(&hi2, ng));
        SNN_TRY(scr.alloc(&items2, ng));
        SNN_TRY(scr.alloc(&off2, ng + 1));
        SNN_LAUNCH(k_group_band, unsigned(cdiv(ng, 128)), 128, 0, s)(sa.tile_lo, sa.tile_hi, sa.ntiles,
                                                                     MT, lo2, hi2, items2, ng);
        SNN_LAUNCH_CHECK();
        SNN_TRY(scan_exclusive<int64_t>(items2, off2, ng, s));
        const int64_t max_items = int64_t(ng) * (cdiv(ix->n, int64_t(kBR) * kChunksPerItem) + 1);
        SNN_TRY(scr.alloc(&it2, max_items));
        SNN_LAUNCH(k_item_tiles, unsigned(cdiv(ng, 128)), 128, 0, s)(off2, ng, it2);
        SNN_LAUNCH_CHECK();
        TileSet ts2{lo2, hi2, off2, it2, ng};
        return nsplit == 2 ? launch_tc<2, 32, 128, true, 1, 16, MT>(ix, *op, sa, qp, K2, K2n, ts2, s, F)
                           : launch_tc<3, 32, 128, true, 1, 16, MT>(ix, *op, sa, qp, K2, K2n, ts2, s, 0);
    }
    // other low-d shapes: two CTAs per SM with a resident query tile, so that
    // one CTA's pipeline bubbles overlap the other's MMAs
    if (kp <= 32)
        return nsplit == 2 ? launch_tc<2, 32, 128, true, 2, 32, 1>(ix, *op, sa, qp, K2, K2n, ts1, s, F)
                           : launch_tc<3, 32, 128, true, 2, 32, 1>(ix, *op, sa, qp, K2, K2n, ts1, s, 0);
    if (kp <= 64)
        return nsplit == 2 ? launch_tc<2, 64, 128, true, 1, 64, 1>(ix, *op, sa, qp, K2, K2n, ts1, s, F)
                           : launch_tc<3, 64, 128, true, 1, 64, 1>(ix, *op, sa, qp, K2, K2n, ts1, s, 0);
    // high d: 128 x 256 accumulators (each query k-block feeds two 128-row
    // halves of the band chunk), 32-column k-blocks, four stages
    return nsplit == 2 ? launch_tc<2, 32, 256, false, 1, 32, 1>(ix, *op, sa, qp, K2, K2n, ts1, s, F)
                       : launch_tc<3, 32, 256, false, 1, 32, 1>(ix, *op, sa, qp, K2, K2n, ts1, s, 0);
}


// ------------------------------------------------ tensor-core groups of a batched query plan
// One out-of-sample query set of a group: the plan's query arrays (sorted
// order), where its rows sit in the group's arrays, and its operand constants
// (as the single-index scorer derives them from the set's index).
struct TcbSet {
    const float *qxc, *qhx, *qnrm;
    int64_t m, xoff, q0g, grp0, tile0, ntiles;
    int d, dp;
    float xscale;
    double fs1, fs2, c, Rx, e_data, abs_n, abs_q;
    DeltaInv di;
};

struct TcBatchGroup {
    int fold_col = 16, MT = 2, K2 = 32, K2n = 16, BK = 32, NW = 16;
    std::vector<int> plan_sets;
    int64_t xrows = 0, ngroups = 0, qrows = 0, max_items = 0;
    TcbSet *d_sets = nullptr;
    int32_t *d_grp_set = nullptr;
    uint16_t *x0 = nullptr, *x1 = nullptr, *q0 = nullptr, *q1 = nullptr;
    int64_t *lo2 = nullptr, *hi2 = nullptr, *items2 = nullptr, *off2 = nullptr;
    int32_t *it2 = nullptr;
    unsigned long long *begin = nullptr;
    CUtensorMap maps[8];
    std::vector<void *> blocks;
};

namespace {

// Query operand rows of a group, one thread per row: row r belongs to tile
// group r / rpg; rows past the set's queries are padding whose folded A' is
// -2^100, so their accumulators are negative and nothing survives.  Otherwise
// the two FP16 parts of the scaled centred query and the query-side folded
// columns, exactly as k_tc_query_consts and k_tc_pack compute them.  A
// scaled coordinate outside the FP16 range sets bit 1 of err.
__global__ void k_tcb_qpack(const TcbSet *__restrict__ sets, const int32_t *__restrict__ grp_set,
                            int64_t qrows, int rpg, int K2, int K2n, int fold_col, uint16_t *__restrict__ q0,
                            uint16_t *__restrict__ q1, int *__restrict__ err) {
    const int64_t r = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (r >= qrows) return;
    const int64_t g = r / rpg;
    const TcbSet &S = sets[grp_set[g]];
    const int64_t i = (g - S.grp0) * rpg + (r - g * rpg);
    uint16_t *o0 = q0 + r * K2, *o1 = q1 + r * K2n;
    for (int k = 0; k < K2; k += 4) *reinterpret_cast<uint2 *>(o0 + k) = make_uint2(0u, 0u);
    for (int k = 0; k < K2n; k += 4) *reinterpret_cast<uint2 *>(o1 + k) = make_uint2(0u, 0u);
    const uint16_t one = bf16_bits(__float2bfloat16_rn(1.0f));
    uint16_t *f = o0 + fold_col;
    uint16_t sp[3], sa[3];
    if (i >= S.m) {
        split3(-0x1p100, sa);
        for (int t = 0; t < 3; ++t) {
            f[t] = one;
            f[6 + t] = sa[t];
        }
        return;
    }
    const int d = S.d;
    const double qn = (double)S.qnrm[i], hy = (double)S.qhx[i];
    const double ei = 1.0001 * (double)kU32 * qn;
    const double rr = S.Rx + S.e_data + ei;
    const double hy_low = hy * (1.0 - 1.05 * (d + 2) * (double)kU32);
    double A = 0.5 * rr * rr - hy_low + (S.abs_n + S.abs_q * qn);
    A += 4.0 * kU64 * (fabs(A) + 0.5 * rr * rr + hy);
    A = A >= 0.0 ? __dmul_ru(A, S.di.inv_m) : __dmul_ru(A, S.di.inv_p);
    A += 0x1p-22 * fabs(A) + 0x1p-100;
    const float *x = S.qxc + i * S.dp;
    bool bad = false;
    for (int k = 0; k < d; ++k) {
        const float v = x[k] * S.xscale;
        bad |= !(fabsf(v) <= 60000.f);
        float hf = __half2float(__float2half_rn(v));
        if (fabsf(hf) < 0x1p-14f) hf = 0.f;
        float lf = __half2float(__float2half_rn(v - hf));
        if (fabsf(lf) < 0x1p-14f) lf = 0.f;
        o0[k] = half_bits(hf);
        o1[k] = half_bits(lf);
    }
    if (bad) atomicOr(err, 2);
    split3(S.c * qn * S.fs1, sp);
    split3(A * S.fs2, sa);
    for (int t = 0; t < 3; ++t) {
        f[t] = one;
        f[3 + t] = sp[t];
        f[6 + t] = sa[t];
    }
}

// Band and work items of every tile group: the union of its plan tiles'
// bands (set-local rows), moved to the group's concatenated rows.
__global__ void k_tcb_groups(const TcbSet *__restrict__ sets, const int32_t *__restrict__ grp_set,
                             int64_t ngroups, int MT, const int64_t *__restrict__ tile_lo,
                             const int64_t *__restrict__ tile_hi, int64_t *__restrict__ lo2,
                             int64_t *__restrict__ hi2, int64_t *__restrict__ items2) {
    const int64_t g = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (g >= ngroups) return;
    const TcbSet &S = sets[grp_set[g]];
    const int64_t t0 = S.tile0 + (g - S.grp0) * MT;
    const int64_t t1 = min(S.tile0 + S.ntiles, t0 + MT);
    int64_t lo = tile_lo[t0], hi = tile_hi[t0];
    for (int64_t t = t0 + 1; t < t1; ++t) {
        lo = min(lo, tile_lo[t]);
        hi = max(hi, tile_hi[t]);
    }
    hi = max(hi, lo);
    lo2[g] = lo + S.xoff;
    hi2[g] = hi + S.xoff;
    items2[g] = cdiv(cdiv(hi - lo, kBR), kChunksPerItem);
}

__global__ void k_tcb_begin(const unsigned long long *__restrict__ count, unsigned long long *__restrict__ begin) {
    *begin = *count;
}

// The group's survivors (appended after *begin) rewritten from (query operand
// row, concatenated row) to (global query number, row of the set's index).
__global__ void k_tcb_convert(uint2 *__restrict__ surv, const unsigned long long *__restrict__ count,
                              int64_t cap, const unsigned long long *__restrict__ begin,
                              const TcbSet *__restrict__ sets, const int32_t *__restrict__ grp_set, int rpg) {
    const int64_t end = min((int64_t)*count, cap);
    for (int64_t k = int64_t(*begin) + int64_t(blockIdx.x) * blockDim.x + threadIdx.x; k < end;
         k += int64_t(gridDim.x) * blockDim.x) {
        const uint2 e = surv[k];
        const int64_t g = int64_t(e.x) / rpg;
        const TcbSet &S = sets[grp_set[g]];
        const int64_t i = (g - S.grp0) * rpg + (int64_t(e.x) - g * rpg);
        surv[k] = make_uint2(unsigned(S.q0g + i), unsigned(int64_t(e.y) - S.xoff));
    }
}

template <typename T>
snn_status tcb_alloc(TcBatchGroup *g, T **p, int64_t count, cudaStream_t s) {
    void *q = nullptr;
    const size_t bytes = (std::max<size_t>(size_t(count) * sizeof(T), 16) + 255) & ~size_t(255);
    if (cudaMallocAsync(&q, bytes, s) != cudaSuccess) {
        cudaGetLastError();
        set_error("tensor-core group allocation of %zu bytes failed", bytes);
        return SNN_ENOMEM;
    }
    g->blocks.push_back(q);
    *p = static_cast<T *>(q);
    return SNN_OK;
}

}  // namespace

void tc_batch_release(TcBatchGroup *g, cudaStream_t s) {
    if (!g) return;
    for (void *b : g->blocks) cudaFreeAsync(b, s);
    delete g;
}

const int *tc_batch_sets(const TcBatchGroup *g, int *nsets) {
    *nsets = int(g->plan_sets.size());
    return g->plan_sets.data();
}

snn_status tc_batch_create(const snn_index *const *idx, const SetDesc *sd, const int *sets, int nsets,
                           int fold_col, cudaStream_t s, TcBatchGroup **out) {
    *out = nullptr;
    if (fold_col != 16 && fold_col != 32 && fold_col != 48) {
        set_error("tensor-core group: fold column %d is not 16, 32 or 48", fold_col);
        return SNN_EINVAL;
    }
    TcBatchGroup *g = new (std::nothrow) TcBatchGroup();
    if (!g) {
        set_error("host allocation failed");
        return SNN_ENOMEM;
    }
    auto fail = [&](snn_status st) {
        tc_batch_release(g, s);
        return st;
    };
    g->fold_col = fold_col;
    g->MT = fold_col == 16 ? 2 : 1;
    g->BK = fold_col == 16 ? 32 : 64;
    g->K2 = g->BK;
    g->NW = fold_col == 16 ? 16 : 64;
    g->K2n = g->NW;
    const int rpg = kTM * g->MT;
    std::vector<TcbSet> hs(nsets);
    std::vector<int32_t> grp_set;
    for (int k = 0; k < nsets; ++k) {
        const int t = sets[k];
        const snn_index *ix = idx[t];
        const SetDesc &d = sd[t];
        TcbSet &S = hs[k];
        S.qxc = d.q_xc;
        S.qhx = d.q_hx;
        S.qnrm = d.q_nrm;
        S.m = d.m;
        S.xoff = g->xrows;
        S.q0g = d.q_glob;
        S.tile0 = d.tile0;
        S.ntiles = cdiv(d.m, int64_t(kBQ));
        S.grp0 = g->ngroups;
        S.d = ix->d;
        S.dp = ix->dp;
        const double Nd = (double)ix->nrm_max;
        const int sigma = Nd > 0.0 ? std::min(120, std::max(-120, 13 - std::ilogb(Nd))) : 0;
        S.fs1 = std::ldexp(1.0, sigma);
        S.fs2 = std::ldexp(1.0, 2 * sigma);
        S.xscale = float(S.fs1);
        double u_k = 0.0;
        S.c = tc_constant(2, ix->d, &u_k, true);
        S.Rx = d.Rx;
        S.e_data = d.e_data;
        S.di = delta_inv(0x1p-23 + u_k);
        S.abs_q = 1.001 * std::sqrt(double(ix->d)) * std::ldexp(1.0, -14 - sigma);
        S.abs_n = S.abs_q * Nd + 2.0 * ix->d * std::ldexp(1.0, -28 - 2 * sigma);
        const int64_t ng = cdiv(S.ntiles, int64_t(g->MT));
        for (int64_t q = 0; q < ng; ++q) grp_set.push_back(k);
        g->ngroups += ng;
        g->xrows += ix->n;
        g->max_items += ng * (cdiv(ix->n, int64_t(kBR) * kChunksPerItem) + 1);
        g->plan_sets.push_back(t);
    }
    g->qrows = g->ngroups * rpg;
#define GTRY(expr)                           \
    do {                                     \
        snn_status _st = (expr);             \
        if (_st != SNN_OK) return fail(_st); \
    } while (0)
    GTRY(tcb_alloc(g, &g->x0, g->xrows * g->K2, s));
    GTRY(tcb_alloc(g, &g->x1, g->xrows * g->K2n, s));
    GTRY(tcb_alloc(g, &g->q0, std::max<int64_t>(g->qrows, 1) * g->K2, s));
    GTRY(tcb_alloc(g, &g->q1, std::max<int64_t>(g->qrows, 1) * g->K2n, s));
    GTRY(tcb_alloc(g, &g->d_sets, nsets, s));
    GTRY(tcb_alloc(g, &g->d_grp_set, std::max<int64_t>(g->ngroups, 1), s));
    GTRY(tcb_alloc(g, &g->lo2, std::max<int64_t>(g->ngroups, 1), s));
    GTRY(tcb_alloc(g, &g->hi2, std::max<int64_t>(g->ngroups, 1), s));
    GTRY(tcb_alloc(g, &g->items2, std::max<int64_t>(g->ngroups, 1), s));
    GTRY(tcb_alloc(g, &g->off2, g->ngroups + 1, s));
    GTRY(tcb_alloc(g, &g->it2, std::max<int64_t>(g->max_items, 1), s));
    GTRY(tcb_alloc(g, &g->begin, 1, s));
    if (cudaMemcpyAsync(g->d_sets, hs.data(), nsets * sizeof(TcbSet), cudaMemcpyHostToDevice, s) != cudaSuccess ||
        (g->ngroups > 0 && cudaMemcpyAsync(g->d_grp_set, grp_set.data(), grp_set.size() * sizeof(int32_t),
                                           cudaMemcpyHostToDevice, s) != cudaSuccess)) {
        set_error("tensor-core group setup copy failed");
        return fail(SNN_ECUDA);
    }
    // the data operands of every set, packed once into the group's rows:
    // one launch over all sets (a job per set, 32 rows per warp)
    {
        std::vector<TcPackJob> jobs(nsets);
        std::vector<int64_t> warp0(nsets + 1, 0);
        for (int k = 0; k < nsets; ++k) {
            const snn_index *ix = idx[sets[k]];
            const TcbSet &S = hs[k];
            jobs[k] = TcPackJob{ix->xc, ix->hx, ix->nrm, g->x0 + S.xoff * g->K2, g->x1 + S.xoff * g->K2n, ix->n,
                                ix->d, ix->dp, S.c, TcPackMode{1, fold_col, S.xscale, S.fs1, S.fs2}};
            warp0[k + 1] = warp0[k] + cdiv(ix->n, 32);
        }
        TcPackJob *d_jobs = nullptr;
        int64_t *d_warp0 = nullptr;
        GTRY(tcb_alloc(g, &d_jobs, nsets, s));
        GTRY(tcb_alloc(g, &d_warp0, nsets + 1, s));
        if (cudaMemcpyAsync(d_jobs, jobs.data(), nsets * sizeof(TcPackJob), cudaMemcpyHostToDevice, s) !=
                cudaSuccess ||
            cudaMemcpyAsync(d_warp0, warp0.data(), (nsets + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s) !=
                cudaSuccess) {
            set_error("tensor-core group setup copy failed");
            return fail(SNN_ECUDA);
        }
        SNN_LAUNCH(k_tc_pack_jobs, unsigned(cdiv(warp0[nsets] * 32, 256)), 256, 0, s)(d_jobs, d_warp0, nsets,
                                                                                   g->K2, g->K2n);
        if (cudaGetLastError() != cudaSuccess) {
            set_error("tensor-core group packing failed");
            return fail(SNN_ECUDA);
        }
        // (copies from pageable host memory have read their source when
        // they return, so the host arrays may go)
    }
    GTRY(make_map(&g->maps[0], g->q0, std::max<int64_t>(g->qrows, 1), g->K2, g->BK, rpg));
    GTRY(make_map(&g->maps[1], g->q1, std::max<int64_t>(g->qrows, 1), g->K2n, g->NW, rpg));
    GTRY(make_map(&g->maps[3], g->x0, g->xrows, g->K2, g->BK, 128));
    GTRY(make_map(&g->maps[4], g->x1, g->xrows, g->K2n, g->NW, 128));
    g->maps[2] = g->maps[0];
    g->maps[5] = g->maps[3];
    g->maps[6] = g->maps[0];
    g->maps[7] = g->maps[3];
#undef GTRY
    *out = g;
    return SNN_OK;
}

snn_status tc_batch_enqueue(TcBatchGroup *g, const int64_t *tile_lo, const int64_t *tile_hi, uint2 *surv,
                            int64_t cap, unsigned long long *count, int *err, cudaStream_t s) {
    if (g->ngroups == 0) return SNN_OK;
    const int rpg = kTM * g->MT;
    SNN_LAUNCH(k_tcb_qpack, unsigned(cdiv(g->qrows, 128)), 128, 0, s)(
        g->d_sets, g->d_grp_set, g->qrows, rpg, g->K2, g->K2n, g->fold_col, g->q0, g->q1, err);
    SNN_LAUNCH(k_tcb_groups, unsigned(cdiv(g->ngroups, 128)), 128, 0, s)(
        g->d_sets, g->d_grp_set, g->ngroups, g->MT, tile_lo, tile_hi, g->lo2, g->hi2, g->items2);
    SNN_LAUNCH_CHECK();
    SNN_TRY(scan_exclusive<int64_t>(g->items2, g->off2, g->ngroups, s));
    SNN_LAUNCH(k_item_tiles, unsigned(cdiv(g->ngroups, 128)), 128, 0, s)(g->off2, int(g->ngroups), g->it2);
    SNN_LAUNCH(k_tcb_begin, 1, 1, 0, s)(count, g->begin);
    SNN_LAUNCH_CHECK();
    TcArgs a;
    std::memset(&a, 0, sizeof(a));
    a.m = g->qrows;
    a.n = g->xrows;
    a.ksteps_data = g->fold_col / 16;
    a.ksteps = a.ksteps_data + 1;
    a.nkb = g->K2 / g->BK;
    a.tile_lo = g->lo2;
    a.tile_hi = g->hi2;
    a.item_off = g->off2;
    a.item_tile = g->it2;
    a.ntiles = int(g->ngroups);
    a.sym = 0;
    a.surv = surv;
    a.cap = cap;
    a.count = count;
    a.err = err;
    a.stall = 0;
    a.f16 = 1;
    ScoreArgs sa;
    snn_status st = g->fold_col == 16 ? run_tc<2, 32, 128, true, 1, 16, 2, 0>(g->maps, a, sa, s)
                                      : run_tc<2, 64, 128, true, 1, 64, 1, 0>(g->maps, a, sa, s);
    if (st != SNN_OK) return st;
    SNN_LAUNCH(k_tcb_convert, unsigned(4 * device_sm_count()), 256, 0, s)(surv, count, cap, g->begin, g->d_sets,
                                                                         g->d_grp_set, rpg);
    SNN_LAUNCH_CHECK();
    return SNN_OK;
}

}  // namespace snn
