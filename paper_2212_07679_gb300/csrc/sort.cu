// Device-wide exclusive scan and stable LSD radix sort of (key, value) pairs.
//
// The radix sort orders the projection scores alpha_i ascending (the sort
// of the index phase, Algorithm 1), the query scores, and long neighbour
// rows.  8-bit digits, one upsweep (per-tile digit histogram), one scan of
// the digit-major histogram, one downsweep that ranks keys stably inside
// each tile with warp match/ballot and scatters.
#include "common.cuh"
#include "radix_kernels.cuh"

namespace snn {

using namespace radix;

template <typename T>
snn_status scan_exclusive(const T *in, T *out, int64_t n, cudaStream_t s) {
    if (n <= 0) {
        SNN_CUDA(cudaMemsetAsync(out, 0, sizeof(T), s));
        return SNN_OK;
    }
    const int64_t nb = cdiv(n, kScanTile);
    if (nb <= 8) {
        SNN_LAUNCH(k_scan_single<T>, 1, kScanThreads, 0, s)(in, out, n);
        SNN_LAUNCH_CHECK();
        return SNN_OK;
    }
    Scratch scr(s);
    T *sums, *offs;
    SNN_TRY(scr.alloc(&sums, nb));
    SNN_TRY(scr.alloc(&offs, nb + 1));
    SNN_LAUNCH(k_scan_reduce<T>, (unsigned)nb, kScanThreads, 0, s)(in, n, sums);
    SNN_LAUNCH_CHECK();
    SNN_TRY(scan_exclusive<T>(sums, offs, nb, s));
    SNN_LAUNCH(k_scan_down<T>, (unsigned)nb, kScanThreads, 0, s)(in, out, n, offs);
    SNN_LAUNCH_CHECK();
    return SNN_OK;
}

template snn_status scan_exclusive<int64_t>(const int64_t *, int64_t *, int64_t, cudaStream_t);
template snn_status scan_exclusive<uint32_t>(const uint32_t *, uint32_t *, int64_t, cudaStream_t);

// ------------------------------------------------------------ radix sort

namespace {

// One read of the keys for every pass's digit histogram (hist: passes x 256,
// zeroed), then each pass's digit bases (exclusive scan of its 256 counts).
template <typename K>
__global__ void __launch_bounds__(kRadixThreads)
k_radix_hist_all(const K *__restrict__ keys, int64_t n, int passes, uint32_t *__restrict__ hist) {
    __shared__ uint32_t h[8][kRadixBuckets];
    for (int i = threadIdx.x; i < passes * kRadixBuckets; i += kRadixThreads) (&h[0][0])[i] = 0u;
    __syncthreads();
    for (int64_t i = int64_t(blockIdx.x) * kRadixThreads + threadIdx.x; i < n;
         i += int64_t(gridDim.x) * kRadixThreads) {
        const K k = keys[i];
        for (int p = 0; p < passes; ++p) atomicAdd(&h[p][(k >> (8 * p)) & 0xff], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < passes * kRadixBuckets; i += kRadixThreads)
        if ((&h[0][0])[i]) atomicAdd(&hist[i], (&h[0][0])[i]);
}

__global__ void __launch_bounds__(kRadixThreads) k_radix_bases(uint32_t *__restrict__ hist, int passes) {
    for (int p = 0; p < passes; ++p) {
        uint32_t total;
        const uint32_t v = hist[p * kRadixBuckets + threadIdx.x];
        hist[p * kRadixBuckets + threadIdx.x] = block_exclusive_scan<uint32_t>(v, &total);
    }
}

// One pass of the sort as one launch: a block takes the next tile (a ticket,
// so every earlier tile belongs to a block already running), ranks its keys
// stably as the downsweep does, publishes its per-digit counts, and sums the
// counts of the earlier tiles by walking back over their published words
// until one carries the inclusive prefix (decoupled look-back); then it
// publishes its own inclusive prefix and scatters.  A tile publishes its
// counts before it looks back, so every walk ends.  status: ntiles x 256
// words, zeroed: flag (bits 30-31: 1 counts, 2 inclusive prefix) | value.
constexpr uint32_t kLbCount = 1u << 30, kLbPrefix = 2u << 30, kLbValue = (1u << 30) - 1u;
constexpr int kLbSpinLimit = 1 << 21;

template <typename K>
__global__ void __launch_bounds__(kRadixThreads)
k_radix_onesweep(const K *__restrict__ kin, const uint32_t *__restrict__ vin, K *__restrict__ kout,
                 uint32_t *__restrict__ vout, int64_t n, int shift, const uint32_t *__restrict__ bases,
                 uint32_t *__restrict__ status, unsigned *__restrict__ ticket, int *__restrict__ err) {
    __shared__ uint32_t wcount[kRadixWarps][kRadixBuckets];
    __shared__ uint32_t goff[kRadixBuckets];
    __shared__ unsigned s_tile;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) s_tile = atomicAdd(ticket, 1u);
    for (int i = threadIdx.x; i < kRadixWarps * kRadixBuckets; i += kRadixThreads)
        (&wcount[0][0])[i] = 0;
    __syncthreads();
    const unsigned tile = s_tile;
    const int64_t base = int64_t(tile) * kRadixTile + int64_t(warp) * 32 * kRadixItems;
    K key[kRadixItems];
    uint32_t val[kRadixItems], rank[kRadixItems];
    int dig[kRadixItems];
    const unsigned lt = lanemask_lt();
#pragma unroll
    for (int s = 0; s < kRadixItems; ++s) {
        const int64_t idx = base + s * 32 + lane;
        const bool valid = idx < n;
        key[s] = valid ? kin[idx] : K(0);
        val[s] = valid ? vin[idx] : 0u;
        dig[s] = valid ? int((key[s] >> shift) & 0xff) : -1;
        const unsigned vmask = __ballot_sync(0xffffffffu, valid);
        if (valid) {
            const unsigned peers = __match_any_sync(vmask, dig[s]);
            const uint32_t before = wcount[warp][dig[s]];
            rank[s] = before + __popc(peers & lt);
            __syncwarp(vmask);
            if ((peers & lt) == 0) wcount[warp][dig[s]] = before + __popc(peers);
        }
        __syncwarp();
    }
    __syncthreads();
    uint32_t run = 0;   // this tile's count of digit threadIdx.x
#pragma unroll
    for (int w = 0; w < kRadixWarps; ++w) {
        const uint32_t c = wcount[w][threadIdx.x];
        wcount[w][threadIdx.x] = run;
        run += c;
    }
    volatile uint32_t *st = status;
    const int64_t me = int64_t(tile) * kRadixBuckets + threadIdx.x;
    uint32_t prefix = 0;
    if (tile == 0) {
        st[me] = kLbPrefix | run;
    } else {
        st[me] = kLbCount | run;
        for (int64_t t = int64_t(tile) - 1; t >= 0; --t) {
            uint32_t v = st[t * kRadixBuckets + threadIdx.x];
            int spins = 0;
            while ((v >> 30) == 0u) {
                if (++spins > kLbSpinLimit) {
                    atomicOr(err, 1);
                    break;
                }
                v = st[t * kRadixBuckets + threadIdx.x];
            }
            prefix += v & kLbValue;
            if ((v >> 30) != 1u) break;   // an inclusive prefix (or a wait that gave up)
        }
        st[me] = kLbPrefix | (prefix + run);
    }
    goff[threadIdx.x] = bases[threadIdx.x] + prefix;
    __syncthreads();
#pragma unroll
    for (int s = 0; s < kRadixItems; ++s) {
        if (dig[s] >= 0) {
            const uint32_t pos = goff[dig[s]] + wcount[warp][dig[s]] + rank[s];
            kout[pos] = key[s];
            vout[pos] = val[s];
        }
    }
}

}  // namespace


template <typename K>
snn_status radix_sort_pairs(K *keys, uint32_t *vals, K *keys_alt, uint32_t *vals_alt,
                            int64_t n, int end_bit, cudaStream_t s, int *err) {
    if (n <= 1) return SNN_OK;
    if (n >= (int64_t(1) << 32) - kRadixTile) {
        set_error("radix sort of %lld keys exceeds 2^32", (long long)n);
        return SNN_ENOTSUP;
    }
    const int64_t nb = cdiv(n, kRadixTile);
    const int npass = (end_bit + 7) / 8;
    if (err && n < int64_t(kLbValue) && npass <= 8) {
        // one histogram launch, one bases launch and one launch per pass
        Scratch scr(s);
        uint32_t *hist, *status;
        unsigned *ticket;
        SNN_TRY(scr.alloc(&hist, size_t(npass) * kRadixBuckets));
        SNN_TRY(scr.alloc(&status, size_t(npass) * nb * kRadixBuckets));
        SNN_TRY(scr.alloc(&ticket, size_t(npass)));
        SNN_CUDA(cudaMemsetAsync(hist, 0, size_t(npass) * kRadixBuckets * sizeof(uint32_t), s));
        SNN_CUDA(cudaMemsetAsync(status, 0, size_t(npass) * nb * kRadixBuckets * sizeof(uint32_t), s));
        SNN_CUDA(cudaMemsetAsync(ticket, 0, size_t(npass) * sizeof(unsigned), s));
        const unsigned hgrid = unsigned(std::min<int64_t>(cdiv(n, kRadixThreads), 4 * device_sm_count()));
        SNN_LAUNCH(k_radix_hist_all<K>, hgrid, kRadixThreads, 0, s)(keys, n, npass, hist);
        SNN_LAUNCH_CHECK();
        SNN_LAUNCH(k_radix_bases, 1, kRadixThreads, 0, s)(hist, npass);
        SNN_LAUNCH_CHECK();
        K *ka = keys, *kb = keys_alt;
        uint32_t *va = vals, *vb = vals_alt;
        for (int p = 0; p < npass; ++p) {
            SNN_LAUNCH(k_radix_onesweep<K>, (unsigned)nb, kRadixThreads, 0, s)(
                ka, va, kb, vb, n, 8 * p, hist + p * kRadixBuckets, status + int64_t(p) * nb * kRadixBuckets,
                ticket + p, err);
            SNN_LAUNCH_CHECK();
            K *tk = ka; ka = kb; kb = tk;
            uint32_t *tv = va; va = vb; vb = tv;
        }
        if (npass & 1) {
            SNN_CUDA(cudaMemcpyAsync(keys, ka, n * sizeof(K), cudaMemcpyDeviceToDevice, s));
            SNN_CUDA(cudaMemcpyAsync(vals, va, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s));
        }
        return SNN_OK;
    }
    const int64_t hn = nb * kRadixBuckets;
    Scratch scr(s);
    uint32_t *hist, *offs;
    SNN_TRY(scr.alloc(&hist, hn));
    SNN_TRY(scr.alloc(&offs, hn + 1));
    K *ka = keys, *kb = keys_alt;
    uint32_t *va = vals, *vb = vals_alt;
    int passes = 0;
    for (int shift = 0; shift < end_bit; shift += 8, ++passes) {
        SNN_LAUNCH(k_radix_upsweep<K>, (unsigned)nb, kRadixThreads, 0, s)(ka, n, shift, hist);
        SNN_LAUNCH_CHECK();
        SNN_TRY(scan_exclusive<uint32_t>(hist, offs, hn, s));
        SNN_LAUNCH(k_radix_downsweep<K>, (unsigned)nb, kRadixThreads, 0, s)(ka, va, kb, vb, n, shift, offs);
        SNN_LAUNCH_CHECK();
        K *tk = ka; ka = kb; kb = tk;
        uint32_t *tv = va; va = vb; vb = tv;
    }
    if (passes & 1) {
        SNN_CUDA(cudaMemcpyAsync(keys, ka, n * sizeof(K), cudaMemcpyDeviceToDevice, s));
        SNN_CUDA(cudaMemcpyAsync(vals, va, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s));
    }
    return SNN_OK;
}

template snn_status radix_sort_pairs<uint32_t>(uint32_t *, uint32_t *, uint32_t *, uint32_t *,
                                               int64_t, int, cudaStream_t, int *);
template snn_status radix_sort_pairs<uint64_t>(uint64_t *, uint32_t *, uint64_t *, uint32_t *,
                                               int64_t, int, cudaStream_t, int *);

}  // namespace snn
