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

template <typename K>
snn_status radix_sort_pairs(K *keys, uint32_t *vals, K *keys_alt, uint32_t *vals_alt,
                            int64_t n, int end_bit, cudaStream_t s) {
    if (n <= 1) return SNN_OK;
    if (n >= (int64_t(1) << 32) - kRadixTile) {
        set_error("radix sort of %lld keys exceeds 2^32", (long long)n);
        return SNN_ENOTSUP;
    }
    const int64_t nb = cdiv(n, kRadixTile);
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
                                               int64_t, int, cudaStream_t);
template snn_status radix_sort_pairs<uint64_t>(uint64_t *, uint32_t *, uint64_t *, uint32_t *,
                                               int64_t, int, cudaStream_t);

}  // namespace snn
