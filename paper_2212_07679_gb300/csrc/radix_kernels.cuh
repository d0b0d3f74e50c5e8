// Kernels of the device-wide exclusive scan and of the stable LSD radix sort
// (8-bit digits: per-tile digit histogram, digit-major scan, stable
// downsweep ranking keys with warp match/ballot), shared by the library's
// pool-backed sort (sort.cu) and the allocation-free score sort
// (noalloc_sort.cu), which differ only in where their scratch lives.
#pragma once
#include "common.cuh"

namespace snn {
namespace radix {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 16;
constexpr int kScanTile = kScanThreads * kScanItems;

template <typename T>
__device__ T block_exclusive_scan(T v, T *total) {
    __shared__ T warp_sums[kScanThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    T x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[warp] = x;
    __syncthreads();
    if (warp == 0) {
        T w = lane < kScanThreads / 32 ? warp_sums[lane] : T(0);
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            T y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < kScanThreads / 32) warp_sums[lane] = w;
    }
    __syncthreads();
    T warp_off = warp ? warp_sums[warp - 1] : T(0);
    *total = warp_sums[kScanThreads / 32 - 1];
    __syncthreads();
    return warp_off + x - v;
}

template <typename T>
__global__ void k_scan_reduce(const T *__restrict__ in, int64_t n, T *__restrict__ sums) {
    const int64_t base = int64_t(blockIdx.x) * kScanTile + threadIdx.x * kScanItems;
    T s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i)
        if (base + i < n) s += in[base + i];
    T total;
    block_exclusive_scan<T>(s, &total);
    if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

template <typename T>
__global__ void k_scan_down(const T *__restrict__ in, T *__restrict__ out, int64_t n,
                            const T *__restrict__ block_off) {
    const int64_t base = int64_t(blockIdx.x) * kScanTile + threadIdx.x * kScanItems;
    T v[kScanItems];
    T s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        v[i] = (base + i < n) ? in[base + i] : T(0);
        s += v[i];
    }
    T total;
    T run = block_exclusive_scan<T>(s, &total) + block_off[blockIdx.x];
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        if (base + i < n) out[base + i] = run;
        run += v[i];
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == kScanThreads - 1) out[n] = run;
}

template <typename T>
__global__ void k_scan_single(const T *__restrict__ in, T *__restrict__ out, int64_t n) {
    // one block, sequential tiles (small n)
    T carry = 0;
    for (int64_t t0 = 0; t0 < n; t0 += kScanTile) {
        const int64_t base = t0 + threadIdx.x * kScanItems;
        T v[kScanItems];
        T s = 0;
#pragma unroll
        for (int i = 0; i < kScanItems; ++i) {
            v[i] = (base + i < n) ? in[base + i] : T(0);
            s += v[i];
        }
        T total;
        T run = block_exclusive_scan<T>(s, &total) + carry;
#pragma unroll
        for (int i = 0; i < kScanItems; ++i) {
            if (base + i < n) out[base + i] = run;
            run += v[i];
        }
        carry += total;
    }
    if (threadIdx.x == 0) out[n] = carry;
}

constexpr int kRadixThreads = 256;
constexpr int kRadixWarps = kRadixThreads / 32;
constexpr int kRadixItems = 8;
constexpr int kRadixTile = kRadixThreads * kRadixItems;  // 2048 keys per tile
constexpr int kRadixBuckets = 256;

template <typename K>
__global__ void __launch_bounds__(kRadixThreads)
k_radix_upsweep(const K *__restrict__ keys, int64_t n, int shift, uint32_t *__restrict__ hist) {
    __shared__ uint32_t h[kRadixBuckets];
    h[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = int64_t(blockIdx.x) * kRadixTile;
#pragma unroll
    for (int i = 0; i < kRadixItems; ++i) {
        int64_t idx = base + i * kRadixThreads + threadIdx.x;
        if (idx < n) atomicAdd(&h[(keys[idx] >> shift) & 0xff], 1u);
    }
    __syncthreads();
    hist[int64_t(threadIdx.x) * gridDim.x + blockIdx.x] = h[threadIdx.x];
}

template <typename K>
__global__ void __launch_bounds__(kRadixThreads)
k_radix_downsweep(const K *__restrict__ kin, const uint32_t *__restrict__ vin, K *__restrict__ kout,
                  uint32_t *__restrict__ vout, int64_t n, int shift,
                  const uint32_t *__restrict__ offs) {
    __shared__ uint32_t wcount[kRadixWarps][kRadixBuckets];
    __shared__ uint32_t goff[kRadixBuckets];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < kRadixWarps * kRadixBuckets; i += kRadixThreads)
        (&wcount[0][0])[i] = 0;
    goff[threadIdx.x] = offs[int64_t(threadIdx.x) * gridDim.x + blockIdx.x];
    __syncthreads();

    // warp w owns keys [base, base + 32*items) of the tile, visited in index
    // order (slot s, then lane), so ranks within a digit follow input order.
    const int64_t base = int64_t(blockIdx.x) * kRadixTile + int64_t(warp) * 32 * kRadixItems;
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
    {   // exclusive prefix over warps, per digit
        uint32_t run = 0;
#pragma unroll
        for (int w = 0; w < kRadixWarps; ++w) {
            uint32_t c = wcount[w][threadIdx.x];
            wcount[w][threadIdx.x] = run;
            run += c;
        }
    }
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

}  // namespace radix
}  // namespace snn
