// Allocation-free variant of the score sort (the radix sort of the scores
// in Algorithm 1) for callers that cannot allocate device memory: code running while
// a CUDA graph is being captured with allocation disallowed, processes that
// run under a fixed device-memory budget set by someone else, or real-time
// loops that must not enter the allocator.  Its scratch lives in one
// file-scope __device__ array of fixed size instead of coming from
// cudaMalloc or the stream-ordered pool.
#include <mutex>

#include "common.cuh"

namespace snn {

namespace {

constexpr int64_t kNoAllocMaxN = SNN_NOALLOC_SORT_MAX_N;
constexpr int kNaThreads = 256;
constexpr int kNaItems = 8;
constexpr int kNaTile = kNaThreads * kNaItems;        // keys per radix tile
constexpr int kNaBuckets = 256;
constexpr int64_t kNaMaxTiles = (kNoAllocMaxN + kNaTile - 1) / kNaTile;
constexpr int64_t kNaHist = kNaMaxTiles * kNaBuckets;  // histogram entries
constexpr int kNaScanTile = 4096;                     // histogram entries per scan block
constexpr int64_t kNaScanBlocks = (kNaHist + kNaScanTile - 1) / kNaScanTile;

// Scratch layout (32-bit words): keys, values, histogram, scanned histogram
// (+1), scan block sums, scanned block sums (+1), a NaN/Inf flag.
constexpr int64_t kOffKeys = 0;
constexpr int64_t kOffVals = kOffKeys + kNoAllocMaxN;
constexpr int64_t kOffHist = kOffVals + kNoAllocMaxN;
constexpr int64_t kOffScan = kOffHist + kNaHist;
constexpr int64_t kOffSums = kOffScan + kNaHist + 1;
constexpr int64_t kOffSumScan = kOffSums + kNaScanBlocks;
constexpr int64_t kOffFlag = kOffSumScan + kNaScanBlocks + 1;   // NaN/Inf flag
constexpr int64_t kScratchWords = kOffFlag + 1;

// Every GPU that loads the library holds this array (about 9 MB) until the
// process exits.
static __device__ __align__(256) uint32_t g_noalloc_scratch[kScratchWords];

__global__ void k_na_keys(const float *__restrict__ alpha, int64_t n, uint32_t *__restrict__ keys,
                          uint32_t *__restrict__ vals, int *__restrict__ bad) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float a = alpha[i];
    if (!isfinite(a)) atomicOr(bad, 1);
    keys[i] = float_to_key(a);
    vals[i] = uint32_t(i);
}

__global__ void __launch_bounds__(kNaThreads)
k_na_upsweep(const uint32_t *__restrict__ keys, int64_t n, int shift, uint32_t *__restrict__ hist) {
    __shared__ uint32_t h[kNaBuckets];
    h[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = int64_t(blockIdx.x) * kNaTile;
    for (int i = 0; i < kNaItems; ++i) {
        const int64_t idx = base + i * kNaThreads + threadIdx.x;
        if (idx < n) atomicAdd(&h[(keys[idx] >> shift) & 0xff], 1u);
    }
    __syncthreads();
    hist[int64_t(threadIdx.x) * gridDim.x + blockIdx.x] = h[threadIdx.x];   // every entry written
}

// Exclusive scan of the digit-major histogram in three steps, all in the
// static scratch: per-block totals, one-block scan of the totals, block scan.
__device__ uint32_t na_block_scan(uint32_t v, uint32_t *total) {
    __shared__ uint32_t ws[kNaThreads / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t x = v;
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) ws[w] = x;
    __syncthreads();
    if (w == 0) {
        uint32_t t = lane < kNaThreads / 32 ? ws[lane] : 0u;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        if (lane < kNaThreads / 32) ws[lane] = t;
    }
    __syncthreads();
    const uint32_t off = w ? ws[w - 1] : 0u;
    *total = ws[kNaThreads / 32 - 1];
    __syncthreads();
    return off + x - v;
}

__global__ void k_na_scan_sums(const uint32_t *__restrict__ in, int64_t n, uint32_t *__restrict__ sums) {
    constexpr int per = kNaScanTile / kNaThreads;
    const int64_t base = int64_t(blockIdx.x) * kNaScanTile + threadIdx.x * per;
    uint32_t s = 0;
    for (int i = 0; i < per; ++i)
        if (base + i < n) s += in[base + i];
    uint32_t total;
    na_block_scan(s, &total);
    if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

__global__ void k_na_scan_top(const uint32_t *__restrict__ sums, int64_t nb, uint32_t *__restrict__ out) {
    // one block; nb <= kNaScanBlocks (a few hundred)
    uint32_t carry = 0;
    for (int64_t t0 = 0; t0 < nb; t0 += kNaThreads) {
        const int64_t i = t0 + threadIdx.x;
        const uint32_t v = i < nb ? sums[i] : 0u;
        uint32_t total;
        const uint32_t ex = na_block_scan(v, &total);
        if (i < nb) out[i] = carry + ex;
        carry += total;
    }
    if (threadIdx.x == 0) out[nb] = carry;
}

__global__ void k_na_scan_down(const uint32_t *__restrict__ in, int64_t n,
                               const uint32_t *__restrict__ block_off, uint32_t *__restrict__ out) {
    constexpr int per = kNaScanTile / kNaThreads;
    const int64_t base = int64_t(blockIdx.x) * kNaScanTile + threadIdx.x * per;
    uint32_t v[per];
    uint32_t s = 0;
    for (int i = 0; i < per; ++i) {
        v[i] = base + i < n ? in[base + i] : 0u;
        s += v[i];
    }
    uint32_t total;
    uint32_t run = na_block_scan(s, &total) + block_off[blockIdx.x];
    for (int i = 0; i < per; ++i) {
        if (base + i < n) out[base + i] = run;
        run += v[i];
    }
}

// Stable scatter of one digit (same ranking as the library's radix sort).
__global__ void __launch_bounds__(kNaThreads)
k_na_downsweep(const uint32_t *__restrict__ kin, const uint32_t *__restrict__ vin,
               uint32_t *__restrict__ kout, uint32_t *__restrict__ vout, int64_t n, int shift,
               const uint32_t *__restrict__ offs) {
    constexpr int W = kNaThreads / 32;
    __shared__ uint32_t wcount[W][kNaBuckets];
    __shared__ uint32_t goff[kNaBuckets];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < W * kNaBuckets; i += kNaThreads) (&wcount[0][0])[i] = 0;
    goff[threadIdx.x] = offs[int64_t(threadIdx.x) * gridDim.x + blockIdx.x];
    __syncthreads();
    const int64_t base = int64_t(blockIdx.x) * kNaTile + int64_t(warp) * 32 * kNaItems;
    uint32_t key[kNaItems], val[kNaItems], rank[kNaItems];
    int dig[kNaItems];
    const unsigned lt = lanemask_lt();
#pragma unroll
    for (int s = 0; s < kNaItems; ++s) {
        const int64_t idx = base + s * 32 + lane;
        const bool valid = idx < n;
        key[s] = valid ? kin[idx] : 0u;
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
    {
        uint32_t run = 0;
        for (int w = 0; w < W; ++w) {
            const uint32_t c = wcount[w][threadIdx.x];
            wcount[w][threadIdx.x] = run;
            run += c;
        }
    }
    __syncthreads();
#pragma unroll
    for (int s = 0; s < kNaItems; ++s) {
        if (dig[s] >= 0) {
            const uint32_t pos = goff[dig[s]] + wcount[warp][dig[s]] + rank[s];
            kout[pos] = key[s];
            vout[pos] = val[s];
        }
    }
}

__global__ void k_na_finish(const uint32_t *__restrict__ keys, const uint32_t *__restrict__ vals,
                            int64_t n, float *__restrict__ alpha_sorted, int32_t *__restrict__ order) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n) return;
    alpha_sorted[i] = key_to_float(keys[i]);
    order[i] = int32_t(vals[i]);
}

// Device address of the static scratch, looked up once per device with that
// device current (host code only sees a stand-in symbol, not the address).
std::mutex g_na_mu;
constexpr int kNaMaxDevices = 64;
uint32_t *g_na_ptr[kNaMaxDevices] = {};

snn_status na_scratch(uint32_t **out) {
    int dev = 0;
    SNN_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kNaMaxDevices) {
        set_error("device ordinal %d out of range", dev);
        return SNN_ENOTSUP;
    }
    std::lock_guard<std::mutex> lk(g_na_mu);
    if (!g_na_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            set_error("cudaGetSymbolAddress of the sort scratch failed: %s", cudaGetErrorString(e));
            return SNN_ECUDA;
        }
        g_na_ptr[dev] = static_cast<uint32_t *>(p);
    }
    *out = g_na_ptr[dev];
    return SNN_OK;
}

}  // namespace

snn_status sort_scores_noalloc(const float *alpha, int64_t n, float *alpha_sorted, int32_t *order,
                               cudaStream_t s) {
    if (n < 0 || n > kNoAllocMaxN) {
        set_error("n = %lld is outside [0, %lld], the size of the static sort scratch",
                  (long long)n, (long long)kNoAllocMaxN);
        return SNN_EINVAL;
    }
    if (n == 0) return SNN_OK;
    if (!alpha || !alpha_sorted || !order) {
        set_error("alpha, alpha_sorted and order must be non-NULL");
        return SNN_EINVAL;
    }
    uint32_t *scr = nullptr;
    SNN_TRY(na_scratch(&scr));
    uint32_t *keys = scr + kOffKeys, *vals = scr + kOffVals;
    uint32_t *hist = scr + kOffHist, *scan = scr + kOffScan;
    uint32_t *sums = scr + kOffSums, *sumscan = scr + kOffSumScan;
    // the flag is the only scratch word read before it is written: clear it
    int *bad = reinterpret_cast<int *>(scr + kOffFlag);
    SNN_CUDA(cudaMemsetAsync(bad, 0, sizeof(int), s));
    // ping-pong between the scratch and the caller's output arrays
    uint32_t *kout = reinterpret_cast<uint32_t *>(alpha_sorted);
    uint32_t *vout = reinterpret_cast<uint32_t *>(order);
    const unsigned g = unsigned(cdiv(n, 256));
    SNN_LAUNCH(k_na_keys, g, 256, 0, s)(alpha, n, keys, vals, bad);
    SNN_LAUNCH_CHECK();
    int hbad = 0;
    SNN_CUDA(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
    SNN_CUDA(cudaStreamSynchronize(s));
    if (hbad) {
        set_error("alpha contains NaN or Inf");
        return SNN_EINVAL;
    }
    const int64_t nt = cdiv(n, kNaTile);
    const int64_t hn = nt * kNaBuckets;
    const int64_t nb = cdiv(hn, kNaScanTile);
    uint32_t *ka = keys, *va = vals, *kb = kout, *vb = vout;
    for (int shift = 0; shift < 32; shift += 8) {
        SNN_LAUNCH(k_na_upsweep, unsigned(nt), kNaThreads, 0, s)(ka, n, shift, hist);
        SNN_LAUNCH(k_na_scan_sums, unsigned(nb), kNaThreads, 0, s)(hist, hn, sums);
        SNN_LAUNCH(k_na_scan_top, 1, kNaThreads, 0, s)(sums, nb, sumscan);
        SNN_LAUNCH(k_na_scan_down, unsigned(nb), kNaThreads, 0, s)(hist, hn, sumscan, scan);
        SNN_LAUNCH(k_na_downsweep, unsigned(nt), kNaThreads, 0, s)(ka, va, kb, vb, n, shift, scan);
        SNN_LAUNCH_CHECK();
        uint32_t *t = ka; ka = kb; kb = t;
        t = va; va = vb; vb = t;
    }
    // four passes end in the scratch; convert into the caller's arrays
    SNN_LAUNCH(k_na_finish, g, 256, 0, s)(ka, va, n, alpha_sorted, order);
    SNN_LAUNCH_CHECK();
    return SNN_OK;
}

}  // namespace snn
