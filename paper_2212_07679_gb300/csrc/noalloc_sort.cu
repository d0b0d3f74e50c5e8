// Allocation-free variant of the score sort (the radix sort of the scores
// in Algorithm 1) for callers that cannot allocate device memory: processes
// that run under a device-memory budget fixed by someone else, or loops that
// must not enter the allocator.  It runs the same scan and radix kernels as
// the library's sort (radix_kernels.cuh); only its scratch differs: one
// file-scope __device__ array of fixed size instead of memory from cudaMalloc
// or the stream-ordered pool.
#include <mutex>

#include "common.cuh"
#include "radix_kernels.cuh"

namespace snn {

namespace {

using namespace radix;

constexpr int64_t kNoAllocMaxN = SNN_NOALLOC_SORT_MAX_N;
constexpr int64_t kNaMaxTiles = (kNoAllocMaxN + kRadixTile - 1) / kRadixTile;
constexpr int64_t kNaHist = kNaMaxTiles * kRadixBuckets;   // histogram entries
constexpr int64_t kNaScanBlocks = (kNaHist + kScanTile - 1) / kScanTile;

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
    const int64_t nt = cdiv(n, kRadixTile);
    const int64_t hn = nt * kRadixBuckets;
    const int64_t nb = cdiv(hn, kScanTile);
    uint32_t *ka = keys, *va = vals, *kb = kout, *vb = vout;
    for (int shift = 0; shift < 32; shift += 8) {
        // digit histogram per tile, its exclusive scan (block totals, one
        // block over the totals, block scans), stable scatter of the digit
        SNN_LAUNCH(k_radix_upsweep<uint32_t>, unsigned(nt), kRadixThreads, 0, s)(ka, n, shift, hist);
        SNN_LAUNCH(k_scan_reduce<uint32_t>, unsigned(nb), kScanThreads, 0, s)(hist, hn, sums);
        SNN_LAUNCH(k_scan_single<uint32_t>, 1, kScanThreads, 0, s)(sums, sumscan, nb);
        SNN_LAUNCH(k_scan_down<uint32_t>, unsigned(nb), kScanThreads, 0, s)(hist, scan, hn, sumscan);
        SNN_LAUNCH(k_radix_downsweep<uint32_t>, unsigned(nt), kRadixThreads, 0, s)(ka, va, kb, vb, n, shift,
                                                                                   scan);
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
