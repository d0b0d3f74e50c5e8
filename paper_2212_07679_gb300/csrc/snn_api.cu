// C ABI of libsnn (include/snn.h): host orchestration of the index phase
// (Algorithm 1), the query phase (Algorithm 2 with Section 4's blocked
// scoring) and DBSCAN on the self-join (Section 6.4).
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <unordered_map>

#include "common.cuh"
#include "dbscan_kernels.cuh"
#include "index_kernels.cuh"
#include "query_kernels.cuh"
#include "tc_score.cuh"
#include "index_struct.cuh"
#include "update_kernels.cuh"
#include "inner_product.cuh"

namespace snn {

namespace {
thread_local char g_err[512] = "";
std::atomic<unsigned long long> g_launches{0};
std::atomic<double> g_surv_hint{0.0};   // survivors per query of the last call

std::mutex g_pool_mu;
uint64_t g_pool_done = 0;   // bit per device: release threshold raised
}  // namespace

// The default pool of the current device keeps freed memory cached (no
// release threshold), so repeated calls reuse it without new allocations.
void ensure_pool() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return;
    std::lock_guard<std::mutex> lk(g_pool_mu);
    if (g_pool_done & (uint64_t(1) << dev)) return;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        uint64_t thr = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    g_pool_done |= uint64_t(1) << dev;
}

void set_error(const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}
void clear_error() { g_err[0] = 0; }

// Output blocks shared by several library-returned pointers (the per-set
// slices of a batched query): each registered pointer holds one reference and
// the block is released when the last one is passed to snn_free.
namespace {
struct SharedBlock {
    void *base;
    int refs;
    cudaStream_t stream;   // stream of the call that allocated the block
};
std::mutex g_blocks_mu;
std::unordered_map<void *, SharedBlock *> g_blocks;
}  // namespace

// Registers library-returned pointers into one pool block allocated on
// stream s; the block is released (stream-ordered, on s) with the last of them.
snn_status register_block(void *block, void *const *ptrs, int count, cudaStream_t s) {
    std::lock_guard<std::mutex> lk(g_blocks_mu);
    SharedBlock *b = new (std::nothrow) SharedBlock{block, 0, s};
    if (!b) {
        set_error("host allocation failed");
        return SNN_ENOMEM;
    }
    for (int i = 0; i < count; ++i) {
        if (!ptrs[i]) continue;
        g_blocks[ptrs[i]] = b;
        ++b->refs;
    }
    if (b->refs == 0) {
        cudaFreeAsync(block, s);
        delete b;
    }
    return SNN_OK;
}

// Pointers the library does not know are left alone.
static void free_device_ptr(void *p) {
    SharedBlock *b = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_blocks_mu);
        auto it = g_blocks.find(p);
        if (it == g_blocks.end()) return;
        b = it->second;
        g_blocks.erase(it);
        if (--b->refs > 0) return;
    }
    cudaFreeAsync(b->base, b->stream);
    delete b;
}
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void note_launches(unsigned long long k) { g_launches.fetch_add(k, std::memory_order_relaxed); }
unsigned long long launch_count_now() { return g_launches.load(std::memory_order_relaxed); }

namespace {
std::atomic<int> g_inject{0};
}
bool take_fault(int which) {
    int expect = which;
    return which != 0 && g_inject.compare_exchange_strong(expect, 0);
}

int device_sm_count() {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 1;
}

namespace {
struct ReadList {
    const unsigned char *src[kMaxHostReads];
    int bytes[kMaxHostReads];
    int off[kMaxHostReads];
    int n;
};

__global__ void k_read_to_mailbox(ReadList L, unsigned char *mbox) {
    for (int i = 0; i < L.n; ++i)
        for (int b = threadIdx.x; b < L.bytes[i]; b += blockDim.x) mbox[L.off[i] + b] = L.src[i][b];
    __threadfence_system();
}

// Mapped pinned buffer of the calling thread (allocated once, kept).
unsigned char *host_mailbox(unsigned char **dev) {
    thread_local unsigned char *host = nullptr, *devp = nullptr;
    if (!host) {
        void *h = nullptr, *d = nullptr;
        if (cudaHostAlloc(&h, kHostReadBytes, cudaHostAllocMapped | cudaHostAllocPortable) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        if (cudaHostGetDevicePointer(&d, h, 0) != cudaSuccess) {
            cudaGetLastError();
            cudaFreeHost(h);
            return nullptr;
        }
        host = static_cast<unsigned char *>(h);
        devp = static_cast<unsigned char *>(d);
    }
    *dev = devp;
    return host;
}
}  // namespace

snn_status read_to_host(const HostRead *reads, int n, cudaStream_t s) {
    if (n < 0 || n > kMaxHostReads) {
        set_error("read_to_host: %d entries (at most %d)", n, kMaxHostReads);
        return SNN_EINVAL;
    }
    unsigned char *dev = nullptr;
    unsigned char *host = host_mailbox(&dev);
    if (!host) {
        set_error("mapped pinned host allocation failed");
        return SNN_ENOMEM;
    }
    ReadList L{};
    int off = 0;
    for (int i = 0; i < n; ++i) {
        L.src[i] = static_cast<const unsigned char *>(reads[i].src);
        L.bytes[i] = reads[i].bytes;
        L.off[i] = off;
        off += (reads[i].bytes + 7) & ~7;
        if (reads[i].bytes < 0 || off > kHostReadBytes) {
            set_error("read_to_host: more than %d bytes", kHostReadBytes);
            return SNN_EINVAL;
        }
    }
    L.n = n;
    SNN_LAUNCH(k_read_to_mailbox, 1, 128, 0, s)(L, dev);
    SNN_LAUNCH_CHECK();
    SNN_CUDA(cudaStreamSynchronize(s));
    for (int i = 0; i < n; ++i) memcpy(reads[i].dst, host + L.off[i], size_t(reads[i].bytes));
    return SNN_OK;
}

static unsigned grid_for(int64_t work, int threads) {
    return (unsigned)std::max<int64_t>(1, cdiv(work, threads));
}

// Library-owned device memory comes from the device's stream-ordered pool
// (no device-wide synchronisation on allocation or release).
template <typename T>
static snn_status dev_alloc(T **p, size_t count, cudaStream_t s) {
    void *q = nullptr;
    size_t bytes = std::max<size_t>(count * sizeof(T), 16);
    bytes = (bytes + 255) & ~size_t(255);
    if (take_fault(SNN_FAULT_DEVICE_ALLOC)) {
        set_error("device allocation of %zu bytes failed: injected test fault", bytes);
        return SNN_ENOMEM;
    }
    cudaError_t e = cudaMallocAsync(&q, bytes, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_error("device allocation of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
        return SNN_ENOMEM;
    }
    *p = static_cast<T *>(q);
    return SNN_OK;
}

// Returns an output array to the pool, or registers it so that snn_free
// releases it (stream-ordered, on the stream of the call that made it).
template <typename T>
static snn_status own_output(T *p, cudaStream_t s) {
    if (!p) return SNN_OK;
    void *ptrs[1] = {p};
    return register_block(p, ptrs, 1, s);
}

void index_release(snn_index *ix) {
    if (!ix) return;
    release_tc_operands(ix, ix->stream);
    if (ix->shared) {
        snn_shared_blocks *sb = ix->shared;
        if (sb->refs.fetch_sub(1) == 1) {
            for (int i = 0; i < sb->nblocks; ++i)
                if (sb->blocks[i]) cudaFreeAsync(sb->blocks[i], sb->stream);
            delete sb;
        }
    } else {
        void *ptrs[] = {ix->mu64, ix->mu32, ix->v64, ix->v32, ix->alpha, ix->order,
                        ix->praw, ix->xc,   ix->hx,  ix->nrm, ix->dconst};
        for (void *p : ptrs)
            if (p) cudaFreeAsync(p, ix->stream);
    }
    delete ix;
}

// ------------------------------------------------- index save / load
// Serialised index: a fixed header, then the arrays of the index record in
// this order, each starting on a 16-byte boundary: mu64[d], mu32[d], v64[d],
// v32[d], dconst[4], alpha[n], order[n], hx[n], nrm[n], praw[n*dp], xc[n*dp].
// Derived operands (the BF16 / e4m3 splits) are not stored: they are rebuilt
// on first use.  Little-endian, as on both host architectures this targets.
namespace {
struct SavedHeader {
    char magic[8];          // "SNNIDX\0\1"
    int32_t version, d;
    int64_t n;
    int32_t dp, reserved;
    float alpha_err, nrm_max;
};
constexpr char kSaveMagic[8] = {'S', 'N', 'N', 'I', 'D', 'X', 0, 1};
constexpr int32_t kSaveVersion = 1;

struct SavedArray {
    size_t off, bytes;
};

// Byte offsets of the arrays after the header (16-byte aligned) and the total.
int64_t saved_layout(int64_t n, int d, int dp, SavedArray (&a)[11]) {
    const size_t sz[11] = {sizeof(double) * d, sizeof(float) * d, sizeof(double) * d, sizeof(float) * d,
                           sizeof(float) * 4,  sizeof(float) * n, sizeof(int32_t) * n, sizeof(float) * n,
                           sizeof(float) * n,  sizeof(float) * n * dp, sizeof(float) * n * dp};
    size_t off = (sizeof(SavedHeader) + 15) & ~size_t(15);
    for (int i = 0; i < 11; ++i) {
        a[i] = {off, sz[i]};
        off = (off + sz[i] + 15) & ~size_t(15);
    }
    return int64_t(off);
}

void *saved_ptr(const snn_index *ix, int i) {
    void *p[11] = {ix->mu64, ix->mu32, ix->v64, ix->v32, ix->dconst, ix->alpha,
                   ix->order, ix->hx, ix->nrm, ix->praw, ix->xc};
    return p[i];
}
}  // namespace

static snn_status index_save(const snn_index *ix, void *buf, int64_t bytes, cudaStream_t s) {
    NvtxPhase nvtx_("snn index save");
    SavedArray a[11];
    const int64_t need = saved_layout(ix->n, ix->d, ix->dp, a);
    if (bytes < need) {
        set_error("the buffer holds %lld bytes, the index needs %lld", (long long)bytes, (long long)need);
        return SNN_EINVAL;
    }
    unsigned char *b = static_cast<unsigned char *>(buf);
    std::memset(b, 0, size_t(need));
    SavedHeader h{};
    std::memcpy(h.magic, kSaveMagic, 8);
    h.version = kSaveVersion;
    h.d = ix->d;
    h.n = ix->n;
    h.dp = ix->dp;
    h.alpha_err = ix->alpha_err;
    h.nrm_max = ix->nrm_max;
    std::memcpy(b, &h, sizeof(h));
    for (int i = 0; i < 11; ++i)
        SNN_CUDA(cudaMemcpyAsync(b + a[i].off, saved_ptr(ix, i), a[i].bytes, cudaMemcpyDeviceToHost, s));
    SNN_CUDA(cudaStreamSynchronize(s));
    return SNN_OK;
}

static snn_status index_load(const void *buf, int64_t bytes, cudaStream_t s, snn_index **out) {
    NvtxPhase nvtx_("snn index load");
    SavedHeader h{};
    if (bytes < int64_t(sizeof(h))) {
        set_error("the buffer is shorter than an index header");
        return SNN_EINVAL;
    }
    std::memcpy(&h, buf, sizeof(h));
    if (std::memcmp(h.magic, kSaveMagic, 8) != 0 || h.version != kSaveVersion) {
        set_error("not a saved index of this format (magic or version differs)");
        return SNN_EINVAL;
    }
    if (h.d < 1 || h.d > 4096 || h.dp != ((h.d + 3) & ~3) || h.n < 1 || h.n >= (int64_t(1) << 31) ||
        !(h.alpha_err >= 0.f) || !(h.nrm_max >= 0.f) || !(double(h.nrm_max) <= kMaxCentredNorm)) {
        set_error("corrupt index header (n %lld, d %d, dp %d)", (long long)h.n, h.d, h.dp);
        return SNN_EINVAL;
    }
    SavedArray a[11];
    const int64_t need = saved_layout(h.n, h.d, h.dp, a);
    if (bytes < need) {
        set_error("the buffer holds %lld bytes, a saved index of n %lld, d %d needs %lld",
                  (long long)bytes, (long long)h.n, h.d, (long long)need);
        return SNN_EINVAL;
    }
    ensure_pool();
    snn_index *ix = new (std::nothrow) snn_index();
    if (!ix) {
        set_error("host allocation failed");
        return SNN_ENOMEM;
    }
    ix->n = h.n;
    ix->d = h.d;
    ix->dp = h.dp;
    ix->stream = s;
    ix->alpha_err = h.alpha_err;
    ix->nrm_max = h.nrm_max;
    cudaGetDevice(&ix->device);
    snn_status st = SNN_OK;
    const int64_t n = h.n, nd = h.n * h.dp;
    const int d = h.d;
    if (st == SNN_OK) st = dev_alloc(&ix->mu64, d, s);
    if (st == SNN_OK) st = dev_alloc(&ix->mu32, d, s);
    if (st == SNN_OK) st = dev_alloc(&ix->v64, d, s);
    if (st == SNN_OK) st = dev_alloc(&ix->v32, d, s);
    if (st == SNN_OK) st = dev_alloc(&ix->dconst, 4, s);
    if (st == SNN_OK) st = dev_alloc(&ix->alpha, n, s);
    if (st == SNN_OK) st = dev_alloc(&ix->order, n, s);
    if (st == SNN_OK) st = dev_alloc(&ix->hx, n, s);
    if (st == SNN_OK) st = dev_alloc(&ix->nrm, n, s);
    if (st == SNN_OK) st = dev_alloc(&ix->praw, nd, s);
    if (st == SNN_OK) st = dev_alloc(&ix->xc, nd, s);
    const unsigned char *b = static_cast<const unsigned char *>(buf);
    for (int i = 0; i < 11 && st == SNN_OK; ++i)
        if (cudaMemcpyAsync(saved_ptr(ix, i), b + a[i].off, a[i].bytes, cudaMemcpyHostToDevice, s) !=
            cudaSuccess) {
            set_error("index load copy failed: %s", cudaGetErrorString(cudaGetLastError()));
            st = SNN_ECUDA;
        }
    if (st == SNN_OK && cudaStreamSynchronize(s) != cudaSuccess) {
        set_error("index load failed: %s", cudaGetErrorString(cudaGetLastError()));
        st = SNN_ECUDA;
    }
    if (st != SNN_OK) {
        cudaStreamSynchronize(s);
        index_release(ix);
        return st;
    }
    *out = ix;
    return SNN_OK;
}

// ---------------------------------------------------------- index build
static snn_status project_sort_gather(const float *X, int64_t n, int d, int64_t ld, int dp,
                                      const float *cvec, const float *v32, cudaStream_t s,
                                      Scratch &scr, float *eps_out, int *bad, int *sort_err, float *alpha,
                                      int32_t *order, float *praw, float *xc, float *hx,
                                      float *nrm) {
    uint32_t *keys, *vals, *ka, *va;
    SNN_TRY(scr.alloc(&keys, n));
    SNN_TRY(scr.alloc(&vals, n));
    SNN_TRY(scr.alloc(&ka, n));
    SNN_TRY(scr.alloc(&va, n));
    const int64_t pthreads = d > 32 ? n * 32 : n;
    // float4 rows when every row starts on a 16-byte boundary and d = 4k
    const int vec = (d % 4 == 0 && ld % 4 == 0 && reinterpret_cast<uintptr_t>(X) % 16 == 0) ? 1 : 0;
    SNN_LAUNCH(k_project, grid_for(pthreads, 256), 256, 0, s)(X, n, d, ld, cvec, v32, keys, vals,
                                                      eps_out, bad, vec);
    SNN_LAUNCH_CHECK();
    SNN_TRY(radix_sort_pairs<uint32_t>(keys, vals, ka, va, n, 32, s, sort_err));
    SNN_LAUNCH(k_gather, grid_for(pthreads, 256), 256, 0, s)(keys, vals, X, n, d, ld, dp, cvec, alpha,
                                                     order, praw, xc, hx, nrm, vec);
    SNN_LAUNCH_CHECK();
    return SNN_OK;
}

__global__ void k_max_nonneg(const float *__restrict__ x, int64_t n, float *__restrict__ out) {
    float m = 0.f;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += int64_t(gridDim.x) * blockDim.x)
        m = fmaxf(m, x[i]);
    for (int o = 16; o; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomic_max_nonneg(out, m);
}

static snn_status first_direction(const double *C, const double *diagC, int d, double *v64,
                                  float *v32, int *err, cudaStream_t s, Scratch &scr) {
    if (d <= kPcSmallMaxD) {
        const size_t smem = (d + 32) * sizeof(double) + (32 + 2 * d) * sizeof(float) +
                            2 * size_t(d) * d * sizeof(float);
        SNN_LAUNCH(k_pc_small, 1, 1024, smem, s)(C, d, v64, v32);
        SNN_LAUNCH_CHECK();
        return SNN_OK;
    }
    return first_direction_tc(C, diagC, d, v64, v32, err, s, scr);
}

static snn_status index_build(const float *X, int64_t n, int d, int64_t ld, cudaStream_t s,
                              snn_index **out) {
    NvtxPhase nvtx_("snn index build");
    ensure_pool();
    snn_index *ix = new (std::nothrow) snn_index();
    if (!ix) {
        set_error("host allocation failed");
        return SNN_ENOMEM;
    }
    ix->n = n;
    ix->d = d;
    ix->dp = (d + 3) & ~3;
    ix->stream = s;
    cudaGetDevice(&ix->device);
    const int dp = ix->dp;
    snn_status st = SNN_OK;
#define TRY_IX(expr)                       \
    do {                                   \
        st = (expr);                       \
        if (st != SNN_OK) {                \
            cudaStreamSynchronize(s);      \
            index_release(ix);             \
            return st;                     \
        }                                  \
    } while (0)
    TRY_IX(dev_alloc(&ix->mu64, d, s));
    TRY_IX(dev_alloc(&ix->mu32, d, s));
    TRY_IX(dev_alloc(&ix->v64, d, s));
    TRY_IX(dev_alloc(&ix->v32, d, s));
    TRY_IX(dev_alloc(&ix->alpha, n, s));
    TRY_IX(dev_alloc(&ix->order, n, s));
    TRY_IX(dev_alloc(&ix->praw, size_t(n) * dp, s));
    TRY_IX(dev_alloc(&ix->xc, size_t(n) * dp, s));
    TRY_IX(dev_alloc(&ix->hx, n, s));
    TRY_IX(dev_alloc(&ix->nrm, n, s));
    TRY_IX(dev_alloc(&ix->dconst, 4, s));
    {
        Scratch scr(s);
        int *bad;   // [0] NaN/Inf seen, [1] a bounded wait expired (tensor-core Gram or score sort)
        TRY_IX(scr.alloc(&bad, 2));
        if (cudaMemsetAsync(bad, 0, 2 * sizeof(int), s) != cudaSuccess ||
            cudaMemsetAsync(ix->dconst, 0, 4 * sizeof(float), s) != cudaSuccess) {
            set_error("cudaMemsetAsync failed");
            TRY_IX(SNN_ECUDA);
        }
        // K1: column means (2-D grid: column chunks x row ranges, about four
        // blocks per SM)
        const int TX = d < 32 ? d : 32, TY = 256 / TX;
        const int64_t ncb = cdiv(d, TX);
        const int64_t nb = std::max<int64_t>(
            1, std::min<int64_t>(cdiv(4 * device_sm_count(), ncb), cdiv(n, 64)));
        const int64_t rows = cdiv(n, nb);
        double *part;
        TRY_IX(scr.alloc(&part, size_t(nb) * d));
        SNN_LAUNCH(k_colsum_partial, dim3(unsigned(nb), unsigned(ncb)), TX * TY,
                   TX * TY * sizeof(double), s)(X, n, d, ld, rows, part, bad);
        if (cudaGetLastError() != cudaSuccess) { set_error("colsum launch"); TRY_IX(SNN_ECUDA); }
        SNN_LAUNCH(k_mean_final, grid_for(int64_t(d) * 32, 128), 128, 0, s)(part, (int)nb, d, n,
                                                                           ix->mu64, ix->mu32);
        // K2: centred Gram matrix
        double *C, *diagC;
        TRY_IX(scr.alloc(&C, size_t(d) * d));
        TRY_IX(scr.alloc(&diagC, d));
        if (d <= kPcSmallMaxD) {
            const int64_t gnb = std::max<int64_t>(
                1, std::min<int64_t>(4 * device_sm_count(), cdiv(n, 256)));
            const int64_t grows = cdiv(n, gnb);
            float *gpart;
            TRY_IX(scr.alloc(&gpart, size_t(gnb) * d * d));
            auto gk = d <= 16 ? k_gram_small16 : (d <= 32 ? k_gram_small32 : k_gram_small64);
            SNN_LAUNCH(gk, unsigned(gnb), 256, 0, s)(X, n, d, ld, ix->mu32, grows, gpart);
            SNN_LAUNCH(k_gram_reduce, grid_for(int64_t(d) * d * 32, 256), 256, 0, s)(gpart, (int)gnb,
                                                                                     d, C);
            if (cudaGetLastError() != cudaSuccess) { set_error("gram launch"); TRY_IX(SNN_ECUDA); }
        } else {
            TRY_IX(gram_tc(X, n, d, ld, ix->mu32, C, diagC, bad + 1, s, scr));
        }
        // K3: first principal direction
        TRY_IX(first_direction(C, diagC, d, ix->v64, ix->v32, bad + 1, s, scr));
        // K4-K6: scores, sort, gather
        TRY_IX(project_sort_gather(X, n, d, ld, dp, ix->mu32, ix->v32, s, scr, ix->dconst + 0, bad, bad + 1,
                                   ix->alpha, ix->order, ix->praw, ix->xc, ix->hx, ix->nrm));
        SNN_LAUNCH(k_max_nonneg, std::min<unsigned>(grid_for(n, 256), 1024), 256, 0, s)(ix->nrm, n,
                                                                                ix->dconst + 1);
        if (cudaGetLastError() != cudaSuccess) { set_error("max launch"); TRY_IX(SNN_ECUDA); }
        float hc[2];
        int hbad[2] = {0, 0};
        {
            const HostRead rd[] = {{ix->dconst, hc, int(sizeof(hc))}, {bad, hbad, int(sizeof(hbad))}};
            TRY_IX(read_to_host(rd, 2, s));
        }
        if (hbad[0]) {
            set_error("X contains NaN or Inf");
            TRY_IX(SNN_EINVAL);
        }
        if (hbad[1]) {
            set_error("index build: a bounded wait expired (tensor-core Gram or score sort)");
            TRY_IX(SNN_ETIMEOUT);
        }
        ix->alpha_err = hc[0];
        ix->nrm_max = hc[1];
        if (!(hc[1] <= kMaxCentredNorm)) {
            set_error("a centred point norm of %g exceeds %g: the FP32 and BF16 scores would "
                      "overflow", (double)hc[1], kMaxCentredNorm);
            TRY_IX(SNN_ENOTSUP);
        }
    }
#undef TRY_IX
    *out = ix;
    return SNN_OK;
}

// ------------------------------------------------------ streaming updates
// Per-position arrays of an index: scores, ids, raw and centred rows, halved
// norms, norm bounds.
struct PosArrays {
    float *alpha = nullptr, *praw = nullptr, *xc = nullptr, *hx = nullptr, *nrm = nullptr;
    int32_t *order = nullptr;
    snn_status alloc(int64_t n, int dp, cudaStream_t s) {
        SNN_TRY(dev_alloc(&alpha, n, s));
        SNN_TRY(dev_alloc(&order, n, s));
        SNN_TRY(dev_alloc(&praw, size_t(n) * dp, s));
        SNN_TRY(dev_alloc(&xc, size_t(n) * dp, s));
        SNN_TRY(dev_alloc(&hx, n, s));
        SNN_TRY(dev_alloc(&nrm, n, s));
        return SNN_OK;
    }
    void release(cudaStream_t s) {
        void *ptrs[] = {alpha, order, praw, xc, hx, nrm};
        for (void *p : ptrs)
            if (p) cudaFreeAsync(p, s);
        *this = PosArrays();
    }
};

// Gives an index of a batched build its own centre, direction and constants
// and drops its reference to the shared blocks (freed in order on s with the
// last reference, after the copies and any kernel already queued on s).
// Returns whether the index was sharing.
static snn_status detach_shared(snn_index *ix, cudaStream_t s, bool *was_shared) {
    *was_shared = ix->shared != nullptr;
    if (!ix->shared) return SNN_OK;
    double *mu64 = nullptr, *v64 = nullptr;
    float *mu32 = nullptr, *v32 = nullptr, *dconst = nullptr;
    snn_status st = SNN_OK;
    if ((st = dev_alloc(&mu64, ix->d, s)) != SNN_OK || (st = dev_alloc(&v64, ix->d, s)) != SNN_OK ||
        (st = dev_alloc(&mu32, ix->d, s)) != SNN_OK || (st = dev_alloc(&v32, ix->d, s)) != SNN_OK ||
        (st = dev_alloc(&dconst, 4, s)) != SNN_OK) {
        void *ptrs[] = {mu64, v64, mu32, v32, dconst};
        for (void *p : ptrs)
            if (p) cudaFreeAsync(p, s);
        return st;
    }
    cudaMemcpyAsync(mu64, ix->mu64, ix->d * sizeof(double), cudaMemcpyDeviceToDevice, s);
    cudaMemcpyAsync(v64, ix->v64, ix->d * sizeof(double), cudaMemcpyDeviceToDevice, s);
    cudaMemcpyAsync(mu32, ix->mu32, ix->d * sizeof(float), cudaMemcpyDeviceToDevice, s);
    cudaMemcpyAsync(v32, ix->v32, ix->d * sizeof(float), cudaMemcpyDeviceToDevice, s);
    cudaMemcpyAsync(dconst, ix->dconst, 4 * sizeof(float), cudaMemcpyDeviceToDevice, s);
    snn_shared_blocks *sb = ix->shared;
    if (sb->refs.fetch_sub(1) == 1) {
        for (int i = 0; i < sb->nblocks; ++i)
            if (sb->blocks[i]) cudaFreeAsync(sb->blocks[i], s);
        delete sb;
    }
    ix->shared = nullptr;
    ix->mu64 = mu64;
    ix->v64 = v64;
    ix->mu32 = mu32;
    ix->v32 = v32;
    ix->dconst = dconst;
    ix->alpha = nullptr;   // slices of the released blocks
    ix->order = nullptr;
    ix->praw = nullptr;
    ix->xc = nullptr;
    ix->hx = nullptr;
    ix->nrm = nullptr;
    return SNN_OK;
}

// Replaces the per-position arrays (the old ones, when the index owns them,
// are freed in order on s) and drops the cached tensor-core operands.
static void install(snn_index *ix, PosArrays &a, int64_t n, cudaStream_t s) {
    std::lock_guard<std::mutex> lk(ix->mu);
    void *old[] = {ix->alpha, ix->order, ix->praw, ix->xc, ix->hx, ix->nrm};
    for (void *p : old)
        if (p) cudaFreeAsync(p, s);
    release_tc_operands(ix, s);
    ix->alpha = a.alpha;
    ix->order = a.order;
    ix->praw = a.praw;
    ix->xc = a.xc;
    ix->hx = a.hx;
    ix->nrm = a.nrm;
    a = PosArrays();
    ix->n = n;
    ix->stream = s;
}

// New points take ids n, n+1, ...: scored with the index's centre and
// direction, sorted, and merged into the sorted order.
static snn_status index_insert(snn_index *ix, const float *X, int64_t k, int64_t ld, cudaStream_t s) {
    NvtxPhase nvtx_("snn index insert");
    ensure_pool();
    const int d = ix->d, dp = ix->dp;
    const int64_t n = ix->n;
    Scratch scr(s);
    PosArrays nw, out;
    int *bad;     // [0] NaN/Inf seen, [1] a bounded wait of the score sort expired
    float *add;   // [0] score error bound of the new points, [1] their largest norm bound
    SNN_TRY(scr.alloc(&bad, 2));
    SNN_TRY(scr.alloc(&add, 2));
    SNN_CUDA(cudaMemsetAsync(bad, 0, 2 * sizeof(int), s));
    SNN_CUDA(cudaMemsetAsync(add, 0, 2 * sizeof(float), s));
    SNN_TRY(scr.alloc(&nw.alpha, k));
    SNN_TRY(scr.alloc(&nw.order, k));
    SNN_TRY(scr.alloc(&nw.praw, size_t(k) * dp));
    SNN_TRY(scr.alloc(&nw.xc, size_t(k) * dp));
    SNN_TRY(scr.alloc(&nw.hx, k));
    SNN_TRY(scr.alloc(&nw.nrm, k));
    SNN_TRY(project_sort_gather(X, k, d, ld, dp, ix->mu32, ix->v32, s, scr, add, bad, bad + 1, nw.alpha,
                                nw.order, nw.praw, nw.xc, nw.hx, nw.nrm));
    SNN_LAUNCH(k_max_nonneg, std::min<unsigned>(grid_for(k, 256), 1024), 256, 0, s)(nw.nrm, k, add + 1);
    SNN_LAUNCH_CHECK();
    int64_t *pos_old, *pos_new;
    SNN_TRY(scr.alloc(&pos_old, n));
    SNN_TRY(scr.alloc(&pos_new, k));
    snn_status st = out.alloc(n + k, dp, s);
    if (st != SNN_OK) {
        out.release(s);
        return st;
    }
    SNN_LAUNCH(k_merge_ranks, grid_for(n + k, 256), 256, 0, s)(ix->alpha, n, nw.alpha, k, pos_old, pos_new);
    SNN_LAUNCH(k_place, grid_for(n * (dp / 4), 256), 256, 0, s)(
        ix->alpha, ix->order, 0, ix->hx, ix->nrm, ix->praw, ix->xc, n, dp, pos_old, out.alpha, out.order,
        out.hx, out.nrm, out.praw, out.xc);
    SNN_LAUNCH(k_place, grid_for(k * (dp / 4), 256), 256, 0, s)(
        nw.alpha, nw.order, int32_t(n), nw.hx, nw.nrm, nw.praw, nw.xc, k, dp, pos_new, out.alpha,
        out.order, out.hx, out.nrm, out.praw, out.xc);
    if (cudaGetLastError() != cudaSuccess) {
        set_error("insert launch failed");
        out.release(s);
        return SNN_ECUDA;
    }
    float hadd[2];
    int hbad[2] = {0, 0};
    {
        const HostRead rd[] = {{add, hadd, int(sizeof(hadd))}, {bad, hbad, int(sizeof(hbad))}};
        const snn_status st = read_to_host(rd, 2, s);
        if (st != SNN_OK) {
            out.release(s);
            return st;
        }
    }
    if (hbad[0]) {
        set_error("X contains NaN or Inf");
        out.release(s);
        return SNN_EINVAL;
    }
    if (hbad[1]) {
        set_error("insert: a bounded wait of the score sort expired");
        out.release(s);
        return SNN_ETIMEOUT;
    }
    if (!(hadd[1] <= kMaxCentredNorm)) {
        set_error("a centred point norm of %g exceeds %g", (double)hadd[1], kMaxCentredNorm);
        out.release(s);
        return SNN_ENOTSUP;
    }
    bool shared = false;
    if ((st = detach_shared(ix, s, &shared)) != SNN_OK) {
        out.release(s);
        return st;
    }
    SNN_LAUNCH(k_update_consts, 1, 32, 0, s)(ix->dconst, add);
    SNN_LAUNCH_CHECK();
    ix->alpha_err = std::max(ix->alpha_err, hadd[0]);
    ix->nrm_max = std::max(ix->nrm_max, hadd[1]);
    install(ix, out, n + k, s);
    return SNN_OK;
}

// Removes the listed ids; the kept points are renumbered 0, 1, ... in their
// previous id order (as if their rows were erased from X).
static snn_status index_delete(snn_index *ix, const int32_t *ids, int64_t cnt, cudaStream_t s) {
    NvtxPhase nvtx_("snn index delete");
    ensure_pool();
    const int dp = ix->dp;
    const int64_t n = ix->n;
    Scratch scr(s);
    uint8_t *del;
    int *bad;
    int64_t *keep_id, *keep_pos, *newid, *newpos;
    SNN_TRY(scr.alloc(&del, n));
    SNN_TRY(scr.alloc(&bad, 1));
    SNN_TRY(scr.alloc(&keep_id, n));
    SNN_TRY(scr.alloc(&keep_pos, n));
    SNN_TRY(scr.alloc(&newid, n + 1));    // exclusive scans: n + 1 entries
    SNN_TRY(scr.alloc(&newpos, n + 1));
    SNN_CUDA(cudaMemsetAsync(del, 0, n, s));
    SNN_CUDA(cudaMemsetAsync(bad, 0, sizeof(int), s));
    SNN_LAUNCH(k_mark_deleted, grid_for(cnt, 256), 256, 0, s)(ids, cnt, n, del, bad);
    SNN_LAUNCH(k_keep_flags, grid_for(n, 256), 256, 0, s)(del, ix->order, n, keep_id, keep_pos);
    SNN_LAUNCH_CHECK();
    SNN_TRY(scan_exclusive<int64_t>(keep_id, newid, n, s));
    SNN_TRY(scan_exclusive<int64_t>(keep_pos, newpos, n, s));
    int64_t kept = 0;
    int hbad = 0;
    {
        const HostRead rd[] = {{newpos + n, &kept, int(sizeof(kept))}, {bad, &hbad, int(sizeof(int))}};
        SNN_TRY(read_to_host(rd, 2, s));
    }
    if (hbad) {
        set_error("an id to delete is outside [0, n)");
        return SNN_EINVAL;
    }
    if (kept < 1) {
        set_error("deleting every point would leave an empty index");
        return SNN_EINVAL;
    }
    if (kept == n) return SNN_OK;
    PosArrays out;
    snn_status st = out.alloc(kept, dp, s);
    if (st != SNN_OK) {
        out.release(s);
        return st;
    }
    SNN_LAUNCH(k_compact, grid_for(n * (dp / 4), 256), 256, 0, s)(
        del, ix->alpha, ix->order, ix->hx, ix->nrm, ix->praw, ix->xc, n, dp, newpos, newid, out.alpha,
        out.order, out.hx, out.nrm, out.praw, out.xc);
    if (cudaGetLastError() != cudaSuccess) {
        set_error("delete launch failed");
        out.release(s);
        return SNN_ECUDA;
    }
    bool shared = false;
    if ((st = detach_shared(ix, s, &shared)) != SNN_OK) {
        out.release(s);
        return st;
    }
    install(ix, out, kept, s);
    return SNN_OK;
}

// ---------------------------------------------------------------- query
// Everything the host needs after the scoring and decision, gathered on the
// device and read back at once (read_to_host).
struct Readback {
    unsigned long long ctr[4];   // survivors, work, band pairs, candidates
    int bad, err;                // NaN/Inf in the queries, expired wait
    int64_t nnz;
    unsigned cls[kSegClasses];   // rows per length class
    int64_t big_total;           // entries in rows longer than 4096
};

__global__ void k_readback(const unsigned long long *__restrict__ ctr, const int *__restrict__ bad,
                           const int *__restrict__ err, const int64_t *__restrict__ nnz,
                           const unsigned *__restrict__ cls, const int64_t *__restrict__ big_total,
                           Readback *__restrict__ rb) {
    const int t = threadIdx.x;
    if (t < 4) rb->ctr[t] = ctr[t];
    if (t < kSegClasses) rb->cls[t] = cls[t];
    if (t == 0) {
        rb->bad = *bad;
        rb->err = *err;
        rb->nnz = *nnz;
        rb->big_total = *big_total;
    }
}


struct QueryScratch {
    float *alpha = nullptr, *raw = nullptr, *xc = nullptr, *hy = nullptr, *nrm = nullptr;
    int32_t *order = nullptr;
    float *eps = nullptr;
    int *bad = nullptr;
};

// Largest true distance the FP64 test S <= fl64(R*R) can still accept:
// S >= D^2 (1 - gamma_{d+2}) and fl64(R*R) <= R^2 (1 + u).
// R: the radius, or with per-query radii Rdev (device, m, query order; out-of-
// sample queries only) the smallest of them, Rmax the largest (host choices:
// the BF16 split, the FP8 availability).  pos_rows: the rows stay in sorted
// positions (row p = the query in sorted position p; columns point ids, rows
// unsorted, no dist2): the internal neighbourhoods of DBSCAN, a self-join
// (Q null).
static snn_status query_impl(const snn_index *ix, const float *Q, int64_t m, int64_t ldq,
                             double R, snn_precision prec, cudaStream_t s, snn_csr *out,
                             snn_query_stats *stats, const double *Rdev = nullptr, double Rmax = 0.0,
                             bool pos_rows = false) {
    NvtxPhase nvtx_("snn query: prepare");
    const bool self = (Q == nullptr);
    if (pos_rows && !self) {
        set_error("internal: position rows need a self-join");
        return SNN_EINVAL;
    }
    double q_nrm_max = self ? (double)ix->nrm_max : 0.0;   // largest centred query norm bound
    if (self) m = ix->n;
    const int d = ix->d, dp = ix->dp;
    out->m = m;
    out->nnz = 0;
    out->offsets = nullptr;
    out->indices = nullptr;
    out->dist2 = nullptr;
    ensure_pool();
    SNN_TRY(dev_alloc(&out->offsets, m + 1, s));
    uint2 *surv = nullptr;
    float *rec_d2 = nullptr;
    int32_t *rec_pos = nullptr;
    auto fail = [&](snn_status st) {
        void *tmp[] = {surv, rec_d2, rec_pos, out->offsets, out->indices, out->dist2};
        for (void *p : tmp)
            if (p) cudaFreeAsync(p, s);
        surv = nullptr;
        rec_d2 = nullptr;
        rec_pos = nullptr;
        out->offsets = nullptr;
        out->indices = nullptr;
        out->dist2 = nullptr;
        out->nnz = 0;
        return st;
    };
#define TRY_Q(expr)                          \
    do {                                     \
        snn_status _st = (expr);             \
        if (_st != SNN_OK) return fail(_st); \
    } while (0)
#define CUDA_Q(call)                                                              \
    do {                                                                          \
        cudaError_t _e = (call);                                                  \
        if (_e != cudaSuccess) {                                                  \
            set_error("%s: %s", #call, cudaGetErrorString(_e));                   \
            return fail(_e == cudaErrorMemoryAllocation ? SNN_ENOMEM : SNN_ECUDA); \
        }                                                                         \
    } while (0)

    if (m == 0) {
        CUDA_Q(cudaMemsetAsync(out->offsets, 0, sizeof(int64_t), s));
        if (stats) std::memset(stats, 0, sizeof(*stats));
        TRY_Q(own_output(out->offsets, s));
        return SNN_OK;
    }
    cudaEvent_t ev[7] = {};
    if (stats) {
        for (auto &e : ev) cudaEventCreate(&e);
        cudaEventRecord(ev[0], s);
    }
    Scratch scr(s);
    QuerySet qs;
    qs.m = m;
    float *eps_q = ix->dconst;   // self-join: the data's own bound
    int *bad = nullptr;   // [0] NaN/Inf in Q, [1] a bounded wait of the query sort expired
    TRY_Q(scr.alloc(&bad, 2));
    CUDA_Q(cudaMemsetAsync(bad, 0, 2 * sizeof(int), s));
    if (self) {
        qs.alpha = ix->alpha;
        qs.order = ix->order;
        qs.raw = ix->praw;
        qs.xc = ix->xc;
        qs.hx = ix->hx;
        qs.nrm = ix->nrm;
    } else {
        float *qa, *qraw, *qxc, *qhy, *qnrm;
        int32_t *qorder;
        TRY_Q(scr.alloc(&qa, m));
        TRY_Q(scr.alloc(&qorder, m));
        TRY_Q(scr.alloc(&qraw, size_t(m) * dp));
        TRY_Q(scr.alloc(&qxc, size_t(m) * dp));
        TRY_Q(scr.alloc(&qhy, m));
        TRY_Q(scr.alloc(&qnrm, m));
        TRY_Q(scr.alloc(&eps_q, 1));
        CUDA_Q(cudaMemsetAsync(eps_q, 0, sizeof(float), s));
        TRY_Q(project_sort_gather(Q, m, d, ldq, dp, ix->mu32, ix->v32, s, scr, eps_q, bad, bad + 1, qa,
                                  qorder, qraw, qxc, qhy, qnrm));
        // NaN/Inf and norm range of the queries, checked before any scoring
        float *qnmax;
        TRY_Q(scr.alloc(&qnmax, 1));
        CUDA_Q(cudaMemsetAsync(qnmax, 0, sizeof(float), s));
        SNN_LAUNCH(k_max_nonneg, std::min<unsigned>(grid_for(m, 256), 1024), 256, 0, s)(qnrm, m, qnmax);
        CUDA_Q(cudaGetLastError());
        float hq = 0.f;
        int hb[2] = {0, 0};
        {
            const HostRead rd[] = {{qnmax, &hq, int(sizeof(float))}, {bad, hb, int(sizeof(hb))}};
            TRY_Q(read_to_host(rd, 2, s));
        }
        if (hb[0]) {
            set_error("Q contains NaN or Inf");
            return fail(SNN_EINVAL);
        }
        if (hb[1]) {
            set_error("query: a bounded wait of the score sort expired");
            return fail(SNN_ETIMEOUT);
        }
        if (!(hq <= kMaxCentredNorm)) {
            set_error("a centred query norm of %g exceeds %g: the FP32 and BF16 scores would "
                      "overflow", (double)hq, kMaxCentredNorm);
            return fail(SNN_ENOTSUP);
        }
        q_nrm_max = (double)hq;
        qs.alpha = qa;
        qs.order = qorder;
        qs.raw = qraw;
        qs.xc = qxc;
        qs.hx = qhy;
        qs.nrm = qnrm;
    }
    DataSet ds{ix->n, d, dp, ix->alpha, ix->order, ix->praw, ix->xc, ix->hx, ix->nrm};

    const double Rx = radius_slack(R, d);
    const double e_data = 1.0001 * (double)kU32 * (double)ix->nrm_max;
    // window half-width: |alpha_j - alpha_q| <= ||v|| D + eps_j + eps_q
    const double Wbase = window_base(R, d);
    // per-query radii, constants and decision constants in sorted order
    double *Rs = nullptr, *R2s = nullptr;
    DecideConsts *dcs = nullptr;
    if (Rdev) {
        TRY_Q(scr.alloc(&Rs, m));
        TRY_Q(scr.alloc(&R2s, m));
        TRY_Q(scr.alloc(&dcs, m));
        SNN_LAUNCH(k_query_radii, grid_for(m, 256), 256, 0, s)(Rdev, qs.order, m, d, Rs, R2s, dcs);
        CUDA_Q(cudaGetLastError());
    }

    // the FP32 scorer's per-query thresholds (computed below when that
    // scorer runs)
    float *thrA;
    TRY_Q(scr.alloc(&thrA, m));

    const int ntiles = (int)cdiv(m, kBQ);
    int64_t *tile_lo, *tile_hi, *items, *item_off;
    // [0] survivors, [1] work, [2] band pairs, [3] candidates, [4] FP64 decisions
    unsigned long long *ctr;
    const int sym = self ? 1 : 0;
    TRY_Q(scr.alloc(&tile_lo, ntiles));
    TRY_Q(scr.alloc(&tile_hi, ntiles));
    TRY_Q(scr.alloc(&items, ntiles));
    TRY_Q(scr.alloc(&item_off, ntiles + 1));
    TRY_Q(scr.alloc(&ctr, 8));
    CUDA_Q(cudaMemsetAsync(ctr, 0, 8 * sizeof(unsigned long long), s));
    SNN_LAUNCH(k_tile_band, grid_for(ntiles, 128), 128, 0, s)(qs.alpha, m, ix->alpha, ix->n, Wbase,
                                                      ix->dconst, eps_q, tile_lo, tile_hi, items,
                                                      ntiles, sym, stats ? ctr + 2 : nullptr, Rs, d);
    CUDA_Q(cudaGetLastError());
    // the candidate-range sizes are counted for the statistics only, unless
    // the caller asked to skip them
    const bool count_cand = stats && !(stats->flags & SNN_STATS_NO_CANDIDATES);
    if (count_cand) {
        SNN_LAUNCH(k_query_windows, grid_for(m, 256), 256, 0, s)(qs.alpha, m, ix->alpha, ix->n, Wbase,
                                                         ix->dconst, eps_q, ctr + 3, Rs, d);
        CUDA_Q(cudaGetLastError());
    }
    TRY_Q(scan_exclusive<int64_t>(items, item_off, ntiles, s));
    // work item -> tile (upper bound on the item count: every tile's band is
    // at most the whole data set)
    const int64_t max_items = int64_t(ntiles) * (cdiv(ix->n, int64_t(kBR) * kChunksPerItem) + 1);
    int32_t *item_tile;
    TRY_Q(scr.alloc(&item_tile, max_items));
    SNN_LAUNCH(k_item_tiles, grid_for(ntiles, 128), 128, 0, s)(item_off, ntiles, item_tile);
    CUDA_Q(cudaGetLastError());

    // scoring with an adaptive survivor buffer; the decision, the row counts,
    // the offsets and the row classes follow without a host round trip, and
    // one synchronisation then reads every count (a survivor overflow is
    // detected there and the phase re-run with the exact size)
    double hint;
    {
        std::lock_guard<std::mutex> lk(ix->mu);
        hint = ix->surv_hint;
    }
    if (!(hint > 0)) hint = g_surv_hint.load(std::memory_order_relaxed);
    // generous first guess (the pool keeps the memory cached); an overflow
    // costs one re-run with the exact count
    int64_t cap = std::max<int64_t>(int64_t(1) << 20,
                                    int64_t(std::ceil((hint > 0 ? hint * 1.25 : 96.0) * m)) + 4096);
    if (take_fault(SNN_FAULT_SMALL_SURVIVOR_BUFFER)) cap = 1;   // forces the overflow re-run
    ScoreArgs sa;
    sa.q = qs;
    sa.x = ds;
    sa.thrA = thrA;
    sa.tile_lo = tile_lo;
    sa.tile_hi = tile_hi;
    sa.item_off = item_off;
    sa.item_tile = item_tile;
    sa.ntiles = ntiles;
    sa.sym = sym;
    sa.c1 = (float)((2.0 * d + 4.0) * (double)kU32 * 1.05);
    sa.count = ctr;
    sa.work = ctr + 1;
    int *dev_err;
    TRY_Q(scr.alloc(&dev_err, 1));
    CUDA_Q(cudaMemsetAsync(dev_err, 0, sizeof(int), s));
    sa.err = dev_err;
    sa.Rq = Rs;
    sa.q_nrm_max = q_nrm_max;
    if (stats) {
        sa.ev_kernel[0] = ev[5];
        sa.ev_kernel[1] = ev[6];
    }
    int32_t *counts, *big_list;
    ulonglong2 *lists;
    int64_t *counts64, *big_len, *toff, *soff;
    unsigned *cls;
    TRY_Q(scr.alloc(&counts, m));
    TRY_Q(scr.alloc(&counts64, m));
    TRY_Q(scr.alloc(&soff, m + 1));
    TRY_Q(scr.alloc(&lists, int64_t(kSegSlotsFine) * m));
    TRY_Q(scr.alloc(&big_list, m));
    TRY_Q(scr.alloc(&big_len, m));
    TRY_Q(scr.alloc(&toff, m + 1));
    TRY_Q(scr.alloc(&cls, kSegClasses));
    uint2 *rinfo;
    TRY_Q(scr.alloc(&rinfo, m));
    const double R2 = R * R;
    // lanes per survivor in the decision: 1 for short rows, 8 up to 128
    // dimensions, 32 beyond (four lanes at d = 16 measured slower: 1.16
    // against 0.85 ms on the 10^6-point self-join)
    const int G = d <= 32 ? 1 : (d <= 128 ? 8 : 32);
    auto dk = G == 1 ? (dp <= 16 ? (sym ? k_decide_sym : k_decide_one) : (sym ? k_decide_sym_w : k_decide_one_w))
                     : (G == 8 ? (sym ? k_decide_sym_g8 : k_decide_one_g8)
                               : (sym ? k_decide_sym_g32 : k_decide_one_g32));
    // one host read-back per attempt (see Readback)
    Readback *dev_rb = nullptr;
    TRY_Q(scr.alloc(&dev_rb, 1));
    Readback hb_store{};
    Readback *hb = &hb_store;
    int64_t mma_fpp = 0;
    int split_used = SNN_SPLIT_NONE;
    // FP8 where its shape and ranges allow it, BF16 otherwise
    const snn_precision used =
        prec == SNN_PREC_FP8E4M3 && !f8_eligible(ix, Rdev ? radius_slack(Rmax, d) : Rx) ? SNN_PREC_BF16 : prec;
    nvtx_.next("snn query: score and decide");
    for (int attempt = 0; attempt < 2; ++attempt) {
        CUDA_Q(cudaMallocAsync(&surv, size_t(cap) * sizeof(uint2), s));
        CUDA_Q(cudaMallocAsync(&rec_d2, size_t(cap) * sizeof(float), s));
        CUDA_Q(cudaMallocAsync(&rec_pos, size_t(sym ? 2 * cap : cap) * sizeof(int32_t), s));
        sa.surv = surv;
        sa.cap = cap;
        if (stats) cudaEventRecord(ev[1], s);
        snn_status st = SNN_OK;
        if (used == SNN_PREC_FP8E4M3) {
            st = f8_score_launch(ix, sa, s, Rx, e_data, scr, &mma_fpp, &split_used);
        } else if (used == SNN_PREC_BF16) {
            // with per-query radii the constants come from Rq; the largest
            // radius sets the operand scaling
            st = tc_score_launch(ix, sa, s, Rdev ? radius_slack(Rmax, d) : Rx, e_data, scr, &mma_fpp,
                                 &split_used);
        } else {
            const int grid = device_sm_count() * 2;
            if (attempt == 0)
                SNN_LAUNCH(k_query_consts, grid_for(m, 256), 256, 0, s)(qs.hx, qs.nrm, m, d, Rx, e_data, thrA,
                                                                        Rs);
            if (stats) cudaEventRecord(ev[5], s);
            if (dp <= 16)
                SNN_LAUNCH(k_score_fp32_single, grid, 256, 0, s)(sa);
            else
                SNN_LAUNCH(k_score_fp32_multi, grid, 256, 0, s)(sa);
            if (stats) cudaEventRecord(ev[6], s);
            if (cudaGetLastError() != cudaSuccess) {
                set_error("score kernel launch failed");
                st = SNN_ECUDA;
            }
        }
        if (st != SNN_OK) return fail(st);
        if (stats) cudaEventRecord(ev[2], s);
        // exact decision for every survivor (compensated FP32, FP64 where
        // needed), sized by the device-side survivor count
        CUDA_Q(cudaMemsetAsync(counts, 0, m * sizeof(int32_t), s));
        const unsigned dgrid =
            std::min<unsigned>(grid_for(cap * G, 256), unsigned(16 * device_sm_count()));
        SNN_LAUNCH(dk, dgrid, 256, 0, s)(surv, ctr, cap, qs.raw, ds.raw, d, dp, R2, decide_consts(d, R2),
                                         R2s, dcs, rec_d2, rec_pos, counts, ctr + 4);
        CUDA_Q(cudaGetLastError());
        if (stats) cudaEventRecord(ev[3], s);
        // row offsets twice: of the staging rows in sorted query positions
        // (soff) and of the output rows by query id (the same offsets when
        // the result stays in positions)
        SNN_LAUNCH(k_counts_to_i64, grid_for(m, 256), 256, 0, s)(counts, m, counts64);
        CUDA_Q(cudaGetLastError());
        CUDA_Q(cudaMemsetAsync(cls, 0, kSegClasses * sizeof(unsigned), s));
        if (pos_rows) {
            soff = out->offsets;
            TRY_Q(scan_exclusive<int64_t>(counts64, soff, m, s));
            SNN_LAUNCH(k_counts_by_id, grid_for(m, 256), 256, 0, s)(counts, qs.order, m, nullptr, soff,
                                                                    rinfo);
            CUDA_Q(cudaGetLastError());
            CUDA_Q(cudaMemsetAsync(toff + m, 0, sizeof(int64_t), s));
        } else {
            TRY_Q(scan_exclusive<int64_t>(counts64, soff, m, s));
            SNN_LAUNCH(k_counts_by_id, grid_for(m, 256), 256, 0, s)(counts, qs.order, m, counts64, soff,
                                                                    rinfo);
            CUDA_Q(cudaGetLastError());
            TRY_Q(scan_exclusive<int64_t>(counts64, out->offsets, m, s));
            // rows by length class (per-row sort below); long rows' sizes scanned
            CUDA_Q(cudaMemsetAsync(big_len, 0, m * sizeof(int64_t), s));
            SNN_LAUNCH(k_seg_classify, grid_for(m, 256), 256, 0, s)(SegMap{soff, out->offsets, qs.order}, m, 1,
                                                                     lists, big_list, big_len, cls);
            CUDA_Q(cudaGetLastError());
            TRY_Q(scan_exclusive<int64_t>(big_len, toff, m, s));
        }
        SNN_LAUNCH(k_readback, 1, 32, 0, s)(ctr, bad, dev_err, out->offsets + m, cls, toff + m, dev_rb);
        CUDA_Q(cudaGetLastError());
        {
            const HostRead rd[] = {{dev_rb, hb, int(sizeof(Readback))}};
            TRY_Q(read_to_host(rd, 1, s));
        }
        if (hb->bad) {
            set_error("Q contains NaN or Inf");
            return fail(SNN_EINVAL);
        }
        if (hb->err) {
            set_error("tensor-core scoring: a bounded wait gave up (pipeline stalled)");
            return fail(SNN_ETIMEOUT);
        }
        if ((int64_t)hb->ctr[0] <= cap) break;
        if (attempt == 1) {
            set_error("survivor buffer overflow after retry");
            return fail(SNN_EOVERFLOW);
        }
        cudaFreeAsync(surv, s);
        cudaFreeAsync(rec_d2, s);
        cudaFreeAsync(rec_pos, s);
        surv = nullptr;
        rec_d2 = nullptr;
        rec_pos = nullptr;
        cap = (int64_t)hb->ctr[0] + 1024;
        CUDA_Q(cudaMemsetAsync(ctr, 0, 8 * sizeof(unsigned long long), s));
        if (stats) {
            // the band and candidate counters are recomputed by the re-run
            SNN_LAUNCH(k_tile_band, grid_for(ntiles, 128), 128, 0, s)(
                qs.alpha, m, ix->alpha, ix->n, Wbase, ix->dconst, eps_q, tile_lo, tile_hi, items,
                ntiles, sym, ctr + 2, Rs, d);
            if (count_cand)
                SNN_LAUNCH(k_query_windows, grid_for(m, 256), 256, 0, s)(qs.alpha, m, ix->alpha, ix->n,
                                                                         Wbase, ix->dconst, eps_q, ctr + 3, Rs, d);
            CUDA_Q(cudaGetLastError());
        }
    }
    const int64_t nsurv = (int64_t)hb->ctr[0];
    {
        std::lock_guard<std::mutex> lk(ix->mu);
        ix->surv_hint = double(nsurv) / double(m);
    }
    g_surv_hint.store(double(nsurv) / double(m), std::memory_order_relaxed);
    const int64_t nnz = hb->nnz;
    if (nnz >= (int64_t(1) << 31)) {
        set_error("%lld neighbour pairs exceed this build's limit of 2^31-1", (long long)nnz);
        return fail(SNN_ENOTSUP);
    }
    out->nnz = nnz;
    nvtx_.next("snn query: CSR");
    if (nnz > 0 && pos_rows) {
        TRY_Q(dev_alloc(&out->indices, nnz, s));
        SNN_LAUNCH(k_scatter_pos, grid_for(nsurv, 1024), 256, 0, s)(surv, rec_pos, nsurv, cap, rinfo,
                                                                   out->indices);
        CUDA_Q(cudaGetLastError());
    } else if (nnz > 0) {
        TRY_Q(dev_alloc(&out->indices, nnz, s));
        TRY_Q(dev_alloc(&out->dist2, nnz, s));
        uint64_t *tmp;
        TRY_Q(scr.alloc(&tmp, nnz));
        SNN_LAUNCH(k_scatter, grid_for(nsurv, 1024), 256, 0, s)(surv, rec_pos, rec_d2, nsurv, cap, sym,
                                                               rinfo, ds.order, tmp);
        CUDA_Q(cudaGetLastError());
        // per-row ascending column ids: staging rows (sorted query positions)
        // to output rows (query ids); classes with no rows are skipped and the
        // grids sized by the class counts
        const unsigned *hc = hb->cls;
        // warps for the rows of a class (rpw rows per warp)
        auto wgrid = [&](unsigned rows, int rpw) {
            return std::min<unsigned>(grid_for(int64_t(cdiv(int64_t(rows), rpw)) * 32, 256), 16384);
        };
        auto lst = [&](int c) { return lists + int64_t(seg_slot(c)) * m; };
        int32_t *oi = out->indices;
        float *od = out->dist2;
        const SegMap oo{soff, out->offsets, qs.order};
        // ids are point ids of the index; SNN_SORT_KEYS64=1 forces the
        // 64-bit sort keys (both widths give the same rows)
        const char *k64 = getenv("SNN_SORT_KEYS64");
        const uint32_t ib = (k64 && k64[0] == '1') ? 0xffffffffu : uint32_t(ix->n);
        if (hc[7]) SNN_LAUNCH(k_seg_sort_s8, wgrid(hc[7], 4), 256, 0, s)(lst(7), cls + 7, tmp, oi, od, ib);
        if (hc[8]) SNN_LAUNCH(k_seg_sort_s16, wgrid(hc[8], 2), 256, 0, s)(lst(8), cls + 8, tmp, oi, od, ib);
        if (hc[0]) SNN_LAUNCH(k_seg_sort_w1, wgrid(hc[0], 1), 256, 0, s)(lst(0), cls, tmp, oi, od, ib);
        if (hc[6]) SNN_LAUNCH(k_seg_sort_w2, wgrid(hc[6], 1), 256, 0, s)(lst(6), cls + 6, tmp, oi, od, ib);
        if (hc[1]) SNN_LAUNCH(k_seg_sort_w4, wgrid(hc[1], 1), 256, 0, s)(lst(1), cls + 1, tmp, oi, od, ib);
        if (hc[5]) SNN_LAUNCH(k_seg_sort_w8, wgrid(hc[5], 1), 256, 0, s)(lst(5), cls + 5, tmp, oi, od, ib);
        if (hc[2]) SNN_LAUNCH(k_seg_sort_w16, wgrid(hc[2], 1), 256, 0, s)(lst(2), cls + 2, tmp, oi, od, ib);
        if (hc[3]) SNN_LAUNCH(k_seg_sort_mid, std::min<unsigned>(hc[3], 4096), 256, 0, s)(lst(3), cls + 3, tmp,
                                                                                       oi, od, ib);
        CUDA_Q(cudaGetLastError());
        const int nbig = (int)hc[4];
        if (nbig > 0) {
            const int64_t tot = hb->big_total;
            uint64_t *bk, *bka;
            uint32_t *bv, *bva;
            float *gd2;
            TRY_Q(scr.alloc(&bk, tot));
            TRY_Q(scr.alloc(&bka, tot));
            TRY_Q(scr.alloc(&bv, tot));
            TRY_Q(scr.alloc(&bva, tot));
            TRY_Q(scr.alloc(&gd2, tot));
            SNN_LAUNCH(k_seg_big_gather, nbig, 256, 0, s)(big_list, nbig, oo, toff, tmp, bk, bv, gd2);
            CUDA_Q(cudaGetLastError());
            int bits = 32;
            while ((int64_t(1) << (bits - 32)) < nbig) ++bits;
            TRY_Q(radix_sort_pairs<uint64_t>(bk, bv, bka, bva, tot, bits, s));
            SNN_LAUNCH(k_seg_big_scatter, grid_for(tot, 256), 256, 0, s)(
                bk, bv, tot, big_list, oo, toff, gd2, out->indices, out->dist2);
            CUDA_Q(cudaGetLastError());
        }
    }
    cudaFreeAsync(surv, s);
    cudaFreeAsync(rec_d2, s);
    cudaFreeAsync(rec_pos, s);
    surv = nullptr;
    rec_d2 = nullptr;
    rec_pos = nullptr;
    if (stats) {
        cudaEventRecord(ev[4], s);
        unsigned long long nf = 0;
        {
            const HostRead rd[] = {{ctr + 4, &nf, int(sizeof(nf))}};
            TRY_Q(read_to_host(rd, 1, s));
        }
        stats->exact_fp64 = (int64_t)nf;
        stats->mma_flops_per_pair = mma_fpp;
        stats->precision_used = (int32_t)used;
        stats->split_used = (int32_t)split_used;
        stats->candidates = count_cand ? (int64_t)hb->ctr[3] : -1;
        stats->band_pairs = (int64_t)hb->ctr[2];
        stats->survivors = nsurv;
        stats->nnz = nnz;
        cudaEventElapsedTime(&stats->ms_prep, ev[0], ev[1]);
        cudaEventElapsedTime(&stats->ms_score, ev[1], ev[2]);
        cudaEventElapsedTime(&stats->ms_recheck, ev[2], ev[3]);
        cudaEventElapsedTime(&stats->ms_csr, ev[3], ev[4]);
        cudaEventElapsedTime(&stats->ms_score_kernel, ev[5], ev[6]);
        for (auto &e : ev) cudaEventDestroy(e);
    }
    // the caller owns the output arrays (released by snn_free)
    TRY_Q(own_output(out->offsets, s));
    TRY_Q(own_output(out->indices, s));
    TRY_Q(own_output(out->dist2, s));
#undef TRY_Q
#undef CUDA_Q
    return SNN_OK;
}

snn_status index_build_batch(int32_t nsets, const float *const *X, const int64_t *n,
                             const int32_t *d, const int64_t *ld, cudaStream_t s, snn_index **out);
snn_status plan_create(int32_t nsets, const snn_index *const *idx, const int64_t *m_in,
                       const double *R_in, snn_precision prec, int64_t surv_cap, int64_t nnz_cap,
                       cudaStream_t s, snn_batch_plan **out);
void plan_release(snn_batch_plan *p, cudaStream_t s);
float *plan_queries(snn_batch_plan *p, int32_t t);
snn_status plan_set_queries(snn_batch_plan *p, const float *const *Q, const int64_t *ldq, cudaStream_t s);
snn_status plan_run(snn_batch_plan *p, cudaStream_t s);
snn_status plan_launch_graph(snn_batch_plan *p, cudaStream_t s);
snn_status plan_result(snn_batch_plan *p, cudaStream_t s, snn_csr *out, int64_t *need_surv,
                       int64_t *need_nnz);
snn_status plan_config(const snn_batch_plan *p, int *cpi, int *ctas, int *ngroups, unsigned *mask,
                       int *from_cache);
snn_status plan_tune(snn_batch_plan *p, cudaStream_t s, int *best_cpi, int *best_ctas,
                     float *best_ms);
snn_status batch_query(int32_t nsets, const snn_index *const *idx, const float *const *Q,
                       const int64_t *m_in, const int64_t *ldq_in, const double *R_in,
                       cudaStream_t s, snn_csr *out);

static snn_status check_finite_r(double R, const char *what) {
    if (!(R >= 0.0) || !std::isfinite(R)) {
        set_error("%s must be finite and >= 0", what);
        return SNN_EINVAL;
    }
    return SNN_OK;
}

// Inner-product threshold search: the Euclidean search on augmented rows
// (p~ = [sqrt(xi^2 - ||p||^2), p], q~ = [0, q]) with a radius for the largest
// query norm gives a superset of the pairs with p.q >= tau; the exact FP64
// dot-product decision then keeps the pairs of the definition, in id order.
static snn_status ip_search(const float *P, int64_t n, int d, int64_t ldp, const float *Q, int64_t m,
                            int64_t ldq, double tau, snn_precision prec, cudaStream_t s, snn_csr *out,
                            snn_ip_stats *st) {
    NvtxPhase nvtx_("snn inner-product search");
    ensure_pool();
    Scratch scr(s);
    double *sqP, *sqQ, *mx;
    int *bad;
    unsigned long long *nf;
    SNN_TRY(scr.alloc(&sqP, n));
    SNN_TRY(scr.alloc(&sqQ, m));
    SNN_TRY(scr.alloc(&mx, 2));
    SNN_TRY(scr.alloc(&bad, 1));
    SNN_TRY(scr.alloc(&nf, 1));
    SNN_CUDA(cudaMemsetAsync(mx, 0, 2 * sizeof(double), s));
    SNN_CUDA(cudaMemsetAsync(bad, 0, sizeof(int), s));
    SNN_CUDA(cudaMemsetAsync(nf, 0, sizeof(unsigned long long), s));
    SNN_LAUNCH(k_row_sq64, grid_for(n, 256), 256, 0, s)(P, n, d, ldp, sqP, mx, bad);
    SNN_LAUNCH(k_row_sq64, grid_for(m, 256), 256, 0, s)(Q, m, d, ldq, sqQ, mx + 1, bad);
    SNN_LAUNCH_CHECK();
    double hm[2];
    int hbad = 0;
    {
        const HostRead rd[] = {{mx, hm, int(sizeof(hm))}, {bad, &hbad, int(sizeof(int))}};
        SNN_TRY(read_to_host(rd, 2, s));
    }
    if (hbad) {
        set_error("P or Q contains NaN or Inf, or a squared norm overflows");
        return SNN_EINVAL;
    }
    // one radius per query (Rq^2 = xi^2 + ||q||^2 - 2 tau plus the slack);
    // the largest for the host choices
    const double R2 = (hm[0] + hm[1] - 2.0 * tau) + 0x1p-20 * (hm[0] + hm[1]);
    const double Rmax = R2 > 0.0 ? std::sqrt(R2) * (1.0 + 0x1p-40) : 0.0;
    if (st) {
        st->xi = std::sqrt(hm[0]);
        st->radius = Rmax;
    }
    double *Rq;
    SNN_TRY(scr.alloc(&Rq, m));
    SNN_LAUNCH(k_ip_radii, grid_for(m, 256), 256, 0, s)(sqQ, m, mx, tau, Rq);
    SNN_LAUNCH_CHECK();
    float *Pa, *Qa;
    SNN_TRY(scr.alloc(&Pa, size_t(n) * (d + 1)));
    SNN_TRY(scr.alloc(&Qa, size_t(m) * (d + 1)));
    SNN_LAUNCH(k_augment, grid_for(n, 256), 256, 0, s)(P, n, d, ldp, sqP, mx, 0, Pa);
    SNN_LAUNCH(k_augment, grid_for(m, 256), 256, 0, s)(Q, m, d, ldq, sqQ, mx, 1, Qa);
    SNN_LAUNCH_CHECK();
    snn_index *ix = nullptr;
    SNN_TRY(index_build(Pa, n, d + 1, d + 1, s, &ix));
    snn_csr cand;
    std::memset(&cand, 0, sizeof(cand));
    snn_query_stats qst{};
    snn_status rc = query_impl(ix, Qa, m, d + 1, Rmax, prec, s, &cand, st ? &qst : nullptr, Rq, Rmax);
    index_release(ix);
    if (rc != SNN_OK) return rc;
    auto drop = [&](snn_csr &c) {
        free_device_ptr(c.offsets);
        if (c.indices) free_device_ptr(c.indices);
        if (c.dist2) free_device_ptr(c.dist2);
        std::memset(&c, 0, sizeof(c));
    };
    const int64_t nnz = cand.nnz;
    if (st) {
        st->candidates = nnz;
        st->survivors = qst.survivors;
        st->band_pairs = qst.band_pairs;
    }
    out->m = m;
    if (nnz == 0) {
        *out = cand;   // every row empty
        if (st) st->nnz = 0, st->exact_fp64 = 0;
        return SNN_OK;
    }
    int64_t *rows, *keep, *pos;
    float *vals;
    SNN_TRY(scr.alloc(&rows, nnz));
    SNN_TRY(scr.alloc(&keep, nnz));
    SNN_TRY(scr.alloc(&pos, nnz + 1));    // exclusive scan: nnz + 1 entries
    SNN_TRY(scr.alloc(&vals, nnz));
    SNN_LAUNCH(k_csr_rows, grid_for(nnz, 256), 256, 0, s)(cand.offsets, m, nnz, rows);
    const int G = d <= 32 ? 1 : (d <= 128 ? 8 : 32);
    auto dk = G == 1 ? k_ip_decide_g1 : (G == 8 ? k_ip_decide_g8 : k_ip_decide_g32);
    const unsigned dgrid = std::min<unsigned>(grid_for(nnz * G, 256), unsigned(16 * device_sm_count()));
    SNN_LAUNCH(dk, dgrid, 256, 0, s)(rows, cand.indices, nnz, P, ldp, Q, ldq, d, tau, keep, vals, nf);
    SNN_LAUNCH_CHECK();
    snn_status st2 = scan_exclusive<int64_t>(keep, pos, nnz, s);
    if (st2 != SNN_OK) { drop(cand); return st2; }
    int64_t *offs = nullptr;
    if ((st2 = dev_alloc(&offs, m + 1, s)) != SNN_OK) { drop(cand); return st2; }
    SNN_LAUNCH(k_ip_offsets, grid_for(m + 1, 256), 256, 0, s)(cand.offsets, m, pos, offs);
    int64_t kept = 0;
    unsigned long long hnf = 0;
    {
        snn_status st = SNN_OK;
        if (cudaGetLastError() != cudaSuccess) {
            set_error("inner-product filter launch failed");
            st = SNN_ECUDA;
        } else {
            const HostRead rd[] = {{offs + m, &kept, int(sizeof(kept))}, {nf, &hnf, int(sizeof(hnf))}};
            st = read_to_host(rd, 2, s);
        }
        if (st != SNN_OK) {
            cudaFreeAsync(offs, s);
            drop(cand);
            return st;
        }
    }
    int32_t *oid = nullptr;
    float *oval = nullptr;
    if (kept > 0) {
        if ((st2 = dev_alloc(&oid, kept, s)) != SNN_OK || (st2 = dev_alloc(&oval, kept, s)) != SNN_OK) {
            if (oid) cudaFreeAsync(oid, s);
            cudaFreeAsync(offs, s);
            drop(cand);
            return st2;
        }
        SNN_LAUNCH(k_ip_compact, grid_for(nnz, 256), 256, 0, s)(cand.indices, vals, keep, pos, nnz, oid, oval);
        SNN_LAUNCH_CHECK();
    }
    drop(cand);
    out->m = m;
    out->nnz = kept;
    out->offsets = offs;
    out->indices = oid;
    out->dist2 = oval;
    SNN_TRY(own_output(offs, s));
    SNN_TRY(own_output(oid, s));
    SNN_TRY(own_output(oval, s));
    if (st) {
        st->nnz = kept;
        st->exact_fp64 = (int64_t)hnf;
    }
    return SNN_OK;
}

static snn_status validate_points(const float *X, int64_t n, int32_t d, int64_t ld) {
    if (!X) { set_error("X is NULL"); return SNN_EINVAL; }
    if (n < 1 || n >= (int64_t(1) << 31)) { set_error("n must be in [1, 2^31)"); return SNN_EINVAL; }
    if (d < 1 || d > 4096) { set_error("d must be in [1, 4096]"); return SNN_EINVAL; }
    if (ld < d) { set_error("ld must be >= d"); return SNN_EINVAL; }
    return SNN_OK;
}

}  // namespace snn

using namespace snn;

extern "C" {

snn_status snn_index_build(const float *X, int64_t n, int32_t d, int64_t ld, void *stream,
                           snn_index **out) {
    clear_error();
    if (!out) { set_error("out is NULL"); return SNN_EINVAL; }
    *out = nullptr;
    SNN_TRY(validate_points(X, n, d, ld));
    return index_build(X, n, d, ld, static_cast<cudaStream_t>(stream), out);
}

snn_status snn_index_build_batch(int32_t nsets, const float *const *X, const int64_t *n,
                                 const int32_t *d, const int64_t *ld, void *stream,
                                 snn_index **out) {
    clear_error();
    if (nsets < 0 || (nsets > 0 && (!X || !n || !d || !ld || !out))) {
        set_error("invalid batch arguments");
        return SNN_EINVAL;
    }
    return index_build_batch(nsets, X, n, d, ld, static_cast<cudaStream_t>(stream), out);
}

snn_status snn_query_radius(const snn_index *idx, const float *Q, int64_t m, int64_t ldq, double R,
                            snn_precision prec, void *stream, snn_csr *out,
                            snn_query_stats *stats) {
    clear_error();
    if (!idx || !out) { set_error("index or out is NULL"); return SNN_EINVAL; }
    std::memset(out, 0, sizeof(*out));
    SNN_TRY(check_finite_r(R, "R"));
    if (Q) {
        if (m < 0 || m >= (int64_t(1) << 31)) { set_error("m must be in [0, 2^31)"); return SNN_EINVAL; }
        if (ldq < idx->d) { set_error("ldq must be >= d"); return SNN_EINVAL; }
    }
    if (prec != SNN_PREC_FP32 && prec != SNN_PREC_BF16 && prec != SNN_PREC_FP8E4M3) {
        set_error("precision %d is not available in this build", (int)prec);
        return SNN_ENOTSUP;
    }
    return query_impl(idx, Q, m, ldq, R, prec, static_cast<cudaStream_t>(stream), out, stats);
}

snn_status snn_query_radius_batch(int32_t nsets, const snn_index *const *idx, const float *const *Q,
                                  const int64_t *m, const int64_t *ldq, const double *R,
                                  snn_precision prec, void *stream, snn_csr *out) {
    clear_error();
    if (nsets < 0 || (nsets > 0 && (!idx || !Q || !m || !ldq || !R || !out))) {
        set_error("invalid batch arguments");
        return SNN_EINVAL;
    }
    if (prec != SNN_PREC_FP32 && prec != SNN_PREC_BF16 && prec != SNN_PREC_FP8E4M3) {
        set_error("precision %d is not available in this build", (int)prec);
        return SNN_ENOTSUP;
    }
    ensure_pool();
    return batch_query(nsets, idx, Q, m, ldq, R, static_cast<cudaStream_t>(stream), out);
}

snn_status snn_batch_plan_create(int32_t nsets, const snn_index *const *idx, const int64_t *m,
                                 const double *R, snn_precision prec, int64_t survivor_capacity,
                                 int64_t nnz_capacity, void *stream, snn_batch_plan **out) {
    clear_error();
    if (!out) { set_error("out is NULL"); return SNN_EINVAL; }
    *out = nullptr;
    if (nsets < 1 || !idx || !m || !R) { set_error("invalid plan arguments"); return SNN_EINVAL; }
    if (prec != SNN_PREC_FP32 && prec != SNN_PREC_BF16 && prec != SNN_PREC_FP8E4M3) {
        set_error("precision %d is not available in this build", (int)prec);
        return SNN_ENOTSUP;
    }
    ensure_pool();
    return plan_create(nsets, idx, m, R, prec, survivor_capacity, nnz_capacity,
                       static_cast<cudaStream_t>(stream), out);
}

float *snn_batch_plan_queries(snn_batch_plan *plan, int32_t set) { return plan_queries(plan, set); }

snn_status snn_batch_plan_set_queries(snn_batch_plan *plan, const float *const *Q, const int64_t *ldq,
                                      void *stream) {
    clear_error();
    if (!plan || !Q || !ldq) {
        set_error("plan, Q or ldq is NULL");
        return SNN_EINVAL;
    }
    return plan_set_queries(plan, Q, ldq, static_cast<cudaStream_t>(stream));
}

snn_status snn_batch_plan_run(snn_batch_plan *plan, void *stream) {
    clear_error();
    if (!plan) { set_error("plan is NULL"); return SNN_EINVAL; }
    return plan_run(plan, static_cast<cudaStream_t>(stream));
}

snn_status snn_batch_plan_launch_graph(snn_batch_plan *plan, void *stream) {
    clear_error();
    if (!plan) { set_error("plan is NULL"); return SNN_EINVAL; }
    return plan_launch_graph(plan, static_cast<cudaStream_t>(stream));
}

snn_status snn_batch_plan_result(snn_batch_plan *plan, void *stream, snn_csr *out,
                                 int64_t *need_survivors, int64_t *need_nnz) {
    clear_error();
    if (!plan || !out) { set_error("plan or out is NULL"); return SNN_EINVAL; }
    return plan_result(plan, static_cast<cudaStream_t>(stream), out, need_survivors, need_nnz);
}

snn_status snn_batch_plan_tune(snn_batch_plan *plan, void *stream, int32_t *chunks_per_item,
                               int32_t *ctas_per_sm, float *ms) {
    clear_error();
    if (!plan) { set_error("plan is NULL"); return SNN_EINVAL; }
    return plan_tune(plan, static_cast<cudaStream_t>(stream), chunks_per_item, ctas_per_sm, ms);
}

snn_status snn_batch_plan_config(const snn_batch_plan *plan, int32_t *chunks_per_item, int32_t *ctas_per_sm,
                                 int32_t *tc_groups, uint32_t *tc_mask, int32_t *from_cache) {
    clear_error();
    if (!plan) { set_error("plan is NULL"); return SNN_EINVAL; }
    int c = 0, t = 0, g = 0, fc = 0;
    unsigned m = 0;
    plan_config(plan, &c, &t, &g, &m, &fc);
    if (chunks_per_item) *chunks_per_item = c;
    if (ctas_per_sm) *ctas_per_sm = t;
    if (tc_groups) *tc_groups = g;
    if (tc_mask) *tc_mask = m;
    if (from_cache) *from_cache = fc;
    return SNN_OK;
}

void snn_batch_plan_free(snn_batch_plan *plan, void *stream) {
    plan_release(plan, static_cast<cudaStream_t>(stream));
}

snn_status snn_dbscan(const float *X, int64_t n, int32_t d, int64_t ld, double eps, int32_t min_pts,
                      snn_precision prec, void *stream, int32_t *labels, uint8_t *is_core) {
    NvtxPhase nvtx_("snn dbscan");
    clear_error();
    SNN_TRY(validate_points(X, n, d, ld));
    SNN_TRY(check_finite_r(eps, "eps"));
    if (min_pts < 1) { set_error("min_pts must be >= 1"); return SNN_EINVAL; }
    if (!labels || !is_core) { set_error("labels/is_core is NULL"); return SNN_EINVAL; }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    snn_index *ix = nullptr;
    SNN_TRY(index_build(X, n, d, ld, s, &ix));
    // the eps-neighbourhoods by sorted position (columns ids, rows unsorted,
    // no distances): the clustering needs no order within a row
    snn_csr csr;
    snn_status st = query_impl(ix, nullptr, 0, 0, eps, prec, s, &csr, nullptr, nullptr, 0.0, true);
    if (st != SNN_OK) {
        index_release(ix);
        return st;
    }
    {
        Scratch scr(s);
        int32_t *parent = nullptr, *owner = nullptr, *minid = nullptr;
        st = scr.alloc(&parent, n);
        if (st == SNN_OK) st = scr.alloc(&owner, n);
        if (st == SNN_OK) st = scr.alloc(&minid, n);
        if (st == SNN_OK) {
            // core flags straight into is_core (by id)
            SNN_LAUNCH(k_db_core, grid_for(n, 256), 256, 0, s)(csr.offsets, ix->order, n, min_pts, is_core,
                                                       parent);
            SNN_LAUNCH(k_db_union, grid_for(n * 32, 256), 256, 0, s)(csr.offsets, csr.indices, n, is_core,
                                                             ix->order, parent);
            SNN_LAUNCH(k_db_init_minid, grid_for(n, 256), 256, 0, s)(minid, n);
            SNN_LAUNCH(k_db_assign, grid_for(n, 256), 256, 0, s)(csr.offsets, csr.indices, n, is_core,
                                                         ix->order, parent, owner, minid);
            SNN_LAUNCH(k_db_label, grid_for(n, 256), 256, 0, s)(owner, minid, ix->order, n, labels);
            cudaError_t e = cudaGetLastError();
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) {
                set_error("dbscan kernels failed: %s", cudaGetErrorString(e));
                st = SNN_ECUDA;
            }
        }
    }
    free_device_ptr(csr.offsets);
    free_device_ptr(csr.indices);
    free_device_ptr(csr.dist2);
    index_release(ix);
    return st;
}

snn_status snn_index_get_view(const snn_index *idx, snn_index_view *view) {
    clear_error();
    if (!idx || !view) { set_error("index or view is NULL"); return SNN_EINVAL; }
    view->n = idx->n;
    view->d = idx->d;
    view->dp = idx->dp;
    view->mu = idx->mu64;
    view->centre = idx->mu32;
    view->v1 = idx->v64;
    view->alpha = idx->alpha;
    view->order = idx->order;
    view->points = idx->praw;
    view->alpha_err = idx->alpha_err;
    return SNN_OK;
}

void snn_free(void *p) {
    if (p) free_device_ptr(p);
}

void snn_index_free(snn_index *idx) { index_release(idx); }

snn_status snn_index_saved_size(const snn_index *idx, int64_t *bytes) {
    clear_error();
    if (!idx || !bytes) { set_error("index or bytes is NULL"); return SNN_EINVAL; }
    SavedArray a[11];
    *bytes = saved_layout(idx->n, idx->d, idx->dp, a);
    return SNN_OK;
}

snn_status snn_index_save(const snn_index *idx, void *buf, int64_t bytes, void *stream) {
    clear_error();
    if (!idx || !buf) { set_error("index or buffer is NULL"); return SNN_EINVAL; }
    return index_save(idx, buf, bytes, static_cast<cudaStream_t>(stream));
}

snn_status snn_index_load(const void *buf, int64_t bytes, void *stream, snn_index **out) {
    clear_error();
    if (!buf || !out) { set_error("buffer or out is NULL"); return SNN_EINVAL; }
    *out = nullptr;
    return index_load(buf, bytes, static_cast<cudaStream_t>(stream), out);
}

snn_status snn_index_insert(snn_index *idx, const float *X, int64_t k, int64_t ld, void *stream) {
    clear_error();
    if (!idx) { set_error("index is NULL"); return SNN_EINVAL; }
    if (k < 0) { set_error("k must be >= 0"); return SNN_EINVAL; }
    if (k == 0) return SNN_OK;
    if (!X) { set_error("X is NULL"); return SNN_EINVAL; }
    if (ld < idx->d) { set_error("ld must be >= d"); return SNN_EINVAL; }
    if (idx->n + k >= (int64_t(1) << 31)) { set_error("n + k must be below 2^31"); return SNN_EINVAL; }
    return index_insert(idx, X, k, ld, static_cast<cudaStream_t>(stream));
}

int64_t snn_index_size(const snn_index *idx) { return idx ? idx->n : -1; }

snn_status snn_query_radius_each(const snn_index *idx, const float *Q, int64_t m, int64_t ldq,
                                 const double *R, snn_precision prec, void *stream, snn_csr *out,
                                 snn_query_stats *stats) {
    clear_error();
    if (!out) { set_error("out is NULL"); return SNN_EINVAL; }
    std::memset(out, 0, sizeof(*out));
    if (!idx) { set_error("index is NULL"); return SNN_EINVAL; }
    if (!Q || m < 1 || m >= (int64_t(1) << 31) || ldq < idx->d || !R) {
        set_error("Q (m in [1, 2^31), ldq >= d) and R must be given");
        return SNN_EINVAL;
    }
    if (prec != SNN_PREC_FP32 && prec != SNN_PREC_BF16 && prec != SNN_PREC_FP8E4M3) {
        set_error("precision %d is not available in this build", (int)prec);
        return SNN_ENOTSUP;
    }
    ensure_pool();
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    double hm[2] = {0.0, 0.0};
    int hbad = 0;
    {
        Scratch scr(s);
        double *mm;
        int *bad;
        SNN_TRY(scr.alloc(&mm, 2));
        SNN_TRY(scr.alloc(&bad, 1));
        const unsigned long long init[2] = {~0ull, 0ull};
        SNN_CUDA(cudaMemcpyAsync(mm, init, sizeof(init), cudaMemcpyHostToDevice, s));
        SNN_CUDA(cudaMemsetAsync(bad, 0, sizeof(int), s));
        SNN_LAUNCH(k_radii_minmax, grid_for(m, 256), 256, 0, s)(R, m, mm, bad);
        SNN_LAUNCH_CHECK();
        const HostRead rd[] = {{mm, hm, int(sizeof(hm))}, {bad, &hbad, int(sizeof(int))}};
        SNN_TRY(read_to_host(rd, 2, s));
    }
    if (hbad) {
        set_error("every radius must be finite and >= 0");
        return SNN_EINVAL;
    }
    return query_impl(idx, Q, m, ldq, hm[0], prec, s, out, stats, R, hm[1]);
}

snn_status snn_inner_product_search(const float *P, int64_t n, int32_t d, int64_t ldp, const float *Q,
                                    int64_t m, int64_t ldq, double tau, snn_precision prec, void *stream,
                                    snn_csr *out, snn_ip_stats *stats) {
    clear_error();
    if (!out) { set_error("out is NULL"); return SNN_EINVAL; }
    std::memset(out, 0, sizeof(*out));
    if (stats) std::memset(stats, 0, sizeof(*stats));
    if (d > 4095) { set_error("d must be at most 4095 (one augmented column)"); return SNN_EINVAL; }
    SNN_TRY(validate_points(P, n, d, ldp));
    if (m < 1 || m >= (int64_t(1) << 31) || !Q || ldq < d) {
        set_error("Q must hold m in [1, 2^31) rows with ldq >= d");
        return SNN_EINVAL;
    }
    if (!std::isfinite(tau)) { set_error("tau must be finite"); return SNN_EINVAL; }
    if (prec != SNN_PREC_FP32 && prec != SNN_PREC_BF16 && prec != SNN_PREC_FP8E4M3) {
        set_error("precision %d is not available in this build", (int)prec);
        return SNN_ENOTSUP;
    }
    return ip_search(P, n, d, ldp, Q, m, ldq, tau, prec, static_cast<cudaStream_t>(stream), out, stats);
}

snn_status snn_index_delete(snn_index *idx, const int32_t *ids, int64_t count, void *stream) {
    clear_error();
    if (!idx) { set_error("index is NULL"); return SNN_EINVAL; }
    if (count < 0) { set_error("count must be >= 0"); return SNN_EINVAL; }
    if (count == 0) return SNN_OK;
    if (!ids) { set_error("ids is NULL"); return SNN_EINVAL; }
    return index_delete(idx, ids, count, static_cast<cudaStream_t>(stream));
}

const char *snn_last_error(void) { return g_err; }

const char *snn_version(void) { return "snn-gb300 0.1 (sm_103a)"; }

uint64_t snn_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

snn_status snn_test_inject(int32_t fault) {
    clear_error();
    if (fault != 0 && fault != SNN_FAULT_STALL_TC_PRODUCER && fault != SNN_FAULT_SMALL_SURVIVOR_BUFFER &&
        fault != SNN_FAULT_DEVICE_ALLOC) {
        set_error("unknown fault %d", (int)fault);
        return SNN_EINVAL;
    }
    g_inject.store(fault);
    return SNN_OK;
}

snn_status snn_sort_scores_noalloc(const float *alpha, int64_t n, float *alpha_sorted,
                                   int32_t *order, void *stream) {
    clear_error();
    return sort_scores_noalloc(alpha, n, alpha_sorted, order, static_cast<cudaStream_t>(stream));
}

}  // extern "C"
