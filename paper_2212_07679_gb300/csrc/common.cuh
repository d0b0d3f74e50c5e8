// Shared helpers for the libsnn CUDA sources (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <cstdio>
#include <cstdarg>
#include <string>

#include <nvtx3/nvToolsExt.h>

#include "snn.h"

namespace snn {

// NVTX ranges over the library's calls and their phases (visible in Nsight
// Systems; without a tool attached each push/pop is a cheap no-op).  The
// range is popped when the object goes out of scope, on every return path.
class NvtxPhase {
  public:
    explicit NvtxPhase(const char *name) { nvtxRangePushA(name); }
    void next(const char *name) {
        nvtxRangePop();
        nvtxRangePushA(name);
    }
    ~NvtxPhase() { nvtxRangePop(); }
    NvtxPhase(const NvtxPhase &) = delete;
    NvtxPhase &operator=(const NvtxPhase &) = delete;
};

// ---------------------------------------------------------------- errors
void set_error(const char *fmt, ...);
void clear_error();

struct Status {
    snn_status code = SNN_OK;
    bool ok() const { return code == SNN_OK; }
};

#define SNN_TRY(expr)                                    \
    do {                                                 \
        snn_status _s = (expr);                          \
        if (_s != SNN_OK) return _s;                     \
    } while (0)

#define SNN_CUDA(call)                                                          \
    do {                                                                        \
        cudaError_t _e = (call);                                                \
        if (_e != cudaSuccess) {                                                \
            ::snn::set_error("%s failed: %s (%s:%d)", #call, cudaGetErrorString(_e), \
                             __FILE__, __LINE__);                               \
            return _e == cudaErrorMemoryAllocation ? SNN_ENOMEM : SNN_ECUDA;    \
        }                                                                       \
    } while (0)

#define SNN_LAUNCH_CHECK()                                                      \
    do {                                                                        \
        cudaError_t _e = cudaGetLastError();                                    \
        if (_e != cudaSuccess) {                                                \
            ::snn::set_error("kernel launch failed: %s (%s:%d)", cudaGetErrorString(_e), \
                             __FILE__, __LINE__);                               \
            return SNN_ECUDA;                                                   \
        }                                                                       \
    } while (0)

// ------------------------------------------------- stream-ordered scratch
// One-shot fault armed by snn_test_inject: true (and disarmed) when fault
// `which` is armed; another armed fault stays armed.
bool take_fault(int which);

// Device scratch taken from the stream-ordered pool and returned on
// destruction (cudaFreeAsync on the same stream).
class Scratch {
  public:
    explicit Scratch(cudaStream_t s) : s_(s) {}
    ~Scratch() { release(); }
    Scratch(const Scratch &) = delete;
    Scratch &operator=(const Scratch &) = delete;

    template <typename T>
    snn_status alloc(T **p, size_t count) {
        void *q = nullptr;
        size_t bytes = count * sizeof(T);
        if (bytes == 0) bytes = 16;
        bytes = (bytes + 255) & ~size_t(255);
        if (take_fault(SNN_FAULT_DEVICE_ALLOC)) {
            set_error("device scratch of %zu bytes: injected test fault", bytes);
            return SNN_ENOMEM;
        }
        cudaError_t e = cudaMallocAsync(&q, bytes, s_);
        if (e != cudaSuccess) {
            set_error("device scratch of %zu bytes: %s", bytes, cudaGetErrorString(e));
            return SNN_ENOMEM;
        }
        if (n_ == kMax) {
            cudaFreeAsync(q, s_);
            set_error("too many scratch buffers");
            return SNN_ENOMEM;
        }
        ptrs_[n_++] = q;
        *p = static_cast<T *>(q);
        return SNN_OK;
    }
    void release() {
        for (int i = n_ - 1; i >= 0; --i) cudaFreeAsync(ptrs_[i], s_);
        n_ = 0;
    }

  private:
    static constexpr int kMax = 64;
    cudaStream_t s_;
    void *ptrs_[kMax];
    int n_ = 0;
};

// ------------------------------------------------------- device helpers
__host__ __device__ inline int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

// Order-preserving map of an FP32 value to uint32 (for radix sorting).
__device__ __forceinline__ uint32_t float_to_key(float f) {
    uint32_t b = __float_as_uint(f);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float key_to_float(uint32_t k) {
    uint32_t b = (k & 0x80000000u) ? (k & 0x7fffffffu) : ~k;
    return __uint_as_float(b);
}

// atomicMax for non-negative floats (their bit patterns order as integers).
__device__ __forceinline__ void atomic_max_nonneg(float *addr, float v) {
    atomicMax(reinterpret_cast<unsigned int *>(addr), __float_as_uint(v));
}

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned r;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(r));
    return r;
}

constexpr float kU32 = 5.9604644775390625e-8f;   // 2^-24, FP32 unit roundoff
// Largest centred norm accepted: products of two such norms stay far below
// the FP32 range, so no score can overflow.
constexpr double kMaxCentredNorm = 1e18;
constexpr double kU64 = 1.1102230246251565e-16;  // 2^-53

// ------------------------------------------------- library-wide primitives
// Exclusive prefix sum: out[0..n] with out[n] = total, so out must hold
// n + 1 entries.  T = int64_t/uint32_t.
template <typename T>
snn_status scan_exclusive(const T *in, T *out, int64_t n, cudaStream_t s);

// Stable LSD radix sort of (key, value) pairs by key bits [0, end_bit).
// Result is left in (keys, vals); (keys_alt, vals_alt) are scratch of n.
// With an error word (err, which the caller reads back) each 8-bit pass is
// one launch with decoupled look-back, whose bounded waits set *err if they
// give up; without one, three to four launches per pass and no waits.
template <typename K>
snn_status radix_sort_pairs(K *keys, uint32_t *vals, K *keys_alt, uint32_t *vals_alt,
                            int64_t n, int end_bit, cudaStream_t s, int *err = nullptr);

int device_sm_count();

// Small device-to-host reads that use no copy engine.  A one-block kernel on
// `s` copies each source into a mapped pinned buffer of the calling host
// thread, the stream is synchronised, and the bytes are copied to the host
// destinations.  A cudaMemcpyAsync read of a few bytes would queue on the
// device-to-host copy engine behind any bulk transfer another stream has
// issued (a CSR read-back of hundreds of MB delays it by milliseconds);
// the kernel's stores reach host memory directly.  At most kMaxHostReads
// entries and kHostReadBytes bytes in total per call.
struct HostRead {
    const void *src;   // device
    void *dst;         // host
    int bytes;
};
constexpr int kMaxHostReads = 8;
constexpr int kHostReadBytes = 2048;
snn_status read_to_host(const HostRead *reads, int n, cudaStream_t s);

// out = max(out, max_i x[i]) for non-negative x (snn_api.cu).
__global__ void k_max_nonneg(const float *x, int64_t n, float *out);


// Allocation-free stable sort of FP32 scores (noalloc_sort.cu).
snn_status sort_scores_noalloc(const float *alpha, int64_t n, float *alpha_sorted, int32_t *order,
                               cudaStream_t s);

// Every kernel launch of the library goes through SNN_LAUNCH, which counts
// it (snn_launch_count() reports the total).
void note_launch();
#define SNN_LAUNCH(kernel, ...) ::snn::note_launch(), kernel<<<__VA_ARGS__>>>

}  // namespace snn
