// Throughput probes for the roofline denominators: back-to-back tcgen05 MMAs
// (kind::f16 BF16 and kind::f8f6f4 e4m3, M = 128, N = 256, K = 16 / 32, one
// CTA per SM issuing into its own TMEM accumulator from fixed shared-memory
// tiles) and FP32 / FP64 fused multiply-add loops on every lane.  Each probe
// is timed with CUDA events on the caller's stream and reports flop/s (an
// MMA of M x N x K counts 2 M N K flop, an FMA 2).
#include <cmath>

#include "common.cuh"
#include "peaks.h"
#include "tc_common.cuh"

namespace snn {
namespace {

constexpr int kPM = 128, kPN = 256;

// kind: 0 = BF16 kind::f16 (K = 16), 1 = e4m3 kind::f8f6f4 (K = 32).  The
// 32-byte rows of A (128 rows) and B (256 rows) hold small finite values of
// either type (no NaN encodings).  MMAs are committed every 64 and the
// thread waits for the previous group (bounded), so that the queue stays
// full without growing.
__global__ void __launch_bounds__(128) k_peak_mma(int kind, int64_t iters, int *err, float *sink) {
    __shared__ __align__(1024) unsigned char sa[kPM * 32];
    __shared__ __align__(1024) unsigned char sb[kPN * 32];
    __shared__ __align__(8) uint64_t bars[2];
    __shared__ uint32_t s_tmem;
    __shared__ int s_abort;
    const int warp = threadIdx.x >> 5;
    // bytes 0x3C / 0x38 are 1.0-ish in both formats' low byte patterns;
    // alternate a few values so the operands are not constant
    for (int i = threadIdx.x; i < kPM * 32; i += blockDim.x) sa[i] = (unsigned char)(0x30 + (i * 7) % 11);
    for (int i = threadIdx.x; i < kPN * 32; i += blockDim.x) sb[i] = (unsigned char)(0x30 + (i * 5) % 13);
    if (threadIdx.x == 0) {
        mbar_init(smem_u32(&bars[0]), 1);
        mbar_init(smem_u32(&bars[1]), 1);
        s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                     "n"(256) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tmem_fence_before();
    __syncthreads();
    tmem_fence_after();
    const uint32_t tmem = s_tmem;
    if (threadIdx.x == 0) {
        const uint64_t ad = smem_desc<32>(smem_u32(sa)), bd = smem_desc<32>(smem_u32(sb));
        constexpr int kGroup = 64;
        int64_t groups = iters / kGroup;
        for (int64_t g = 0; g < groups && !s_abort; ++g) {
            for (int i = 0; i < kGroup; ++i) {
                const uint32_t acc = (g | i) != 0 ? 1u : 0u;
                if (kind == 1) mma_e4m3(tmem, ad, bd, idesc_e4m3<kPM, kPN>(), acc);
                else mma_bf16(tmem, ad, bd, idesc_bf16<kPM, kPN>(), acc);
            }
            mma_commit(smem_u32(&bars[g & 1]));
            // wait for the group before the previous one (two in flight)
            if (g >= 1 && !mbar_wait(smem_u32(&bars[(g - 1) & 1]), uint32_t((g - 1) >> 1) & 1u, &s_abort, err))
                break;
        }
        if (groups >= 1 && !s_abort)
            mbar_wait(smem_u32(&bars[(groups - 1) & 1]), uint32_t((groups - 1) >> 1) & 1u, &s_abort, err);
    }
    tmem_fence_before();
    __syncthreads();
    tmem_fence_after();
    if (!s_abort) {
        uint32_t r[64];
        tmem_ld64(tmem + (uint32_t(warp * 32) << 16), r);
        if (__uint_as_float(r[0]) == 12345.f) sink[blockIdx.x] = __uint_as_float(r[1]);   // keep the work
    }
    tmem_fence_before();
    __syncthreads();
    tmem_fence_after();
    if (warp == 1)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "n"(256) : "memory");
}

// Eight independent FMA chains per thread.
__global__ void __launch_bounds__(256) k_peak_ffma(int64_t iters, float *sink) {
    float a[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) a[j] = 1.0f + 1e-7f * float(threadIdx.x + j);
    const float b = 0.9999999f, c = 1e-8f;
    for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < 8; ++j) a[j] = fmaf(a[j], b, c);
    }
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < 8; ++j) s += a[j];
    if (s == 12345.f) sink[blockIdx.x] = s;
}

__global__ void __launch_bounds__(256) k_peak_dfma(int64_t iters, double *sink) {
    double a[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) a[j] = 1.0 + 1e-15 * double(threadIdx.x + j);
    const double b = 0.9999999999, c = 1e-16;
    for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < 8; ++j) a[j] = fma(a[j], b, c);
    }
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < 8; ++j) s += a[j];
    if (s == 12345.0) sink[blockIdx.x] = s;
}

}  // namespace
}  // namespace snn

using namespace snn;

extern "C" snn_status snn_measure_peak(int32_t kind, int64_t iters, void *stream, double *flops_per_s) {
    clear_error();
    if (!flops_per_s || kind < 0 || kind > 3 || iters < 64) {
        set_error("kind must be 0..3, iters >= 64 and flops_per_s non-NULL");
        return SNN_EINVAL;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int sms = device_sm_count();
    Scratch scr(s);
    int *err;
    double *sink;
    SNN_TRY(scr.alloc(&err, 1));
    SNN_TRY(scr.alloc(&sink, size_t(sms) * 8));
    SNN_CUDA(cudaMemsetAsync(err, 0, sizeof(int), s));
    cudaEvent_t e0, e1;
    SNN_CUDA(cudaEventCreate(&e0));
    SNN_CUDA(cudaEventCreate(&e1));
    double flops = 0.0;
    const int64_t groups = iters / 64;
    SNN_CUDA(cudaEventRecord(e0, s));
    if (kind <= 1) {
        SNN_LAUNCH(k_peak_mma, sms, 128, 0, s)(kind, iters, err, reinterpret_cast<float *>(sink));
        flops = 2.0 * kPM * kPN * (kind == 1 ? 32 : 16) * double(groups * 64) * sms;
    } else if (kind == 2) {
        const int blocks = sms * 8;
        SNN_LAUNCH(k_peak_ffma, blocks, 256, 0, s)(iters, reinterpret_cast<float *>(sink));
        flops = 2.0 * 8 * double(iters) * blocks * 256;
    } else {
        const int blocks = sms * 8;
        SNN_LAUNCH(k_peak_dfma, blocks, 256, 0, s)(iters, sink);
        flops = 2.0 * 8 * double(iters) * blocks * 256;
    }
    SNN_LAUNCH_CHECK();
    SNN_CUDA(cudaEventRecord(e1, s));
    int herr = 0;
    SNN_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s));
    SNN_CUDA(cudaEventSynchronize(e1));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (herr) {
        set_error("peak probe: a bounded wait expired");
        return SNN_ETIMEOUT;
    }
    *flops_per_s = flops / (double(ms) * 1e-3);
    return SNN_OK;
}
