/* Bench-only throughput probes of the arithmetic units (libsnn_probes.so,
 * linked against libsnn.so for its error state and launch helpers).  Not part
 * of the search library's boundary: the benchmark uses them to check the
 * ratios its rooflines rely on. */
#pragma once
#include "snn.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Throughput probe for roofline denominators (the paper has no counterpart).
 * Runs one kernel that keeps one arithmetic unit of every SM busy and returns
 * its rate in flop/s, timed with CUDA events on `stream`:
 *  kind 0  tcgen05.mma kind::f16, BF16 operands, FP32 accumulation,
 *          M = 128, N = 256, K = 16 per instruction, one CTA per SM;
 *  kind 1  tcgen05.mma kind::f8f6f4, e4m3 operands, same shape with K = 32;
 *  kind 2  FP32 fused multiply-add on every lane (8 warps x 8 CTAs per SM);
 *  kind 3  FP64 fused multiply-add, same launch.
 * An MMA of M x N x K counts 2MNK flop and an FMA 2.  `iters` (>= 64) is the
 * number of instructions per issuing thread (MMAs are issued in groups of 64,
 * so kinds 0 and 1 round it down to a multiple of 64).  The operands are
 * fixed finite values; the results are discarded.  Synchronises `stream`.
 * Errors: SNN_EINVAL for kind outside 0..3, iters < 64 or a NULL output;
 * SNN_ETIMEOUT if a bounded MMA completion wait (about 2 s) expired;
 * SNN_ENOMEM / SNN_ECUDA on device failures. */
snn_status snn_measure_peak(int32_t kind, int64_t iters, void *stream, double *flops_per_s);

#ifdef __cplusplus
}
#endif
