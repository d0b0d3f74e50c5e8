// Declarations of the index-phase kernels (Algorithm 1).
#pragma once
#include "common.cuh"

namespace snn {

__global__ void k_colsum_partial(const float *X, int64_t n, int d, int64_t ld, int64_t rows,
                                 double *part, int *bad);
__global__ void k_mean_final(const double *part, int nb, int d, int64_t n, double *mu64,
                             float *mu32);
// Small-d Gram partials for d <= 16 / 32 / 64 (one TG x TG tile per block).
__global__ void k_gram_small16(const float *X, int64_t n, int d, int64_t ld, const float *cvec,
                               int64_t rows, float *part);
__global__ void k_gram_small32(const float *X, int64_t n, int d, int64_t ld, const float *cvec,
                               int64_t rows, float *part);
__global__ void k_gram_small64(const float *X, int64_t n, int d, int64_t ld, const float *cvec,
                               int64_t rows, float *part);
__global__ void k_gram_reduce(const float *part, int nchunk, int d, double *C);
__global__ void k_pc_small(const double *C, int d, double *v64, float *v32);
__global__ void k_matvec64(const double *C, int d, const double *v, double *w);
__global__ void k_normalise64(const double *w, int d, double *v, float *v32, int final_);
__global__ void k_project(const float *X, int64_t n, int d, int64_t ld, const float *cvec,
                          const float *v32, uint32_t *keys, uint32_t *vals, float *eps_max,
                          int *bad, int vec);
__global__ void k_gather(const uint32_t *skeys, const uint32_t *order, const float *X, int64_t n,
                         int d, int64_t ld, int dp, const float *cvec, float *alpha,
                         int32_t *order_out, float *praw, float *xc, float *hx, float *nrm,
                         int vec);

constexpr int kPcSmallMaxD = 64;

// ------------------------------------------------ batched index build
// One set of a batched build (d <= kPcSmallMaxD): its input, the offsets of
// its partial sums in the shared scratch arrays, and its output slices.
struct BSet {
    const float *X;
    int64_t n, ld;
    int d, dp;
    int64_t p0;                  // global index of the set's first point
    int nb;                      // row blocks of the partial sums
    int64_t part_off;            // colsum partials: nb x d doubles
    int64_t gpart_off;           // Gram partials: nb x d x d floats
    int64_t c_off;               // C: d x d doubles
    double *mu64, *v64;
    float *mu32, *v32, *alpha, *praw, *xc, *hx, *nrm, *dconst;
    int32_t *order;
    int vec;                     // rows are float4-aligned
};
// A block's unit of work: rows [r0, r1) of set `set`, row block rb, column
// chunk cb (colsum only).
struct BBlk {
    int set, rb, cb;
    int64_t r0, r1;
};
__global__ void k_colsum_batch(const BSet *sets, const BBlk *blks, double *part, int *bad);
__global__ void k_mean_final_batch(const BSet *sets, const double *part);
__global__ void k_gram_batch16(const BSet *sets, const BBlk *blks, float *gpart);
__global__ void k_gram_batch32(const BSet *sets, const BBlk *blks, float *gpart);
__global__ void k_gram_batch64(const BSet *sets, const BBlk *blks, float *gpart);
__global__ void k_gram_reduce_batch(const BSet *sets, const float *gpart, double *C);
__global__ void k_pc_small_batch(const BSet *sets, const double *C);
__global__ void k_project_batch(const BSet *sets, const BBlk *blks, uint64_t *keys, uint32_t *vals,
                                int *bad);
__global__ void k_gather_batch(const BSet *sets, const uint64_t *skeys, const uint32_t *svals,
                               int64_t total);

// Tensor-core Gram matrix and first direction for d > kPcSmallMaxD
// (gram_tc.cu).  gram_tc: C (d x d, FP64, full) = sum_r x_r x_r^T over the
// centred rows x = fl32(p - c), and diag[i] = C[i][i].  first_direction_tc:
// v1 from C and its diagonal (FP64 and FP32 copies).  Stream-ordered; a
// bounded wait that expires sets *err (device) to nonzero, which the caller
// reads with its other device flags.  Scratch memory comes from `scr`.
snn_status gram_tc(const float *X, int64_t n, int d, int64_t ld, const float *cvec, double *C,
                   double *diag, int *err, cudaStream_t s, Scratch &scr);
snn_status first_direction_tc(const double *C, const double *diagC, int d, double *v64,
                              float *v32, int *err, cudaStream_t s, Scratch &scr);

}  // namespace snn
