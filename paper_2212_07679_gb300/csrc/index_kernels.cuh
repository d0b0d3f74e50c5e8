// Declarations of the index-phase kernels (Algorithm 1).
#pragma once
#include "common.cuh"

namespace snn {

__global__ void k_colsum_partial(const float *X, int64_t n, int d, int64_t ld, int64_t rows,
                                 double *part, int *bad);
__global__ void k_mean_final(const double *part, int nb, int d, int64_t n, double *mu64,
                             float *mu32);
__global__ void k_gram_partial(const float *X, int64_t n, int d, int64_t ld, const float *mu32,
                               int64_t rows, int ntile, float *part);
__global__ void k_gram_reduce(const float *part, int nchunk, int d, double *C);
__global__ void k_pc_small(const double *C, int d, double *v64, float *v32);
__global__ void k_pc_init(const double *C, int d, float *M, double *trace_out);
__global__ void k_scale_from_double(const double *C, int64_t count, const double *tr, float *M);
__global__ void k_square(const float *M, int d, float *T);
__global__ void k_trace_f(const float *T, int d, float *scale);
__global__ void k_scale_f(const float *T, int64_t count, const float *scale, float *M);
__global__ void k_pick_column(const float *M, int d, const double *tr, double *v);
__global__ void k_matvec64(const double *C, int d, const double *v, double *w);
__global__ void k_normalise64(const double *w, int d, double *v, float *v32, int final_);
__global__ void k_project(const float *X, int64_t n, int d, int64_t ld, const double *mu64,
                          const float *v32, uint32_t *keys, uint32_t *vals, float *eps_max,
                          int *bad);
__global__ void k_gather(const uint32_t *skeys, const uint32_t *order, const float *X, int64_t n,
                         int d, int64_t ld, int dp, const double *mu64, float *alpha,
                         int32_t *order_out, float *praw, float *xc, float *hx, float *nrm);

constexpr int kPcSmallMaxD = 64;
constexpr int kGramTile = 64;

}  // namespace snn
