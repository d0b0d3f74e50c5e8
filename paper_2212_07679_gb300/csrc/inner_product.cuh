// Kernels of the inner-product threshold search (see inner_product.cu).
#pragma once
#include "common.cuh"

namespace snn {

// sq[i] = sum over ascending k of x_ik^2 in FP64; *sq_max (zero-initialised)
// receives the largest finite value; a non-finite row sets *bad.
__global__ void k_row_sq64(const float *X, int64_t n, int d, int64_t ld, double *sq, double *sq_max,
                           int *bad);

// Augmented rows of d + 1 floats: [fl32(sqrt(max(0, xi2 - sq[i]))), x_i] for
// points, [0, x_i] for queries (query != 0).
__global__ void k_augment(const float *X, int64_t n, int d, int64_t ld, const double *sq,
                          const double *xi2, int query, float *out);

// mm[0] = min, mm[1] = max of R (mm preset to +inf bits / 0); a negative,
// NaN or infinite radius sets *bad.
__global__ void k_radii_minmax(const double *R, int64_t m, double *mm, int *bad);

// Per-query radius of the augmented Euclidean search for threshold tau.
__global__ void k_ip_radii(const double *sqQ, int64_t m, const double *xi2, double tau, double *R);

// rows[e] = the CSR row holding entry e.
__global__ void k_csr_rows(const int64_t *offsets, int64_t m, int64_t nnz, int64_t *rows);

// Exact decision D(point ids[e], query rows[e]) >= tau with value fl32(D);
// 1, 8 or 32 lanes per candidate.
__global__ void k_ip_decide_g1(const int64_t *rows, const int32_t *ids, int64_t nnz, const float *P,
                               int64_t ldp, const float *Q, int64_t ldq, int d, double tau, int64_t *keep,
                               float *vals, unsigned long long *n_fp64);
__global__ void k_ip_decide_g8(const int64_t *rows, const int32_t *ids, int64_t nnz, const float *P,
                               int64_t ldp, const float *Q, int64_t ldq, int d, double tau, int64_t *keep,
                               float *vals, unsigned long long *n_fp64);
__global__ void k_ip_decide_g32(const int64_t *rows, const int32_t *ids, int64_t nnz, const float *P,
                                int64_t ldp, const float *Q, int64_t ldq, int d, double tau, int64_t *keep,
                                float *vals, unsigned long long *n_fp64);

// Offsets of the kept entries (pos = exclusive scan of keep, nnz + 1
// entries) and their compaction; the kept entries of a row stay in id order.
__global__ void k_ip_offsets(const int64_t *offsets, int64_t m, const int64_t *pos, int64_t *out_offsets);
__global__ void k_ip_compact(const int32_t *ids, const float *vals, const int64_t *keep, const int64_t *pos,
                             int64_t nnz, int32_t *out_ids, float *out_vals);

}  // namespace snn
