/*
 * Plain FP64 brute-force fixed-radius search: the ground truth that every
 * GPU result is compared against.  TEST INFRASTRUCTURE ONLY: nothing on the
 * product path may link, load or call this file; only the tests, the smoke
 * check and the CPU-baseline leg of the benchmark do.
 *
 * What it computes (problem statement of Section 3 and Section 3.2; the
 * direct form Eq. (3)):
 *
 *     S(j, q) = sum_{k=0}^{d-1} (p_jk - q_k)^2,
 *
 * with every FP32 input widened exactly to FP64, the sum taken in ascending
 * k, each subtraction, product and addition rounded to nearest on its own
 * (built with -ffp-contract=off so no FMA is formed).  A point j is a
 * neighbour of q iff S(j, q) <= R2 (inclusive, as "||p_i - q|| <= R" in
 * Section 3.2 and the final test of Algorithm 2), where R2 = fl64(R * R) is passed in.
 * Neighbour ids are reported in ascending order and the squared distance is
 * reported as (float)S.  The raw, uncentred points are used: centring
 * preserves distances only in exact arithmetic (Section 3.1).
 *
 * Queries are split across OpenMP threads; each (query, point) pair is still
 * evaluated by the plain loop above, so the thread count changes no result.
 */
#include <stdint.h>
#include <stddef.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* Eq. (3): squared Euclidean distance by direct differences, FP64. */
double snn_oracle_dist2(const float *a, const float *b, int32_t d)
{
    double s = 0.0;
    for (int32_t k = 0; k < d; ++k) {
        double t = (double)a[k] - (double)b[k];
        double sq = t * t;
        s = s + sq;
    }
    return s;
}

/* counts[i] = number of points j with S(j, q_i) <= R2.  Returns the total. */
int64_t snn_oracle_count(const float *P, int64_t n, int32_t d, int64_t ldp,
                         const float *Q, int64_t m, int64_t ldq, double R2,
                         int64_t *counts)
{
    int64_t total = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : total)
    for (int64_t i = 0; i < m; ++i) {
        const float *q = Q + i * ldq;
        int64_t c = 0;
        for (int64_t j = 0; j < n; ++j) {
            if (snn_oracle_dist2(P + j * ldp, q, d) <= R2)
                ++c;
        }
        counts[i] = c;
        total += c;
    }
    return total;
}

/* Fills row i of a CSR whose offsets come from snn_oracle_count: ids in
 * ascending order (the scan over j is ascending) and dist2 = (float)S. */
void snn_oracle_fill(const float *P, int64_t n, int32_t d, int64_t ldp,
                     const float *Q, int64_t m, int64_t ldq, double R2,
                     const int64_t *offsets, int32_t *ids, float *dist2)
{
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < m; ++i) {
        const float *q = Q + i * ldq;
        int64_t o = offsets[i];
        for (int64_t j = 0; j < n; ++j) {
            double s = snn_oracle_dist2(P + j * ldp, q, d);
            if (s <= R2) {
                ids[o] = (int32_t)j;
                dist2[o] = (float)s;
                ++o;
            }
        }
    }
}

/* Same definition for an explicit list of (query row, point row) pairs, in
 * FP64: out[t] = S(pj[t], q_{qi[t]}).  Used for sampled checks at full size. */
void snn_oracle_pairs(const float *P, int32_t d, int64_t ldp,
                      const float *Q, int64_t ldq,
                      const int64_t *qi, const int64_t *pj, int64_t npairs,
                      double *out)
{
#pragma omp parallel for schedule(static)
    for (int64_t t = 0; t < npairs; ++t)
        out[t] = snn_oracle_dist2(P + pj[t] * ldp, Q + qi[t] * ldq, d);
}

int32_t snn_oracle_threads(void)
{
#ifdef _OPENMP
    return (int32_t)omp_get_max_threads();
#else
    return 1;
#endif
}
