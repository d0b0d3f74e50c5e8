/*
 * snn.h -- C ABI of libsnn: exact fixed-radius neighbour search by sorting
 * (SNN, Chen & Guettel, arXiv 2212.07679) on one NVIDIA GB300 (sm_103a).
 *
 * Problem (Section 3, Section 3.2): given points p_1..p_n in R^d, a query q
 * and a radius R, return every i with ||p_i - q|| <= R (inclusive), and the
 * squared distances (Section 3: "can also return the corresponding
 * distances").
 *
 * Exactness contract.  A point j is reported for query q iff the FP64 value
 *     S(j, q) = sum_{k=0..d-1} (p_jk - q_k)^2
 * (FP32 inputs widened exactly, ascending k, every operation rounded to
 * nearest, no fused multiply-add) satisfies S <= fl64(R*R); the reported
 * squared distance is (float)S.  Faster low-precision scoring only rejects
 * pairs that a rigorous rounding bound proves to be outside the radius; every
 * other pair is decided by S itself.
 *
 * Conventions for every entry point:
 *  - Pointers named "device" are CUDA device pointers on the current device;
 *    "host" pointers are ordinary host memory.
 *  - Points and queries are FP32, row-major, with a leading dimension (row
 *    stride, in elements) >= d.  The library reads them during the call only
 *    and never retains them.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  All device work of a call is ordered on that stream.  Calls
 *    that must size their outputs synchronise the stream once to read a count.
 *  - Every function returns a status and never aborts, traps or prints.  On a
 *    non-OK status, snn_last_error() gives a message for the calling thread
 *    and no output is owned by the caller.
 *  - Limits: 1 <= d <= 4096, 1 <= n < 2^31, m < 2^31, total neighbour pairs
 *    of one call < 2^31 (SNN_ENOTSUP beyond that).
 *  - Environment variables (read at each call; none changes any result):
 *    SNN_TC_SPLIT = bf16x2, bf16x3 or fp16x2 and SNN_FP8_PRODUCTS = 3, 4 or 6
 *    fix the tensor-core split (see snn_precision); SNN_SORT_KEYS64 = 1 makes the
 *    per-row sort of the CSR build use 64-bit keys even where 32-bit keys
 *    (id and position in the row) fit.
 */
#ifndef SNN_H
#define SNN_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SNN_OK = 0,
    SNN_EINVAL = 1,     /* invalid argument, or NaN/Inf in the data        */
    SNN_ENOMEM = 2,     /* device or host allocation failed                */
    SNN_ECUDA = 3,      /* a CUDA runtime call failed                      */
    SNN_ETIMEOUT = 4,   /* a bounded device wait gave up                   */
    SNN_EOVERFLOW = 5,  /* a device buffer stayed too small after a retry  */
    SNN_ENOTSUP = 6     /* size or feature beyond this build's limits      */
} snn_status;

/* Arithmetic used to reject candidate pairs before the exact FP64 decision
 * (Section 4, Eq. (4): x_j^T x_j/2 - x_j^T x_q <= (R^2 - x_q^T x_q)/2).
 * The output is identical for every precision; only the speed differs. */
typedef enum {
    SNN_PREC_FP32 = 0,      /* FP32 CUDA-core dot products                  */
    SNN_PREC_BF16 = 1,      /* 16-bit tcgen05 tensor-core dot products: two
                               BF16 parts of each value where that bound is
                               tight enough for the norms and R, else two
                               FP16 parts of the rows scaled by a power of
                               two (folded threshold columns in BF16); the
                               environment variable SNN_TC_SPLIT = bf16x2,
                               bf16x3 or fp16x2 overrides                   */
    SNN_PREC_FP8E4M3 = 2    /* FP8 e4m3 tcgen05 dot products, each row
                               scaled by its own power of two; used for
                               d > 55 with norms and R below 2^20, BF16
                               elsewhere (see precision_used).  Two e4m3
                               parts (3 or 4 products per k-step) where the
                               largest norm is within about 2R, else three
                               (6 products); the environment variable
                               SNN_FP8_PRODUCTS = 3, 4 or 6 overrides       */
} snn_precision;

/* Opaque index (Algorithm 1 output): mean mu, first principal direction v1,
 * points sorted by their score alpha_i = (p_i - mu)^T v1, halved squared
 * norms of the centred points, and the sort permutation.  Library-owned;
 * release with snn_index_free. */
typedef struct snn_index snn_index;

/* Neighbour lists in CSR form.  Row r (r = 0..m-1) holds the neighbours of
 * query r at indices[offsets[r] .. offsets[r+1]-1], as ORIGINAL point ids
 * (row numbers of the X given to snn_index_build) in ascending order, with
 * dist2[] the matching (float)S.  All three arrays are DEVICE memory
 * allocated by the library; release each with snn_free.  offsets has m+1
 * entries; indices/dist2 are NULL when nnz == 0. */
typedef struct {
    int64_t m;
    int64_t nnz;
    int64_t *offsets;
    int32_t *indices;
    float *dist2;
} snn_csr;

/* Optional per-call counters (pass NULL to skip; a non-NULL pointer adds a
 * few small kernels and one extra stream synchronisation).
 *  candidates  sum over queries of |J_q|, the candidate range of Algorithm 2
 *              (with the rounding-safe widening);
 *  band_pairs  pairs actually scored (query tiles score the union of their
 *              queries' ranges, Section 4's gemm over the union of J);
 *  survivors   pairs the low-precision test could not reject, all of which
 *              were decided exactly (recheck count; a symmetric self-join
 *              counts each unordered pair once);
 *  nnz         neighbour pairs returned;
 *  exact_fp64  survivors whose decision or distance needed the FP64 loop
 *              itself (the compensated FP32 evaluation settles the rest);
 *  mma_flops_per_pair  tensor-core flops executed per scored pair (BF16
 *              or e4m3 split products and folded threshold columns; 0 for
 *              FP32);
 *  precision_used  the rejection arithmetic that ran (an FP8 request runs
 *              BF16 where FP8 is not available);
 *  split_used  operand split of the tensor-core scorer: SNN_SPLIT_NONE (FP32
 *              scoring), SNN_SPLIT_BF16X2, SNN_SPLIT_BF16X3, SNN_SPLIT_FP16X2,
 *              SNN_SPLIT_FP16X1, or for e4m3 SNN_SPLIT_E4M3 + products per
 *              k-step (3, 4, 6);
 *  ms_*        device time of the phases (CUDA events on `stream`);
 *              ms_score covers the operand packing and the scoring launch,
 *              ms_score_kernel the scoring launch alone;
 *  flags       read on input (zero-initialise the struct): with
 *              SNN_STATS_NO_CANDIDATES set the per-query candidate-range
 *              sizes are not counted (one kernel of FP64 range arithmetic
 *              fewer) and candidates is returned as -1. */
typedef struct {
    int64_t candidates;
    int64_t band_pairs;
    int64_t survivors;
    int64_t nnz;
    int64_t exact_fp64;
    int64_t mma_flops_per_pair;
    float ms_prep;
    float ms_score;
    float ms_recheck;
    float ms_csr;
    int32_t precision_used;
    int32_t split_used;
    float ms_score_kernel;
    int32_t flags;
} snn_query_stats;

#define SNN_STATS_NO_CANDIDATES 1

#define SNN_SPLIT_NONE 0
#define SNN_SPLIT_BF16X2 1
#define SNN_SPLIT_BF16X3 2
#define SNN_SPLIT_FP16X2 3
#define SNN_SPLIT_FP16X1 4
#define SNN_SPLIT_E4M3 10

/* Algorithm 1 (Section 3.1): centre, first principal direction, scores,
 * sort, halved norms.
 *  X      device, n x d FP32 row-major, row stride ld (elements, >= d).
 *  out    host pointer receiving a new index (caller frees with
 *         snn_index_free).
 * Errors: SNN_EINVAL for n < 1, d < 1, d > 4096, ld < d, n >= 2^31, X NULL or
 * any NaN/Inf in X; SNN_ENOMEM / SNN_ECUDA on device failures.  Synchronises
 * `stream` once (to check the data for NaN/Inf). */
snn_status snn_index_build(const float *X, int64_t n, int32_t d, int64_t ld,
                           void *stream, snn_index **out);

/* Algorithm 1 for nsets independent sets at once (many small problems of
 * uneven n and d): one launch per step over every set and one sort of all
 * scores by the composite key (set, score); the result is nsets ordinary
 * indices (each freed with snn_index_free; their arrays are slices of shared
 * blocks released with the last one).  The scores may differ from a
 * per-set snn_index_build in the last bits (partial sums are grouped
 * differently); every query result is exact either way.
 *  X, n, d, ld  host arrays of nsets entries; X[t] device, n[t] x d[t] FP32,
 *               row stride ld[t].  1 <= d[t] <= 64, n[t] >= 1, total points
 *               < 2^31.
 *  out          host array of nsets index pointers (all NULL on error).
 * Errors: SNN_EINVAL for invalid sizes or NaN/Inf in any set; SNN_ENOTSUP
 * when a centred norm exceeds 1e18.  Synchronises `stream` once. */
snn_status snn_index_build_batch(int32_t nsets, const float *const *X, const int64_t *n,
                                 const int32_t *d, const int64_t *ld, void *stream,
                                 snn_index **out);

/* Algorithm 2 (Section 3.2) for m queries at once (Section 4: one gemm over
 * the union of candidate ranges of a tile of queries sorted by score).
 *  Q      device, m x d FP32 row-major, stride ldq; NULL means the self-join:
 *         the queries are the index's own points, row r of the result is
 *         point r (m and ldq are then ignored).  An empty query set is m == 0
 *         with any non-NULL Q (it is not read).
 *  R      radius, finite and >= 0 (double); the test is S <= fl64(R*R).
 *  prec   rejection arithmetic (see snn_precision).
 *  out    host struct receiving library-allocated device arrays.
 *  stats  optional host struct (NULL to skip).
 * Errors: SNN_EINVAL for a NULL index/out, m < 0, ldq < d, R < 0 or
 * non-finite, NaN/Inf in Q; SNN_ENOTSUP for an unavailable precision or more
 * than 2^31-1 result pairs; SNN_ENOMEM / SNN_ECUDA on device failures.
 * m == 0 returns SNN_OK with offsets = {0}. */
snn_status snn_query_radius(const snn_index *idx, const float *Q, int64_t m, int64_t ldq,
                            double R, snn_precision prec, void *stream,
                            snn_csr *out, snn_query_stats *stats);

/* Many independent (index, queries, radius) problems in one call (ragged n,
 * d and m).  Arrays of length nsets; Q[s] may be NULL (self-join of set s);
 * ldq[s] is ignored for a self-join.  out[s] receives the CSR of set s.
 * Errors: as snn_query_radius for each set; on error no out[s] is owned by
 * the caller. */
snn_status snn_query_radius_batch(int32_t nsets, const snn_index *const *idx,
                                  const float *const *Q, const int64_t *m,
                                  const int64_t *ldq, const double *R,
                                  snn_precision prec, void *stream, snn_csr *out);

/* Radius search with one radius per query (out-of-sample queries): query i
 * takes the points with S <= fl64(R[i]*R[i]) (S as in snn_query_radius).
 *  R       device, m FP64 radii in query order (finite, >= 0).
 * Other arguments, output and errors as snn_query_radius (Q must be given);
 * SNN_EINVAL also for a negative, NaN or infinite radius.  Synchronises
 * `stream` once more (the radii are validated first). */
snn_status snn_query_radius_each(const snn_index *idx, const float *Q, int64_t m, int64_t ldq,
                                 const double *R, snn_precision prec, void *stream, snn_csr *out,
                                 snn_query_stats *stats);

/* Inner-product threshold search (the maximum-inner-product variant of
 * Section 3).  Returns, for every query q (row of Q), the points p (rows of
 * P) with D(p, q) >= tau, where D is the FP64 dot product summed over
 * ascending k with every product and sum rounded to nearest and no fused
 * multiply-add; ids ascending, and the CSR's dist2 array holds fl32(D).
 * Section 3 turns p.q into a Euclidean distance of augmented rows,
 * ||p~ - q~||^2 = xi^2 + ||q||^2 - 2 p.q with p~ = [sqrt(xi^2 - ||p||^2), p],
 * q~ = [0, q], xi = max ||p||; the search prunes with SNN on those rows
 * (one radius, for the largest query norm, widened by the rounding of the
 * augmented coordinate) and decides every remaining pair on the exact dot
 * product.
 *  P, Q    device FP32, n x d and m x d, row strides ldp, ldq (>= d).
 *  tau     finite threshold.
 *  prec    rejection arithmetic of the Euclidean stage (see snn_precision).
 *  out     host struct receiving the CSR (device arrays; free each with
 *          snn_free).
 *  stats   optional: xi, the Euclidean radius, the Euclidean candidates and
 *          their survivors, the pairs returned and those the FP64 loop decided.
 * Errors: SNN_EINVAL for NULL arguments, n or m outside [1, 2^31), d outside
 * [1, 4095], ld < d, a non-finite tau, NaN/Inf in P or Q; as
 * snn_query_radius otherwise.  Synchronises `stream`. */
typedef struct {
    double xi;
    double radius;
    int64_t band_pairs;
    int64_t survivors;
    int64_t candidates;
    int64_t nnz;
    int64_t exact_fp64;
} snn_ip_stats;
snn_status snn_inner_product_search(const float *P, int64_t n, int32_t d, int64_t ldp, const float *Q,
                                    int64_t m, int64_t ldq, double tau, snn_precision prec, void *stream,
                                    snn_csr *out, snn_ip_stats *stats);

/* Streaming updates of a built index (Section 1: the index suits an online
 * setting).  Algorithm 2 is exact for any unit direction v and any centre, so
 * new points are scored with the index's own centre and direction (no PCA
 * refresh; a stale direction only weakens the pruning) and merged into the
 * sorted order, and deleted points are compacted out.  The result of every
 * later query equals that of an index built on the updated point set.
 * The caller orders an update after every query that uses the index (the
 * index's arrays are replaced in order on `stream`); cached tensor-core
 * operands are rebuilt by the next query.  Both calls synchronise `stream`
 * once (to validate before the index is changed); on an error the index is
 * unchanged.
 *
 * snn_index_insert: the k rows of X (device, k x d FP32, row stride ld >= d)
 * become points n, n+1, ..., n+k-1.
 * Errors: SNN_EINVAL for k < 0, NULL arguments, ld < d, n + k >= 2^31 or a
 * NaN/Inf in X; SNN_ENOTSUP for a centred norm above 1e18; SNN_ENOMEM /
 * SNN_ECUDA on device failures.  k = 0 does nothing.
 *
 * snn_index_delete: removes the points whose ids are listed in ids (device,
 * count int32; repeats allowed).  The remaining points are renumbered
 * 0, 1, ... in their previous id order, as if their rows had been erased from
 * X.  Errors: SNN_EINVAL for count < 0, NULL arguments, an id outside [0, n)
 * or a deletion of every point. */
snn_status snn_index_insert(snn_index *idx, const float *X, int64_t k, int64_t ld, void *stream);
snn_status snn_index_delete(snn_index *idx, const int32_t *ids, int64_t count, void *stream);

/* Number of points of an index (host value; -1 for NULL). */
int64_t snn_index_size(const snn_index *idx);

/* Cosine and angular distances (Section 3): for unit vectors u, v the
 * cosine distance 1 - u.v equals ||u - v||^2 / 2, and the angle between them
 * is at most alpha exactly when ||u - v||^2 <= 2 - 2 cos(alpha).  A cosine or
 * angular search is the Euclidean search (snn_index_build, snn_query_radius)
 * on rows normalised by snn_normalize_rows, with the radius from
 * snn_radius_for_cosine_distance or snn_radius_for_cosine_similarity; the
 * returned dist2 is then twice the cosine distance of the normalised rows.
 *
 * snn_normalize_rows: row i of X becomes u_k = fl32(x_k * r), r =
 * 1 / sqrt(sum over ascending k of x_k^2), all in FP64 with every operation
 * rounded to nearest and no fused multiply-add; a row of zeros stays zero, a
 * NaN or infinity makes its row NaN (which the index build then rejects).
 *  X, out  device, n x d FP32 with row strides ld, ldo (elements, >= d); out
 *          may be X (in place, ldo == ld).
 *  stream  cudaStream_t; the call is stream-ordered and does not synchronise.
 * Errors: SNN_EINVAL for n < 0, d < 1, ld or ldo < d, NULL arrays (n > 0);
 * SNN_ECUDA if the launch fails. */
snn_status snn_normalize_rows(const float *X, int64_t n, int32_t d, int64_t ld, float *out,
                              int64_t ldo, void *stream);

/* Radius of the Euclidean search on normalised rows: sqrt(2 c) for a cosine
 * distance bound c in [0, 2]; sqrt(2 - 2 t) for a cosine similarity bound t
 * in [-1, 1] (t = cos(alpha) for an angle bound alpha).  FP64, correctly
 * rounded square root; NaN outside the ranges. */
double snn_radius_for_cosine_distance(double c);
double snn_radius_for_cosine_similarity(double t);

/* DBSCAN with SNN as its neighbour search (Section 6.4).
 *  X        device, n x d FP32, stride ld.
 *  eps      neighbourhood radius (inclusive, S <= fl64(eps*eps)).
 *  min_pts  a point is core iff its eps-neighbourhood, itself included,
 *           has >= min_pts points.
 *  labels   device, n int32 (caller-allocated): -1 for noise, otherwise the
 *           smallest point id of the point's cluster.  Clusters are the
 *           connected components of core points joined by neighbour pairs;
 *           a non-core point with a core neighbour joins the cluster of its
 *           smallest-id core neighbour.
 *  is_core  device, n uint8 (caller-allocated): 1 for core points.
 * Errors: as snn_index_build, plus SNN_EINVAL for eps < 0/non-finite or
 * min_pts < 1, or NULL outputs. */
snn_status snn_dbscan(const float *X, int64_t n, int32_t d, int64_t ld, double eps,
                      int32_t min_pts, snn_precision prec, void *stream,
                      int32_t *labels, uint8_t *is_core);

/* Plan of a batched query (Algorithm 2 for nsets independent problems; the
 * paper has no counterpart) whose runs are pure stream-ordered device work:
 * every size is fixed at creation (queries per set, survivor and neighbour
 * capacities), so a run never synchronises and can be captured into a CUDA
 * graph and replayed with new query values.  One persistent FP32 scoring
 * launch covers every (set, query tile, band chunk group) item of the batch
 * through a device work counter.  With prec SNN_PREC_BF16 (or FP8, which
 * takes the same path here) the out-of-sample sets of d <= 48 are scored on
 * the tensor cores instead, one launch per group of sets with the same
 * rounded width (d <= 16, <= 32, <= 48): two FP16 parts of each set's rows
 * scaled by its own power of two, packed once at creation (Eq. (4) with the
 * same rejection bound as snn_query_radius); results are exact either way.
 *  idx, m, R  host arrays of nsets entries: m[t] queries for set t (written
 *             into the plan's buffer, snn_batch_plan_queries) or m[t] < 0 for
 *             the self-join of idx[t].  The indices must outlive the plan.
 *  survivor_capacity, nnz_capacity  sizes of the survivor list and of the
 *             result (all sets together); a run that needs more reports
 *             SNN_EOVERFLOW from snn_batch_plan_result with the sizes needed.
 * Synchronises `stream` once (setup). */
typedef struct snn_batch_plan snn_batch_plan;
snn_status snn_batch_plan_create(int32_t nsets, const snn_index *const *idx, const int64_t *m,
                                 const double *R, snn_precision prec, int64_t survivor_capacity,
                                 int64_t nnz_capacity, void *stream, snn_batch_plan **out);

/* Device buffer of set t's queries (m[t] x d FP32 rows, stride d), read by
 * every run; NULL for a self-join set or an invalid t. */
float *snn_batch_plan_queries(snn_batch_plan *plan, int32_t set);

/* Copies every out-of-sample set's queries into the plan's buffers in one
 * launch on `stream` (instead of one copy per set).
 *  Q    host array of nsets device pointers: Q[t] holds m[t] x d FP32 rows
 *       with stride ldq[t] >= d; ignored (may be NULL) for self-join sets and
 *       sets of no query.
 *  ldq  host array of nsets row strides (elements).
 * Errors: SNN_EINVAL for a NULL plan, Q or ldq, a NULL Q[t] or ldq[t] < d of
 * an out-of-sample set with queries; SNN_ECUDA on a device failure.  No
 * synchronisation; NaN or Inf values are reported by the next run's
 * snn_batch_plan_result. */
snn_status snn_batch_plan_set_queries(snn_batch_plan *plan, const float *const *Q, const int64_t *ldq,
                                      void *stream);

/* Enqueues one run on `stream` (no synchronisation). */
snn_status snn_batch_plan_run(snn_batch_plan *plan, void *stream);

/* One run as a CUDA graph launch: the run is captured into a graph on the
 * first call (after any snn_batch_plan_tune) and the graph replayed. */
snn_status snn_batch_plan_launch_graph(snn_batch_plan *plan, void *stream);

/* Synchronises `stream` and returns the last run's result: out[t] views the
 * plan's own arrays (valid until the next run or snn_batch_plan_free; do not
 * pass them to snn_free).  need_survivors / need_nnz (nullable) receive the
 * sizes the run needed.  Errors: SNN_EOVERFLOW (a capacity was too small),
 * SNN_EINVAL (NaN/Inf queries), SNN_ENOTSUP (a query norm beyond 1e18, or a
 * row longer than 4096 neighbours: use snn_query_radius_batch). */
snn_status snn_batch_plan_result(snn_batch_plan *plan, void *stream, snn_csr *out,
                                 int64_t *need_survivors, int64_t *need_nnz);

/* Autotuner: runs the plan on its current queries, the median of three timed
 * runs per candidate: first every combination of tensor-core groups scoring
 * their sets on the tensor cores or leaving them to the FP32 scorer, then
 * every FP32 work granularity (band chunks per scoring item: 4, 8, 16, 32)
 * and grid (1 or 2 CTAs per SM); keeps the fastest and reports the FP32 part
 * (nullable outputs; snn_batch_plan_config reports the rest).  When the
 * environment variable SNN_TUNE_CACHE names a file (JSON Lines: one object
 * per plan key of row and query size buckets per group), a plan whose key is
 * stored takes that choice without timing (ms = 0), and a tuned choice is
 * stored.  Synchronises `stream`; drops a previously captured graph. */
snn_status snn_batch_plan_tune(snn_batch_plan *plan, void *stream, int32_t *chunks_per_item,
                               int32_t *ctas_per_sm, float *ms);

/* The plan's current scoring configuration (nullable outputs): FP32 work
 * granularity and grid, the number of tensor-core groups and the mask of
 * those that score on the tensor cores (bit k: group k), and whether the last
 * snn_batch_plan_tune took its choice from the tuning cache. */
snn_status snn_batch_plan_config(const snn_batch_plan *plan, int32_t *chunks_per_item,
                                 int32_t *ctas_per_sm, int32_t *tc_groups, uint32_t *tc_mask,
                                 int32_t *from_cache);

/* Releases the plan (stream-ordered on `stream`; NULL is a no-op). */
void snn_batch_plan_free(snn_batch_plan *plan, void *stream);

/* Read-only view of an index's device arrays (for inspection and tests).
 * All pointers are device memory owned by the index and valid until
 * snn_index_free.  alpha is sorted ascending; order[r] is the original id of
 * sorted position r. */
typedef struct {
    int64_t n;
    int32_t d;
    int32_t dp;              /* padded row stride of the sorted copies      */
    const double *mu;        /* d, FP64 column means                        */
    const double *v1;        /* d, FP64 unit first principal direction      */
    const float *alpha;      /* n, sorted FP32 scores                       */
    const int32_t *order;    /* n, original id of each sorted position      */
    const float *points;     /* n x dp, raw points in sorted order          */
    double alpha_err;        /* bound on |computed alpha_i - exact alpha_i|,
                                alpha_i = (p_i - centre) . v1 exactly       */
    const float *centre;     /* d, the centre c = fl32(mu) every point and
                                query is shifted by before scoring (any fixed
                                centre leaves distances unchanged,
                                Section 3.1)                                 */
} snn_index_view;

snn_status snn_index_get_view(const snn_index *idx, snn_index_view *view);

/* Releases a device buffer returned in an snn_csr (NULL, and pointers the
 * library did not return, are no-ops).  Library buffers come from the
 * device's stream-ordered memory pool and are released in order on the
 * stream of the call that returned them: that stream must still exist, and
 * work on other streams that reads the buffer must be ordered before the
 * release (for example through an event). */
void snn_free(void *p);

/* Releases an index and all its device memory (NULL is a no-op), in order on
 * the stream the index was built on (same rules as snn_free). */
void snn_index_free(snn_index *idx);

/* Index checkpoint (the paper has no counterpart): the index record of
 * Algorithm 1 -- n, d, the centre mu, the direction v1, the sorted scores,
 * the permutation, the halved norms, the norm bounds and the sorted raw and
 * centred rows -- as one little-endian byte image in caller-owned host
 * memory.  The tensor-core operands derived from it are not stored; a loaded
 * index rebuilds them on first use, and every query on it returns exactly
 * what the saved index returned.
 * snn_index_saved_size: *bytes = the image size of idx.
 * snn_index_save: writes the image into buf (host, >= that size), with
 *   device-to-host copies on `stream`, which it synchronises.
 * snn_index_load: a new index (free with snn_index_free) on the current
 *   device from an image in buf (host, `bytes` long), with host-to-device
 *   copies on `stream`, which it synchronises.
 * Errors: SNN_EINVAL for NULL arguments, a buffer shorter than the image, or
 * an image whose magic, version or sizes do not match this format (checked on
 * the host before any device work); SNN_ENOMEM / SNN_ECUDA on device
 * failures. */
snn_status snn_index_saved_size(const snn_index *idx, int64_t *bytes);
snn_status snn_index_save(const snn_index *idx, void *buf, int64_t bytes, void *stream);
snn_status snn_index_load(const void *buf, int64_t bytes, void *stream, snn_index **out);

/* Message for the calling thread's last non-OK status ("" if none). */
const char *snn_last_error(void);

/* Library version string. */
const char *snn_version(void);

/* Largest n accepted by snn_sort_scores_noalloc. */
#define SNN_NOALLOC_SORT_MAX_N (1 << 20)

/* Allocation-free sort of scores (the paper has no counterpart: this entry
 * point exists for callers that cannot allocate device memory).  Some
 * callers cannot call cudaMalloc or use a memory pool: a process whose device
 * memory budget is fixed by someone else (every byte already handed out), or
 * a latency-critical loop that must never enter the allocator.  This call
 * sorts n FP32 values ascending with a stable LSD radix sort -- the same
 * kernels and the same result as the index build's sort of alpha (Algorithm
 * 1) -- using only a static device array compiled into the library (about
 * 9 MB, held by every GPU that loads the library until the process exits).
 *  alpha         device, n FP32 values (NaN/Inf rejected); may equal
 *                alpha_sorted (in place).
 *  n             0 <= n <= SNN_NOALLOC_SORT_MAX_N; larger n returns
 *                SNN_EINVAL with a message naming the limit.
 *  alpha_sorted  device, n FP32 outputs, ascending in the order of the
 *                values' order-preserving 32-bit keys (so -0.0 sorts before
 *                +0.0); caller-allocated.
 *  order         device, n int32 outputs: order[r] is the input position of
 *                alpha_sorted[r]; equal keys keep their input order.
 * The call allocates nothing.  It copies a NaN/Inf flag to the host and
 * synchronises `stream` once, before sorting.  The first call on a device
 * looks up the device address of the static array.  All calls share the one
 * array and it keeps the last call's contents, so calls whose device work
 * overlaps (different streams, or different host threads on one device)
 * race: serialise them. */
snn_status snn_sort_scores_noalloc(const float *alpha, int64_t n, float *alpha_sorted,
                                   int32_t *order, void *stream);

/* Test-only fault injection (the paper has no counterpart): arms a one-shot
 * fault for the next call that reaches it, to exercise failure detection
 * without faulting the GPU (one fault is armed at a time).
 *  SNN_FAULT_STALL_TC_PRODUCER  the next tensor-core scoring launch issues no
 *      TMA loads; its consumers' bounded waits (about 2 s of SM clock) expire,
 *      the kernel frees its TMEM and exits, and the query returns
 *      SNN_ETIMEOUT with the CUDA context still usable.
 *  SNN_FAULT_SMALL_SURVIVOR_BUFFER  the next query sizes its survivor buffer
 *      at one entry: the scoring overflows it (counting, never writing past
 *      the end) and the query re-runs with the exact size; the result is
 *      unchanged.
 *  SNN_FAULT_DEVICE_ALLOC  the next library device allocation fails: the
 *      call returns SNN_ENOMEM and releases what it had allocated.
 * 0 disarms.  Returns SNN_EINVAL for an unknown fault. */
#define SNN_FAULT_STALL_TC_PRODUCER 1
#define SNN_FAULT_SMALL_SURVIVOR_BUFFER 2
#define SNN_FAULT_DEVICE_ALLOC 3
snn_status snn_test_inject(int32_t fault);

/* Number of CUDA kernels this library has launched in this process so far
 * (diagnostics: the difference around a call is that call's launch count). */
uint64_t snn_launch_count(void);

#ifdef __cplusplus
}
#endif

#endif /* SNN_H */
