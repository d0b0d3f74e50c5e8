// Kernels of the streaming index updates (see update_kernels.cu).
#pragma once
#include "common.cuh"

namespace snn {

// Positions in the merged sorted order: pos_old[i] for the n existing
// entries, pos_new[j] for the k new ones (existing entries precede new
// entries of equal score).  One thread per entry of either array.
__global__ void k_merge_ranks(const float *aold, int64_t n, const float *anew, int64_t k,
                              int64_t *pos_old, int64_t *pos_new);

// Entry i of the sorted arrays (score, id + id_off, halved norm, norm bound,
// raw row, centred row; rows of dp floats) to position pos[i] of the output
// arrays; one thread per 4-float quad of a row.
__global__ void k_place(const float *alpha, const int32_t *order, int32_t id_off, const float *hx,
                        const float *nrm, const float *praw, const float *xc, int64_t rows, int dp,
                        const int64_t *pos, float *alpha_o, int32_t *order_o, float *hx_o, float *nrm_o,
                        float *praw_o, float *xc_o);

// dconst[0..1] = max(dconst[0..1], add[0..1]) (score error bound, norm bound).
__global__ void k_update_consts(float *dconst, const float *add);

// del[id] = 1 for every listed id; an id outside [0, n) sets *bad.
__global__ void k_mark_deleted(const int32_t *ids, int64_t cnt, int64_t n, uint8_t *del, int *bad);

// keep_id[id] = 1 unless id is deleted; keep_pos[p] = 1 unless the point at
// sorted position p is deleted.
__global__ void k_keep_flags(const uint8_t *del, const int32_t *order, int64_t n, int64_t *keep_id,
                             int64_t *keep_pos);

// Kept entry at sorted position i to position newpos[i], its id renumbered to
// newid[id] (the kept ids in ascending order become 0, 1, ...).
__global__ void k_compact(const uint8_t *del, const float *alpha, const int32_t *order, const float *hx,
                          const float *nrm, const float *praw, const float *xc, int64_t n, int dp,
                          const int64_t *newpos, const int64_t *newid, float *alpha_o, int32_t *order_o,
                          float *hx_o, float *nrm_o, float *praw_o, float *xc_o);

}  // namespace snn
