// Kernels of the streaming index updates (insert and delete).  New points are
// scored with the index's own centre and direction and merged into the sorted
// order; deleted points are compacted out.  Algorithm 2 stays exact for any
// unit direction and any centre, so a direction that is no longer the first
// principal component of the current points only weakens the pruning.
#include "update_kernels.cuh"

namespace snn {

namespace {
// Number of entries of the sorted score array a (n entries, ascending by
// float_to_key) whose key is below `key` (strict) or at most `key`.
__device__ __forceinline__ int64_t count_below(const float *__restrict__ a, int64_t n, uint32_t key,
                                               bool inclusive) {
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        const uint32_t k = float_to_key(a[mid]);
        if (inclusive ? k <= key : k < key) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}
}  // namespace

__global__ void k_merge_ranks(const float *__restrict__ aold, int64_t n, const float *__restrict__ anew,
                              int64_t k, int64_t *__restrict__ pos_old, int64_t *__restrict__ pos_new) {
    const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (t < n) {
        pos_old[t] = t + count_below(anew, k, float_to_key(aold[t]), false);
    } else if (t < n + k) {
        const int64_t j = t - n;
        pos_new[j] = j + count_below(aold, n, float_to_key(anew[j]), true);
    }
}

__global__ void k_place(const float *__restrict__ alpha, const int32_t *__restrict__ order, int32_t id_off,
                        const float *__restrict__ hx, const float *__restrict__ nrm,
                        const float *__restrict__ praw, const float *__restrict__ xc, int64_t rows, int dp,
                        const int64_t *__restrict__ pos, float *__restrict__ alpha_o,
                        int32_t *__restrict__ order_o, float *__restrict__ hx_o, float *__restrict__ nrm_o,
                        float *__restrict__ praw_o, float *__restrict__ xc_o) {
    const int q4 = dp / 4;
    const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (t >= rows * q4) return;
    const int64_t i = t / q4;
    const int q = int(t - i * q4);
    const int64_t p = pos[i];
    reinterpret_cast<float4 *>(praw_o + p * dp)[q] = reinterpret_cast<const float4 *>(praw + i * dp)[q];
    reinterpret_cast<float4 *>(xc_o + p * dp)[q] = reinterpret_cast<const float4 *>(xc + i * dp)[q];
    if (q == 0) {
        alpha_o[p] = alpha[i];
        order_o[p] = order[i] + id_off;
        hx_o[p] = hx[i];
        nrm_o[p] = nrm[i];
    }
}

__global__ void k_update_consts(float *__restrict__ dconst, const float *__restrict__ add) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        dconst[0] = fmaxf(dconst[0], add[0]);
        dconst[1] = fmaxf(dconst[1], add[1]);
    }
}

__global__ void k_mark_deleted(const int32_t *__restrict__ ids, int64_t cnt, int64_t n,
                               uint8_t *__restrict__ del, int *__restrict__ bad) {
    const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (t >= cnt) return;
    const int32_t id = ids[t];
    if (id < 0 || int64_t(id) >= n) {
        atomicOr(bad, 1);
        return;
    }
    del[id] = 1;
}

__global__ void k_keep_flags(const uint8_t *__restrict__ del, const int32_t *__restrict__ order, int64_t n,
                             int64_t *__restrict__ keep_id, int64_t *__restrict__ keep_pos) {
    const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (t >= n) return;
    keep_id[t] = del[t] ? 0 : 1;
    keep_pos[t] = del[order[t]] ? 0 : 1;
}

__global__ void k_compact(const uint8_t *__restrict__ del, const float *__restrict__ alpha,
                          const int32_t *__restrict__ order, const float *__restrict__ hx,
                          const float *__restrict__ nrm, const float *__restrict__ praw,
                          const float *__restrict__ xc, int64_t n, int dp, const int64_t *__restrict__ newpos,
                          const int64_t *__restrict__ newid, float *__restrict__ alpha_o,
                          int32_t *__restrict__ order_o, float *__restrict__ hx_o, float *__restrict__ nrm_o,
                          float *__restrict__ praw_o, float *__restrict__ xc_o) {
    const int q4 = dp / 4;
    const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (t >= n * q4) return;
    const int64_t i = t / q4;
    const int q = int(t - i * q4);
    const int32_t id = order[i];
    if (del[id]) return;
    const int64_t p = newpos[i];
    reinterpret_cast<float4 *>(praw_o + p * dp)[q] = reinterpret_cast<const float4 *>(praw + i * dp)[q];
    reinterpret_cast<float4 *>(xc_o + p * dp)[q] = reinterpret_cast<const float4 *>(xc + i * dp)[q];
    if (q == 0) {
        alpha_o[p] = alpha[i];
        order_o[p] = int32_t(newid[id]);
        hx_o[p] = hx[i];
        nrm_o[p] = nrm[i];
    }
}

}  // namespace snn
