// DBSCAN on the SNN self-join (Section 6.4: the neighbour search inside
// DBSCAN is replaced by SNN).  From the eps-neighbourhoods (self included) of
// the points in sorted position p (row p: the point of id order[p]; rows
// unsorted, columns point ids): core flags by id, union-find over core-core
// neighbour pairs (on point ids, hooking the larger root under the smaller
// with atomicCAS, path halving: the ids are in the caller's order, where a
// cluster is not one contiguous run as it is in sorted positions), border
// points joined to the cluster of their smallest-id core neighbour, and
// cluster labels canonicalised to the smallest member id.
#include "dbscan_kernels.cuh"

namespace snn {

// Core flags by point id (into the caller's is_core), parent[] over ids.
__global__ void k_db_core(const int64_t *__restrict__ offsets, const int32_t *__restrict__ order, int64_t n,
                          int32_t min_pts, uint8_t *__restrict__ core, int32_t *__restrict__ parent) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n) return;
    core[order[i]] = (offsets[i + 1] - offsets[i]) >= min_pts ? 1 : 0;
    parent[i] = (int32_t)i;
}

__device__ __forceinline__ int32_t uf_find(int32_t *parent, int32_t x) {
    // path halving; every write moves a pointer to an ancestor, so concurrent
    // finds and hooks stay consistent
    int32_t p = parent[x];
    while (p != x) {
        const int32_t g = parent[p];
        if (g != p) parent[x] = g;
        x = p;
        p = parent[x];
    }
    return x;
}

// One warp per core point (row i, id order[i]): unions its id with each core
// neighbour of smaller id (each pair once).
__global__ void k_db_union(const int64_t *__restrict__ offsets, const int32_t *__restrict__ idx,
                           int64_t n, const uint8_t *__restrict__ core, const int32_t *__restrict__ order,
                           int32_t *__restrict__ parent) {
    const int64_t i = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (i >= n) return;
    const int32_t id = order[i];
    if (!core[id]) return;
    const int64_t o0 = offsets[i], o1 = offsets[i + 1];
    for (int64_t o = o0 + lane; o < o1; o += 32) {
        const int32_t jd = idx[o];
        if (jd >= id || !core[jd]) continue;
        int32_t a = id, b = jd;
        for (;;) {
            a = uf_find(parent, a);
            b = uf_find(parent, b);
            if (a == b) break;
            const int32_t hi = max(a, b), lo = min(a, b);
            if (atomicCAS(&parent[hi], hi, lo) == hi) break;
            a = hi;
            b = lo;
        }
    }
}

// The root of row i's cluster: its own for cores, that of the core neighbour
// of smallest id for border points (a minimum over the whole unsorted row);
// -1 for noise.  The cluster's label candidate is the smallest member id.
__global__ void k_db_assign(const int64_t *__restrict__ offsets, const int32_t *__restrict__ idx,
                            int64_t n, const uint8_t *__restrict__ core, const int32_t *__restrict__ order,
                            int32_t *__restrict__ parent, int32_t *__restrict__ owner,
                            int32_t *__restrict__ minid) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int32_t id = order[i];
    int32_t r = -1;
    if (core[id]) {
        r = uf_find(parent, id);
    } else {
        int32_t best = INT32_MAX;
        for (int64_t o = offsets[i]; o < offsets[i + 1]; ++o) {
            const int32_t jd = idx[o];
            if (core[jd]) best = min(best, jd);
        }
        if (best != INT32_MAX) r = uf_find(parent, best);
    }
    owner[i] = r;
    if (r >= 0) atomicMin(&minid[r], id);
}

__global__ void k_db_init_minid(int32_t *__restrict__ minid, int64_t n) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i < n) minid[i] = INT32_MAX;
}

// labels[order[i]] (the core flags are already by id).
__global__ void k_db_label(const int32_t *__restrict__ owner, const int32_t *__restrict__ minid,
                           const int32_t *__restrict__ order, int64_t n, int32_t *__restrict__ labels) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int32_t r = owner[i];
    labels[order[i]] = r >= 0 ? minid[r] : -1;
}

}  // namespace snn
