// DBSCAN kernels on the SNN self-join (Section 6.4).
#pragma once
#include "common.cuh"

namespace snn {

__global__ void k_db_core(const int64_t *offsets, const int32_t *order, int64_t n, int32_t min_pts,
                          uint8_t *core, int32_t *parent);
__global__ void k_db_union(const int64_t *offsets, const int32_t *idx, int64_t n,
                           const uint8_t *core, const int32_t *order, int32_t *parent);
__global__ void k_db_assign(const int64_t *offsets, const int32_t *idx, int64_t n,
                            const uint8_t *core, const int32_t *order, int32_t *parent,
                            int32_t *owner, int32_t *minid);
__global__ void k_db_init_minid(int32_t *minid, int64_t n);
__global__ void k_db_label(const int32_t *owner, const int32_t *minid, const int32_t *order, int64_t n,
                           int32_t *labels);

}  // namespace snn
