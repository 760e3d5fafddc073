// tc.cuh -- internal interface of the tcgen05 (tensor-core) screen passes.
#pragma once

#include "dbscan.cuh"

namespace mgb {

// Runs passes 1-3 (count, core flags, unions, flatten, border) with the BF16
// tensor-core screen. Returns a mapper_status.
int tc_cluster_passes(const PassArgs& a, int64_t n_pairs, int32_t min_pts, cudaStream_t s);

}  // namespace mgb
