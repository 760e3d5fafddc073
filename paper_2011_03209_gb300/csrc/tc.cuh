// tc.cuh -- internal interface of the tcgen05 (tensor-core) screening passes.
#pragma once

#include "dbscan.cuh"

namespace mgb {

// Operands of the tensor-core screen: rows centred on their segment's
// centroid, split into BF16 hi and lo parts (R x dp each, row-major), with
// |a|^2 (FP32, to nearest) and |a| (FP32, rounded up) per row.
struct TcArgs {
    const void* Ah;
    const void* Al;
    const float* rn2;
    const float* rn;
    int64_t R;
    int ns;                          // BF16 products per pair: 3 (hi.hi + hi.lo + lo.hi) or 1
    int num_sms;                     // persistent grid size
    uint2* queue;                    // band pairs for the FP64 recheck
    unsigned long long* queue_n;     // entries pushed (may exceed queue_cap)
    unsigned long long queue_cap;
    int* err;                        // set to 1 if a bounded wait ran out
    cudaEvent_t ev_begin, ev_end;    // if set: recorded around the tensor-core kernel
    const int2* groups;              // pass 1, if set: pair groups sharing tile A (tc_groups)
    int64_t n_groups;                //   capacity of groups
    const unsigned long long* groups_dev;   // ... and their number on the device
    const unsigned long long* n_dev; // ungrouped, if set: the pair count on the device
                                     //   (n_pairs then bounds it)
};

// Groups the pair list (sorted by tile A, then tile B) into work items of
// one or two pairs sharing tile A: groups[k] = (pair index, pair index or -1).
// Allocates *groups (capacity n) and *pos ([n + 1] int64; pos[n] = the number
// of groups) on stream s, without a host round trip. Returns a mapper_status.
int tc_groups(const int2* pairs, int64_t n, Buf* groups, Buf* pos, cudaStream_t s);

// Pass `mode` (1 = counts and neighbour lists, 2 = unions) over the tile
// pairs a.pairs[0 .. n_pairs) on tensor cores. Returns a mapper_status.
int tc_pass(int mode, const PassArgs& a, const TcArgs& t, int64_t n_pairs, cudaStream_t s);

// Nearest of K <= 256 pivots (rows of Pv, pitch dp) for every point of X, on
// tensor cores (rows centred and rounded to BF16, one MMA of N = 256 per 16
// columns); near ties may resolve either way, which only orders the layout.
// Returns a mapper_status.
int assign_pivots_tc(const float* X, int64_t n, int d, int64_t ld, int dp, const float* Pv, int K,
                     int num_sms, int32_t* piv, float* pd2, cudaStream_t s);

// Runs the passes' bounded mbarrier wait on a barrier that is never
// completed: MAPPER_ETIMEOUT once it gives up (after 4 s), as designed.
int tc_wait_selftest(cudaStream_t s);

// Constants of the screen's error bound E = A1 |a||b| + A2 (|a|^2 + |b|^2) + A3.
void tc_bound(int ns, int dp, double eps2, double* A1, double* A2, double* A3);

}  // namespace mgb
