// dbscan.cuh -- internal interface of the per-element DBSCAN passes and of
// graph assembly (k_dbscan.cu, k_tc.cu).
#pragma once

#include "common.cuh"

namespace mgb {

enum : int { kStatBand = 0, kStatTies = 1, kStatScreened = 2, kStatCore = 3, kStatTileOut = 4,
             kStatTileIn = 5, kStatCount = 8 };

// Arguments of one screening pass over all tile pairs of all elements.
struct PassArgs {
    const float* G;              // gathered rows, one per membership slot, pitch dp floats
    int dp;                      // row pitch (multiple of 32, zero padded)
    int d;                       // true dimension
    const int64_t* elem_off;     // [E+1] slot offsets of the elements
    const int64_t* pair_off;     // [E+1] tile-pair offsets of the elements
    int E;
    float lo_thr, hi_thr;        // FP32 screen: in if s <= lo_thr, out if s > hi_thr
    double eps2;                 // eps * eps in double
    double tie_thr;              // 1e-12 * eps2
    int32_t* count;              // pass 1 output
    const uint8_t* core;         // passes 2, 3
    int32_t* parent;             // pass 2 union-find
    const int32_t* root;         // pass 3 (flattened)
    int32_t* border;             // pass 3 output (root slot or INT_MAX)
    unsigned long long* stats;   // kStat* counters
};

// FP32 screen thresholds for eps2 at dimension d: a pair is certainly a
// neighbour when the FP32 screen value is <= *lo, certainly not when > *hi.
void fp32_thresholds(double eps2, int d, float* lo, float* hi);

cudaError_t gather_rows(const float* X, int64_t ld, int d, int dp, const int32_t* slot_point,
                        int64_t M, float* G, int* nonfinite, cudaStream_t s);
cudaError_t element_offsets(const uint64_t* keys, int64_t M, int64_t E, int64_t* elem_off,
                            cudaStream_t s);
cudaError_t tile_pair_offsets(const int64_t* elem_off, int64_t E, int64_t* pair_off, cudaStream_t s);
cudaError_t simt_pass(int mode, const PassArgs& a, int64_t n_pairs, cudaStream_t s);
cudaError_t core_flags(const int32_t* count, int64_t M, int32_t min_pts, uint8_t* core,
                       int32_t* parent, int32_t* border, unsigned long long* stats, cudaStream_t s);
cudaError_t flatten(const int32_t* parent, const uint8_t* core, int64_t M, int32_t* root,
                    cudaStream_t s);
cudaError_t labels(const uint8_t* core, const int32_t* root, const int32_t* border,
                   const int32_t* slot_point, int64_t M, int32_t* lab, int32_t* is_root,
                   int32_t* is_member, int64_t* slot_label, cudaStream_t s);
cudaError_t member_keys(const int32_t* lab, const int64_t* nid, const int64_t* mpos,
                        const int32_t* slot_point, const int32_t* slot_elem, int64_t M,
                        uint64_t* keys, int32_t* node_elem, cudaStream_t s);
cudaError_t node_offsets(const uint64_t* keys, int64_t G, int64_t* node_off, int32_t* members,
                         uint64_t* keys2, cudaStream_t s);
cudaError_t run_pairs(const uint64_t* keys2, int64_t G, int64_t* cnt, cudaStream_t s);
cudaError_t emit_pairs(const uint64_t* keys2, int64_t G, const int64_t* pos, uint64_t* out,
                       cudaStream_t s);
cudaError_t unique_flags(const uint64_t* k, int64_t P, int32_t* flag, cudaStream_t s);
cudaError_t unique_emit(const uint64_t* k, const int32_t* flag, const int64_t* pos, int64_t P,
                        int32_t* edges, cudaStream_t s);

}  // namespace mgb
