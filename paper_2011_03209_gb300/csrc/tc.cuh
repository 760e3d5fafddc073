// tc.cuh -- internal interface of the tcgen05 (tensor-core) screening passes.
#pragma once

#include "dbscan.cuh"

namespace mgb {

// Count pass over several radii of one cover (mode 5 of tc_pass): one
// contraction whose epilogue decides every pair against each radius in turn,
// writing each radius's counts, lists, hit flags and band queue (the FP64
// recheck then runs per radius). Radii ascending, at most kMaxRadii.
constexpr int kMaxRadii = 4;
struct RadiusOut {
    int32_t* count;                  // [R] neighbour counts, zeroed by the caller
    int32_t* nbr;                    // [R * cap] first cap neighbours (cap of the PassArgs), or nullptr
    uint8_t* pair_hit;               // per tile pair of the list: holds a neighbour pair (nullable)
    uint2* queue;                    // band pairs of this radius (capacity TcArgs::queue_cap)
    unsigned long long* queue_n;     // entries pushed (may exceed the capacity)
    unsigned long long* stats;       // this radius's kStat* counters (band, ties, FP64, index checks)
    double eps2;
};

// Operands of the tensor-core screen: rows centred on their segment's
// centroid, split into BF16 hi and lo parts (R x dp each, row-major), with
// |a|^2 (FP32, to nearest) and |a| (FP32, rounded up) per row.
struct TcArgs {
    const void* Ah;
    const void* Al;
    const float* rn2;
    const float* rn;
    const float* rl;                 // |a - hi| per row (rounded up): the tighter bound; or nullptr
    const float4* tmax;              // per tile: largest |a|^2, |a|, |a - hi| (count pass)
    const float* tn2min;             // per tile: smallest |a|^2 of the valid rows (count pass)
    int64_t R;
    int ns;                          // products per pair: 3 (hi.hi + hi.lo + lo.hi) or 1
    bool f8;                         // count pass on FP8 E4M3 operands (Ah, Al: R x dp bytes, per-tile
                                     //   scale in tmax[t].w; rl: |a - s hi|), ns = 3
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
    // pass 1 with ns = 1 only: the first phase of the two-phase count pass.
    // Each 32 x 32 sub-block (TMEM lane quadrant, column part) of a tile pair
    // with no pair in the one-product band is counted; the others set their
    // bit (quadrant * 4 + part) in redo_mask[q] (one word per pair of the
    // list, zeroed by the caller), and their pair is flagged in pair_hit.
    // tc_redo_list then lists the pairs with deferred sub-blocks, and the
    // second phase (ns = 3) runs over that list with sub_mask = redo_mask and
    // sub_q = its first-phase indices, counting only those sub-blocks.
    bool defer;
    bool defer_mixed;                // first phase: defer every block with a row neither all in nor
                                     // all out (decided from the rows' extremes alone)
    uint32_t* redo_mask;
    const uint32_t* sub_mask;
    const int32_t* sub_q;
    // mode 5: the radii (ascending) and their outputs; the PassArgs' count,
    // nbr, pair_hit, eps2 and this struct's queue are not used then
    int n_radii;
    RadiusOut radii[kMaxRadii];
};

// The pairs q of pairs[0 .. n) with mask[q] != 0, in list order: redo[k] =
// pairs[q_k], redo_q[k] = q_k (capacity n each); *pos receives [n + 1] int64
// with their number at pos[n]. stats (nullable, two counters): += the
// deferred blocks and the 32-column parts holding one. Returns a mapper_status.
int tc_redo_list(const int2* pairs, const uint32_t* mask, int64_t n, int2* redo, int32_t* redo_q, Buf* pos,
                 cudaStream_t s, unsigned long long* stats = nullptr);
// out[j] = pairs[j * stride] for j < n. Returns a mapper_status.
int tc_sample_pairs(const int2* pairs, int64_t stride, int64_t n, int2* out, cudaStream_t s);

// tc_groups over the first *n_dev entries of a list of capacity n (number of
// groups at (*pos)[n]). Returns a mapper_status.
int tc_groups_dev(const int2* pairs, int64_t n, const unsigned long long* n_dev, Buf* groups, Buf* pos,
                  cudaStream_t s);

// Groups the pair list (sorted by tile A, then tile B) into work items of
// one or two pairs sharing tile A: groups[k] = (pair index, pair index or -1).
// Allocates *groups (capacity n) and *pos ([n + 1] int64; pos[n] = the number
// of groups) on stream s, without a host round trip. Returns a mapper_status.
int tc_groups(const int2* pairs, int64_t n, Buf* groups, Buf* pos, cudaStream_t s);

// Pass `mode` (1 = counts and neighbour lists, 2 = unions, 5 = counts and
// lists for each of t.radii, BF16 operands) over the tile pairs a.pairs[0 ..
// n_pairs) on tensor cores. Returns a mapper_status.
int tc_pass(int mode, const PassArgs& a, const TcArgs& t, int64_t n_pairs, cudaStream_t s);

// Nearest of K <= 256 pivots (rows of Pv, pitch dp) for every point of X, on
// tensor cores (rows centred and rounded to BF16, one MMA of N = 256 per 16
// columns); near ties may resolve either way, which only orders the layout.
// pre (nullable): the points already centred on c and split (xh: BF16 rows
// of pitch dp, n_tiles * 128 of them, the rows past n zero; xn2: |x - c|^2),
// c (dp floats) being the pivots' centre of this call. Returns a mapper_status.
struct PivotSplit {
    const float* c;
    const void* xh;
    const float* xn2;
};
int assign_pivots_tc(const float* X, int64_t n, int d, int64_t ld, int dp, const float* Pv, int K,
                     int num_sms, int32_t* piv, float* pd2, cudaStream_t s, const PivotSplit* pre = nullptr);

// Entries per list of the k-distance tensor-core screen (k <= this).
constexpr int kKnnList = 8;

// k-distance screen on tensor cores. Operand rows (BF16 hi + lo of the rows
// centred on one centre, |row|^2 in rn2) hold the points in order (row =
// point index, tile_n marking the valid rows of each 128-row tile), then the
// q queries from tile q_tile0 on. CTA (query tile u, chunk c) screens query
// tile u against screened point tiles c chunk_tiles .. (c + 1) chunk_tiles - 1
// of n_tiles (screened tile b = operand tile b tile_stride), three products
// per tile pair. For query row a and point b the screen's key
//   key = RD(RD(|a|^2 m - A3f) + RD(c2 acc + RD(|b|^2 m)))
// is a lower bound of d^2 (FAR: of -d^2) when the host sets m = RD(1 - K),
// c2 = -2 (FAR: m = -RU(1 + K), c2 = 2), with K (|a|^2 + |b|^2) + A3f a bound of
// the error of |a|^2 + |b|^2 - 2 acc.
//   List mode (tau null): per query row and 32-column part of the chunk, the
//   kKnnList smallest keys with their points, cand_v / cand_i[((query *
//   chunks + c) * 4 + part) * kKnnList + i], ascending, padded with +inf / -1.
//   Append mode: every key <= tau[query] with its point at cand_v / cand_i[query
//   * cap + slot], slot < count[query] (count, zeroed by the caller, counts
//   every such key, also those beyond cap); with off set, at off[query] + slot,
//   slot < off[query + 1] - off[query].
// *err = 1 if a bounded wait ran out. Returns a mapper_status.
struct KnnScreen {
    const void* Ah;
    const void* Al;
    const float* rn2;
    const int32_t* tile_n;
    int64_t rows;                 // operand rows (a multiple of 128)
    int64_t n_tiles, tile_stride, q_tile0, q;
    int dp, chunk_tiles, chunks;
    float m, c2, A3f;
    const float* tau;
    int cap;
    const int64_t* off;
    int* count;
    float* cand_v;
    int32_t* cand_i;
    int* err;
};
int tc_knn_screen(const KnnScreen& k, cudaStream_t s);

// Accumulation probe: random BF16 rows (values 2^-4 .. 2^5 in magnitude,
// random signs) through the screen's tcgen05 path (ns products, row pitch
// dp, M = N = 128, four tile pairs); *observed = the largest |acc - exact|
// over the accumulators, relative to the sum of the magnitudes of the
// products, and *modelled = the accumulation term of the screen's error bound
// relative to the same sum. Returns a mapper_status.
// fmt: 0 = BF16 rows (kind::f16), 1 = FP8 E4M3 rows (kind::f8f6f4, the
// FP8 screen's model).
int tc_mma_probe(int ns, int fmt, int dp, uint64_t seed, int num_sms, double* observed, double* modelled,
                 cudaStream_t s);

// Runs the passes' bounded mbarrier wait on a barrier that is never
// completed: MAPPER_ETIMEOUT once it gives up (after 4 s), as designed.
int tc_wait_selftest(cudaStream_t s);

// Constants of the screen's error bound E = A1 |a||b| + A2 (|a|^2 + |b|^2) + A3.
void tc_bound(int ns, int dp, double eps2, double* A1, double* A2, double* A3);

}  // namespace mgb
