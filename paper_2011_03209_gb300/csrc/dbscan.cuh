// dbscan.cuh -- internal interface of the per-element DBSCAN stage: tile
// layout (k_tiles.cu), screening passes (k_dbscan.cu, k_tc.cu) and graph
// assembly (k_nerve.cu).
#pragma once

#include "common.cuh"

namespace mgb {

constexpr int kTile = 128;          // rows per tile (one tcgen05 M block)

// A union-pass list entry may carry a flag in bit 30 of its second tile:
// the A-tile cores already share one root and the B-tile cores another, so
// one neighbour pair between them is enough (no per-pair unions).
constexpr int kPairOneEach = 1 << 30;
constexpr int kPairTileMask = kPairOneEach - 1;

enum : int { kStatBand = 0, kStatTies = 1, kStatScreened = 2, kStatCore = 3, kStatTileOut = 4,
             kStatTileIn = 5, kStatSkipped = 6, kStatTcPairs = 7, kStatSimtPairs = 8, kStatFp64 = 9,
             kStatUnion = 10, kStatRedo = 11, kStatOob = 12, kStatRedoBlocks = 13, kStatRedoParts = 14,
             kStatCount = 15 };

// Work lists of tile pairs, classified by bounding spheres.
enum : int { kListAllIn = 0, kListTC = 1, kListSimt = 2, kListCount = 3 };

// Arguments of one screening pass. Rows are points of one element laid out
// in tiles of kTile rows; a tile pair (a, b), a <= b, belongs to one element.
//   explicit mode (pairs != nullptr): tile pair q is pairs[q] (tile indices),
//     tile t spans rows [t*kTile, t*kTile + tile_n[t]);
//   implicit mode: every tile pair of every element, elements given by
//     elem_off (rows) and pair_off (tile pairs), rows = cover slots.
struct PassArgs {
    const float* G;              // FP32 rows, pitch dp floats (zero padded), or nullptr:
    const float* X;              //   then row r is X + row_pt[r] * ld (d columns)
    int64_t ld;
    bool xvec;                   //   X rows 16-byte aligned (float4 loads)
    int dp;                      // row pitch (multiple of 32)
    int d;                       // true dimension
    const int2* pairs;           // explicit list, or nullptr
    const unsigned long long* n_dev;   // explicit list: its length on the device, if set
                                       //   (launches cover an upper bound; the rest exit)
    const int32_t* tile_n;       // valid rows per tile (explicit mode)
    const int64_t* elem_off;     // implicit mode: [E+1] row offsets of the elements
    const int64_t* pair_off;     // implicit mode: [E+1] tile-pair offsets
    int E;
    float lo_thr, hi_thr;        // FP32 screen: in if s <= lo_thr, out if s > hi_thr
    double eps2;                 // eps * eps in double
    double tie_thr;              // 1e-12 * eps2
    const int32_t* row_pt;       // point index of each row (nullptr: the row index)
    int32_t* count;              // pass 1 output, per row
    int32_t* nbr;                // pass 1: first `cap` neighbour rows of each row
    int cap;                     //   (0: no lists)
    uint8_t* pair_hit;           // pass 1 (explicit mode, optional): set to 1 for each tile
                                 //   pair with a neighbour pair, or one left to the recheck
    const uint8_t* core;         // passes 2, 3
    int32_t* parent;             // pass 2 union-find over rows
    const int32_t* root;         // pass 3 (flattened)
    unsigned long long* border;  // pass 3 output: (canonical point << 32 | root row), min
    unsigned long long* stats;   // kStat* counters
    int64_t n_rows, n_tiles;     // rows and tiles of the layout (index checks of the checked build)
};

// Row `row` of a pass (the tile layout's FP32 rows, or the input rows).
__device__ __forceinline__ const float* pass_row(const PassArgs& A, int64_t row)
{
    return A.G ? A.G + row * A.dp : A.X + (int64_t)A.row_pt[row] * A.ld;
}

// Columns 4 k4 .. 4 k4 + 3 of a row from pass_row (zero from column d on).
__device__ __forceinline__ float4 pass_ld4(const PassArgs& A, const float* p, int k4)
{
    if (A.G) return reinterpret_cast<const float4*>(p)[k4];
    const int k = 4 * k4;
    if (A.xvec && k + 3 < A.d) return *reinterpret_cast<const float4*>(p + k);
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (k < A.d) v.x = p[k];
    if (k + 1 < A.d) v.y = p[k + 1];
    if (k + 2 < A.d) v.z = p[k + 2];
    if (k + 3 < A.d) v.w = p[k + 3];
    return v;
}

// FP32 screen thresholds for eps2 at dimension d: a pair is certainly a
// neighbour when the FP32 screen value is <= *lo, certainly not when > *hi.
void fp32_thresholds(double eps2, int d, float* lo, float* hi);

// --- screening passes (k_dbscan.cu)
cudaError_t simt_pass(int mode, const PassArgs& a, int64_t n_pairs, cudaStream_t s);
cudaError_t allin_pass(int mode, const PassArgs& a, int64_t n_pairs, cudaStream_t s);
cudaError_t core_flags(const int32_t* count, int64_t R, int32_t min_pts, uint8_t* core,
                       int32_t* parent, unsigned long long* border, unsigned long long* stats,
                       cudaStream_t s);
cudaError_t flatten(const int32_t* parent, const uint8_t* core, int64_t R, int32_t* root,
                    cudaStream_t s);
cudaError_t border_from_lists(const int32_t* count, const int32_t* nbr, int cap,
                              const uint8_t* core, const int32_t* root, const int32_t* row_pt,
                              int64_t R, unsigned long long* border, cudaStream_t s,
                              unsigned long long* oob = nullptr);
// Row space -> cover-slot space: per slot the root slot of its node (or -1),
// canonical point id (or -1), root flag, member flag and core flag.
// Unions of each core row with the core rows of its pass-1 neighbour list.
cudaError_t list_unions(const int32_t* count, const int32_t* nbr, int cap, const uint8_t* core, int32_t* parent,
                        const int32_t* row_pt, int64_t R, cudaStream_t s, unsigned long long* oob = nullptr);
cudaError_t rows_to_slots(const int32_t* row_slot, const int32_t* row_pt, const uint8_t* core,
                          const int32_t* root, const unsigned long long* border, int64_t R,
                          int32_t* lab, int32_t* is_root, int32_t* is_member,
                          int64_t* slot_label, uint8_t* slot_core, cudaStream_t s);
cudaError_t element_offsets(const uint64_t* keys, int64_t M, int64_t E, int64_t* elem_off,
                            cudaStream_t s);
// f[row_pt[row] * m + j] = count[row] for every non-padding row (the rows of
// a one-element cover of the whole cloud: the density filter).
cudaError_t counts_to_lens(const int32_t* row_slot, const int32_t* row_pt, const int32_t* count, int64_t R,
                           double* f, int m, int j, cudaStream_t s);
// Appends to `out` the tile pairs of `pairs` whose hit flag is set; *count
// receives the size.
cudaError_t select_hit(const int2* pairs, const uint8_t* hit, int64_t n, int2* out,
                       unsigned long long* count, cudaStream_t s);
// *dst += *src (one device counter into another).
cudaError_t add_counter(unsigned long long* dst, const unsigned long long* src, cudaStream_t s);
// Appends to `out` the tile pairs (a, b) of pairs[0 .. *n_dev) (at most n)
// with lo < b - a <= hi; *count receives the size.
cudaError_t select_delta(const int2* pairs, int64_t n, const unsigned long long* n_dev, int lo, int hi, int2* out,
                         unsigned long long* count, cudaStream_t s);
// Keeps the union-pass tile pairs of pairs[0 .. *n_dev) (at most n) whose
// core rows do not all share one root yet (flagging kPairOneEach pairs);
// *count receives the size. tile_roots: scratch of T entries (the current
// root range of each of the T tiles).
cudaError_t filter_joined(const PassArgs& a, int64_t T, int2* tile_roots, const int2* pairs, int64_t n,
                          const unsigned long long* n_dev, int2* out, unsigned long long* count, cudaStream_t s);

// --- single-linkage forest (k_mst.cu)
// Edges of the minimum spanning forests of the eps-graphs of all elements:
// points u < v, element, the two cover slots (su < sv) and the FP64 d2; n
// edges (capacity M), in no particular order.
struct ForestOut {
    Buf u, v, elem, su, sv, d2;
    int64_t n = 0;
};
// a: the rows of a tile layout (G or X via row_pt, dp, d, tile_n, row_pt,
// eps2, hi_thr of fp32_thresholds) and a.pairs[0 .. n_pairs) the element tile
// pairs not certified all-out at eps. Returns a mapper_status.
int msf_forest(const PassArgs& a, const int32_t* row_slot, const int32_t* slot_point, const int32_t* slot_elem,
               int64_t M, int64_t R, int64_t T, int64_t n_pairs, ForestOut* out, cudaStream_t s);
// Single-linkage clusters at height h (edges with d2 <= h^2) in cover-slot
// space, in the layout of rows_to_slots (every slot a member and core).
int msf_cut(const ForestOut& f, const int32_t* slot_point, int64_t M, double h, int32_t* lab, int32_t* is_root,
            int32_t* is_member, int64_t* slot_label, uint8_t* core, cudaStream_t s);

// --- nodes and nerve (k_nerve.cu)
// Nerve keys (point << 32 | node) of the members of nodes given by offsets.
cudaError_t node_member_keys(const int64_t* node_off, int64_t N, int64_t G, const int32_t* members,
                             uint64_t* keys2, cudaStream_t s);
// slot_elem[i] = the element e with elem_off[e] <= i < elem_off[e + 1].
cudaError_t fill_slot_elem(const int64_t* elem_off, int32_t k, int64_t M, int32_t* slot_elem, cudaStream_t s);
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

// --- tile layout (k_tiles.cu)
struct TileLayout {
    int64_t R = 0;               // rows (multiple of kTile)
    int64_t T = 0;               // tiles
    int64_t n_seg = 0;           // (element, group) segments
    int n_groups = 0;            // pivot groups (outliers form group n_groups)
    Buf row_slot;                // [R] int32 cover slot, -1 for padding
    Buf row_pt;                  // [R] int32 point, INT32_MAX for padding
    Buf G;                       // [R x dp] FP32 rows (unset on the tensor-core path for dp <= 256)
    Buf tile_n, tile_seg, tile_elem;      // [T] int32
    Buf tile_cent;               // [T x dp] FP32 centre
    Buf tile_rad;                // [T] FP64 upper bound of the rows' distance to it
    Buf seg_cent;                // [n_seg x dp] FP32 centre of each segment
    Buf seg_outlier;             // [n_seg] int32: 1 if the segment holds outliers
    Buf seg_elem;                // [n_seg] int32 element of each segment
    Buf seg_toff;                // [n_seg + 1] int64 first tile of each segment
    Buf seg_rad;                 // [n_seg] FP64 upper bound of its rows' distance to its centre
    Buf Ah, Al;                  // [R x dp] BF16 centred rows (hi and lo parts)
    Buf rn2, rn;                 // [R] FP32 |a|^2 and |a| (rounded up)
    Buf rl;                      // [R] FP32 |a - hi| (rounded up): the residual of the hi part
    Buf tmax;                    // [T] float4: largest |a|^2, |a|, |a - hi| of each tile's rows
    Buf tn2min;                  // [T] smallest |a|^2 of each tile's valid rows
    Buf Fh, Fl;                  // [R x dp] FP8 E4M3 parts of a / s (s: the tile's scale), if built
    Buf frl;                     // [R] |a - s hi| (FP8 hi part), rounded up
    Buf ftmax;                   // [T] float4: largest |a|^2, |a|, frl of each tile, and its scale s
};

struct PairLists {
    Buf list[kListCount];        // int2 tile pairs
    int64_t n[kListCount] = {0, 0, 0};
    int64_t n_candidates = 0, n_out = 0;
};

// The pivots of the tile layout and every point's nearest one: K pivots
// (points floor(k n / K)), Pv their FP32 rows (K x dp), piv[n] the nearest
// pivot and pd2[n] an FP32 squared distance to it. They depend on X only, so
// one set serves every layout of the cloud.
struct PivotSet {
    int K = 0;
    Buf Pv, piv, pd2;
    // set by pivot_prepare: the pivots' centre c and the points' split for
    // the tensor-core assignment (written by the lens pass, lens_l2_split)
    bool split = false;
    Buf c, xh, xn2;
};
// Allocates the set on stream `alloc_s` (where it is later freed) and
// computes it on stream `s` (which must wait for alloc_s).
cudaError_t pivot_alloc(int64_t n, int dp, PivotSet* P, cudaStream_t alloc_s);
int pivot_assign(const float* X, int64_t n, int32_t d, int64_t ld, int dp, bool bf16, int num_sms, PivotSet* P,
                 cudaStream_t s);
// Before the lens pass (P from pivot_alloc): the pivot rows (X's rows
// k n / K; X in host memory when `host`), their FP32 centre c, and room for the
// points' BF16 split (rows past n zeroed), which lens_l2_split then writes;
// pivot_assign afterwards skips its own split. A mapper_status.
int pivot_prepare(const float* X, int64_t n, int32_t d, int64_t ld, int dp, bool host, PivotSet* P, cudaStream_t s);

// Orders every element's points by pivot group, lays them out in tiles
// (a tile never mixes groups) and gathers rows. tau: distance under which two
// pivots join a group and beyond which a point is an outlier. bf16: also
// build the tensor-core operands (and assign pivots on tensor cores).
// pre: the pivot set, computed beforehand (stream-ordered before s), or null.
int build_tiles(const float* X, int64_t n, int32_t d, int64_t ld, int dp, const int32_t* slot_point,
                const int32_t* slot_elem, int64_t M, int64_t E, double tau, bool bf16, int num_sms,
                TileLayout* L, int* nonfinite, cudaStream_t s, const PivotSet* pre = nullptr);
// Classifies every tile pair of every element by bounding spheres: out (no
// pair within eps), all-in, or mixed (to the tensor-core list when both tiles
// are one non-outlier segment and use_tc, else to the CUDA-core list).
// X, ld, d: the rows (read for the outlier tiles' distance bounds when G is
// not gathered). eps_all_in (if > 0, <= eps): the radius a pair must be all in
// at to go to the all-in list (the smallest of several radii sharing the
// lists; out stays decided at eps, the largest).
int classify_pairs(const TileLayout& L, const float* X, int64_t ld, int d, int dp, int64_t E, double eps,
                   bool use_tc, PairLists* P, cudaStream_t s, double eps_all_in = 0.0);
// Count-pass phase choice per tile pair: bin[q] (< kPairBins) of the pair's
// statistic (|c_a - c_b|^2 + r_a^2 + r_b^2) / eps^2 from the layout's tile
// spheres, on a log2 scale of 8 bins per octave from 2^-4.
constexpr int kPairBins = 64;
cudaError_t pair_bins(const TileLayout& L, const int2* pairs, int64_t n, int dp, double eps, uint8_t* bin,
                      cudaStream_t s);
// Tally of a sample of the list (sample pair j = list pair j * stride, mask[j]
// its first phase's deferred blocks): cnt[2 b] sampled pairs of bin b,
// cnt[2 b + 1] of them that deferred a block (2 kPairBins counters, zeroed here).
cudaError_t sample_bins(const uint32_t* mask, int64_t n_s, const uint8_t* bin, int64_t stride,
                        unsigned long long* cnt, cudaStream_t s);
// Stable partition of pairs[0 .. n): those whose bin is chosen (chosen: kPairBins
// bytes on the device) first, then the rest, into out; *pos receives [n + 1]
// int64 with their number at pos[n].
cudaError_t partition_pairs(const int2* pairs, const uint8_t* bin, const uint8_t* chosen, int64_t n, int2* out,
                            Buf* pos, cudaStream_t s);
// FP8 E4M3 operands of a tile layout built with BF16 operands (needs its
// centres and tmax): per tile a power-of-two scale s, hi and lo parts of a / s
// (Fh, Fl), frl and ftmax. A no-op when already built. Returns a mapper_status.
int fp8_operands(TileLayout* L, const float* X, int64_t ld, int d, int dp, cudaStream_t s);
// BF16 hi + lo operands of rows row_pt[.] of X (T tiles of 128 rows, the
// first tile_n[t] of tile t valid, the rest zero), centred on cents[tile_cent[t]]
// (dp floats each), with FP32 |a|^2 and |a| rounded up. nonfinite (nullable):
// set to 1 when a valid row's |a|^2 is not finite (a NaN or Inf in the row, or
// a norm beyond FP32).
cudaError_t centred_operands(const float* X, int64_t ld, int d, int dp, const int32_t* row_pt, const int32_t* tile_n,
                             const int32_t* tile_cent, const float* cents, int64_t T, void* Ah, void* Al, float* rn2,
                             float* rn, cudaStream_t s, int* nonfinite = nullptr);
// Tensor-core operands for the CUDA-core list (tile pairs of one element, two
// segments): every row centred on its element's centre, BF16 hi + lo, with
// FP32 |a|^2, and |a| and |a - hi| rounded up (R rows each), their largest
// values per tile (T float4) and the smallest |a|^2 per tile.
int cross_operands(const TileLayout& L, const float* X, int64_t ld, int d, int dp, int64_t E, Buf* Ah, Buf* Al,
                   Buf* rn2, Buf* rn, Buf* rl, Buf* tmax, Buf* tn2min, cudaStream_t s);

}  // namespace mgb
