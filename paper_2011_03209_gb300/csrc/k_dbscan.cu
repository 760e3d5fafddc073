// k_dbscan.cu -- per-cover-element DBSCAN on CUDA cores.
//
// "Mapper Interactive" §3: DBSCAN(eps, minPts) clusters the points of each
// cover element; §4.3 parallelises over elements and precomputes each
// element's distance matrix. Here the distance matrix is never stored: the
// rows of an element are cut into tiles of 128 and each tile pair (a <= b) is
// one CTA that recomputes the pair's squared distances in registers and
// consumes them at once:
//   pass 1  neighbour counts (and the first minPts-1 neighbours of each row,
//           enough to hold every neighbour of a non-core row)
//   pass 2  core-core unions: lock-free union-find whose roots are the
//           component's smallest point index (the canonical id)
//   pass 3  border rows: the smallest canonical id among core neighbours,
//           from the stored neighbours (or a third contraction when minPts
//           is too large to store them)
// Screen: the FP32 sum of squared differences s has |s - d2| <= eta d2 + tiny
// (fp32_thresholds); a pair is in when s <= eps^2(1-eta) - tiny, out when
// s > eps^2(1+eta) + tiny, else it is re-decided in FP64 by the defining
// expression (k ascending, one rounding per operation), so every decision
// equals the FP64 definition.
#include <cfloat>
#include <climits>
#include <cmath>

#include "dbscan.cuh"

namespace mgb {

namespace {

constexpr int kT = kTile;      // tile rows
constexpr int kK = 32;         // k chunk
constexpr int kPad = 132;      // smem row pitch (floats)

__device__ __forceinline__ int64_t upper_bound_i64(const int64_t* a, int64_t n, int64_t v)
{
    int64_t l = 0, r = n;
    while (l < r) {
        const int64_t m = (l + r) >> 1;
        if (a[m] <= v) l = m + 1; else r = m;
    }
    return l;
}

// q-th entry of the upper triangle of a T x T grid: rows of cum(a) = aT -
// a(a-1)/2 entries (a, a), (a, a+1), ...
__device__ __forceinline__ void decode_pair(int64_t q, int64_t T, int* ta, int* tb)
{
    int64_t l = 0, r = T - 1;
    while (l < r) {
        const int64_t m = (l + r + 1) >> 1;
        const int64_t cum = m * T - m * (m - 1) / 2;
        if (cum <= q) l = m; else r = m - 1;
    }
    *ta = (int)l;
    *tb = (int)(l + (q - (l * T - l * (l - 1) / 2)));
}

__device__ __forceinline__ double exact_sqdist(const float* __restrict__ x, const float* __restrict__ y,
                                               int d)
{
    double s = 0.0;
    for (int k = 0; k < d; ++k) {
        const double t = __dsub_rn((double)x[k], (double)y[k]);
        s = __dadd_rn(s, __dmul_rn(t, t));
    }
    return s;
}

__device__ __forceinline__ int key_of(const int32_t* row_pt, int row)
{
    return row_pt ? __ldg(row_pt + row) : row;
}

// Global union-find over rows. Parents always carry a smaller key (point
// index) than their child, so every chain ends and a root is the smallest
// key of its component. Path halving only ever points a node at an ancestor.
__device__ __forceinline__ int gfind(int32_t* parent, int x)
{
    volatile int32_t* par = parent;
    int p = par[x];
    while (p != x) {
        const int gp = par[p];
        if (gp != p) par[x] = gp;
        x = p;
        p = par[x];
    }
    return x;
}

__device__ __forceinline__ void gunion(int32_t* parent, const int32_t* row_pt, int a, int b)
{
    while (true) {
        a = gfind(parent, a);
        b = gfind(parent, b);
        if (a == b) return;
        if (key_of(row_pt, a) < key_of(row_pt, b)) { const int t = a; a = b; b = t; }
        if (atomicCAS(&parent[a], a, b) == a) return;
    }
}

// Shared-memory union-find over the 256 rows of a tile pair, same rules with
// the local index as key.
__device__ __forceinline__ int lfind(volatile int* par, int x)
{
    int p = par[x];
    while (p != x) {
        const int gp = par[p];
        if (gp != p) par[x] = gp;
        x = p;
        p = par[x];
    }
    return x;
}

__device__ __forceinline__ void lunion(int* par, int a, int b)
{
    volatile int* vp = par;
    while (true) {
        a = lfind(vp, a);
        b = lfind(vp, b);
        if (a == b) return;
        if (a < b) { const int t = a; a = b; b = t; }
        if (atomicCAS(&par[a], a, b) == a) return;
    }
}

struct Decider {
    const PassArgs& A;
    __device__ __forceinline__ bool operator()(float s, int64_t row_a, int64_t row_b,
                                               bool count_tie) const
    {
        if (s <= A.lo_thr) return true;
        if (s > A.hi_thr && s <= FLT_MAX) return false;
        const double d2 = exact_sqdist(pass_row(A, row_a), pass_row(A, row_b), A.d);
        atomicAdd(&A.stats[kStatBand], 1ull);
        atomicAdd(&A.stats[kStatFp64], 1ull);
        if (count_tie && fabs(d2 - A.eps2) <= A.tie_thr) atomicAdd(&A.stats[kStatTies], 1ull);
        return d2 <= A.eps2;
    }
};

// Rows, sizes and diagonal flag of this CTA's tile pair.
struct PairRows {
    int64_t sa, sb;
    int na, nb;
    bool diag;
};

__device__ __forceinline__ PairRows pair_rows(const PassArgs& A, int64_t q)
{
    PairRows P;
    if (A.pairs) {
        const int2 p = A.pairs[q];
        int ta = p.x, tb = p.y & kPairTileMask;
        bool ok = true;
        unsigned long long* oob = A.stats ? A.stats + kStatOob : nullptr;
        (void)oob;
        if (!MGB_IN_RANGE(ta, A.n_tiles, oob) || !MGB_IN_RANGE(tb, A.n_tiles, oob)) {
            ta = tb = 0;
            ok = false;
        }
        P.sa = (int64_t)ta * kT;
        P.sb = (int64_t)tb * kT;
        P.na = ok ? A.tile_n[ta] : 0;
        P.nb = ok ? A.tile_n[tb] : 0;
        P.diag = ta == tb;
    } else {
        const int64_t e = upper_bound_i64(A.pair_off, (int64_t)A.E + 1, q) - 1;
        const int64_t qq = q - A.pair_off[e];
        const int64_t base = A.elem_off[e], ne = A.elem_off[e + 1] - base;
        const int64_t T = (ne + kT - 1) / kT;
        int ta, tb;
        decode_pair(qq, T, &ta, &tb);
        P.sa = base + (int64_t)ta * kT;
        P.sb = base + (int64_t)tb * kT;
        P.na = (int)(ne - (int64_t)ta * kT < kT ? ne - (int64_t)ta * kT : kT);
        P.nb = (int)(ne - (int64_t)tb * kT < kT ? ne - (int64_t)tb * kT : kT);
        P.diag = ta == tb;
    }
    return P;
}

__device__ __forceinline__ unsigned long long root_code(const PassArgs& A, int row)
{
    const int r = A.root[row];
    return ((unsigned long long)(unsigned)key_of(A.row_pt, r) << 32) | (unsigned)r;
}

// Before a union pass on a tile pair: how many core rows each side holds,
// and whether all of them already share one root (nothing left to join).
// Fills s_core. Must be reached by all threads.
__device__ __forceinline__ bool union_prologue(const PassArgs& A, const PairRows& P,
                                               unsigned char* s_core, int* s_mm)
{
    const int tid = threadIdx.x;
    const bool valid = tid < kT ? tid < P.na : (!P.diag && tid - kT < P.nb);
    const int64_t row = tid < kT ? P.sa + tid : P.sb + (tid - kT);
    const bool c = valid && A.core[row];
    s_core[tid] = c;
    if (tid == 0) { s_mm[0] = INT_MAX; s_mm[1] = -1; }
    const int nca = __syncthreads_count(tid < kT && c);
    const int ncb = __syncthreads_count(tid >= kT && c);
    const bool work = P.diag ? nca >= 2 : (nca > 0 && ncb > 0);
    if (!work) return false;
    if (c) {
        const int r = gfind(A.parent, (int)row);
        atomicMin(&s_mm[0], r);
        atomicMax(&s_mm[1], r);
    }
    __syncthreads();
    const bool joined = s_mm[0] == s_mm[1];
    if (joined && tid == 0) atomicAdd(&A.stats[kStatSkipped], 1ull);
    return !joined;
}

template <int MODE>
__global__ void __launch_bounds__(256, 2) simt_pass_kernel(const PassArgs A)
{
    __shared__ __align__(16) float As[kK][kPad];
    __shared__ __align__(16) float Bs[kK][kPad];
    __shared__ int s_aux[2 * kT];                  // 1: column counts; 2: local parents
    __shared__ int s_old[kT];                      // 1: count of each column before this pair
    __shared__ unsigned long long s_code[2 * kT];  // 3: root code of each core row, then best
    __shared__ unsigned char s_core[2 * kT];
    __shared__ int s_mm[2];

    const int tid = threadIdx.x;
    if (A.n_dev && (unsigned long long)blockIdx.x >= *A.n_dev) return;
    const PairRows P = pair_rows(A, blockIdx.x);
    const int64_t sa = P.sa, sb = P.sb;
    const int na = P.na, nb = P.nb;
    const bool diag = P.diag;

    if (MODE == 1) {
        if (tid < kT) s_aux[tid] = 0;
    } else if (MODE == 2) {
        if (!union_prologue(A, P, s_core, s_mm)) return;
        s_aux[tid] = tid;
    } else {
        const bool valid = tid < kT ? tid < na : tid - kT < nb;
        const int64_t row = tid < kT ? sa + tid : sb + (tid - kT);
        const bool c = valid && A.core[row];
        s_core[tid] = c;
        const int nca = __syncthreads_count(tid < kT && c);
        const int ncb = __syncthreads_count(tid >= kT && c);
        const bool work = (ncb > 0 && nca < na) || (!diag && nca > 0 && ncb < nb);
        if (!work) return;
        s_code[tid] = c ? root_code(A, (int)row) : ~0ull;
    }

    const int tx = tid & 15, ty = tid >> 4;
    float acc[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;

    for (int k0 = 0; k0 < A.dp; k0 += kK) {
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const int idx = tid + 256 * v;       // float4 index in the 128 x 32 chunk
            const int r = idx >> 3, k4 = (idx & 7) * 4;
            float4 xa = make_float4(0.f, 0.f, 0.f, 0.f), xb = xa;
            if (r < na) xa = pass_ld4(A, pass_row(A, sa + r), (k0 + k4) >> 2);
            if (r < nb) xb = pass_ld4(A, pass_row(A, sb + r), (k0 + k4) >> 2);
            As[k4 + 0][r] = xa.x; As[k4 + 1][r] = xa.y; As[k4 + 2][r] = xa.z; As[k4 + 3][r] = xa.w;
            Bs[k4 + 0][r] = xb.x; Bs[k4 + 1][r] = xb.y; Bs[k4 + 2][r] = xb.z; Bs[k4 + 3][r] = xb.w;
        }
        __syncthreads();
#pragma unroll 8
        for (int k = 0; k < kK; ++k) {
            const float4 a0 = *reinterpret_cast<const float4*>(&As[k][ty * 4]);
            const float4 a1 = *reinterpret_cast<const float4*>(&As[k][64 + ty * 4]);
            const float4 b0 = *reinterpret_cast<const float4*>(&Bs[k][tx * 4]);
            const float4 b1 = *reinterpret_cast<const float4*>(&Bs[k][64 + tx * 4]);
            const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            const float b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const float t = a[i] - b[j];
                    acc[i][j] = fmaf(t, t, acc[i][j]);
                }
        }
        __syncthreads();
    }

    const Decider decide{A};
    if (MODE == 1) {
        // decide every pair once; bit (i*8 + j) = pair (row i, column j) is in
        unsigned long long inb = 0ull;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int r = i < 4 ? ty * 4 + i : 64 + ty * 4 + i - 4;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int c = j < 4 ? tx * 4 + j : 64 + tx * 4 + j - 4;
                if (r < na && c < nb && decide(acc[i][j], sa + r, sb + c, !diag || r < c))
                    inb |= 1ull << (i * 8 + j);
            }
        }
        // rows: counts and list positions from a scan over the 16 lanes of a row
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const unsigned bits = (unsigned)(inb >> (i * 8)) & 0xffu;
            const int own = __popc(bits);
            int incl = own;
#pragma unroll
            for (int o = 1; o < 16; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, incl, o, 16);
                if (tx >= o) incl += y;
            }
            const int total = __shfl_sync(0xffffffffu, incl, 15, 16);
            const int r = i < 4 ? ty * 4 + i : 64 + ty * 4 + i - 4;
            int old = 0;
            if (tx == 0 && total > 0) old = atomicAdd(&A.count[sa + r], total);
            old = __shfl_sync(0xffffffffu, old, 0, 16);
            if (A.cap > 0 && total > 0 && old < A.cap && bits) {
                int pos = old + incl - own;
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    if (!((bits >> j) & 1u)) continue;
                    if (pos < A.cap) {
                        const int c = j < 4 ? tx * 4 + j : 64 + tx * 4 + j - 4;
                        A.nbr[(sa + r) * A.cap + pos] = (int32_t)(sb + c);
                    }
                    ++pos;
                }
            }
        }
        if (!diag) {
            // columns: counts gathered in shared memory, then one atomic each
            int pos_local[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                unsigned colbits = 0;
#pragma unroll
                for (int i = 0; i < 8; ++i) colbits |= (unsigned)((inb >> (i * 8 + j)) & 1ull) << i;
                const int c = j < 4 ? tx * 4 + j : 64 + tx * 4 + j - 4;
                pos_local[j] = colbits ? atomicAdd(&s_aux[c], __popc(colbits)) : 0;
            }
            __syncthreads();
            if (tid < kT) s_old[tid] = (tid < nb && s_aux[tid]) ? atomicAdd(&A.count[sb + tid], s_aux[tid]) : 0;
            __syncthreads();
            if (A.cap > 0) {
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const int c = j < 4 ? tx * 4 + j : 64 + tx * 4 + j - 4;
                    int pos = s_old[c] + pos_local[j];
                    if (pos >= A.cap) continue;
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        if (!((inb >> (i * 8 + j)) & 1ull)) continue;
                        if (pos < A.cap) {
                            const int r = i < 4 ? ty * 4 + i : 64 + ty * 4 + i - 4;
                            A.nbr[(sb + c) * A.cap + pos] = (int32_t)(sa + r);
                        }
                        ++pos;
                    }
                }
            }
        }
        if (A.pair_hit && inb && A.pairs) A.pair_hit[blockIdx.x] = 1;
        if (tid == 0) {
            const int64_t pairs = diag ? (int64_t)na * (na + 1) / 2 : (int64_t)na * nb;
            atomicAdd(&A.stats[kStatScreened], (unsigned long long)pairs);
            atomicAdd(&A.stats[kStatSimtPairs], (unsigned long long)pairs);
        }
    } else if (MODE == 2) {
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int r = i < 4 ? ty * 4 + i : 64 + ty * 4 + i - 4;
            if (r >= na || !s_core[r]) continue;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int c = j < 4 ? tx * 4 + j : 64 + tx * 4 + j - 4;
                if (diag) {
                    if (c <= r || c >= na || !s_core[c]) continue;
                } else if (c >= nb || !s_core[kT + c]) {
                    continue;
                }
                const int lr = r, lc = diag ? c : kT + c;
                if (lfind(s_aux, lr) == lfind(s_aux, lc)) continue;
                if (decide(acc[i][j], sa + r, sb + c, false)) lunion(s_aux, lr, lc);
            }
        }
        __syncthreads();
        const int x = tid;
        if (s_core[x]) {
            const int rx = lfind(s_aux, x);
            if (rx != x) {
                const int64_t row_x = x < kT ? sa + x : sb + (x - kT);
                const int64_t row_r = rx < kT ? sa + rx : sb + (rx - kT);
                gunion(A.parent, A.row_pt, (int)row_x, (int)row_r);
            }
        }
    } else {
        __shared__ unsigned long long s_best[2 * kT];
        s_best[tid] = ~0ull;
        __syncthreads();
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int r = i < 4 ? ty * 4 + i : 64 + ty * 4 + i - 4;
            if (r >= na) continue;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int c = j < 4 ? tx * 4 + j : 64 + tx * 4 + j - 4;
                if (c >= nb) continue;
                const bool need_a = !s_core[r] && s_core[kT + c];
                const bool need_b = !diag && !s_core[kT + c] && s_core[r];
                if (!(need_a || need_b)) continue;
                if (decide(acc[i][j], sa + r, sb + c, false)) {
                    if (need_a) atomicMin(&s_best[r], s_code[kT + c]);
                    if (need_b) atomicMin(&s_best[kT + c], s_code[r]);
                }
            }
        }
        __syncthreads();
        const int x = tid;
        if (s_best[x] != ~0ull) {
            const int64_t row_x = x < kT ? sa + x : sb + (x - kT);
            atomicMin(&A.border[row_x], s_best[x]);
        }
    }
}

// Tile pairs certified all-in by bounding spheres: every pair is a
// neighbour pair, nothing to screen.
template <int MODE>
__global__ void __launch_bounds__(256) allin_kernel(const PassArgs A)
{
    __shared__ unsigned char s_core[2 * kT];
    __shared__ int s_mm[2];
    __shared__ int s_first;
    __shared__ unsigned long long s_min[2];
    const int tid = threadIdx.x;
    const PairRows P = pair_rows(A, blockIdx.x);
    const bool side_b = tid >= kT;
    const int x = side_b ? tid - kT : tid;
    const bool valid = side_b ? (!P.diag && x < P.nb) : x < P.na;
    const int64_t row = side_b ? P.sb + x : P.sa + x;
    if (MODE == 1) {
        if (!valid) return;
        const int k = side_b ? P.na : (P.diag ? P.na : P.nb);
        const int old = atomicAdd(&A.count[row], k);
        if (A.cap > 0 && old < A.cap) {
            const int64_t other = side_b ? P.sa : (P.diag ? P.sa : P.sb);
            for (int i = 0; i < k && old + i < A.cap; ++i)
                A.nbr[row * A.cap + old + i] = (int32_t)(other + i);
        }
        if (tid == 0) {
            const int64_t pairs = P.diag ? (int64_t)P.na * (P.na + 1) / 2 : (int64_t)P.na * P.nb;
            atomicAdd(&A.stats[kStatScreened], (unsigned long long)pairs);
        }
    } else if (MODE == 2) {
        if (!union_prologue(A, P, s_core, s_mm)) return;
        if (tid == 0) s_first = INT_MAX;
        __syncthreads();
        if (s_core[tid]) atomicMin(&s_first, tid);
        __syncthreads();
        const int f = s_first;
        if (s_core[tid] && tid != f) {
            const int64_t row_f = f < kT ? P.sa + f : P.sb + (f - kT);
            gunion(A.parent, A.row_pt, (int)row, (int)row_f);
        }
    } else {
        const bool c = valid && A.core[row];
        if (tid < 2) s_min[tid] = ~0ull;
        __syncthreads();
        if (c) atomicMin(&s_min[side_b ? 1 : 0], root_code(A, (int)row));
        __syncthreads();
        if (valid && !c) {
            const unsigned long long best = P.diag ? s_min[0] : s_min[side_b ? 0 : 1];
            if (best != ~0ull) atomicMin(&A.border[row], best);
        }
    }
}

__global__ void core_kernel(const int32_t* __restrict__ count, int64_t R, int32_t min_pts,
                            uint8_t* __restrict__ core, int32_t* __restrict__ parent,
                            unsigned long long* __restrict__ border, unsigned long long* stats)
{
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    bool c = false;
    if (s < R) {
        c = count[s] >= min_pts;
        core[s] = c;
        parent[s] = (int32_t)s;
        border[s] = ~0ull;
    }
    const int nc = __syncthreads_count(c);
    if (threadIdx.x == 0 && nc) atomicAdd(&stats[kStatCore], (unsigned long long)nc);
}

__global__ void flatten_kernel(const int32_t* __restrict__ parent, const uint8_t* __restrict__ core,
                               int64_t R, int32_t* __restrict__ root)
{
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= R) return;
    int r = (int)s;
    if (core[s])
        while (parent[r] != r) r = parent[r];
    root[s] = r;
}

// A non-core row holds fewer than minPts neighbours, all of them stored by
// pass 1: its label is the smallest canonical id among its core neighbours.
__global__ void border_lists_kernel(const int32_t* __restrict__ count, const int32_t* __restrict__ nbr,
                                    int cap, const uint8_t* __restrict__ core,
                                    const int32_t* __restrict__ root, const int32_t* __restrict__ row_pt,
                                    int64_t R, unsigned long long* __restrict__ border, unsigned long long* oob)
{
    (void)oob;
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= R || core[s]) return;
    const int k = min(count[s], cap);
    unsigned long long best = ~0ull;
    for (int i = 0; i < k; ++i) {
        const int q = nbr[s * cap + i];
        if (q < 0 || !MGB_IN_RANGE(q, R, oob) || !core[q]) continue;
        const int r = root[q];
        const unsigned long long code =
            ((unsigned long long)(unsigned)(row_pt ? row_pt[r] : r) << 32) | (unsigned)r;
        best = code < best ? code : best;
    }
    border[s] = best;
}

// Unions along the neighbour lists of pass 1: a core row's list holds its
// first cap neighbours, every one a certified neighbour pair; joining the
// core ones merges most of each cluster before the union pass, which then
// skips every tile pair whose core rows already share one root.
__global__ void list_unions_kernel(const int32_t* __restrict__ count, const int32_t* __restrict__ nbr, int cap,
                                   const uint8_t* __restrict__ core, int32_t* __restrict__ parent,
                                   const int32_t* __restrict__ row_pt, int64_t R, unsigned long long* oob)
{
    (void)oob;
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= R || !core[s]) return;
    const int k = min(count[s], cap);
    for (int i = 0; i < k; ++i) {
        const int q = nbr[s * cap + i];
        if (q >= 0 && MGB_IN_RANGE(q, R, oob) && core[q]) gunion(parent, row_pt, (int)s, q);
    }
}

__global__ void rows_to_slots_kernel(const int32_t* __restrict__ row_slot, const int32_t* __restrict__ row_pt,
                                     const uint8_t* __restrict__ core, const int32_t* __restrict__ root,
                                     const unsigned long long* __restrict__ border, int64_t R,
                                     int32_t* __restrict__ lab, int32_t* __restrict__ is_root,
                                     int32_t* __restrict__ is_member, int64_t* __restrict__ slot_label,
                                     uint8_t* __restrict__ slot_core)
{
    const int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= R) return;
    const int slot = row_slot[row];
    if (slot < 0) return;
    const bool c = core[row];
    int l = -1;
    if (c) l = root[row];
    else if (border[row] != ~0ull) l = (int)(unsigned)(border[row] & 0xffffffffull);
    lab[slot] = l >= 0 ? row_slot[l] : -1;
    slot_label[slot] = l >= 0 ? (int64_t)row_pt[l] : -1;
    is_root[slot] = c && root[row] == (int32_t)row;
    is_member[slot] = l >= 0;
    slot_core[slot] = c;
}

__global__ void counts_to_lens_kernel(const int32_t* __restrict__ row_slot, const int32_t* __restrict__ row_pt,
                                      const int32_t* __restrict__ count, int64_t R, double* __restrict__ f, int m,
                                      int j)
{
    const int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= R || row_slot[row] < 0) return;
    f[(int64_t)row_pt[row] * m + j] = (double)count[row];
}

__global__ void elem_offsets_kernel(const uint64_t* __restrict__ keys, int64_t M, int64_t E,
                                    int64_t* __restrict__ elem_off)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e > E) return;
    int64_t l = 0, r = M;                      // first slot whose element >= e
    while (l < r) {
        const int64_t m = (l + r) >> 1;
        if ((int64_t)(keys[m] >> 32) < e) l = m + 1; else r = m;
    }
    elem_off[e] = l;
}

__global__ void select_hit_kernel(const int2* __restrict__ pairs, const uint8_t* __restrict__ hit, int64_t n,
                                  int2* __restrict__ out, unsigned long long* __restrict__ count)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || !hit[i]) return;
    out[atomicAdd(count, 1ull)] = pairs[i];
}

// Tile pairs whose tile distance b - a lies in (lo, hi].
__global__ void select_delta_kernel(const int2* __restrict__ pairs, int64_t n,
                                    const unsigned long long* __restrict__ n_dev, int lo, int hi,
                                    int2* __restrict__ out, unsigned long long* __restrict__ count)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || (n_dev && (unsigned long long)i >= *n_dev)) return;
    const int2 p = pairs[i];
    const int delta = p.y - p.x;
    if (delta > lo && delta <= hi) out[atomicAdd(count, 1ull)] = p;
}

// Smallest and largest current root over each tile's core rows (INT_MAX,
// -1 for a tile without core rows); one warp per tile.
__global__ void tile_roots_kernel(const PassArgs A, int64_t T, int2* __restrict__ tr)
{
    const int lane = threadIdx.x & 31;
    const int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (t >= T) return;
    const int nt = A.tile_n[t];
    int lo = INT_MAX, hi = -1;
    for (int x = lane; x < nt; x += 32) {
        const int64_t row = t * kT + x;
        if (!A.core[row]) continue;
        const int r = gfind(A.parent, (int)row);
        lo = min(lo, r);
        hi = max(hi, r);
    }
    for (int o = 16; o; o >>= 1) {
        lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    if (lane == 0) tr[t] = make_int2(lo, hi);
}

// A tile pair is kept if the roots of its core rows differ (read from the
// tiles' root ranges); an off-diagonal pair whose A cores share one root and
// whose B cores share another is flagged (kPairOneEach): one neighbour pair
// joins them. One thread per pair.
__global__ void filter_joined_kernel(const int2* __restrict__ pairs, int64_t n,
                                     const unsigned long long* __restrict__ n_dev, const int2* __restrict__ tr,
                                     int2* __restrict__ out, unsigned long long* __restrict__ count,
                                     unsigned long long* __restrict__ stats)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (n_dev) n = min(n, (int64_t)*n_dev);
    bool keep = false, skipped = false;
    int2 p = make_int2(0, 0);
    if (i < n) {
        p = pairs[i];
        const bool diag = p.x == p.y;
        const int2 a = tr[p.x], b = tr[p.y];
        bool work, one_each = false;
        if (diag) {
            work = a.y >= 0 && a.x != a.y;
        } else {
            work = a.y >= 0 && b.y >= 0 && (a.x != a.y || b.x != b.y || a.x != b.x);
            one_each = work && a.x == a.y && b.x == b.y;
        }
        keep = work;
        skipped = !work && a.y >= 0;
        if (one_each) p.y |= kPairOneEach;
    }
    // one output atomic per warp
    const unsigned m = __ballot_sync(0xffffffffu, keep);
    unsigned long long base = 0;
    const int lane = threadIdx.x & 31;
    if (lane == 0 && m) base = atomicAdd(count, (unsigned long long)__popc(m));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (keep) out[base + __popc(m & ((1u << lane) - 1u))] = p;
    const unsigned ms = __ballot_sync(0xffffffffu, skipped);
    if (lane == 0 && ms) atomicAdd(&stats[kStatSkipped], (unsigned long long)__popc(ms));
}

inline unsigned grid_for(int64_t n, int t = 256) { return (unsigned)std::max<int64_t>(1, div_up(n, t)); }

}  // namespace

cudaError_t select_hit(const int2* pairs, const uint8_t* hit, int64_t n, int2* out,
                       unsigned long long* count, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    select_hit_kernel<<<grid_for(n), 256, 0, s>>>(pairs, hit, n, out, count);
    note_launch();
    return cudaGetLastError();
}

__global__ void add_counter_kernel(unsigned long long* dst, const unsigned long long* src) { *dst += *src; }

cudaError_t add_counter(unsigned long long* dst, const unsigned long long* src, cudaStream_t s)
{
    add_counter_kernel<<<1, 1, 0, s>>>(dst, src);
    note_launch();
    return cudaGetLastError();
}

cudaError_t select_delta(const int2* pairs, int64_t n, const unsigned long long* n_dev, int lo, int hi, int2* out,
                         unsigned long long* count, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    select_delta_kernel<<<grid_for(n), 256, 0, s>>>(pairs, n, n_dev, lo, hi, out, count);
    note_launch();
    return cudaGetLastError();
}

cudaError_t filter_joined(const PassArgs& a, int64_t T, int2* tile_roots, const int2* pairs, int64_t n,
                          const unsigned long long* n_dev, int2* out, unsigned long long* count, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    tile_roots_kernel<<<grid_for(T * 32), 256, 0, s>>>(a, T, tile_roots);
    filter_joined_kernel<<<grid_for(n), 256, 0, s>>>(pairs, n, n_dev, tile_roots, out, count, a.stats);
    note_launch(2);
    return cudaGetLastError();
}

// FP32 screen thresholds. The sum of d squared differences accumulated by
// FMA in FP32 satisfies |s - d2| <= ((1+u)^2 (1+gamma_d) - 1) d2 + tiny
// (u = 2^-24, gamma_d = d u / (1 - d u); all terms are nonnegative, the
// subtraction rounds once, each FMA once, subnormal results add at most
// 2^-149 each). With eta = 1.5 (d + 4) u the pair is certainly inside when
// s <= eps2 (1 - eta) - tiny and certainly outside when s > eps2 (1 + eta)
// + tiny; the bounds are rounded outward to float.
void fp32_thresholds(double eps2, int d, float* lo, float* hi)
{
    const double u = std::ldexp(1.0, -24);
    const double eta = 1.5 * (d + 4) * u;
    const double tiny = 3.0 * (d + 2) * std::ldexp(1.0, -149);
    const double l = eps2 * (1.0 - eta) - tiny;
    const double h = eps2 * (1.0 + eta) + tiny;
    float lf = (float)l;
    if ((double)lf > l) lf = std::nextafter(lf, -INFINITY);
    if (l <= 0.0) lf = -1.0f;
    float hf = (float)h;
    if ((double)hf < h) hf = std::nextafter(hf, INFINITY);
    *lo = lf;
    *hi = hf;
}

cudaError_t simt_pass(int mode, const PassArgs& a, int64_t n_pairs, cudaStream_t s)
{
    if (n_pairs == 0) return cudaSuccess;
    if (mode == 1) simt_pass_kernel<1><<<(unsigned)n_pairs, 256, 0, s>>>(a);
    else if (mode == 2) simt_pass_kernel<2><<<(unsigned)n_pairs, 256, 0, s>>>(a);
    else simt_pass_kernel<3><<<(unsigned)n_pairs, 256, 0, s>>>(a);
    note_launch();
    return cudaGetLastError();
}

cudaError_t allin_pass(int mode, const PassArgs& a, int64_t n_pairs, cudaStream_t s)
{
    if (n_pairs == 0) return cudaSuccess;
    if (mode == 1) allin_kernel<1><<<(unsigned)n_pairs, 256, 0, s>>>(a);
    else if (mode == 2) allin_kernel<2><<<(unsigned)n_pairs, 256, 0, s>>>(a);
    else allin_kernel<3><<<(unsigned)n_pairs, 256, 0, s>>>(a);
    note_launch();
    return cudaGetLastError();
}

cudaError_t core_flags(const int32_t* count, int64_t R, int32_t min_pts, uint8_t* core,
                       int32_t* parent, unsigned long long* border, unsigned long long* stats,
                       cudaStream_t s)
{
    if (R == 0) return cudaSuccess;
    core_kernel<<<grid_for(R), 256, 0, s>>>(count, R, min_pts, core, parent, border, stats);
    note_launch();
    return cudaGetLastError();
}

cudaError_t flatten(const int32_t* parent, const uint8_t* core, int64_t R, int32_t* root,
                    cudaStream_t s)
{
    if (R == 0) return cudaSuccess;
    flatten_kernel<<<grid_for(R), 256, 0, s>>>(parent, core, R, root);
    note_launch();
    return cudaGetLastError();
}

cudaError_t border_from_lists(const int32_t* count, const int32_t* nbr, int cap,
                              const uint8_t* core, const int32_t* root, const int32_t* row_pt,
                              int64_t R, unsigned long long* border, cudaStream_t s, unsigned long long* oob)
{
    if (R == 0 || cap <= 0) return cudaSuccess;
    border_lists_kernel<<<grid_for(R), 256, 0, s>>>(count, nbr, cap, core, root, row_pt, R, border, oob);
    note_launch();
    return cudaGetLastError();
}

cudaError_t list_unions(const int32_t* count, const int32_t* nbr, int cap, const uint8_t* core, int32_t* parent,
                        const int32_t* row_pt, int64_t R, cudaStream_t s, unsigned long long* oob)
{
    if (R == 0 || cap == 0) return cudaSuccess;
    list_unions_kernel<<<grid_for(R), 256, 0, s>>>(count, nbr, cap, core, parent, row_pt, R, oob);
    note_launch();
    return cudaGetLastError();
}

cudaError_t rows_to_slots(const int32_t* row_slot, const int32_t* row_pt, const uint8_t* core,
                          const int32_t* root, const unsigned long long* border, int64_t R,
                          int32_t* lab, int32_t* is_root, int32_t* is_member,
                          int64_t* slot_label, uint8_t* slot_core, cudaStream_t s)
{
    if (R == 0) return cudaSuccess;
    rows_to_slots_kernel<<<grid_for(R), 256, 0, s>>>(row_slot, row_pt, core, root, border, R, lab,
                                                     is_root, is_member, slot_label, slot_core);
    note_launch();
    return cudaGetLastError();
}

cudaError_t counts_to_lens(const int32_t* row_slot, const int32_t* row_pt, const int32_t* count, int64_t R,
                           double* f, int m, int j, cudaStream_t s)
{
    counts_to_lens_kernel<<<grid_for(R), 256, 0, s>>>(row_slot, row_pt, count, R, f, m, j);
    note_launch();
    return cudaGetLastError();
}

cudaError_t element_offsets(const uint64_t* keys, int64_t M, int64_t E, int64_t* elem_off,
                            cudaStream_t s)
{
    elem_offsets_kernel<<<grid_for(E + 1), 256, 0, s>>>(keys, M, E, elem_off);
    note_launch();
    return cudaGetLastError();
}

}  // namespace mgb
