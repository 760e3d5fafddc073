// k_tiles.cu -- spatially coherent tiles for the per-element DBSCAN passes,
// and bounding-sphere classification of their tile pairs.
//
// The per-element DBSCAN of "Mapper Interactive" (§3; parallel per interval
// in §4.3) needs, for each element, every point pair within eps. Points of an
// element sit in a few dense regions far apart; if consecutive rows of a tile
// come from one region, most tile pairs are provably all-out (or all-in) by
// the triangle inequality and need no distance at all. The layout:
//   1. K pivots (points floor(k n / K)); every point goes to its nearest
//      pivot; pivots closer than tau join one group (connected components);
//      a point farther than tau from every pivot is an outlier.
//   2. Each element's slots are sorted by (group, pivot), stably, so points
//      stay ascending inside a pivot; each (element, group) segment is cut
//      into tiles of 128 rows (the last one padded), so no tile mixes groups.
//   3. Per tile: rows gathered (FP32, zero padded), FP64 centroid and radius.
//      Per segment: FP64 centroid; rows centred on it are split into BF16
//      hi + lo parts with |a|^2 and |a| for the tensor-core screen.
// Only speed depends on this ordering; every decision stays exact.
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include <cfloat>
#include <climits>
#include <cmath>
#include <vector>

#include "../../include/mapper.h"
#include "tc.cuh"

namespace mgb {

namespace {

constexpr int kPiv = 256;      // most pivots
constexpr int kT = kTile;

inline unsigned grid_for(int64_t n, int t = 256) { return (unsigned)std::max<int64_t>(1, div_up(n, t)); }

int bits_for(int64_t n)        // bits to hold values 0 .. n-1
{
    int b = 1;
    while (b < 63 && (int64_t(1) << b) < n) ++b;
    return b;
}

__global__ void pivot_gather_kernel(const float* __restrict__ X, int64_t n, int d, int64_t ld, int dp,
                                    int K, float* __restrict__ Pv)
{
    const int k = blockIdx.x;
    const int64_t p = (int64_t)k * n / K;
    for (int j = threadIdx.x; j < dp; j += blockDim.x) Pv[(int64_t)k * dp + j] = j < d ? X[p * ld + j] : 0.f;
}

// c[k] = the FP32 sum of the K pivots' column k in pivot order, / K
__global__ void pivot_mean_kernel(const float* __restrict__ Pv, int K, int dp, float* __restrict__ c)
{
    for (int k = threadIdx.x; k < dp; k += blockDim.x) {
        float s = 0.f;
        for (int i = 0; i < K; ++i) s += Pv[(int64_t)i * dp + k];
        c[k] = s / (float)K;
    }
}

// Nearest pivot of every point (FP32 distances; ties to the lower index).
// CTA: 128 points x 128 pivots per step, 32 dimensions staged at a time.
__global__ void __launch_bounds__(256, 2) assign_kernel(const float* __restrict__ X, int64_t n, int d,
                                                        int64_t ld, const float* __restrict__ Pv, int dp,
                                                        int K, int32_t* __restrict__ piv,
                                                        float* __restrict__ pd2)
{
    __shared__ __align__(16) float As[32][132];
    __shared__ __align__(16) float Bs[32][132];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int64_t p0 = (int64_t)blockIdx.x * kT;
    float best[8];
    int bidx[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) { best[i] = FLT_MAX; bidx[i] = INT_MAX; }
    for (int c0 = 0; c0 < K; c0 += kT) {
        float acc[8][8];
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
            for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
        for (int k0 = 0; k0 < d; k0 += 32) {
#pragma unroll 4
            for (int v = 0; v < 16; ++v) {
                const int idx = tid + 256 * v;
                const int r = idx >> 5, k = idx & 31;
                float x = 0.f;
                if (p0 + r < n && k0 + k < d) x = X[(p0 + r) * ld + k0 + k];
                As[k][r] = x;
            }
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                const int idx = tid + 256 * v;
                const int r = idx >> 3, k4 = (idx & 7) * 4;
                float4 b = make_float4(0.f, 0.f, 0.f, 0.f);
                if (c0 + r < K) b = *reinterpret_cast<const float4*>(Pv + (int64_t)(c0 + r) * dp + k0 + k4);
                Bs[k4 + 0][r] = b.x; Bs[k4 + 1][r] = b.y; Bs[k4 + 2][r] = b.z; Bs[k4 + 3][r] = b.w;
            }
            __syncthreads();
#pragma unroll 8
            for (int k = 0; k < 32; ++k) {
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
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int c = c0 + (j < 4 ? tx * 4 + j : 64 + tx * 4 + j - 4);
                if (c < K && (acc[i][j] < best[i] || (acc[i][j] == best[i] && c < bidx[i]))) {
                    best[i] = acc[i][j];
                    bidx[i] = c;
                }
            }
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
#pragma unroll
        for (int o = 1; o < 16; o <<= 1) {
            const float ov = __shfl_xor_sync(0xffffffffu, best[i], o);
            const int oi = __shfl_xor_sync(0xffffffffu, bidx[i], o);
            if (ov < best[i] || (ov == best[i] && oi < bidx[i])) { best[i] = ov; bidx[i] = oi; }
        }
        const int r = i < 4 ? ty * 4 + i : 64 + ty * 4 + i - 4;
        if (tx == 0 && p0 + r < n) {
            piv[p0 + r] = bidx[i] == INT_MAX ? 0 : bidx[i];       // NaN rows: any pivot
            pd2[p0 + r] = best[i];
        }
    }
}

// Pivot adjacency: bit j of adj[i] set when |p_i - p_j| <= tau (FP32).
// One warp per pivot pair i <= j.
__global__ void pivot_adj_kernel(const float* __restrict__ Pv, int dp, int K, float tau2,
                                 unsigned* __restrict__ adj)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarp = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t npairs = (int64_t)K * K;
    for (int64_t e = warp; e < npairs; e += nwarp) {
        const int i = (int)(e / K), j = (int)(e - (int64_t)i * K);
        if (j < i) continue;
        float s = 0.f;
        for (int k = lane; k < dp; k += 32) {
            const float t = Pv[(int64_t)i * dp + k] - Pv[(int64_t)j * dp + k];
            s = fmaf(t, t, s);
        }
        for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0 && s <= tau2) {
            atomicOr(&adj[i * (kPiv / 32) + (j >> 5)], 1u << (j & 31));
            atomicOr(&adj[j * (kPiv / 32) + (i >> 5)], 1u << (i & 31));
        }
    }
}

// Pivot groups: connected components of the adjacency, numbered 0.. in
// order of their smallest pivot. One CTA.
__global__ void __launch_bounds__(256) group_kernel(const unsigned* __restrict__ adj_g, int K,
                                                    int32_t* __restrict__ gid, int32_t* __restrict__ n_groups)
{
    __shared__ unsigned adj[kPiv][kPiv / 32];
    __shared__ int lab[kPiv];
    __shared__ int changed;
    const int tid = threadIdx.x;
    for (int e = tid; e < kPiv * kPiv / 32; e += blockDim.x) (&adj[0][0])[e] = adj_g[e];
    if (tid < K) lab[tid] = tid;
    __syncthreads();
    for (int it = 0; it <= K; ++it) {
        if (tid == 0) changed = 0;
        __syncthreads();
        if (tid < K) {
            int m = lab[tid];
            for (int w = 0; w < (K + 31) / 32; ++w) {
                unsigned bits = adj[tid][w];
                while (bits) {
                    const int j = w * 32 + __ffs(bits) - 1;
                    bits &= bits - 1;
                    m = min(m, lab[j]);
                }
            }
            if (m < lab[tid]) { lab[tid] = m; changed = 1; }
        }
        __syncthreads();
        if (!changed) break;
        __syncthreads();
    }
    if (tid < K) {
        const int l = lab[tid];
        int g = 0;
        for (int j = 0; j < l; ++j) g += lab[j] == j;
        gid[tid] = g;
        if (tid == K - 1) {
            int ng = 0;
            for (int j = 0; j < K; ++j) ng += lab[j] == j;
            *n_groups = ng;
        }
    }
}

// Sort key of a slot: (element, group, pivot) above the slot index.
__global__ void key_kernel(const int32_t* __restrict__ slot_point, const int32_t* __restrict__ slot_elem,
                           int64_t M, const int32_t* __restrict__ piv, const float* __restrict__ pd2,
                           const int32_t* __restrict__ gid, float tau2, int K, int gbits, int pbits,
                           uint64_t* __restrict__ keys)
{
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= M) return;
    const int pt = slot_point[s];
    const int pv = piv[pt];
    const bool outlier = !(pd2[pt] <= tau2);
    uint64_t g = 0, pf = 0;
    if (gbits) g = outlier ? (uint64_t)K : (uint64_t)gid[pv];
    if (pbits && !outlier) pf = (uint64_t)pv;
    const uint64_t hi = ((uint64_t)slot_elem[s] << (gbits + pbits)) | (g << pbits) | pf;
    keys[s] = (hi << 32) | (uint64_t)(uint32_t)s;
}

__global__ void seg_flag_kernel(const uint64_t* __restrict__ keys, int64_t M, int shift,
                                int32_t* __restrict__ flag)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= M) return;
    flag[i] = i == 0 || (keys[i] >> shift) != (keys[i - 1] >> shift);
}

// seg_start[nseg+1], seg_elem, seg_out (outlier segment) from the flags' scan
__global__ void seg_start_kernel(const uint64_t* __restrict__ keys, const int32_t* __restrict__ flag,
                                 const int64_t* __restrict__ segpos, int64_t M, int gbits, int pbits,
                                 int K, int64_t* __restrict__ seg_start, int32_t* __restrict__ seg_elem,
                                 int32_t* __restrict__ seg_out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= M) return;
    if (flag[i]) {
        const int64_t sg = segpos[i];
        const uint64_t hi = keys[i] >> 32;
        seg_start[sg] = i;
        seg_elem[sg] = (int32_t)(hi >> (gbits + pbits));
        seg_out[sg] = gbits ? (int32_t)(((hi >> pbits) & ((1ull << gbits) - 1)) == (uint64_t)K) : 0;
    }
    if (i == M - 1) seg_start[segpos[M]] = M;
}

__global__ void seg_tiles_kernel(const int64_t* __restrict__ seg_start, int64_t nseg,
                                 int64_t* __restrict__ seg_tiles)
{
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= nseg) return;
    seg_tiles[g] = (seg_start[g + 1] - seg_start[g] + kT - 1) / kT;
}

__global__ void row_map_kernel(const uint64_t* __restrict__ keys, const int64_t* __restrict__ segpos,
                               const int64_t* __restrict__ seg_start, const int64_t* __restrict__ seg_toff,
                               int64_t M, int32_t* __restrict__ row_slot)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= M) return;
    const int64_t sg = segpos[i + 1] - 1;
    const int64_t row = seg_toff[sg] * kT + (i - seg_start[sg]);
    row_slot[row] = (int32_t)(uint32_t)keys[i];
}

__global__ void tile_info_kernel(const int64_t* __restrict__ seg_start, const int64_t* __restrict__ seg_toff,
                                 const int32_t* __restrict__ seg_elem, int64_t nseg,
                                 int32_t* __restrict__ tile_n, int32_t* __restrict__ tile_seg,
                                 int32_t* __restrict__ tile_elem)
{
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= nseg) return;
    const int64_t len = seg_start[g + 1] - seg_start[g];
    for (int64_t t = seg_toff[g]; t < seg_toff[g + 1]; ++t) {
        const int64_t first = (t - seg_toff[g]) * kT;
        tile_n[t] = (int32_t)(len - first < kT ? len - first : kT);
        tile_seg[t] = (int32_t)g;
        tile_elem[t] = seg_elem[g];
    }
}

// One CTA per tile: gather rows, FP32 centroid (any centre serves the
// sphere test) and a radius that bounds every row's distance to it: the FP32
// sum of d squares of rounded differences is within (d/32 + 10) 2^-24 of the
// exact one, so sqrt(sum) (1 + (d + 64) 2^-23), rounded up, is an upper bound.
__global__ void __launch_bounds__(256) tile_prep_kernel(const float* __restrict__ X, int d, int64_t ld, int dp,
                                                        const int32_t* __restrict__ slot_point,
                                                        const int32_t* __restrict__ row_slot,
                                                        const int32_t* __restrict__ tile_n,
                                                        float* __restrict__ G, int32_t* __restrict__ row_pt,
                                                        float* __restrict__ cent, double* __restrict__ rad,
                                                        int* nonfinite)
{
    __shared__ float s_c[1024];
    __shared__ unsigned s_rad;
    const int t = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t row0 = (int64_t)t * kT;
    const int nt = tile_n[t];
    bool bad = false;
    for (int r = warp; r < kT; r += 8) {
        const int64_t row = row0 + r;
        const int slot = row_slot[row];
        const int64_t pt = slot >= 0 ? slot_point[slot] : -1;
        for (int k = lane; k < dp; k += 32) {
            float v = 0.f;
            if (pt >= 0 && k < d) {
                v = X[pt * ld + k];
                bad |= !isfinite(v);
            }
            G[row * dp + k] = v;
        }
        if (lane == 0) row_pt[row] = pt >= 0 ? (int32_t)pt : INT_MAX;
    }
    if (tid == 0) s_rad = 0u;
    if (__syncthreads_or(bad) && tid == 0) atomicOr(nonfinite, 1);
    for (int k = tid; k < dp; k += blockDim.x) {
        float s = 0.f;
        for (int r = 0; r < nt; ++r) s += G[(row0 + r) * dp + k];
        const float c = s / (float)nt;
        cent[(int64_t)t * dp + k] = c;
        if (k < 1024) s_c[k] = c;
    }
    __syncthreads();
    const float infl = 1.0f + (float)(d + 64) * 1.1920929e-7f;
    for (int r = warp; r < nt; r += 8) {
        const int64_t row = row0 + r;
        float s = 0.f;
        for (int k = lane; k < d; k += 32) {
            const float c = k < 1024 ? s_c[k] : cent[(int64_t)t * dp + k];
            const float u = G[row * dp + k] - c;
            s = fmaf(u, u, s);
        }
        for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) atomicMax(&s_rad, __float_as_uint(__fmul_ru(__fsqrt_ru(s), infl)));
    }
    __syncthreads();
    if (tid == 0) rad[t] = (double)__uint_as_float(s_rad);
}

// tile_prep_kernel for dp <= 256 with the tile held in registers: 16 warps,
// warp w owns rows w, w + 16, ..; lane l holds columns 4l .. 4l + 3 and
// 128 + 4l .. 131 + 4l of each. X is read once and G written once; centroid
// and radius come from the registers (same FP32 radius bound: each lane sums
// at most dp/32 squares before the shuffle tree).
constexpr int kPrepWarps = 16;
constexpr int kPrepRows = kT / kPrepWarps;

__global__ void __launch_bounds__(32 * kPrepWarps, 1) tile_prep_reg_kernel(
    const float* __restrict__ X, int d, int64_t ld, int dp, bool vec, const int32_t* __restrict__ slot_point,
    const int32_t* __restrict__ row_slot, const int32_t* __restrict__ tile_n, float* __restrict__ G,
    int32_t* __restrict__ row_pt, float* __restrict__ cent, double* __restrict__ rad, int* nonfinite)
{
    __shared__ float4 s_part[kPrepWarps][64];
    __shared__ float4 s_c[64];
    __shared__ unsigned s_rad;
    const int t = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t row0 = (int64_t)t * kT;
    const int nt = tile_n[t];
    float4 v[kPrepRows][2];
    bool bad = false;
    int pt_l = -1;                                  // lane i < kPrepRows: point of row warp + 16 i
    if (lane < kPrepRows) {
        const int64_t row = row0 + warp + kPrepWarps * lane;
        const int slot = row_slot[row];
        pt_l = slot >= 0 ? slot_point[slot] : -1;
        row_pt[row] = pt_l >= 0 ? pt_l : INT_MAX;
    }
#pragma unroll
    for (int i = 0; i < kPrepRows; ++i) {
        const int64_t pt = __shfl_sync(0xffffffffu, pt_l, i);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int k = h * 128 + 4 * lane;
            float4 x = make_float4(0.f, 0.f, 0.f, 0.f);
            if (pt >= 0 && k < d) {
                const float* src = X + pt * ld + k;
                if (vec && k + 3 < d) {
                    x = __ldg(reinterpret_cast<const float4*>(src));
                } else {
                    x.x = src[0];
                    if (k + 1 < d) x.y = src[1];
                    if (k + 2 < d) x.z = src[2];
                    if (k + 3 < d) x.w = src[3];
                }
            }
            v[i][h] = x;
        }
    }
    if (tid == 0) s_rad = 0u;
    float4 part[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        part[h] = make_float4(0.f, 0.f, 0.f, 0.f);
        const int k = h * 128 + 4 * lane;
#pragma unroll
        for (int i = 0; i < kPrepRows; ++i) {
            const float4 x = v[i][h];
            bad |= !isfinite(x.x) || !isfinite(x.y) || !isfinite(x.z) || !isfinite(x.w);
            if (G && k < dp)
                *reinterpret_cast<float4*>(G + (row0 + warp + kPrepWarps * i) * dp + k) = x;
            part[h].x += x.x;
            part[h].y += x.y;
            part[h].z += x.z;
            part[h].w += x.w;
        }
        s_part[warp][h * 32 + lane] = part[h];
    }
    if (__syncthreads_or(bad) && tid == 0) atomicOr(nonfinite, 1);
    if (tid < 64) {
        float4 c = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int w = 0; w < kPrepWarps; ++w) {
            const float4 q = s_part[w][tid];
            c.x += q.x; c.y += q.y; c.z += q.z; c.w += q.w;
        }
        const float inv = (float)nt;
        c.x /= inv; c.y /= inv; c.z /= inv; c.w /= inv;
        s_c[tid] = c;
        const int k = (tid >> 5) * 128 + 4 * (tid & 31);
        if (k < dp) *reinterpret_cast<float4*>(cent + (int64_t)t * dp + k) = c;
    }
    __syncthreads();
    const float infl = 1.0f + (float)(d + 64) * 1.1920929e-7f;
    const float4 c0 = s_c[lane], c1 = s_c[32 + lane];
#pragma unroll
    for (int i = 0; i < kPrepRows; ++i) {
        if (warp + kPrepWarps * i >= nt) continue;                 // warp-uniform
        float s = 0.f;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const float4 x = v[i][h], c = h ? c1 : c0;
            const int k = h * 128 + 4 * lane;
            float u;
            if (k < d)     { u = x.x - c.x; s = fmaf(u, u, s); }
            if (k + 1 < d) { u = x.y - c.y; s = fmaf(u, u, s); }
            if (k + 2 < d) { u = x.z - c.z; s = fmaf(u, u, s); }
            if (k + 3 < d) { u = x.w - c.w; s = fmaf(u, u, s); }
        }
        for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) atomicMax(&s_rad, __float_as_uint(__fmul_ru(__fsqrt_ru(s), infl)));
    }
    __syncthreads();
    if (tid == 0) rad[t] = (double)__uint_as_float(s_rad);
}

// Segment centre: the row-weighted mean of its tile centres, in double.
// With dp <= 512 the CTA splits the tiles over blockDim / dp thread groups
// (one thread per column in each) and adds the group sums at the end.
__global__ void __launch_bounds__(1024) seg_cent_kernel(const float* __restrict__ cent,
                                                        const int32_t* __restrict__ tile_n,
                                                        const int64_t* __restrict__ seg_toff, int dp,
                                                        float* __restrict__ seg_cent)
{
    __shared__ double s_sum[2][1024];
    const int64_t g = blockIdx.x;
    const int W = dp <= 512 ? (int)blockDim.x / dp : 1;
    const int w = dp <= 512 ? (int)threadIdx.x / dp : 0;
    const int64_t t0 = seg_toff[g], t1 = seg_toff[g + 1];
    for (int k0 = 0; k0 < dp; k0 += (dp <= 512 ? dp : (int)blockDim.x)) {
        const int k = dp <= 512 ? (int)threadIdx.x % dp : k0 + (int)threadIdx.x;
        double sum = 0.0, wt = 0.0;
        if (w < W && k < dp) {
            for (int64_t t = t0 + w; t < t1; t += W) {
                sum += (double)cent[t * dp + k] * (double)tile_n[t];
                wt += (double)tile_n[t];
            }
        }
        if (W > 1) {
            if (w < W) {
                s_sum[0][threadIdx.x] = sum;
                s_sum[1][threadIdx.x] = wt;
            }
            __syncthreads();
            if (w == 0) {
                for (int v = 1; v < W; ++v) {
                    sum += s_sum[0][v * dp + k];
                    wt += s_sum[1][v * dp + k];
                }
            }
            __syncthreads();
        }
        if (w == 0 && k < dp) seg_cent[g * dp + k] = (float)(sum / wt);
    }
}

// BF16 operands centred on the segment centre c (FP32): a = fl(x - c),
// hi = bf16(a), lo = bf16(a - hi) (a - hi is exact in FP32); |a|^2 summed in
// FP32 (lane partials of at most dp/32 squares, then a shuffle tree) and |a|
// rounded up; if rl is set, also |a - hi| (the residual the hi part leaves,
// summed the same way) rounded up; if tmax is set, the largest |a|^2, |a| and
// |a - hi| of the tile's rows (x, y, z) and the smallest |a|^2 of its valid
// rows (tn2min). A warp per row, a lane per 8
// consecutive columns (16-byte stores); rows come from G when it is set, else
// from X.
__global__ void __launch_bounds__(256) operand_kernel(const float* __restrict__ G, const float* __restrict__ X,
                                                      int64_t ld, bool xvec, const int32_t* __restrict__ row_pt,
                                                      int d, int dp, const int32_t* __restrict__ tile_n,
                                                      const int32_t* __restrict__ tile_seg,
                                                      const float* __restrict__ seg_cent,
                                                      __nv_bfloat16* __restrict__ Ah,
                                                      __nv_bfloat16* __restrict__ Al,
                                                      float* __restrict__ rn2, float* __restrict__ rn,
                                                      float* __restrict__ rl, float4* __restrict__ tmax,
                                                      float* __restrict__ tn2min, float norm_infl,
                                                      int* __restrict__ nonfinite = nullptr)
{
    const int t = blockIdx.x, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __shared__ unsigned smax[4];                          // non-negative floats compare as their bits
    if (threadIdx.x < 3) smax[threadIdx.x] = 0u;
    if (threadIdx.x == 3) smax[3] = 0x7f800000u;          // +inf: the smallest |a|^2 of the valid rows
    __syncthreads();
    const int nt = tile_n[t];
    const float* c = seg_cent + (int64_t)tile_seg[t] * dp;
    const bool vec = G ? true : xvec;
    for (int r = warp; r < kT; r += 8) {
        const int64_t row = (int64_t)t * kT + r;
        const bool valid = r < nt;
        const float* xr = !valid ? nullptr : (G ? G + row * dp : X + (int64_t)row_pt[row] * ld);
        float s = 0.f, sr = 0.f;
        for (int k0 = 0; k0 < dp; k0 += 256) {
            const int k = k0 + lane * 8;
            if (k >= dp) continue;
            float a[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) a[u] = 0.f;
            if (valid) {
                if (vec && k + 7 < d) {
                    const float4 x0 = *reinterpret_cast<const float4*>(xr + k);
                    const float4 x1 = *reinterpret_cast<const float4*>(xr + k + 4);
                    a[0] = x0.x; a[1] = x0.y; a[2] = x0.z; a[3] = x0.w;
                    a[4] = x1.x; a[5] = x1.y; a[6] = x1.z; a[7] = x1.w;
                } else {
#pragma unroll
                    for (int u = 0; u < 8; ++u) if (k + u < d) a[u] = xr[k + u];
                }
                const float4 c0 = *reinterpret_cast<const float4*>(c + k);
                const float4 c1 = *reinterpret_cast<const float4*>(c + k + 4);
                const float cc[8] = {c0.x, c0.y, c0.z, c0.w, c1.x, c1.y, c1.z, c1.w};
#pragma unroll
                for (int u = 0; u < 8; ++u) a[u] = k + u < d ? a[u] - cc[u] : 0.f;
            }
            uint32_t wh[4], wl[4];
#pragma unroll
            for (int u = 0; u < 8; u += 2) {
                const __nv_bfloat162 h = __floats2bfloat162_rn(a[u], a[u + 1]);
                const float2 hf = __bfloat1622float2(h);
                const float r0 = a[u] - hf.x, r1 = a[u + 1] - hf.y;          // exact
                const __nv_bfloat162 l = __floats2bfloat162_rn(r0, r1);
                wh[u >> 1] = *reinterpret_cast<const uint32_t*>(&h);
                wl[u >> 1] = *reinterpret_cast<const uint32_t*>(&l);
                s = fmaf(a[u], a[u], s);
                s = fmaf(a[u + 1], a[u + 1], s);
                sr = fmaf(r0, r0, sr);
                sr = fmaf(r1, r1, sr);
            }
            *reinterpret_cast<uint4*>(Ah + row * dp + k) = make_uint4(wh[0], wh[1], wh[2], wh[3]);
            if (Al) *reinterpret_cast<uint4*>(Al + row * dp + k) = make_uint4(wl[0], wl[1], wl[2], wl[3]);
        }
        for (int o = 16; o; o >>= 1) {
            s += __shfl_xor_sync(0xffffffffu, s, o);
            sr += __shfl_xor_sync(0xffffffffu, sr, o);
        }
        // a NaN or Inf in the row (or |row - c|^2 beyond FLT_MAX) leaves s non-finite
        if (nonfinite && lane == 0 && valid && !(s <= FLT_MAX)) *nonfinite = 1;
        if (lane == 0) {
            const float n1 = __fmul_ru(__fsqrt_ru(s), norm_infl), l1 = __fmul_ru(__fsqrt_ru(sr), norm_infl);
            rn2[row] = s;
            rn[row] = n1;
            if (rl) rl[row] = l1;
            if (tmax) {
                atomicMax(&smax[0], __float_as_uint(s));
                atomicMax(&smax[1], __float_as_uint(n1));
                atomicMax(&smax[2], __float_as_uint(l1));
                if (valid) atomicMin(&smax[3], __float_as_uint(s));
            }
        }
    }
    if (tmax) {
        __syncthreads();
        if (threadIdx.x == 0) {
            tmax[t] = make_float4(__uint_as_float(smax[0]), __uint_as_float(smax[1]), __uint_as_float(smax[2]), 0.f);
            tn2min[t] = __uint_as_float(smax[3]);
        }
    }
}

// FP8 E4M3 operands with one power-of-two scale per tile: the rows of tile t
// centred on its segment centre (a = fl(x - c), FP32 as for the BF16
// operands), M = the largest |a_k| of the tile, s = 2^e with 2^e > M / 448
// (frexp), hi = e4m3(a / s), lo = e4m3(a / s - hi) (the difference exact in
// FP32); per row |a - s hi| rounded up (frl); per tile (max |a|^2, max |a|,
// max frl, s) in ftmax. |a|^2 and |a| are those of the BF16 operands (same
// centred rows), read from tmax. A CTA per tile: the first sweep finds M,
// the second writes the bytes.
__global__ void __launch_bounds__(256) fp8_operand_kernel(const float* __restrict__ G, const float* __restrict__ X,
                                                          int64_t ld, bool xvec, const int32_t* __restrict__ row_pt,
                                                          int d, int dp, const int32_t* __restrict__ tile_n,
                                                          const int32_t* __restrict__ tile_seg,
                                                          const float* __restrict__ seg_cent,
                                                          const float4* __restrict__ tmax,
                                                          uint8_t* __restrict__ Fh, uint8_t* __restrict__ Fl,
                                                          float* __restrict__ frl, float4* __restrict__ ftmax,
                                                          float norm_infl)
{
    const int t = blockIdx.x, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nt = tile_n[t];
    const float* c = seg_cent + (int64_t)tile_seg[t] * dp;
    const bool vec = G ? true : xvec;
    __shared__ unsigned smax, lmax;
    if (threadIdx.x == 0) { smax = 0u; lmax = 0u; }
    __syncthreads();
    // a = fl(x - c) of 8 columns k .. k + 7 of row r (zero past d and for padding rows)
    auto centred = [&](int r, int k, float (&a)[8]) {
#pragma unroll
        for (int u = 0; u < 8; ++u) a[u] = 0.f;
        if (r >= nt) return;
        const int64_t row = (int64_t)t * kT + r;
        const float* xr = G ? G + row * dp : X + (int64_t)row_pt[row] * ld;
        if (vec && k + 7 < d) {
            const float4 x0 = *reinterpret_cast<const float4*>(xr + k);
            const float4 x1 = *reinterpret_cast<const float4*>(xr + k + 4);
            a[0] = x0.x; a[1] = x0.y; a[2] = x0.z; a[3] = x0.w;
            a[4] = x1.x; a[5] = x1.y; a[6] = x1.z; a[7] = x1.w;
        } else {
#pragma unroll
            for (int u = 0; u < 8; ++u) if (k + u < d) a[u] = xr[k + u];
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) a[u] = k + u < d ? a[u] - c[k + u] : 0.f;
    };
    float m = 0.f;
    for (int r = warp; r < kT; r += 8)
        for (int k = lane * 8; k < dp; k += 256) {
            float a[8];
            centred(r, k, a);
#pragma unroll
            for (int u = 0; u < 8; ++u) m = fmaxf(m, fabsf(a[u]));
        }
    for (int o = 16; o; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) atomicMax(&smax, __float_as_uint(m));
    __syncthreads();
    const float M = __uint_as_float(smax);
    int e = 0;
    if (M > 0.f) {
        frexpf(M / 448.f, &e);                            // M / 448 < 2^e, up to the division's rounding
        if (M * ldexpf(1.f, -e) >= 448.f) ++e;           // (exact test)
    }
    const float sc = ldexpf(1.f, e), inv = ldexpf(1.f, -e);
    for (int r = warp; r < kT; r += 8) {
        const int64_t row = (int64_t)t * kT + r;
        float sr = 0.f;
        for (int k = lane * 8; k < dp; k += 256) {
            float a[8];
            centred(r, k, a);
            uint32_t wh[2] = {0u, 0u}, wl[2] = {0u, 0u};
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const float x = a[u] * inv;                   // exact (power of two)
                const __nv_fp8_storage_t h = __nv_cvt_float_to_fp8(x, __NV_SATFINITE, __NV_E4M3);
                const float hf = __half2float(__half(__nv_cvt_fp8_to_halfraw(h, __NV_E4M3)));
                const float rr = x - hf;                      // exact
                const __nv_fp8_storage_t l = __nv_cvt_float_to_fp8(rr, __NV_SATFINITE, __NV_E4M3);
                wh[u >> 2] |= (uint32_t)h << (8 * (u & 3));
                wl[u >> 2] |= (uint32_t)l << (8 * (u & 3));
                sr = fmaf(rr, rr, sr);
            }
            *reinterpret_cast<uint2*>(Fh + row * dp + k) = make_uint2(wh[0], wh[1]);
            *reinterpret_cast<uint2*>(Fl + row * dp + k) = make_uint2(wl[0], wl[1]);
        }
        for (int o = 16; o; o >>= 1) sr += __shfl_xor_sync(0xffffffffu, sr, o);
        if (lane == 0) {
            const float l1 = __fmul_ru(__fmul_ru(__fsqrt_ru(sr), norm_infl), sc);
            frl[row] = l1;
            atomicMax(&lmax, __float_as_uint(l1));
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const float4 tm = tmax[t];
        ftmax[t] = make_float4(tm.x, tm.y, __uint_as_float(lmax), sc);
    }
}

__global__ void elem_tiles_kernel(const int32_t* __restrict__ tile_elem, int64_t T, int64_t E,
                                  int64_t* __restrict__ etile_off)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e > E) return;
    int64_t l = 0, r = T;                      // first tile whose element >= e
    while (l < r) {
        const int64_t m = (l + r) >> 1;
        if (tile_elem[m] < e) l = m + 1; else r = m;
    }
    etile_off[e] = l;
}

__global__ void cand_count_kernel(const int64_t* __restrict__ etile_off, int64_t E, int64_t* __restrict__ cnt)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= E) return;
    const int64_t T = etile_off[e + 1] - etile_off[e];
    cnt[e] = T * (T + 1) / 2;
}

// Upper bound of the distance between two centres from an FP32 sum of
// squares s: the sum of d rounded squares of rounded differences (lane
// partials, then a shuffle tree) is within (d/32 + 12) 2^-23 of the exact one.
__device__ __forceinline__ float dist_sum32(const float* __restrict__ x, const float* __restrict__ y, int dp,
                                            int lane)
{
    float s = 0.f;
    for (int k = lane; k < dp; k += 32) {
        const float u = x[k] - y[k];
        s = fmaf(u, u, s);
    }
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    return s;
}

// Segment radius: max over its tiles of |c_t - c_seg| + r_t (upper bounds).
__global__ void __launch_bounds__(1024) seg_rad_kernel(const float* __restrict__ cent,
                                                       const double* __restrict__ rad,
                                                       const float* __restrict__ seg_cent,
                                                       const int64_t* __restrict__ seg_toff, int dp,
                                                       double rel, double* __restrict__ seg_rad)
{
    __shared__ double s_max[32];
    const int64_t g = blockIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    double m = 0.0;
    for (int64_t t = seg_toff[g] + warp; t < seg_toff[g + 1]; t += nw) {
        const float ssum = dist_sum32(cent + t * dp, seg_cent + g * dp, dp, lane);
        m = fmax(m, sqrt((double)ssum * (1.0 + rel)) * (1.0 + 1e-15) + rad[t]);
    }
    if (lane == 0) s_max[warp] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < nw; ++w) m = fmax(m, s_max[w]);
        seg_rad[g] = m * (1.0 + 1e-15);
    }
}

__global__ void elem_segs_kernel(const int32_t* __restrict__ seg_elem, int64_t nseg, int64_t E,
                                 int64_t* __restrict__ eseg_off)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e > E) return;
    int64_t l = 0, r = nseg;                   // first segment whose element >= e
    while (l < r) {
        const int64_t m = (l + r) >> 1;
        if (seg_elem[m] < e) l = m + 1; else r = m;
    }
    eseg_off[e] = l;
}

// One CTA per tile a. Its centre is staged in shared memory; the segments of
// its element that cannot hold a point within eps of the segment of a (by
// segment spheres) are skipped whole; every tile b >= a of the others is
// classified by tile spheres: out, all-in, or mixed (tensor-core list when
// a and b share a segment, hence a centre, else CUDA-core list).
// Outlier tiles (rows that no pivot group took) have wide spheres, so their
// pairs with the tiles of other segments stay mixed. For each outlier tile t
// and each segment g of its element, tsm[t * smax + (g - first segment)] is a
// lower bound of the smallest distance from t's rows to g's centre (FP32
// lane-split sums with relative error at most rel, rounded down): no point of
// g lies within eps of t when that bound minus g's radius exceeds eps.
__global__ void __launch_bounds__(256) outlier_seg_kernel(const float* __restrict__ G, const float* __restrict__ X,
                                                          int64_t ld, int d, int dp, const int32_t* __restrict__ row_pt,
                                                          const int32_t* __restrict__ tile_n,
                                                          const int32_t* __restrict__ tile_seg,
                                                          const int32_t* __restrict__ tile_elem,
                                                          const int32_t* __restrict__ seg_out,
                                                          const int64_t* __restrict__ eseg_off,
                                                          const float* __restrict__ seg_cent, double rel, int smax,
                                                          float* __restrict__ tsm)
{
    __shared__ float s_min[8];
    const int t = blockIdx.x;
    if (!seg_out[tile_seg[t]]) return;                   // whole block
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int e = tile_elem[t];
    const int64_t g0 = eseg_off[e], g1 = eseg_off[e + 1];
    const int nt = tile_n[t];
    for (int64_t g = g0; g < g1 && g - g0 < smax; ++g) {
        const float* c = seg_cent + g * dp;
        float mn = INFINITY;
        for (int r = warp; r < nt; r += 8) {
            const int64_t row = (int64_t)t * kT + r;
            const float* x = G ? G + row * dp : X + (int64_t)row_pt[row] * ld;
            float ss = 0.f;
            for (int k = lane; k < d; k += 32) {
                const float u = x[k] - c[k];
                ss = fmaf(u, u, ss);
            }
            for (int o = 16; o; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
            mn = fminf(mn, ss);
        }
        if (lane == 0) s_min[warp] = mn;
        __syncthreads();
        if (threadIdx.x == 0) {
            float m = s_min[0];
            for (int w = 1; w < 8; ++w) m = fminf(m, s_min[w]);
            tsm[(int64_t)t * smax + (g - g0)] = __double2float_rd(sqrt((double)m * (1.0 - rel)) * (1.0 - 1e-15));
        }
        __syncthreads();
    }
}

constexpr int kMaxSegList = 1024;

// Tile-pair classification by bounding spheres, with the centres of up to
// kClsA tiles A of one segment per CTA (in shared memory) against one tile B
// per lane: each
// tile B's centre is read once per CTA instead of once per tile A, and a
// lane keeps the kClsA sums itself (a sequential FMA chain over dp columns:
// the true squared distance lies in [ssum c_lo, ssum c_hi]). CTA c takes block c of the blocks of kClsA tiles
// that blk_off (exclusive prefix of ceil(tiles / kClsA) per segment) numbers.
constexpr int kClsA = 8;

__global__ void __launch_bounds__(256) classify_blk_kernel(const int64_t* __restrict__ blk_off, int64_t n_seg,
                                                           const int64_t* __restrict__ eseg_off,
                                                           const int64_t* __restrict__ seg_toff,
                                                           const int32_t* __restrict__ seg_elem,
                                                           const float* __restrict__ seg_cent,
                                                           const double* __restrict__ seg_rad,
                                                           const float* __restrict__ cent,
                                                           const double* __restrict__ rad,
                                                           const int32_t* __restrict__ seg_out, int dp, double rel,
                                                           double c_lo, double c_hi, double eps_out, double eps_in,
                                                           int use_tc,
                                                           const float* __restrict__ tsm, int smax,
                                                           int2* __restrict__ l_in, int2* __restrict__ l_tc,
                                                           int2* __restrict__ l_simt,
                                                           unsigned long long* __restrict__ counts)
{
    extern __shared__ float4 s_ca4[];                    // [kClsA][dp / 4]
    __shared__ int s_seg[kMaxSegList];
    __shared__ int s_nseg;
    __shared__ unsigned long long s_out;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t c = blockIdx.x;
    if (c >= blk_off[n_seg]) return;
    // the block's segment: the last g with blk_off[g] <= c
    int64_t lo = 0, hi = n_seg - 1;
    while (lo < hi) {
        const int64_t mid = (lo + hi + 1) / 2;
        if (blk_off[mid] <= c) lo = mid;
        else hi = mid - 1;
    }
    const int64_t ga = lo;
    const int64_t ta0 = seg_toff[ga] + (c - blk_off[ga]) * kClsA;
    const int64_t left_a = seg_toff[ga + 1] - ta0;
    const int na = (int)(left_a < kClsA ? left_a : kClsA);
    const int dq = dp / 4;
    for (int k = threadIdx.x; k < kClsA * dq; k += blockDim.x) {
        const int a = k / dq, kk = k % dq;
        s_ca4[k] = reinterpret_cast<const float4*>(cent + (ta0 + (a < na ? a : 0)) * dp)[kk];
    }
    const int64_t g_end = eseg_off[seg_elem[ga] + 1];
    const int64_t g_first = eseg_off[seg_elem[ga]];
    if (threadIdx.x == 0) { s_nseg = 0; s_out = 0ull; }
    __syncthreads();
    const bool listed = g_end - ga <= kMaxSegList;
    for (int64_t gb = ga + warp; gb < g_end && listed; gb += 8) {
        bool keep = gb == ga;
        if (!keep) {
            const float ssum = dist_sum32(seg_cent + ga * dp, seg_cent + gb * dp, dp, lane);
            const double Dlo = sqrt((double)ssum * (1.0 - rel)) * (1.0 - 1e-15);
            keep = !(Dlo - seg_rad[ga] - seg_rad[gb] > eps_out);
        }
        if (lane == 0) {
            if (keep) s_seg[atomicAdd(&s_nseg, 1)] = (int)gb;
            else atomicAdd(&s_out, (unsigned long long)na * (unsigned long long)(seg_toff[gb + 1] - seg_toff[gb]));
        }
    }
    __syncthreads();
    const int nlist = listed ? s_nseg : (int)(g_end - ga);
    double ra[kClsA];
#pragma unroll
    for (int a = 0; a < kClsA; ++a) ra[a] = a < na ? rad[ta0 + a] : 0.0;
    int64_t n_out = 0;
    for (int li = 0; li < nlist; ++li) {
        const int64_t gb = listed ? s_seg[li] : ga + li;
        const int64_t t0 = gb == ga ? ta0 : seg_toff[gb], t1 = seg_toff[gb + 1];
        const int gbi = (int)gb;
        for (int64_t tb0 = t0 + warp * 32; tb0 < t1; tb0 += 8 * 32) {
            const int64_t tb = tb0 + lane;
            const bool live = tb < t1;
            const float4* cb = reinterpret_cast<const float4*>(cent + (live ? tb : t0) * dp);
            float acc[kClsA];
#pragma unroll
            for (int a = 0; a < kClsA; ++a) acc[a] = 0.f;
#pragma unroll 4
            for (int kk = 0; kk < dq; ++kk) {
                const float4 b = __ldg(cb + kk);
#pragma unroll
                for (int a = 0; a < kClsA; ++a) {
                    const float4 x = s_ca4[a * dq + kk];
                    float u = x.x - b.x;
                    acc[a] = fmaf(u, u, acc[a]);
                    u = x.y - b.y;
                    acc[a] = fmaf(u, u, acc[a]);
                    u = x.z - b.z;
                    acc[a] = fmaf(u, u, acc[a]);
                    u = x.w - b.w;
                    acc[a] = fmaf(u, u, acc[a]);
                }
            }
            const double rb = live ? rad[tb] : 0.0;
#pragma unroll
            for (int a = 0; a < kClsA; ++a) {
                const int64_t ta = ta0 + a;
                const bool pair = live && a < na && !(gb == ga && tb < ta);
                // squared bounds with outward rounding (no square root):
                // D^2 >= ssum c_lo, D^2 <= ssum c_hi for the true centre distance D
                const double ssum = tb == ta ? 0.0 : (double)acc[a];
                const double t_out = __dadd_ru(__dadd_ru(eps_out, ra[a]), rb);
                const double w_in = __dsub_rd(__dsub_rd(eps_in, ra[a]), rb);
                int cls;
                if (!pair) cls = -2;                      // (no memory reads for lanes without a pair)
                else if (__dmul_rd(ssum, c_lo) > __dmul_ru(t_out, t_out)) cls = -1;
                else if (w_in > 0.0 && __dadd_ru(__dmul_ru(ssum, c_hi), 1e-36) < __dmul_rd(w_in, w_in))
                    cls = kListAllIn;                         // (1e-36: the FP32 subnormal roundings)
                else if (tsm && gbi != (int)ga &&
                         ((seg_out[ga] && (double)tsm[ta * smax + (gbi - g_first)] - seg_rad[gbi] > eps_out) ||
                          (seg_out[gbi] && (double)tsm[tb * smax + (ga - g_first)] - seg_rad[ga] > eps_out)))
                    cls = -1;
                else if (use_tc && gbi == (int)ga) cls = kListTC;
                else cls = kListSimt;
                if (cls == -1) ++n_out;
                // one atomic per warp and list: the lanes of a class take
                // consecutive slots
#pragma unroll
                for (int k3 = 0; k3 < kListCount; ++k3) {
                    const unsigned m = __ballot_sync(0xffffffffu, cls == k3);
                    if (!m) continue;
                    const int leader = __ffs(m) - 1;
                    unsigned long long at = 0;
                    if (lane == leader) at = atomicAdd(&counts[k3], (unsigned long long)__popc(m));
                    at = __shfl_sync(0xffffffffu, at, leader);
                    if (cls == k3) {
                        int2* dst = k3 == kListAllIn ? l_in : (k3 == kListTC ? l_tc : l_simt);
                        dst[at + __popc(m & ((1u << lane) - 1u))] = make_int2((int)ta, (int)tb);
                    }
                }
            }
        }
    }
    if (n_out) atomicAdd(&s_out, (unsigned long long)n_out);
    __syncthreads();
    if (threadIdx.x == 0 && s_out) atomicAdd(&counts[3], s_out);
}

// Bin of a tile pair's statistic s = (|c_a - c_b|^2 + r_a^2 + r_b^2) / eps^2
// (tile centres and radii): where rows concentrate around their tile centre,
// as in high dimension, s is about the typical squared distance of the
// pair's rows over eps^2, so s near 1 means rows whose distances straddle
// eps. bin = floor(8 (log2 s + 4)) clamped to [0, kPairBins), in FP32 (a
// binning, decided by no result; FP64 on one lane would cost the FP64 pipe a
// whole warp's issue). A warp per pair.
__global__ void __launch_bounds__(256) pair_bin_kernel(const int2* __restrict__ pairs, int64_t n,
                                                       const float* __restrict__ cent,
                                                       const double* __restrict__ rad, int dp, float inv_eps2,
                                                       uint8_t* __restrict__ bin)
{
    const int lane = threadIdx.x & 31;
    const int64_t q = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (q >= n) return;
    const int2 tp = pairs[q];
    const int a = tp.x, b = tp.y & kPairTileMask;
    const float* ca = cent + (int64_t)a * dp;
    const float* cb = cent + (int64_t)b * dp;
    float d2 = 0.f;
    for (int k = lane; k < dp; k += 32) {
        const float t = ca[k] - cb[k];
        d2 = fmaf(t, t, d2);
    }
    for (int o = 16; o; o >>= 1) d2 += __shfl_xor_sync(0xffffffffu, d2, o);
    if (lane == 0) {
        const float ra = (float)rad[a], rb = (float)rad[b];
        const float s = (d2 + ra * ra + rb * rb) * inv_eps2;
        const float l = s > 0.f ? 8.f * (__log2f(s) + 4.f) : 0.f;        // NaN and below 0: bin 0
        bin[q] = (uint8_t)(!(l >= 0.f) ? 0 : (l >= (float)kPairBins ? kPairBins - 1 : (int)l));
    }
}

// Per bin of the sampled pairs (pair j of the sample is pairs[j * stride] of
// the list): cnt[2 b] sampled pairs, cnt[2 b + 1] of them with a deferred block.
__global__ void sample_bin_kernel(const uint32_t* __restrict__ mask, int64_t n_s, const uint8_t* __restrict__ bin,
                                  int64_t stride, unsigned long long* __restrict__ cnt)
{
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n_s) return;
    const int b = bin[j * stride];
    atomicAdd(&cnt[2 * b], 1ull);
    if (mask[j]) atomicAdd(&cnt[2 * b + 1], 1ull);
}

// flag[q] = chosen[bin[q]]
__global__ void bin_flag_kernel(const uint8_t* __restrict__ bin, int64_t n, const uint8_t* __restrict__ chosen,
                                int32_t* __restrict__ flag)
{
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q < n) flag[q] = chosen[bin[q]];
}

// Stable partition: the flagged pairs first (pos = their exclusive prefix,
// pos[n] their number), then the others, each in list order.
__global__ void partition_kernel(const int2* __restrict__ in, int64_t n, const int32_t* __restrict__ flag,
                                 const int64_t* __restrict__ pos, int2* __restrict__ out)
{
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    out[flag[q] ? pos[q] : pos[n] + (q - pos[q])] = in[q];
}

// blocks of kClsA tiles per segment: cnt[g] = ceil(tiles(g) / kClsA)
__global__ void seg_blocks_kernel(const int64_t* __restrict__ seg_toff, int64_t n_seg, int64_t* __restrict__ cnt)
{
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g < n_seg) cnt[g] = (seg_toff[g + 1] - seg_toff[g] + kClsA - 1) / kClsA;
}

}  // namespace

cudaError_t pair_bins(const TileLayout& L, const int2* pairs, int64_t n, int dp, double eps, uint8_t* bin,
                      cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    pair_bin_kernel<<<grid_for(n * 32), 256, 0, s>>>(pairs, n, L.tile_cent.as<float>(), L.tile_rad.as<double>(),
                                                     dp, (float)(1.0 / (eps * eps)), bin);
    note_launch();
    return cudaGetLastError();
}

cudaError_t sample_bins(const uint32_t* mask, int64_t n_s, const uint8_t* bin, int64_t stride,
                        unsigned long long* cnt, cudaStream_t s)
{
    MGB_TRY(cudaMemsetAsync(cnt, 0, sizeof(unsigned long long) * 2 * kPairBins, s));
    if (n_s == 0) return cudaSuccess;
    sample_bin_kernel<<<grid_for(n_s), 256, 0, s>>>(mask, n_s, bin, stride, cnt);
    note_launch();
    return cudaGetLastError();
}

cudaError_t partition_pairs(const int2* pairs, const uint8_t* bin, const uint8_t* chosen, int64_t n, int2* out,
                            Buf* pos, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    Buf flag;
    MGB_TRY(flag.alloc(sizeof(int32_t) * n, s));
    MGB_TRY(pos->alloc(sizeof(int64_t) * (n + 1), s));
    bin_flag_kernel<<<grid_for(n), 256, 0, s>>>(bin, n, chosen, flag.as<int32_t>());
    note_launch();
    MGB_TRY(cudaGetLastError());
    MGB_TRY(exclusive_scan_i32_to_i64(flag.as<int32_t>(), pos->as<int64_t>(), n, s));
    partition_kernel<<<grid_for(n), 256, 0, s>>>(pairs, n, flag.as<int32_t>(), pos->as<int64_t>(), out);
    note_launch();
    return cudaGetLastError();
}

cudaError_t pivot_alloc(int64_t n, int dp, PivotSet* P, cudaStream_t alloc_s)
{
    P->K = (int)std::min<int64_t>(kPiv, n);
    cudaError_t e = P->Pv.alloc(sizeof(float) * (size_t)P->K * dp, alloc_s);
    if (e == cudaSuccess) e = P->piv.alloc(sizeof(int32_t) * n, alloc_s);
    if (e == cudaSuccess) e = P->pd2.alloc(sizeof(float) * n, alloc_s);
    return e;
}

int pivot_assign(const float* X, int64_t n, int32_t d, int64_t ld, int dp, bool bf16, int num_sms, PivotSet* P,
                 cudaStream_t s)
{
    const int K = P->K;
    if (!P->split) {
        pivot_gather_kernel<<<K, 128, 0, s>>>(X, n, d, ld, dp, K, P->Pv.as<float>());
        note_launch();
    }
    if (bf16) {
        const PivotSplit pre{P->c.as<float>(), P->xh.p, P->xn2.as<float>()};
        const int rc = assign_pivots_tc(X, n, d, ld, dp, P->Pv.as<float>(), K, num_sms, P->piv.as<int32_t>(),
                                        P->pd2.as<float>(), s, P->split ? &pre : nullptr);
        if (rc) return rc;
    } else {
        assign_kernel<<<grid_for(n, kT), 256, 0, s>>>(X, n, d, ld, P->Pv.as<float>(), dp, K, P->piv.as<int32_t>(),
                                                     P->pd2.as<float>());
        note_launch();
    }
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error(std::string("pivot assignment: ") + cudaGetErrorString(e));
        return MAPPER_ECUDA;
    }
    return MAPPER_OK;
}

int pivot_prepare(const float* X, int64_t n, int32_t d, int64_t ld, int dp, bool host, PivotSet* P, cudaStream_t s)
{
#define PK(expr)                                                                      \
    do {                                                                              \
        cudaError_t e_ = (expr);                                                      \
        if (e_ != cudaSuccess) {                                                      \
            set_error(std::string("pivot_prepare: ") + cudaGetErrorString(e_));       \
            return e_ == cudaErrorMemoryAllocation ? MAPPER_ENOMEM : MAPPER_ECUDA;    \
        }                                                                             \
    } while (0)
    const int K = P->K;
    const int64_t rows = div_up(n, kT) * kT;
    PK(P->c.alloc(sizeof(float) * dp, s));
    PK(P->xh.alloc(sizeof(uint16_t) * (size_t)rows * dp, s));
    PK(P->xn2.alloc(sizeof(float) * rows, s));
    if (rows > n) {
        PK(cudaMemsetAsync(static_cast<uint16_t*>(P->xh.p) + n * dp, 0, sizeof(uint16_t) * (size_t)(rows - n) * dp, s));
        PK(cudaMemsetAsync(P->xn2.as<float>() + n, 0, sizeof(float) * (rows - n), s));
    }
    if (!host) {
        pivot_gather_kernel<<<K, 128, 0, s>>>(X, n, d, ld, dp, K, P->Pv.as<float>());
        pivot_mean_kernel<<<1, 256, 0, s>>>(P->Pv.as<float>(), K, dp, P->c.as<float>());
        note_launch(2);
        PK(cudaGetLastError());
    } else {
        // the same rows and sums on the host (X there); two pageable copies
        std::vector<float> pv((size_t)K * dp, 0.f), c(dp, 0.f);
        for (int k = 0; k < K; ++k) {
            const float* x = X + ((int64_t)k * n / K) * ld;
            for (int j = 0; j < d; ++j) pv[(size_t)k * dp + j] = x[j];
        }
        for (int j = 0; j < dp; ++j) {
            float sum = 0.f;
            for (int k = 0; k < K; ++k) sum += pv[(size_t)k * dp + j];
            c[j] = sum / (float)K;
        }
        PK(cudaMemcpyAsync(P->Pv.p, pv.data(), sizeof(float) * pv.size(), cudaMemcpyHostToDevice, s));
        PK(cudaMemcpyAsync(P->c.p, c.data(), sizeof(float) * dp, cudaMemcpyHostToDevice, s));
        PK(cudaStreamSynchronize(s));                  // the host vectors go out of scope
    }
    P->split = true;
    return MAPPER_OK;
#undef PK
}

int build_tiles(const float* X, int64_t n, int32_t d, int64_t ld, int dp, const int32_t* slot_point,
                const int32_t* slot_elem, int64_t M, int64_t E, double tau, bool bf16, int num_sms,
                TileLayout* L, int* nonfinite, cudaStream_t s, const PivotSet* pre)
{
#define TK(expr)                                                                      \
    do {                                                                              \
        cudaError_t e_ = (expr);                                                      \
        if (e_ != cudaSuccess) {                                                      \
            set_error(std::string("build_tiles: ") + cudaGetErrorString(e_));         \
            return e_ == cudaErrorMemoryAllocation ? MAPPER_ENOMEM : MAPPER_ECUDA;    \
        }                                                                             \
    } while (0)
    PivotSet own;
    if (!pre) {
        TK(pivot_alloc(n, dp, &own, s));
        const int rc = pivot_assign(X, n, d, ld, dp, bf16, num_sms, &own, s);
        if (rc) return rc;
        pre = &own;
    }
    const int K = pre->K;
    const Buf& Pv = pre->Pv;
    const Buf& piv = pre->piv;
    const Buf& pd2 = pre->pd2;
    Buf gid, ngrp, adj;
    TK(gid.alloc(sizeof(int32_t) * kPiv, s));
    TK(ngrp.alloc(sizeof(int32_t), s));
    TK(adj.alloc(sizeof(unsigned) * kPiv * (kPiv / 32), s));
    TK(cudaMemsetAsync(adj.p, 0, sizeof(unsigned) * kPiv * (kPiv / 32), s));
    const float tau2 = (float)(tau * tau);
    pivot_adj_kernel<<<grid_for((int64_t)K * K * 32, 256), 256, 0, s>>>(Pv.as<float>(), dp, K, tau2,
                                                                       adj.as<unsigned>());
    group_kernel<<<1, 256, 0, s>>>(adj.as<unsigned>(), K, gid.as<int32_t>(), ngrp.as<int32_t>());
    note_launch(2);
    TK(cudaGetLastError());

    int ebits = bits_for(E), gbits = bits_for(K + 1), pbits = bits_for(K);
    if (ebits + gbits + pbits > 32) pbits = 0;
    if (ebits + gbits + pbits > 32) gbits = 0;
    Buf keys, tmp, flag, segpos;
    TK(keys.alloc(sizeof(uint64_t) * M, s));
    TK(tmp.alloc(sizeof(uint64_t) * M, s));
    key_kernel<<<grid_for(M), 256, 0, s>>>(slot_point, slot_elem, M, piv.as<int32_t>(), pd2.as<float>(),
                                          gid.as<int32_t>(), tau2, K, gbits, pbits, keys.as<uint64_t>());
    note_launch();
    TK(cudaGetLastError());
    TK(radix_sort_u64(keys.as<uint64_t>(), tmp.as<uint64_t>(), M, 32, 32 + ebits + gbits + pbits, s));
    TK(flag.alloc(sizeof(int32_t) * M, s));
    TK(segpos.alloc(sizeof(int64_t) * (M + 1), s));
    seg_flag_kernel<<<grid_for(M), 256, 0, s>>>(keys.as<uint64_t>(), M, 32 + pbits, flag.as<int32_t>());
    note_launch();
    TK(cudaGetLastError());
    TK(exclusive_scan_i32_to_i64(flag.as<int32_t>(), segpos.as<int64_t>(), M, s));
    int64_t nseg = 0;
    int32_t ng = 0;
    TK(cudaMemcpyAsync(&nseg, segpos.as<int64_t>() + M, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    TK(cudaMemcpyAsync(&ng, ngrp.p, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    TK(cudaStreamSynchronize(s));
    L->n_seg = nseg;
    L->n_groups = gbits ? ng : 1;

    Buf seg_start, seg_tiles;
    Buf& seg_elem = L->seg_elem;
    Buf& seg_toff = L->seg_toff;
    TK(seg_start.alloc(sizeof(int64_t) * (nseg + 1), s));
    TK(seg_elem.alloc(sizeof(int32_t) * nseg, s));
    TK(L->seg_outlier.alloc(sizeof(int32_t) * nseg, s));
    TK(seg_tiles.alloc(sizeof(int64_t) * nseg, s));
    TK(seg_toff.alloc(sizeof(int64_t) * (nseg + 1), s));
    seg_start_kernel<<<grid_for(M), 256, 0, s>>>(keys.as<uint64_t>(), flag.as<int32_t>(), segpos.as<int64_t>(),
                                                M, gbits, pbits, K, seg_start.as<int64_t>(),
                                                seg_elem.as<int32_t>(), L->seg_outlier.as<int32_t>());
    seg_tiles_kernel<<<grid_for(nseg), 256, 0, s>>>(seg_start.as<int64_t>(), nseg, seg_tiles.as<int64_t>());
    note_launch(2);
    TK(cudaGetLastError());
    TK(exclusive_scan_i64(seg_tiles.as<int64_t>(), seg_toff.as<int64_t>(), nseg, s));
    int64_t T = 0;
    TK(cudaMemcpyAsync(&T, seg_toff.as<int64_t>() + nseg, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    TK(cudaStreamSynchronize(s));
    L->T = T;
    L->R = T * kT;
    const int64_t R = L->R;

    TK(L->row_slot.alloc(sizeof(int32_t) * R, s));
    TK(L->row_pt.alloc(sizeof(int32_t) * R, s));
    // FP32 rows gathered in layout order for the CUDA-core passes (and the
    // tile statistics of rows wider than 256); the tensor-core path reads the
    // few rows it rechecks from X instead
    if (!bf16 || dp > 256) TK(L->G.alloc(sizeof(float) * (size_t)R * dp, s));
    TK(L->tile_n.alloc(sizeof(int32_t) * T, s));
    TK(L->tile_seg.alloc(sizeof(int32_t) * T, s));
    TK(L->tile_elem.alloc(sizeof(int32_t) * T, s));
    TK(L->tile_cent.alloc(sizeof(float) * (size_t)T * dp, s));
    TK(L->tile_rad.alloc(sizeof(double) * T, s));
    TK(L->seg_cent.alloc(sizeof(float) * (size_t)nseg * dp, s));
    TK(cudaMemsetAsync(L->row_slot.p, 0xff, sizeof(int32_t) * R, s));
    row_map_kernel<<<grid_for(M), 256, 0, s>>>(keys.as<uint64_t>(), segpos.as<int64_t>(), seg_start.as<int64_t>(),
                                              seg_toff.as<int64_t>(), M, L->row_slot.as<int32_t>());
    tile_info_kernel<<<grid_for(nseg), 256, 0, s>>>(seg_start.as<int64_t>(), seg_toff.as<int64_t>(),
                                                    seg_elem.as<int32_t>(), nseg, L->tile_n.as<int32_t>(),
                                                    L->tile_seg.as<int32_t>(), L->tile_elem.as<int32_t>());
    if (dp <= 256) {
        const bool vec = ld % 4 == 0 && ((uintptr_t)X & 15) == 0;
        tile_prep_reg_kernel<<<(unsigned)T, 32 * kPrepWarps, 0, s>>>(
            X, d, ld, dp, vec, slot_point, L->row_slot.as<int32_t>(), L->tile_n.as<int32_t>(), L->G.as<float>(),
            L->row_pt.as<int32_t>(), L->tile_cent.as<float>(), L->tile_rad.as<double>(), nonfinite);
    } else {
        tile_prep_kernel<<<(unsigned)T, 256, 0, s>>>(X, d, ld, dp, slot_point, L->row_slot.as<int32_t>(),
                                                     L->tile_n.as<int32_t>(), L->G.as<float>(),
                                                     L->row_pt.as<int32_t>(), L->tile_cent.as<float>(),
                                                     L->tile_rad.as<double>(), nonfinite);
    }
    seg_cent_kernel<<<(unsigned)nseg, 1024, 0, s>>>(L->tile_cent.as<float>(), L->tile_n.as<int32_t>(),
                                                  seg_toff.as<int64_t>(), dp, L->seg_cent.as<float>());
    note_launch(4);
    TK(cudaGetLastError());
    TK(L->seg_rad.alloc(sizeof(double) * nseg, s));
    const double rel = (double)(dp / 32 + 12) * std::ldexp(1.0, -23);
    seg_rad_kernel<<<(unsigned)nseg, 1024, 0, s>>>(L->tile_cent.as<float>(), L->tile_rad.as<double>(),
                                                 L->seg_cent.as<float>(), seg_toff.as<int64_t>(), dp, rel,
                                                 L->seg_rad.as<double>());
    note_launch();
    TK(cudaGetLastError());
    if (bf16) {
        TK(L->Ah.alloc(sizeof(__nv_bfloat16) * (size_t)R * dp, s));
        TK(L->Al.alloc(sizeof(__nv_bfloat16) * (size_t)R * dp, s));
        TK(L->rn2.alloc(sizeof(float) * R, s));
        TK(L->rn.alloc(sizeof(float) * R, s));
        TK(L->rl.alloc(sizeof(float) * R, s));
        TK(L->tmax.alloc(sizeof(float4) * T, s));
        TK(L->tn2min.alloc(sizeof(float) * T, s));
        const float norm_infl = 1.0f + (float)(dp / 32 + 16) * 5.9604645e-8f;
        const bool xvec = ld % 4 == 0 && ((uintptr_t)X & 15) == 0;
        operand_kernel<<<(unsigned)T, 256, 0, s>>>(L->G.as<float>(), X, ld, xvec, L->row_pt.as<int32_t>(), d, dp,
                                                   L->tile_n.as<int32_t>(),
                                                   L->tile_seg.as<int32_t>(), L->seg_cent.as<float>(),
                                                   L->Ah.as<__nv_bfloat16>(), L->Al.as<__nv_bfloat16>(),
                                                   L->rn2.as<float>(), L->rn.as<float>(), L->rl.as<float>(),
                                                   L->tmax.as<float4>(), L->tn2min.as<float>(), norm_infl);
        note_launch();
        TK(cudaGetLastError());
    }
    return MAPPER_OK;
}

int fp8_operands(TileLayout* L, const float* X, int64_t ld, int d, int dp, cudaStream_t s)
{
    if (L->T == 0 || L->Fh.p) return MAPPER_OK;
    const int64_t R = L->R, T = L->T;
    cudaError_t e = L->Fh.alloc((size_t)R * dp, s);
    if (e == cudaSuccess) e = L->Fl.alloc((size_t)R * dp, s);
    if (e == cudaSuccess) e = L->frl.alloc(sizeof(float) * R, s);
    if (e == cudaSuccess) e = L->ftmax.alloc(sizeof(float4) * T, s);
    if (e == cudaSuccess) {
        const float norm_infl = 1.0f + (float)(dp / 32 + 16) * 5.9604645e-8f;
        const bool xvec = ld % 4 == 0 && ((uintptr_t)X & 15) == 0;
        fp8_operand_kernel<<<(unsigned)T, 256, 0, s>>>(L->G.as<float>(), X, ld, xvec, L->row_pt.as<int32_t>(), d, dp,
                                                       L->tile_n.as<int32_t>(), L->tile_seg.as<int32_t>(),
                                                       L->seg_cent.as<float>(), L->tmax.as<float4>(),
                                                       L->Fh.as<uint8_t>(), L->Fl.as<uint8_t>(), L->frl.as<float>(),
                                                       L->ftmax.as<float4>(), norm_infl);
        note_launch();
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        set_error(std::string("fp8_operands: ") + cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? MAPPER_ENOMEM : MAPPER_ECUDA;
    }
    return MAPPER_OK;
}

cudaError_t centred_operands(const float* X, int64_t ld, int d, int dp, const int32_t* row_pt, const int32_t* tile_n,
                             const int32_t* tile_cent, const float* cents, int64_t T, void* Ah, void* Al, float* rn2,
                             float* rn, cudaStream_t s, int* nonfinite)
{
    if (T == 0) return cudaSuccess;
    const float norm_infl = 1.0f + (float)(dp / 32 + 16) * 5.9604645e-8f;
    const bool xvec = ld % 4 == 0 && ((uintptr_t)X & 15) == 0;
    operand_kernel<<<(unsigned)T, 256, 0, s>>>(nullptr, X, ld, xvec, row_pt, d, dp, tile_n, tile_cent, cents,
                                               static_cast<__nv_bfloat16*>(Ah), static_cast<__nv_bfloat16*>(Al), rn2,
                                               rn, nullptr, nullptr, nullptr, norm_infl, nonfinite);
    note_launch();
    return cudaGetLastError();
}

// Operands for tile pairs of one element but two segments (two centres):
// rows centred on their element's centre (the row-weighted mean of its tile
// centres), split as by operand_kernel. |a| is larger than with the segment
// centre, so the screen's error bound, and its band, are wider; pairs far
// apart are still decided at once.
int cross_operands(const TileLayout& L, const float* X, int64_t ld, int d, int dp, int64_t E, Buf* Ah, Buf* Al,
                   Buf* rn2, Buf* rn, Buf* rl, Buf* tmax, Buf* tn2min, cudaStream_t s)
{
#define XK(expr)                                                                      \
    do {                                                                              \
        cudaError_t e_ = (expr);                                                      \
        if (e_ != cudaSuccess) {                                                      \
            set_error(std::string("cross_operands: ") + cudaGetErrorString(e_));      \
            return e_ == cudaErrorMemoryAllocation ? MAPPER_ENOMEM : MAPPER_ECUDA;    \
        }                                                                             \
    } while (0)
    const int64_t R = L.R, T = L.T;
    Buf etile_off, ecent;
    XK(etile_off.alloc(sizeof(int64_t) * (E + 1), s));
    XK(ecent.alloc(sizeof(float) * (size_t)E * dp, s));
    XK(Ah->alloc(sizeof(__nv_bfloat16) * (size_t)R * dp, s));
    XK(Al->alloc(sizeof(__nv_bfloat16) * (size_t)R * dp, s));
    XK(rn2->alloc(sizeof(float) * R, s));
    XK(rn->alloc(sizeof(float) * R, s));
    XK(rl->alloc(sizeof(float) * R, s));
    XK(tmax->alloc(sizeof(float4) * T, s));
    XK(tn2min->alloc(sizeof(float) * T, s));
    elem_tiles_kernel<<<grid_for(E + 1), 256, 0, s>>>(L.tile_elem.as<int32_t>(), T, E, etile_off.as<int64_t>());
    seg_cent_kernel<<<(unsigned)E, 1024, 0, s>>>(L.tile_cent.as<float>(), L.tile_n.as<int32_t>(),
                                               etile_off.as<int64_t>(), dp, ecent.as<float>());
    const float norm_infl = 1.0f + (float)(dp / 32 + 16) * 5.9604645e-8f;
    const bool xvec = ld % 4 == 0 && ((uintptr_t)X & 15) == 0;
    operand_kernel<<<(unsigned)T, 256, 0, s>>>(L.G.as<float>(), X, ld, xvec, L.row_pt.as<int32_t>(), d, dp,
                                               L.tile_n.as<int32_t>(), L.tile_elem.as<int32_t>(), ecent.as<float>(),
                                               Ah->as<__nv_bfloat16>(), Al->as<__nv_bfloat16>(), rn2->as<float>(),
                                               rn->as<float>(), rl->as<float>(), tmax->as<float4>(),
                                               tn2min->as<float>(), norm_infl);
    note_launch(3);
    XK(cudaGetLastError());
    return MAPPER_OK;
#undef XK
}

int classify_pairs(const TileLayout& L, const float* X, int64_t ld, int d, int dp, int64_t E, double eps, bool use_tc,
                   PairLists* P, cudaStream_t s, double eps_all_in)
{
    if (!(eps_all_in > 0.0)) eps_all_in = eps;
    Buf etile_off, cnt, cand_off, counts, eseg_off;
    TK(etile_off.alloc(sizeof(int64_t) * (E + 1), s));
    TK(eseg_off.alloc(sizeof(int64_t) * (E + 1), s));
    TK(cnt.alloc(sizeof(int64_t) * std::max<int64_t>(E, 1), s));
    TK(cand_off.alloc(sizeof(int64_t) * (E + 1), s));
    TK(counts.alloc(sizeof(unsigned long long) * 4, s));
    TK(cudaMemsetAsync(counts.p, 0, sizeof(unsigned long long) * 4, s));
    elem_tiles_kernel<<<grid_for(E + 1), 256, 0, s>>>(L.tile_elem.as<int32_t>(), L.T, E, etile_off.as<int64_t>());
    elem_segs_kernel<<<grid_for(E + 1), 256, 0, s>>>(L.seg_elem.as<int32_t>(), L.n_seg, E, eseg_off.as<int64_t>());
    cand_count_kernel<<<grid_for(E), 256, 0, s>>>(etile_off.as<int64_t>(), E, cnt.as<int64_t>());
    note_launch(3);
    TK(cudaGetLastError());
    TK(exclusive_scan_i64(cnt.as<int64_t>(), cand_off.as<int64_t>(), E, s));
    int64_t C = 0;
    TK(cudaMemcpyAsync(&C, cand_off.as<int64_t>() + E, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    TK(cudaStreamSynchronize(s));
    P->n_candidates = C;
    for (int k = 0; k < kListCount; ++k) TK(P->list[k].alloc(sizeof(int2) * std::max<int64_t>(C, 1), s));
    // blocks of kClsA tiles A per segment for classify_blk_kernel
    Buf blk_cnt, blk_off;
    TK(blk_cnt.alloc(sizeof(int64_t) * std::max<int64_t>(L.n_seg, 1), s));
    TK(blk_off.alloc(sizeof(int64_t) * (L.n_seg + 1), s));
    if (L.n_seg > 0) {
        seg_blocks_kernel<<<grid_for(L.n_seg), 256, 0, s>>>(L.seg_toff.as<int64_t>(), L.n_seg,
                                                            blk_cnt.as<int64_t>());
        note_launch();
        TK(cudaGetLastError());
    }
    TK(exclusive_scan_i64(blk_cnt.as<int64_t>(), blk_off.as<int64_t>(), L.n_seg, s));
    const unsigned cls_grid = (unsigned)(div_up(L.T, kClsA) + L.n_seg);
    const size_t cls_smem = sizeof(float) * kClsA * dp;
    if (cls_smem > 48 * 1024)
        TK(cudaFuncSetAttribute(classify_blk_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cls_smem));
    // segment distances: lane partial sums and a shuffle tree (dist_sum32);
    // tile distances: one FMA chain over dp columns
    const double rel = (double)(dp / 32 + 12) * std::ldexp(1.0, -23);
    // |ssum - D^2| <= rel_tile D^2, so D^2 is in [ssum c_lo, ssum c_hi] with
    // c_lo <= 1 - rel_tile and c_hi >= 1 / (1 - rel_tile) (outward rounding)
    const double rel_tile = (double)(dp + 24) * std::ldexp(1.0, -24);
    const double c_lo = std::nextafter(1.0 - rel_tile, 0.0);
    const double c_hi = std::nextafter(1.0 / (1.0 - rel_tile), INFINITY);
    const double eps_out = eps * (1.0 + 1e-9), eps_in = eps_all_in * (1.0 - 1e-9);
    auto classify = [&](const float* tsm, int smax) -> int {
        classify_blk_kernel<<<cls_grid, 256, cls_smem, s>>>(
            blk_off.as<int64_t>(), L.n_seg, eseg_off.as<int64_t>(), L.seg_toff.as<int64_t>(),
            L.seg_elem.as<int32_t>(), L.seg_cent.as<float>(), L.seg_rad.as<double>(), L.tile_cent.as<float>(),
            L.tile_rad.as<double>(), L.seg_outlier.as<int32_t>(), dp, rel, c_lo, c_hi, eps_out, eps_in, use_tc ? 1 : 0,
            tsm, smax, P->list[kListAllIn].as<int2>(), P->list[kListTC].as<int2>(), P->list[kListSimt].as<int2>(),
            counts.as<unsigned long long>());
        note_launch();
        TK(cudaGetLastError());
        return MAPPER_OK;
    };
    if (C > 0) {
        const int rc = classify(nullptr, 0);
        if (rc) return rc;
    }
    unsigned long long h[4] = {0, 0, 0, 0};
    TK(cudaMemcpyAsync(h, counts.p, sizeof(h), cudaMemcpyDeviceToHost, s));
    TK(cudaStreamSynchronize(s));
    // Many mixed pairs across segments (a cover element holding scattered
    // points): bound the outlier tiles' distance to every segment of their
    // element and classify again, certifying more pairs all-out.
    if (C > 0 && (int64_t)h[kListSimt] * 32 >= L.R) {
        const int smax = L.n_groups + 1;
        Buf tsm;
        TK(tsm.alloc(sizeof(float) * (size_t)L.T * smax, s));
        outlier_seg_kernel<<<(unsigned)L.T, 256, 0, s>>>(L.G.as<float>(), X, ld, d, dp, L.row_pt.as<int32_t>(),
                                                          L.tile_n.as<int32_t>(), L.tile_seg.as<int32_t>(),
                                                          L.tile_elem.as<int32_t>(), L.seg_outlier.as<int32_t>(),
                                                          eseg_off.as<int64_t>(), L.seg_cent.as<float>(), rel, smax,
                                                          tsm.as<float>());
        note_launch();
        TK(cudaMemsetAsync(counts.p, 0, sizeof(unsigned long long) * 4, s));
        const int rc = classify(tsm.as<float>(), smax);
        if (rc) return rc;
        TK(cudaMemcpyAsync(h, counts.p, sizeof(h), cudaMemcpyDeviceToHost, s));
        TK(cudaStreamSynchronize(s));
    }
    for (int k = 0; k < kListCount; ++k) P->n[k] = (int64_t)h[k];
    P->n_out = (int64_t)h[3];
    return MAPPER_OK;
#undef TK
}

}  // namespace mgb
