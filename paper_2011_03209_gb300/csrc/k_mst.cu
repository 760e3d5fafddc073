// k_mst.cu -- single-linkage forest of every cover element.
//
// "Mapper Interactive" §5: Lum et al. cluster each cover element by single
// linkage, where the tool uses DBSCAN. Single linkage cut at a height h gives
// the connected components of the h-graph; the whole dendrogram up to eps is
// the minimum spanning forest of the element's eps-graph (pairs with d2 <=
// eps^2, the DBSCAN distance). Edges are ordered by the key (d2, smaller
// point, larger point), so the forest is unique when distances tie.
//
// Borůvka rounds over the tile pairs of the element (those not certified
// all-out at eps by the tile layout's bounding spheres), every round on CUDA
// cores:
//   1. the FP32 sum of squared differences s of every pair whose rows lie in
//      two components and which may be within eps (s <= the FP32 screen's
//      upper limit): the smallest s of each component (atomicMin);
//   2. the same pairs again: those whose s lies within the FP32 error of
//      their component's smallest s (|s - d2| <= eta d2 + tiny, so the
//      lightest edge is among them) get their FP64 d2 by the defining
//      expression, and, when d2 <= eps^2, their key competes for the
//      component's lightest edge (a 128-bit atomic minimum of (d2, slots));
//   3. every component adds its lightest edge to the forest (once for an
//      edge two components chose) and joins the other component
//      (lock-free union-find whose roots are the smallest point index).
// Within an element the cover slots are in ascending point order, so slot
// indices order the ties as point indices do. Tile pairs whose rows all share
// one component drop out of later rounds.
#include <cfloat>
#include <climits>
#include <cmath>
#include <string>

#include "../../include/mapper.h"
#include "dbscan.cuh"

namespace mgb {

namespace {

constexpr int kT = kTile;
constexpr int kK = 32;
constexpr int kPad = 132;

__device__ __forceinline__ int mfind(int32_t* parent, int x)
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

// Joins two components; the root of larger point index goes under the other.
__device__ __forceinline__ void munion(int32_t* parent, const int32_t* row_pt, int a, int b)
{
    while (true) {
        a = mfind(parent, a);
        b = mfind(parent, b);
        if (a == b) return;
        if (row_pt[a] < row_pt[b]) { const int t = a; a = b; b = t; }
        if (atomicCAS(&parent[a], a, b) == a) return;
    }
}

__device__ __forceinline__ double msf_sqdist(const float* __restrict__ x, const float* __restrict__ y, int d)
{
    double s = 0.0;
    for (int k = 0; k < d; ++k) {
        const double t = __dsub_rn((double)x[k], (double)y[k]);
        s = __dadd_rn(s, __dmul_rn(t, t));
    }
    return s;
}

// 128-bit keys: y = bits of d2 (non-negative doubles order as their bits),
// x = (smaller slot << 32) | larger slot; the minimum is lexicographic in (y, x).
__device__ __forceinline__ bool key_less(ulonglong2 a, ulonglong2 b)
{
    return a.y < b.y || (a.y == b.y && a.x < b.x);
}

__device__ __forceinline__ ulonglong2 cas128(ulonglong2* addr, ulonglong2 cmp, ulonglong2 val)
{
    unsigned long long lo, hi;
    asm volatile(
        "{\n .reg .b128 c, v, o;\n mov.b128 c, {%2, %3};\n mov.b128 v, {%4, %5};\n"
        " atom.relaxed.gpu.global.cas.b128 o, [%6], c, v;\n mov.b128 {%0, %1}, o;\n}"
        : "=l"(lo), "=l"(hi)
        : "l"(cmp.x), "l"(cmp.y), "l"(val.x), "l"(val.y), "l"(addr)
        : "memory");
    return make_ulonglong2(lo, hi);
}

__device__ __forceinline__ void key_min(ulonglong2* addr, ulonglong2 k)
{
    const volatile unsigned long long* va = reinterpret_cast<const volatile unsigned long long*>(addr);
    ulonglong2 cur = make_ulonglong2(va[0], va[1]);       // may be torn: the CAS returns the true value
    while (key_less(k, cur)) {
        const ulonglong2 old = cas128(addr, cur, k);
        if (old.x == cur.x && old.y == cur.y) return;
        cur = old;
    }
}

struct MsfArgs {
    PassArgs A;                     // rows (G or X via row_pt), dp, d, pairs, tile_n, eps2, hi_thr
    const int32_t* root;            // component root row of every row (this round)
    const int32_t* row_slot;
    unsigned* cmin;                 // per root row: the smallest FP32 s of its candidate pairs (as bits)
    ulonglong2* ckey;               // per root row: the lightest candidate edge's key
    float eta, tiny;                // |s - d2| <= eta d2 + tiny
    unsigned long long* oob;        // checked build: indices found out of range
};

// STAGE 1: component minima of s; STAGE 2: exact keys of the pairs near them.
template <int STAGE>
__global__ void __launch_bounds__(256, 2) msf_screen_kernel(const MsfArgs M)
{
    __shared__ __align__(16) float As[kK][kPad];
    __shared__ __align__(16) float Bs[kK][kPad];
    __shared__ int s_root[2 * kT];
    const PassArgs& A = M.A;
    const int tid = threadIdx.x;
    if (A.n_dev && (unsigned long long)blockIdx.x >= *A.n_dev) return;
    const int2 p = A.pairs[blockIdx.x];
    int ta = p.x, tb = p.y & kPairTileMask;
    bool ok = true;
    if (!MGB_IN_RANGE(ta, A.n_tiles, M.oob) || !MGB_IN_RANGE(tb, A.n_tiles, M.oob)) {
        ta = tb = 0;                                       // checked build: counted, then skipped
        ok = false;
    }
    const int64_t sa = (int64_t)ta * kT, sb = (int64_t)tb * kT;
    const int na = ok ? A.tile_n[ta] : 0, nb = ok ? A.tile_n[tb] : 0;
    const bool diag = ta == tb;
    s_root[tid] = tid < kT ? (tid < na ? M.root[sa + tid] : -1) : (tid - kT < nb ? M.root[sb + tid - kT] : -2);

    const int tx = tid & 15, ty = tid >> 4;
    float acc[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
    for (int k0 = 0; k0 < A.dp; k0 += kK) {
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const int idx = tid + 256 * v;
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

    float rmin[8], cmin[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) { rmin[i] = INFINITY; cmin[i] = INFINITY; }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int r = i < 4 ? ty * 4 + i : 64 + ty * 4 + i - 4;
        const int ra = s_root[r];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int c = j < 4 ? tx * 4 + j : 64 + tx * 4 + j - 4;
            const int rb = s_root[kT + c];
            const float s = acc[i][j];
            // a pair of rows in two components that may lie within eps (diagonal: once)
            if (r >= na || c >= nb || (diag && c <= r) || ra == rb || !(s <= A.hi_thr)) continue;
            if (STAGE == 1) {
                rmin[i] = fminf(rmin[i], s);
                cmin[j] = fminf(cmin[j], s);
            } else {
                // thresholds: s of the lightest edge is at most m (1 + eta)^2 / (1 - eta) + 2 tiny
                const float ma = __uint_as_float(M.cmin[ra]), mb = __uint_as_float(M.cmin[rb]);
                const float lim_a = __fmaf_ru(ma, 4.f * M.eta, __fadd_ru(ma, 2.f * M.tiny));
                const float lim_b = __fmaf_ru(mb, 4.f * M.eta, __fadd_ru(mb, 2.f * M.tiny));
                const bool ca = s <= lim_a, cb = s <= lim_b;
                if (!ca && !cb) continue;
                const double d2 = msf_sqdist(pass_row(A, sa + r), pass_row(A, sb + c), A.d);
                if (!(d2 <= A.eps2)) continue;
                const unsigned s1 = (unsigned)M.row_slot[sa + r], s2 = (unsigned)M.row_slot[sb + c];
                const ulonglong2 key = make_ulonglong2(
                    ((unsigned long long)min(s1, s2) << 32) | (unsigned long long)max(s1, s2),
                    (unsigned long long)__double_as_longlong(d2));
                if (ca) key_min(&M.ckey[ra], key);
                if (cb) key_min(&M.ckey[rb], key);
            }
        }
    }
    if (STAGE == 1) {
        // one atomic per row and per column of this thread (roots differ per row)
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int r = i < 4 ? ty * 4 + i : 64 + ty * 4 + i - 4;
            if (rmin[i] < INFINITY) atomicMin(&M.cmin[s_root[r]], __float_as_uint(rmin[i]));
            const int c = i < 4 ? tx * 4 + i : 64 + tx * 4 + i - 4;
            if (cmin[i] < INFINITY) atomicMin(&M.cmin[s_root[kT + c]], __float_as_uint(cmin[i]));
        }
    }
}

// Each component root with a candidate adds its lightest edge (once when
// both components chose the same edge) and joins the other component.
__global__ void msf_pick_kernel(const int32_t* __restrict__ root, const ulonglong2* __restrict__ ckey,
                                const int32_t* __restrict__ slot_row, const int32_t* __restrict__ slot_point,
                                const int32_t* __restrict__ slot_elem, const int32_t* __restrict__ row_pt, int64_t R,
                                int32_t* parent, int32_t* __restrict__ e_u, int32_t* __restrict__ e_v,
                                int32_t* __restrict__ e_elem, int32_t* __restrict__ e_su, int32_t* __restrict__ e_sv,
                                double* __restrict__ e_d2, unsigned long long* n_edges, unsigned long long* picks)
{
    const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= R || root[x] != (int32_t)x) return;
    const ulonglong2 k = ckey[x];
    if (k.y == ~0ull) return;
    const int s1 = (int)(k.x >> 32), s2 = (int)(k.x & 0xffffffffull);
    const int r1 = slot_row[s1], r2 = slot_row[s2];
    const int other = root[r1] == (int32_t)x ? root[r2] : root[r1];
    atomicAdd(picks, 1ull);
    const ulonglong2 ko = ckey[other];
    if (!(ko.x == k.x && ko.y == k.y) || x < other) {
        const unsigned long long at = atomicAdd(n_edges, 1ull);
        e_u[at] = slot_point[s1];
        e_v[at] = slot_point[s2];
        e_elem[at] = slot_elem[s1];
        e_su[at] = s1;
        e_sv[at] = s2;
        e_d2[at] = __longlong_as_double((long long)k.y);
    }
    munion(parent, row_pt, (int)x, other);
}

__global__ void msf_flatten_kernel(int32_t* parent, const int32_t* __restrict__ row_slot, int64_t R,
                                   int32_t* __restrict__ root, unsigned* __restrict__ cmin,
                                   ulonglong2* __restrict__ ckey)
{
    const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= R) return;
    root[x] = row_slot[x] >= 0 ? mfind(parent, (int)x) : (int32_t)x;
    cmin[x] = 0x7f800000u;                                 // +inf
    ckey[x] = make_ulonglong2(~0ull, ~0ull);
}

__global__ void msf_init_kernel(const int32_t* __restrict__ row_slot, int64_t R, int32_t* __restrict__ parent,
                                int32_t* __restrict__ slot_row)
{
    const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= R) return;
    parent[x] = (int32_t)x;
    if (row_slot[x] >= 0) slot_row[row_slot[x]] = (int32_t)x;
}

// Per tile: the smallest and largest root of its valid rows.
__global__ void msf_tile_roots_kernel(const int32_t* __restrict__ root, const int32_t* __restrict__ tile_n,
                                      int64_t T, int2* __restrict__ tr)
{
    const int64_t t = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (t >= T) return;
    int lo = INT_MAX, hi = INT_MIN;
    for (int r = lane; r < tile_n[t]; r += 32) {
        const int v = root[t * kT + r];
        lo = min(lo, v);
        hi = max(hi, v);
    }
    for (int o = 16; o; o >>= 1) {
        lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    if (lane == 0) tr[t] = make_int2(lo, hi);
}

// Keeps the tile pairs whose rows are not all in one component.
__global__ void msf_filter_kernel(const int2* __restrict__ pairs, int64_t n, const unsigned long long* __restrict__ n_in,
                                  const int2* __restrict__ tr, int2* __restrict__ out, unsigned long long* n_out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || (n_in && (unsigned long long)i >= *n_in)) return;
    const int2 p = pairs[i];
    const int2 a = tr[p.x], b = tr[p.y & kPairTileMask];
    if (a.x == a.y && b.x == b.y && a.x == b.x) return;
    out[atomicAdd(n_out, 1ull)] = p;
}

// Single-linkage cut in cover-slot space: slots of one component (edges
// with d2 <= h^2) take the smallest slot as root (slot order = point order
// within an element).
__global__ void cut_init_kernel(int64_t M, int32_t* __restrict__ parent)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < M) parent[i] = (int32_t)i;
}

__device__ __forceinline__ void slot_union(int32_t* parent, int a, int b)
{
    while (true) {
        a = mfind(parent, a);
        b = mfind(parent, b);
        if (a == b) return;
        if (a < b) { const int t = a; a = b; b = t; }
        if (atomicCAS(&parent[a], a, b) == a) return;
    }
}

__global__ void cut_union_kernel(const int32_t* __restrict__ e_su, const int32_t* __restrict__ e_sv,
                                 const double* __restrict__ e_d2, int64_t n, double h2, int32_t* parent)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && e_d2[i] <= h2) slot_union(parent, e_su[i], e_sv[i]);
}

__global__ void cut_labels_kernel(int32_t* parent, const int32_t* __restrict__ slot_point, int64_t M,
                                  int32_t* __restrict__ lab, int32_t* __restrict__ is_root,
                                  int32_t* __restrict__ is_member, int64_t* __restrict__ slot_label,
                                  uint8_t* __restrict__ core)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= M) return;
    const int r = mfind(parent, (int)i);
    lab[i] = r;
    slot_label[i] = slot_point[r];
    is_root[i] = r == (int)i;
    is_member[i] = 1;
    core[i] = 1;
}

}  // namespace

int msf_forest(const PassArgs& a, const int32_t* row_slot, const int32_t* slot_point, const int32_t* slot_elem,
               int64_t M, int64_t R, int64_t T, int64_t n_pairs, ForestOut* out, cudaStream_t s)
{
#define MK(expr)                                                                   \
    do {                                                                           \
        cudaError_t e_ = (expr);                                                   \
        if (e_ != cudaSuccess) {                                                   \
            set_error(std::string("single linkage: ") + cudaGetErrorString(e_));   \
            return e_ == cudaErrorMemoryAllocation ? MAPPER_ENOMEM : MAPPER_ECUDA;  \
        }                                                                          \
    } while (0)
    out->n = 0;
    const int64_t cap = std::max<int64_t>(M, 1);
    MK(out->u.alloc(sizeof(int32_t) * cap, s));
    MK(out->v.alloc(sizeof(int32_t) * cap, s));
    MK(out->elem.alloc(sizeof(int32_t) * cap, s));
    MK(out->su.alloc(sizeof(int32_t) * cap, s));
    MK(out->sv.alloc(sizeof(int32_t) * cap, s));
    MK(out->d2.alloc(sizeof(double) * cap, s));
    if (R == 0 || n_pairs == 0) return MAPPER_OK;           // no pair can lie within eps
    Buf parent, root, slot_row, cmin, ckey, tr, lists[2], counts;
    MK(parent.alloc(sizeof(int32_t) * R, s));
    MK(root.alloc(sizeof(int32_t) * R, s));
    MK(slot_row.alloc(sizeof(int32_t) * cap, s));
    MK(cmin.alloc(sizeof(unsigned) * R, s));
    MK(ckey.alloc(sizeof(ulonglong2) * R, s));
    MK(tr.alloc(sizeof(int2) * std::max<int64_t>(T, 1), s));
    MK(lists[0].alloc(sizeof(int2) * std::max<int64_t>(n_pairs, 1), s));
    MK(lists[1].alloc(sizeof(int2) * std::max<int64_t>(n_pairs, 1), s));
    MK(counts.alloc(sizeof(unsigned long long) * 5, s));       // n_edges, picks, list lengths, index checks
    unsigned long long* n_edges = counts.as<unsigned long long>();
    unsigned long long* picks = n_edges + 1;
    unsigned long long* len = n_edges + 2;
    unsigned long long* oob = n_edges + 4;
    MK(cudaMemsetAsync(counts.p, 0, sizeof(unsigned long long) * 5, s));
    const unsigned gR = (unsigned)div_up(R, 256);
    msf_init_kernel<<<gR, 256, 0, s>>>(row_slot, R, parent.as<int32_t>(), slot_row.as<int32_t>());
    MK(cudaGetLastError());
    MK(cudaMemcpyAsync(lists[0].p, a.pairs, sizeof(int2) * n_pairs, cudaMemcpyDeviceToDevice, s));
    MK(cudaMemcpyAsync(len, &n_pairs, sizeof(unsigned long long), cudaMemcpyHostToDevice, s));
    MsfArgs m{};
    m.A = a;
    m.root = root.as<int32_t>();
    m.row_slot = row_slot;
    m.cmin = cmin.as<unsigned>();
    m.ckey = ckey.as<ulonglong2>();
    m.eta = (float)(1.5 * (a.d + 4) * std::ldexp(1.0, -24));
    m.oob = oob;
    m.tiny = (float)(3.0 * (a.d + 2) * std::ldexp(1.0, -149));
    if (m.tiny == 0.f) m.tiny = std::ldexp(1.0f, -149);
    int cur = 0;
    for (int round = 0; round < 64; ++round) {
        msf_flatten_kernel<<<gR, 256, 0, s>>>(parent.as<int32_t>(), row_slot, R, root.as<int32_t>(), cmin.as<unsigned>(),
                                             ckey.as<ulonglong2>());
        // drop the tile pairs whose rows are all in one component
        msf_tile_roots_kernel<<<(unsigned)div_up(T, 8), 256, 0, s>>>(root.as<int32_t>(), a.tile_n, T, tr.as<int2>());
        MK(cudaMemsetAsync(len + 1 - cur, 0, sizeof(unsigned long long), s));
        msf_filter_kernel<<<(unsigned)div_up(n_pairs, 256), 256, 0, s>>>(lists[cur].as<int2>(), n_pairs, len + cur,
                                                                           tr.as<int2>(), lists[1 - cur].as<int2>(),
                                                                           len + 1 - cur);
        cur = 1 - cur;
        MK(cudaMemsetAsync(picks, 0, sizeof(unsigned long long), s));
        note_launch(3);
        m.A.pairs = lists[cur].as<int2>();
        m.A.n_dev = len + cur;
        msf_screen_kernel<1><<<(unsigned)n_pairs, 256, 0, s>>>(m);
        msf_screen_kernel<2><<<(unsigned)n_pairs, 256, 0, s>>>(m);
        msf_pick_kernel<<<gR, 256, 0, s>>>(root.as<int32_t>(), ckey.as<ulonglong2>(), slot_row.as<int32_t>(), slot_point,
                                           slot_elem, a.row_pt, R, parent.as<int32_t>(), out->u.as<int32_t>(),
                                           out->v.as<int32_t>(), out->elem.as<int32_t>(), out->su.as<int32_t>(),
                                           out->sv.as<int32_t>(), out->d2.as<double>(), n_edges, picks);
        note_launch(3);
        MK(cudaGetLastError());
        unsigned long long h = 0;
        MK(cudaMemcpyAsync(&h, picks, sizeof(h), cudaMemcpyDeviceToHost, s));
        MK(cudaStreamSynchronize(s));
        if (h == 0) break;
    }
    unsigned long long ne = 0, h_oob = 0;
    MK(cudaMemcpyAsync(&ne, n_edges, sizeof(ne), cudaMemcpyDeviceToHost, s));
    MK(cudaMemcpyAsync(&h_oob, oob, sizeof(h_oob), cudaMemcpyDeviceToHost, s));
    MK(cudaStreamSynchronize(s));
    out->n = (int64_t)ne;
    if (h_oob) {
        set_error("single linkage: a device-side index check failed");
        return MAPPER_EINTERNAL;
    }
#undef MK
    return MAPPER_OK;
}

int msf_cut(const ForestOut& f, const int32_t* slot_point, int64_t M, double h, int32_t* lab, int32_t* is_root,
            int32_t* is_member, int64_t* slot_label, uint8_t* core, cudaStream_t s)
{
    if (M == 0) return MAPPER_OK;
    Buf parent;
    cudaError_t e = parent.alloc(sizeof(int32_t) * M, s);
    if (e == cudaSuccess) {
        cut_init_kernel<<<(unsigned)div_up(M, 256), 256, 0, s>>>(M, parent.as<int32_t>());
        if (f.n > 0)
            cut_union_kernel<<<(unsigned)div_up(f.n, 256), 256, 0, s>>>(f.su.as<int32_t>(), f.sv.as<int32_t>(),
                                                                         f.d2.as<double>(), f.n, h * h,
                                                                         parent.as<int32_t>());
        cut_labels_kernel<<<(unsigned)div_up(M, 256), 256, 0, s>>>(parent.as<int32_t>(), slot_point, M, lab, is_root,
                                                                     is_member, slot_label, core);
        note_launch(3);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        set_error(std::string("single-linkage cut: ") + cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? MAPPER_ENOMEM : MAPPER_ECUDA;
    }
    return MAPPER_OK;
}

}  // namespace mgb
