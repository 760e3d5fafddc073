// k_dbscan.cu -- per-cover-element DBSCAN and graph assembly.
//
// "Mapper Interactive" §3: DBSCAN(eps, minPts) clusters the points of each
// cover element; §4.3 parallelises over elements and precomputes each
// element's distance matrix. Here the distance matrix is never stored: every
// element's membership slots are cut into 128-row tiles and each pair of
// tiles (a <= b) is one CTA that recomputes the tile's squared distances and
// consumes them at once:
//   pass 1  neighbour counts      count[s] = |N(s)|           (core: >= minPts)
//   pass 2  core-core unions      lock-free union-find, root = smallest slot
//   pass 3  border assignment     smallest root among core neighbours
// Screen: the FP32 sum of squared differences has a rigorous relative error
// bound eta (see pass thresholds in capi.cu); a pair is "in" when the screen
// value is <= eps^2 (1 - eta), "out" when > eps^2 (1 + eta), and otherwise
// it is re-decided in FP64 with the defining expression (k ascending, one
// rounding per operation), so decisions equal the FP64 definition exactly.
#include <cfloat>
#include <cmath>
#include <climits>

#include "dbscan.cuh"

namespace mgb {

namespace {

constexpr int kT = 128;        // tile rows
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

// q-th entry of the upper triangle (a <= b) of a T x T grid, row-major
__device__ __forceinline__ void decode_pair(int64_t q, int64_t T, int* ta, int* tb)
{
    int64_t l = 0, r = T - 1;                  // largest a with cum(a) <= q
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

__device__ __forceinline__ int gfind(int32_t* parent, int x)
{
    volatile int32_t* par = parent;
    int p = par[x];
    while (p != x) {
        const int gp = par[p];
        if (gp != p) par[x] = gp;             // path halving: any ancestor is a valid parent
        x = p;
        p = par[x];
    }
    return x;
}

__device__ __forceinline__ void gunion(int32_t* parent, int a, int b)
{
    while (true) {
        a = gfind(parent, a);
        b = gfind(parent, b);
        if (a == b) return;
        if (a < b) { const int t = a; a = b; b = t; }
        // link the larger root under the smaller: roots stay component minima
        if (atomicCAS(&parent[a], a, b) == a) return;
    }
}

__device__ __forceinline__ int lfind(volatile int* par, int x)
{
    int p = par[x];
    while (p != x) { x = p; p = par[x]; }
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
    __device__ __forceinline__ bool operator()(float s, int64_t slot_a, int64_t slot_b,
                                               bool count_tie) const
    {
        if (s <= A.lo_thr) return true;
        if (s > A.hi_thr && s <= FLT_MAX) return false;
        const double d2 = exact_sqdist(A.G + slot_a * A.dp, A.G + slot_b * A.dp, A.d);
        atomicAdd(&A.stats[kStatBand], 1ull);
        if (count_tie && fabs(d2 - A.eps2) <= A.tie_thr) atomicAdd(&A.stats[kStatTies], 1ull);
        return d2 <= A.eps2;
    }
};

template <int MODE>
__global__ void __launch_bounds__(256, 2) simt_pass_kernel(const PassArgs A)
{
    __shared__ __align__(16) float As[kK][kPad];
    __shared__ __align__(16) float Bs[kK][kPad];
    __shared__ int s_aux[2 * kT];              // pass 1: column counts; 2: local parents; 3: best roots
    __shared__ int s_root[2 * kT];             // pass 3: roots of A (0..127) and B (128..255)
    __shared__ unsigned char s_core[2 * kT];

    const int tid = threadIdx.x;
    const int64_t e = upper_bound_i64(A.pair_off, (int64_t)A.E + 1, (int64_t)blockIdx.x) - 1;
    const int64_t q = (int64_t)blockIdx.x - A.pair_off[e];
    const int64_t base = A.elem_off[e], ne = A.elem_off[e + 1] - base;
    const int64_t T = (ne + kT - 1) / kT;
    int ta, tb;
    decode_pair(q, T, &ta, &tb);
    const bool diag = ta == tb;
    const int64_t sa = base + (int64_t)ta * kT, sb = base + (int64_t)tb * kT;
    const int na = (int)(ne - (int64_t)ta * kT < kT ? ne - (int64_t)ta * kT : kT);
    const int nb = (int)(ne - (int64_t)tb * kT < kT ? ne - (int64_t)tb * kT : kT);

    if (MODE == 1) {
        if (tid < kT) s_aux[tid] = 0;
    } else {
        bool ca = false, cb = false;
        if (tid < kT) {
            ca = tid < na && A.core[sa + tid];
            s_core[tid] = ca;
        } else {
            const int c = tid - kT;
            cb = c < nb && A.core[sb + c];
            s_core[tid] = cb;
        }
        const int n_core_a = __syncthreads_count(tid < kT && ca);
        const int n_core_b = __syncthreads_count(tid >= kT && cb);
        if (MODE == 2) {
            if (n_core_a == 0 || n_core_b == 0) return;
            s_aux[tid] = tid;
        } else {
            const bool work = (n_core_b > 0 && n_core_a < na) || (!diag && n_core_a > 0 && n_core_b < nb);
            if (!work) return;
            s_aux[tid] = INT_MAX;
            if (tid < kT) s_root[tid] = (tid < na && ca) ? A.root[sa + tid] : INT_MAX;
            else s_root[tid] = (tid - kT < nb && cb) ? A.root[sb + tid - kT] : INT_MAX;
        }
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
            if (r < na) xa = *reinterpret_cast<const float4*>(A.G + (sa + r) * A.dp + k0 + k4);
            if (r < nb) xb = *reinterpret_cast<const float4*>(A.G + (sb + r) * A.dp + k0 + k4);
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
        int rc[8], cc[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) cc[j] = 0;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            rc[i] = 0;
            const int r = i < 4 ? ty * 4 + i : 64 + ty * 4 + i - 4;
            if (r >= na) continue;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int c = j < 4 ? tx * 4 + j : 64 + tx * 4 + j - 4;
                if (c >= nb) continue;
                const bool in = decide(acc[i][j], sa + r, sb + c, !diag || r < c);
                rc[i] += in;
                cc[j] += in;
            }
        }
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            int v = rc[i];
            v += __shfl_xor_sync(0xffffffffu, v, 1);
            v += __shfl_xor_sync(0xffffffffu, v, 2);
            v += __shfl_xor_sync(0xffffffffu, v, 4);
            v += __shfl_xor_sync(0xffffffffu, v, 8);
            const int r = i < 4 ? ty * 4 + i : 64 + ty * 4 + i - 4;
            if (tx == 0 && r < na && v) atomicAdd(&A.count[sa + r], v);
        }
        if (!diag) {
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int c = j < 4 ? tx * 4 + j : 64 + tx * 4 + j - 4;
                if (c < nb && cc[j]) atomicAdd(&s_aux[c], cc[j]);
            }
            __syncthreads();
            if (tid < nb && s_aux[tid]) atomicAdd(&A.count[sb + tid], s_aux[tid]);
        }
        if (tid == 0) {
            const int64_t pairs = diag ? (int64_t)na * (na + 1) / 2 : (int64_t)na * nb;
            atomicAdd(&A.stats[kStatScreened], (unsigned long long)pairs);
        }
    } else if (MODE == 2) {
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int r = i < 4 ? ty * 4 + i : 64 + ty * 4 + i - 4;
            if (r >= na || !s_core[r]) continue;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int c = j < 4 ? tx * 4 + j : 64 + tx * 4 + j - 4;
                if (c >= nb || !s_core[kT + c]) continue;
                if (diag && c <= r) continue;
                if (decide(acc[i][j], sa + r, sb + c, false)) lunion(s_aux, r, diag ? c : kT + c);
            }
        }
        __syncthreads();
        {
            const int x = tid;
            const bool live = x < kT ? (x < na && s_core[x]) : (!diag && x - kT < nb && s_core[x]);
            if (live) {
                const int rx = lfind(s_aux, x);
                if (rx != x) {
                    const int64_t slot_x = x < kT ? sa + x : sb + (x - kT);
                    const int64_t slot_r = rx < kT ? sa + rx : sb + (rx - kT);
                    gunion(A.parent, (int)slot_x, (int)slot_r);
                }
            }
        }
    } else {
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
                    if (need_a) atomicMin(&s_aux[r], s_root[kT + c]);
                    if (need_b) atomicMin(&s_aux[kT + c], s_root[r]);
                }
            }
        }
        __syncthreads();
        const int x = tid;
        if (s_aux[x] != INT_MAX) {
            const int64_t slot_x = x < kT ? sa + x : sb + (x - kT);
            atomicMin(&A.border[slot_x], s_aux[x]);
        }
    }
}

// ------------------------------------------------------------- small kernels
__global__ void gather_kernel(const float* __restrict__ X, int64_t ld, int d, int dp,
                              const int32_t* __restrict__ slot_point, int64_t M,
                              float* __restrict__ G, int* nonfinite)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarp = ((int64_t)gridDim.x * blockDim.x) >> 5;
    bool bad = false;
    for (int64_t s = warp; s < M; s += nwarp) {
        const int64_t p = slot_point[s];
        for (int k = lane; k < dp; k += 32) {
            float v = 0.f;
            if (k < d) {
                v = X[p * ld + k];
                bad |= !isfinite(v);
            }
            G[s * dp + k] = v;
        }
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(nonfinite, 1);
}

__global__ void elem_offsets_kernel(const uint64_t* __restrict__ keys, int64_t M, int64_t E,
                                    int64_t* __restrict__ elem_off)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e > E) return;
    // first slot whose element >= e
    int64_t l = 0, r = M;
    while (l < r) {
        const int64_t m = (l + r) >> 1;
        if ((int64_t)(keys[m] >> 32) < e) l = m + 1; else r = m;
    }
    elem_off[e] = l;
}

__global__ void pair_counts_kernel(const int64_t* __restrict__ elem_off, int64_t E,
                                   int64_t* __restrict__ pairs)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= E) return;
    const int64_t T = (elem_off[e + 1] - elem_off[e] + kT - 1) / kT;
    pairs[e] = T * (T + 1) / 2;
}

__global__ void core_kernel(const int32_t* __restrict__ count, int64_t M, int32_t min_pts,
                            uint8_t* __restrict__ core, int32_t* __restrict__ parent,
                            int32_t* __restrict__ border, unsigned long long* stats)
{
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    bool c = false;
    if (s < M) {
        c = count[s] >= min_pts;
        core[s] = c;
        parent[s] = (int32_t)s;
        border[s] = INT_MAX;
    }
    const int nc = __syncthreads_count(c);
    if (threadIdx.x == 0 && nc) atomicAdd(&stats[kStatCore], (unsigned long long)nc);
}

__global__ void flatten_kernel(const int32_t* __restrict__ parent, const uint8_t* __restrict__ core,
                               int64_t M, int32_t* __restrict__ root)
{
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= M) return;
    int r = (int)s;
    if (core[s])
        while (parent[r] != r) r = parent[r];
    root[s] = r;
}

// label[s] = root slot of the node holding s, or -1
__global__ void label_kernel(const uint8_t* __restrict__ core, const int32_t* __restrict__ root,
                             const int32_t* __restrict__ border, const int32_t* __restrict__ slot_point,
                             int64_t M, int32_t* __restrict__ lab, int32_t* __restrict__ is_root,
                             int32_t* __restrict__ is_member, int64_t* __restrict__ slot_label)
{
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= M) return;
    int l = -1;
    if (core[s]) l = root[s];
    else if (border[s] != INT_MAX) l = border[s];
    lab[s] = l;
    slot_label[s] = l >= 0 ? (int64_t)slot_point[l] : -1;
    is_root[s] = core[s] && root[s] == (int32_t)s;
    is_member[s] = l >= 0;
}

__global__ void member_keys_kernel(const int32_t* __restrict__ lab, const int64_t* __restrict__ nid,
                                   const int64_t* __restrict__ mpos,
                                   const int32_t* __restrict__ slot_point,
                                   const int32_t* __restrict__ slot_elem, int64_t M,
                                   uint64_t* __restrict__ keys, int32_t* __restrict__ node_elem)
{
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= M) return;
    const int l = lab[s];
    if (l < 0) return;
    const int64_t node = nid[l];
    keys[mpos[s]] = ((uint64_t)node << 32) | (uint64_t)(uint32_t)slot_point[s];
    if (l == (int)s) node_elem[node] = slot_elem[s];
}

__global__ void node_offsets_kernel(const uint64_t* __restrict__ keys, int64_t G,
                                    int64_t* __restrict__ node_off, int32_t* __restrict__ members,
                                    uint64_t* __restrict__ keys2)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= G) return;
    const uint64_t k = keys[i];
    const int64_t node = (int64_t)(k >> 32);
    members[i] = (int32_t)(uint32_t)k;
    keys2[i] = ((k & 0xffffffffull) << 32) | (uint64_t)node;
    if (i == 0 || (int64_t)(keys[i - 1] >> 32) != node) node_off[node] = i;
}

__global__ void run_pairs_kernel(const uint64_t* __restrict__ keys2, int64_t G,
                                 int64_t* __restrict__ cnt)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= G) return;
    const uint64_t pt = keys2[i] >> 32;
    int64_t c = 0;
    if (i == 0 || (keys2[i - 1] >> 32) != pt) {
        int64_t len = 1;
        while (i + len < G && (keys2[i + len] >> 32) == pt) ++len;
        c = len * (len - 1) / 2;
    }
    cnt[i] = c;
}

__global__ void emit_pairs_kernel(const uint64_t* __restrict__ keys2, int64_t G,
                                  const int64_t* __restrict__ pos, uint64_t* __restrict__ out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= G) return;
    const uint64_t pt = keys2[i] >> 32;
    if (!(i == 0 || (keys2[i - 1] >> 32) != pt)) return;
    int64_t len = 1;
    while (i + len < G && (keys2[i + len] >> 32) == pt) ++len;
    int64_t o = pos[i];
    for (int64_t a = 0; a < len; ++a)
        for (int64_t b = a + 1; b < len; ++b)
            out[o++] = ((keys2[i + a] & 0xffffffffull) << 32) | (keys2[i + b] & 0xffffffffull);
}

__global__ void unique_flags_kernel(const uint64_t* __restrict__ k, int64_t P,
                                    int32_t* __restrict__ flag)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P) return;
    flag[i] = (i == 0 || k[i] != k[i - 1]);
}

__global__ void unique_emit_kernel(const uint64_t* __restrict__ k, const int32_t* __restrict__ flag,
                                   const int64_t* __restrict__ pos, int64_t P,
                                   int32_t* __restrict__ edges)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P || !flag[i]) return;
    const int64_t o = pos[i];
    edges[2 * o] = (int32_t)(k[i] >> 32);
    edges[2 * o + 1] = (int32_t)(uint32_t)k[i];
}

inline unsigned grid_for(int64_t n, int t = 256) { return (unsigned)std::max<int64_t>(1, div_up(n, t)); }

}  // namespace

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

cudaError_t gather_rows(const float* X, int64_t ld, int d, int dp, const int32_t* slot_point,
                        int64_t M, float* G, int* nonfinite, cudaStream_t s)
{
    if (M == 0) return cudaSuccess;
    const int64_t blocks = std::min<int64_t>(div_up(M, 8), 152 * 16);
    { gather_kernel<<<(unsigned)blocks, 256, 0, s>>>(X, ld, d, dp, slot_point, M, G, nonfinite); note_launch(); }
    return cudaGetLastError();
}

cudaError_t element_offsets(const uint64_t* keys, int64_t M, int64_t E, int64_t* elem_off,
                            cudaStream_t s)
{
    { elem_offsets_kernel<<<grid_for(E + 1), 256, 0, s>>>(keys, M, E, elem_off); note_launch(); }
    return cudaGetLastError();
}

cudaError_t tile_pair_offsets(const int64_t* elem_off, int64_t E, int64_t* pair_off, cudaStream_t s)
{
    Buf cnt;
    MGB_TRY(cnt.alloc(sizeof(int64_t) * std::max<int64_t>(E, 1), s));
    if (E) { pair_counts_kernel<<<grid_for(E), 256, 0, s>>>(elem_off, E, cnt.as<int64_t>()); note_launch(); }
    MGB_TRY(cudaGetLastError());
    return exclusive_scan_i64(cnt.as<int64_t>(), pair_off, E, s);
}

cudaError_t simt_pass(int mode, const PassArgs& a, int64_t n_pairs, cudaStream_t s)
{
    if (n_pairs == 0) return cudaSuccess;
    if (mode == 1) { simt_pass_kernel<1><<<(unsigned)n_pairs, 256, 0, s>>>(a); note_launch(); }
    else if (mode == 2) { simt_pass_kernel<2><<<(unsigned)n_pairs, 256, 0, s>>>(a); note_launch(); }
    else { simt_pass_kernel<3><<<(unsigned)n_pairs, 256, 0, s>>>(a); note_launch(); }
    return cudaGetLastError();
}

cudaError_t core_flags(const int32_t* count, int64_t M, int32_t min_pts, uint8_t* core,
                       int32_t* parent, int32_t* border, unsigned long long* stats, cudaStream_t s)
{
    if (M == 0) return cudaSuccess;
    { core_kernel<<<grid_for(M), 256, 0, s>>>(count, M, min_pts, core, parent, border, stats); note_launch(); }
    return cudaGetLastError();
}

cudaError_t flatten(const int32_t* parent, const uint8_t* core, int64_t M, int32_t* root,
                    cudaStream_t s)
{
    if (M == 0) return cudaSuccess;
    { flatten_kernel<<<grid_for(M), 256, 0, s>>>(parent, core, M, root); note_launch(); }
    return cudaGetLastError();
}

cudaError_t labels(const uint8_t* core, const int32_t* root, const int32_t* border,
                   const int32_t* slot_point, int64_t M, int32_t* lab, int32_t* is_root,
                   int32_t* is_member, int64_t* slot_label, cudaStream_t s)
{
    if (M == 0) return cudaSuccess;
    { label_kernel<<<grid_for(M), 256, 0, s>>>(core, root, border, slot_point, M, lab, is_root,
                                             is_member, slot_label); note_launch(); }
    return cudaGetLastError();
}

cudaError_t member_keys(const int32_t* lab, const int64_t* nid, const int64_t* mpos,
                        const int32_t* slot_point, const int32_t* slot_elem, int64_t M,
                        uint64_t* keys, int32_t* node_elem, cudaStream_t s)
{
    if (M == 0) return cudaSuccess;
    { member_keys_kernel<<<grid_for(M), 256, 0, s>>>(lab, nid, mpos, slot_point, slot_elem, M, keys,
                                                   node_elem); note_launch(); }
    return cudaGetLastError();
}

cudaError_t node_offsets(const uint64_t* keys, int64_t G, int64_t* node_off, int32_t* members,
                         uint64_t* keys2, cudaStream_t s)
{
    if (G == 0) return cudaSuccess;
    { node_offsets_kernel<<<grid_for(G), 256, 0, s>>>(keys, G, node_off, members, keys2); note_launch(); }
    return cudaGetLastError();
}

cudaError_t run_pairs(const uint64_t* keys2, int64_t G, int64_t* cnt, cudaStream_t s)
{
    if (G == 0) return cudaSuccess;
    { run_pairs_kernel<<<grid_for(G), 256, 0, s>>>(keys2, G, cnt); note_launch(); }
    return cudaGetLastError();
}

cudaError_t emit_pairs(const uint64_t* keys2, int64_t G, const int64_t* pos, uint64_t* out,
                       cudaStream_t s)
{
    if (G == 0) return cudaSuccess;
    { emit_pairs_kernel<<<grid_for(G), 256, 0, s>>>(keys2, G, pos, out); note_launch(); }
    return cudaGetLastError();
}

cudaError_t unique_flags(const uint64_t* k, int64_t P, int32_t* flag, cudaStream_t s)
{
    if (P == 0) return cudaSuccess;
    { unique_flags_kernel<<<grid_for(P), 256, 0, s>>>(k, P, flag); note_launch(); }
    return cudaGetLastError();
}

cudaError_t unique_emit(const uint64_t* k, const int32_t* flag, const int64_t* pos, int64_t P,
                        int32_t* edges, cudaStream_t s)
{
    if (P == 0) return cudaSuccess;
    { unique_emit_kernel<<<grid_for(P), 256, 0, s>>>(k, flag, pos, P, edges); note_launch(); }
    return cudaGetLastError();
}

}  // namespace mgb
