// k_knn.cu -- k-th nearest-neighbour distances ("Mapper Interactive" §5,
// "Visualizing Class Separation via Neuron Activations": a module plots the
// distribution of the distances to the k-th nearest neighbours, k = 5, to
// choose eps for DBSCAN), and the farthest-point distance of the
// L-infinity-centrality filter (§5), the same computation with the largest
// distance.
//
// For each query point p, the k-th smallest distance d(p, y) over all points
// y of the cloud, p itself included (distance 0): p is a core point of
// DBSCAN(eps, k) on the whole cloud iff that distance is <= eps. The result is
// the FP64 distance of the defining expression (double sum of squared
// differences, k ascending, then sqrt). Two screens find it exactly:
//
// Tensor cores (k <= 8, knn_select_tc): rows centred on a sampled mean and
// split into BF16 hi + lo, three products per tile pair in the count pass's
// kernel (tc_kernel, MODE 3), whose epilogue keeps per query row and 32-point
// part of each chunk the 8 smallest lower bounds s - E of the squared
// distance (E bounds the screen's error for that pair of rows);
// knn_merge_abs_kernel settles each query from those lists (its comment gives
// the argument).
//
// CUDA cores (knn_select): FP32 squared distances (FMA sum of squared
// differences, relative error at most eta = 1.5 (d + 4) 2^-24 plus a
// subnormal term), then
//   A. the k-th smallest FP32 value T;
//   B. every point with FP32 value <= B = (T + tiny)(1 + eta) / (1 - eta) +
//      tiny (rounded up) gets its exact FP64 squared distance; the k smallest
//      of those are the k smallest overall: the k points behind T are within
//      (T + tiny) / (1 - eta) exactly, so the true k-th D* is too, and a point
//      with true value <= D* has an FP32 value <= (1 + eta) D* + tiny <= B.
// Pass A runs register-tiled: a CTA screens 64 queries against tiles of 128
// points (each thread 4 x 8 distances, columns staged 64 at a time in shared
// memory), CTAs split the points into chunks, and every (query, chunk, part)
// keeps its 16 smallest values with their points; a part is a 32-point slice
// of each tile. The union of those lists holds the 16 smallest values of the
// whole cloud, so when the 16th of them exceeds B every point below B is in
// it, and pass B reduces to the exact distances of at most 16 candidates per
// query. Queries whose 16th value is within B (many near ties, or k = 16 with
// a tie at the k-th value) take the two streaming passes: one warp per query,
// 16 queries per CTA, 32 points per shared-memory tile.
#include <cfloat>
#include <cmath>

#include "../../include/mapper.h"
#include "common.cuh"
#include "tc.cuh"

namespace mgb {

namespace {

constexpr int kQ = 16;            // queries per CTA (one warp each)
constexpr int kP = 32;            // points per tile (one per lane)
constexpr int kKMax = 16;         // largest k

template <class T, int N>
__device__ __forceinline__ void topk_insert(T (&top)[N], int k, T v, T& worst)
{
    if (!(v < worst)) return;
#pragma unroll
    for (int i = 0; i < N; ++i) {
        if (i < k && v < top[i]) {
            const T t = top[i];
            top[i] = v;
            v = t;
        }
    }
#pragma unroll
    for (int i = 0; i < N; ++i)
        if (i == k - 1) worst = top[i];
}

// k-th smallest of the warp's lane lists (each ascending, k entries)
template <class T, int N>
__device__ __forceinline__ T warp_kth(T (&top)[N], int k, int lane)
{
    T v = top[0];
    for (int r = 0; r < k; ++r) {
        v = top[0];
        T m = v;
        for (int o = 16; o; o >>= 1) {
            const T other = __shfl_xor_sync(0xffffffffu, m, o);
            m = other < m ? other : m;
        }
        const unsigned owners = __ballot_sync(0xffffffffu, top[0] == m);
        if (lane == __ffs(owners) - 1) {
#pragma unroll
            for (int i = 0; i + 1 < N; ++i) top[i] = top[i + 1];
            top[N - 1] = (T)INFINITY;
        }
        v = m;
    }
    return v;
}

// The same sums with 16-byte loads (rows 16-byte aligned, d a multiple of 4):
// columns still ascending, one rounding per operation.
__device__ __forceinline__ double exact_sqdist_rows4(const float* __restrict__ x, const float* __restrict__ y, int d)
{
    double s = 0.0;
    const float4* x4 = reinterpret_cast<const float4*>(x);
    const float4* y4 = reinterpret_cast<const float4*>(y);
    for (int k = 0; k < d / 4; ++k) {
        const float4 a = x4[k], b = __ldg(y4 + k);
        const float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const double t = __dsub_rn((double)av[u], (double)bv[u]);
            s = __dadd_rn(s, __dmul_rn(t, t));
        }
    }
    return s;
}

__device__ __forceinline__ double exact_sqdist_rows(const float* __restrict__ x, const float* __restrict__ y, int d)
{
    double s = 0.0;
    for (int k = 0; k < d; ++k) {
        const double t = __dsub_rn((double)x[k], (double)y[k]);
        s = __dadd_rn(s, __dmul_rn(t, t));
    }
    return s;
}

// The fallback streaming passes over the queries at positions pos[0 .. q)
// of the query list (all of them when pos is null); columns staged kFC at a
// time, so any row length. FAR: the k-th largest distance instead (values
// negated in the lists), with the lower bound of the candidates' FP32 values.
constexpr int kFC = 192;

template <int PASS, bool FAR>
__global__ void __launch_bounds__(32 * kQ, 1) knn_kernel(const float* __restrict__ X, int64_t n, int d, int64_t ld,
                                                          const int32_t* __restrict__ queries,
                                                          const int32_t* __restrict__ pos, int64_t q,
                                                          int k, float eta_lo, float eta_hi, float tiny,
                                                          float* __restrict__ thr, double* __restrict__ out)
{
    __shared__ float qrow[kQ][kFC];
    __shared__ float prow[kP][kFC + 1];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t qi = (int64_t)blockIdx.x * kQ + w;
    const bool live = qi < q;
    const int64_t qpos = live ? (pos ? pos[qi] : qi) : 0;
    const int64_t qp = live ? queries[qpos] : 0;
    float bound = 0.f;
    if (PASS == 1 && live) {
        const float t = thr[qi];
        // nearest: B = (T + tiny)(1 + eta) / (1 - eta) + tiny, each step rounded up;
        // farthest: B = (T - tiny)(1 - eta) / (1 + eta) - tiny, each step rounded down
        bound = FAR ? __fsub_rd(__fdiv_rd(__fmul_rd(__fsub_rd(t, tiny), eta_lo), eta_hi), tiny)
                    : __fadd_ru(__fdiv_ru(__fmul_ru(__fadd_ru(t, tiny), eta_hi), eta_lo), tiny);
    }
    float topf[kKMax];
    double topd[kKMax];
#pragma unroll
    for (int i = 0; i < kKMax; ++i) {
        topf[i] = INFINITY;
        topd[i] = INFINITY;
    }
    float worstf = INFINITY;
    double worstd = INFINITY;
    for (int64_t j0 = 0; j0 < n; j0 += kP) {
        const int64_t j = j0 + lane;
        const bool act = live && j < n;
        float s = 0.f;
        for (int k0 = 0; k0 < d; k0 += kFC) {
            const int kc = d - k0 < kFC ? d - k0 : kFC;
            __syncthreads();
            for (int c = lane; c < kc; c += 32) qrow[w][c] = live ? X[qp * ld + k0 + c] : 0.f;
            for (int e = threadIdx.x; e < kP * kc; e += blockDim.x) {
                const int r = e / kc, c = e - r * kc;
                const int64_t jr = j0 + r;
                prow[r][c] = jr < n ? X[jr * ld + k0 + c] : 0.f;
            }
            __syncthreads();
            if (act) {
                for (int c = 0; c < kc; ++c) {
                    const float t = qrow[w][c] - prow[lane][c];
                    s = fmaf(t, t, s);
                }
            }
        }
        if (!act) continue;
        if (PASS == 0) {
            topk_insert(topf, k, FAR ? -s : s, worstf);
        } else if (FAR ? s >= bound : s <= bound) {
            const double e2 = exact_sqdist_rows(X + qp * ld, X + j * ld, d);
            topk_insert(topd, k, FAR ? -e2 : e2, worstd);
        }
    }
    if (!live) return;                           // whole warp: qi is per warp
    if (PASS == 0) {
        const float t = warp_kth(topf, k, lane);
        if (lane == 0) thr[qi] = FAR ? -t : t;
    } else {
        const double t = warp_kth(topd, k, lane);
        if (lane == 0) out[qpos] = __dsqrt_rn(FAR ? -t : t);
    }
}

// ------------------------------------------------------ register-tiled pass A
constexpr int kTQ = 64;                          // queries per CTA
constexpr int kTP = 128;                         // points per tile
constexpr int kKC = 64;                          // columns per staged chunk
constexpr int kL = kKMax;                        // candidates per list
constexpr int kParts = kTP / 32;                 // lists per query and CTA
constexpr int kDS = kParts * 33;                 // distance-tile row stride (floats)
constexpr int kPS = (kTP * (kKC + 1) > kTQ * kDS) ? kTP * (kKC + 1) : kTQ * kDS;

// acc_i += (a - b_i)^2 for i = 0, 1 with the packed FP32 pair instructions:
// each lane rounds as the scalar subtract and FMA do.
__device__ __forceinline__ void sqdiff2(float& acc0, float& acc1, float a, float b0, float b1)
{
    asm("{.reg .b64 A, B, T, S;\n\t"
        "mov.b64 A, {%2, %2};\n\t"
        "mov.b64 B, {%3, %4};\n\t"
        "sub.rn.f32x2 T, A, B;\n\t"
        "mov.b64 S, {%0, %1};\n\t"
        "fma.rn.f32x2 S, T, T, S;\n\t"
        "mov.b64 {%0, %1}, S;}\n"
        : "+f"(acc0), "+f"(acc1) : "f"(a), "f"(b0), "f"(b1));
}

// Insert (v, j) into an ascending list of kL entries (v below the last).
__device__ __forceinline__ void list_insert(float (&lv)[kL], int (&li)[kL], float v, int j)
{
#pragma unroll
    for (int i = kL - 1; i > 0; --i) {
        const bool sh = v < lv[i - 1];
        const bool here = !sh && v < lv[i];
        lv[i] = sh ? lv[i - 1] : (here ? v : lv[i]);
        li[i] = sh ? li[i - 1] : (here ? j : li[i]);
    }
    if (v < lv[0]) { lv[0] = v; li[0] = j; }
}

// Grid (query tiles, point chunks). Thread (tq, tp) = (tid / 16, tid % 16)
// computes queries tq + 16 u (u < 4) against points tp + 16 v (v < 8) of each
// tile: FP32 sums of squared differences, columns ascending (the same chain
// as the fallback pass, so the same error bound), two points per packed
// instruction. The tile of distances then
// goes through shared memory to thread (qq, part) = (tid / 4, tid % 4), which
// keeps the kL smallest of query qq over points 32 part .. 32 part + 31 of
// every tile of the chunk.
template <bool FAR>
__global__ void __launch_bounds__(256, 2) knn_screen_kernel(const float* __restrict__ X, int64_t n, int d,
                                                             int64_t ld, bool xvec,
                                                             const int32_t* __restrict__ queries, int64_t q,
                                                             int64_t chunk, float* __restrict__ cand_v,
                                                             int32_t* __restrict__ cand_i)
{
    __shared__ float qs[kTQ][kKC + 1];
    __shared__ __align__(16) float ps[kPS];
    const int tid = threadIdx.x, tq = tid >> 4, tp = tid & 15;
    const int qq = tid >> 2, part = tid & 3;
    const int64_t q0 = (int64_t)blockIdx.x * kTQ;
    const int64_t p_begin = (int64_t)blockIdx.y * chunk;
    const int64_t p_end = p_begin + chunk < n ? p_begin + chunk : n;
    float lv[kL];
    int li[kL];
#pragma unroll
    for (int i = 0; i < kL; ++i) { lv[i] = INFINITY; li[i] = -1; }
    for (int64_t p0 = p_begin; p0 < p_end; p0 += kTP) {
        float acc[4][8];
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 8; ++v) acc[u][v] = 0.f;
        for (int k0 = 0; k0 < d; k0 += kKC) {
            __syncthreads();
            // queries: thread = (row tid / 64 + 4 r, column tid % 64)
            {
                const int c = tid & 63;
                for (int r = tid >> 6; r < kTQ; r += 4) {
                    const int64_t qi = q0 + r;
                    float x = 0.f;
                    if (qi < q && k0 + c < d) x = __ldg(X + (int64_t)queries[qi] * ld + k0 + c);
                    qs[r][c] = x;
                }
            }
            // points: 16 float4 per row chunk
            {
                const int c4 = (tid & 15) * 4;
                for (int r = tid >> 4; r < kTP; r += 16) {
                    const int64_t j = p0 + r;
                    float4 x = make_float4(0.f, 0.f, 0.f, 0.f);
                    if (j < p_end) {
                        const float* src = X + j * ld + k0 + c4;
                        if (xvec && k0 + c4 + 3 < d) {
                            x = __ldg(reinterpret_cast<const float4*>(src));
                        } else {
                            if (k0 + c4 < d) x.x = __ldg(src);
                            if (k0 + c4 + 1 < d) x.y = __ldg(src + 1);
                            if (k0 + c4 + 2 < d) x.z = __ldg(src + 2);
                            if (k0 + c4 + 3 < d) x.w = __ldg(src + 3);
                        }
                    }
                    float* dst = ps + r * (kKC + 1) + c4;
                    dst[0] = x.x; dst[1] = x.y; dst[2] = x.z; dst[3] = x.w;
                }
            }
            __syncthreads();
            const int kc = d - k0 < kKC ? d - k0 : kKC;
#pragma unroll 4
            for (int c = 0; c < kc; ++c) {
                float a[4], b[8];
#pragma unroll
                for (int u = 0; u < 4; ++u) a[u] = qs[tq + 16 * u][c];
#pragma unroll
                for (int v = 0; v < 8; ++v) b[v] = ps[(tp + 16 * v) * (kKC + 1) + c];
#pragma unroll
                for (int u = 0; u < 4; ++u)
#pragma unroll
                    for (int v = 0; v < 8; v += 2) sqdiff2(acc[u][v], acc[u][v + 1], a[u], b[v], b[v + 1]);
            }
        }
        __syncthreads();
        // distance tile: row r (query), part p (32 points), column c at
        // r * kDS + 33 p + c; +inf past the chunk's end
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 8; ++v) {
                const int col = tp + 16 * v;
                ps[(tq + 16 * u) * kDS + (col >> 5) * 33 + (col & 31)] =
                    p0 + col < p_end ? (FAR ? -acc[u][v] : acc[u][v]) : INFINITY;
            }
        __syncthreads();
        const float* row = ps + qq * kDS + part * 33;
#pragma unroll 4
        for (int c = 0; c < 32; ++c) {
            const float v = row[c];
            if (v < lv[kL - 1]) list_insert(lv, li, v, (int)(p0 + part * 32 + c));
        }
    }
    const int64_t qi = q0 + qq;
    if (qi >= q) return;
    const int64_t base = ((qi * gridDim.y + blockIdx.y) * kParts + part) * kL;
#pragma unroll
    for (int i = 0; i < kL; ++i) {
        cand_v[base + i] = lv[i];
        cand_i[base + i] = li[i];
    }
}

// One warp per query: the kL smallest of the query's lists (each lane keeps
// the smallest of a strided share, then kL rounds of a warp minimum), the
// bound B from the k-th of them, and, when the kL-th exceeds B, the exact
// FP64 distances of the candidates below B and their k-th smallest. Else the
// query goes to the fallback list.
template <bool FAR>
__global__ void __launch_bounds__(256) knn_merge_kernel(const float* __restrict__ X, int d, int64_t ld,
                                                        const int32_t* __restrict__ queries, int64_t q,
                                                        int n_lists, const float* __restrict__ cand_v,
                                                        const int32_t* __restrict__ cand_i, int k, float eta_lo,
                                                        float eta_hi, float tiny, double* __restrict__ out,
                                                        int32_t* __restrict__ redo,
                                                        unsigned long long* __restrict__ n_redo)
{
    const int lane = threadIdx.x & 31;
    const int64_t qi = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (qi >= q) return;                         // whole warp
    float lv[kL];
    int li[kL];
#pragma unroll
    for (int i = 0; i < kL; ++i) { lv[i] = INFINITY; li[i] = -1; }
    const int64_t total = (int64_t)n_lists * kL;
    const float* cv = cand_v + qi * total;
    const int32_t* ci = cand_i + qi * total;
    for (int64_t e = lane; e < total; e += 32) {
        const float v = cv[e];
        if (v < lv[kL - 1]) list_insert(lv, li, v, ci[e]);
    }
    // kL rounds: lane r keeps the r-th smallest (value, point)
    float my_v = INFINITY;
    int my_i = -1;
    for (int r = 0; r < kL; ++r) {
        float m = lv[0];
#pragma unroll
        for (int o = 16; o; o >>= 1) m = fminf(m, __shfl_xor_sync(0xffffffffu, m, o));
        const unsigned owners = __ballot_sync(0xffffffffu, lv[0] == m);
        const int src = __ffs(owners) - 1;
        const int j = __shfl_sync(0xffffffffu, li[0], src);
        if (lane == src) {
#pragma unroll
            for (int i = 0; i + 1 < kL; ++i) { lv[i] = lv[i + 1]; li[i] = li[i + 1]; }
            lv[kL - 1] = INFINITY;
            li[kL - 1] = -1;
        }
        if (lane == r) { my_v = m; my_i = j; }
    }
    // the lists hold negated values when FAR: v = -s
    const float t = __shfl_sync(0xffffffffu, my_v, k - 1);
    const float last = __shfl_sync(0xffffffffu, my_v, kL - 1);
    bool cand, redo_q;
    if (!FAR) {
        const float bound = __fadd_ru(__fdiv_ru(__fmul_ru(__fadd_ru(t, tiny), eta_hi), eta_lo), tiny);
        redo_q = !(last > bound);
        cand = lane < kL && my_v <= bound && my_i >= 0;
    } else {
        const float bound = __fsub_rd(__fdiv_rd(__fmul_rd(__fsub_rd(-t, tiny), eta_lo), eta_hi), tiny);
        redo_q = !(-last < bound);
        cand = lane < kL && -my_v >= bound && my_i >= 0;
    }
    if (redo_q) {
        if (lane == 0) redo[atomicAdd(n_redo, 1ull)] = (int32_t)qi;
        return;
    }
    const double none = FAR ? -INFINITY : INFINITY;
    double e = none;
    if (cand) e = exact_sqdist_rows(X + (int64_t)queries[qi] * ld, X + (int64_t)my_i * ld, d);
    // rank among the candidates, ascending (descending when FAR), ties by lane
    int rank = 0;
    for (int j = 0; j < kL; ++j) {
        const double o = __shfl_sync(0xffffffffu, e, j);
        rank += ((FAR ? o > e : o < e) || (o == e && j < lane)) ? 1 : 0;
    }
    if (cand && rank == k - 1) out[qi] = __dsqrt_rn(e);
}

}  // namespace

namespace {

__global__ void iota_kernel(int64_t n, int32_t* __restrict__ v)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) v[i] = (int32_t)i;
}

// FP32 sum of squared differences of two rows, columns ascending (the chain
// of the CUDA-core screen: relative error at most eta, subnormals below tiny).
__device__ __forceinline__ float fp32_sqdist_rows4(const float* __restrict__ x, const float* __restrict__ y, int d)
{
    float s = 0.f;
    const float4* x4 = reinterpret_cast<const float4*>(x);
    const float4* y4 = reinterpret_cast<const float4*>(y);
    for (int k = 0; k < d / 4; ++k) {
        const float4 a = x4[k], b = __ldg(y4 + k);
        float t = a.x - b.x;
        s = fmaf(t, t, s);
        t = a.y - b.y;
        s = fmaf(t, t, s);
        t = a.z - b.z;
        s = fmaf(t, t, s);
        t = a.w - b.w;
        s = fmaf(t, t, s);
    }
    return s;
}

__device__ __forceinline__ float fp32_sqdist_rows(const float* __restrict__ x, const float* __restrict__ y, int d)
{
    float s = 0.f;
    for (int k = 0; k < d; ++k) {
        const float t = x[k] - y[k];
        s = fmaf(t, t, s);
    }
    return s;
}

// Merge for the tensor-core screen. Its lists hold lower bounds l = key - E
// of the exact key (d^2, or -d^2 for FAR) with E = A1 |a||b| + A2 (|a|^2 +
// |b|^2) + A3 for that pair of rows, so u = l + 2E bounds it from above. The
// k-th smallest exact key is at most U = the k-th smallest u over the lists,
// and every point that can reach it has l <= U. Each list (kTL smallest l of a
// 32-point part of a chunk) holds every point of its part below its last l;
// the candidates are the entries below U of the lists whose last l exceeds U,
// and every point of the parts whose list does not (the warp screens those
// together). The candidates are then screened
// again by their FP32 sums (relative error eta): with T32 the k-th smallest
// of those keys, only candidates within B32 = (T32 + tiny)(1 + eta) / (1 - eta)
// + tiny (FAR: the mirror bound) can hold the k-th exact key, and those few
// get the FP64 defining expression. One warp per query, lane i takes lists
// i, i + 32, ..
constexpr int kTL = kKnnList;

template <bool FAR>
__global__ void __launch_bounds__(256) knn_merge_abs_kernel(const float* __restrict__ X, int d, int64_t ld,
                                                            const int32_t* __restrict__ queries, int64_t q,
                                                            int n_lists, const float* __restrict__ cand_v,
                                                            const int32_t* __restrict__ cand_i, int k,
                                                            const float* __restrict__ rn2, const float* __restrict__ rn,
                                                            int64_t q_row0, float A1, float A2, float A3,
                                                            float eta_lo, float eta_hi, float tiny, int64_t n,
                                                            int64_t Tp, int chunk_tiles, bool vec4,
                                                            double* __restrict__ out)
{
    constexpr int kCache = 8;                    // candidates cached per lane
    __shared__ float c_f[8][kCache][32];
    __shared__ int c_j[8][kCache][32];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int64_t qi = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (qi >= q) return;                         // whole warp
    const float* cv = cand_v + qi * (int64_t)n_lists * kTL;
    const int32_t* ci = cand_i + qi * (int64_t)n_lists * kTL;
    const float na2 = rn2[q_row0 + qi], nra = rn[q_row0 + qi];
    float top[kTL];
#pragma unroll
    for (int i = 0; i < kTL; ++i) top[i] = INFINITY;
    float worst = INFINITY, mlast = INFINITY;
    for (int l = lane; l < n_lists; l += 32) {
        const int64_t e0 = (int64_t)l * kTL;
        mlast = fminf(mlast, cv[e0 + kTL - 1]);
        for (int i = 0; i < kTL; ++i) {
            const float lo = cv[e0 + i];
            if (!(lo < worst)) break;            // ascending list; u >= l
            const int j = ci[e0 + i];
            const float E = __fmaf_ru(A1, __fmul_ru(nra, rn[j]), __fmaf_ru(A2, __fadd_ru(na2, rn2[j]), A3));
            topk_insert(top, k, __fadd_ru(lo, __fmul_ru(2.f, E)), worst);
        }
    }
    const float U = warp_kth(top, k, lane);
#pragma unroll
    for (int o = 16; o; o >>= 1) mlast = fminf(mlast, __shfl_xor_sync(0xffffffffu, mlast, o));
    const bool all_complete = U < mlast;
    const float* xq = X + (int64_t)queries[qi] * ld;
    // Visits every candidate once: entries below U of complete lists (lane
    // by list), then all points of the incomplete lists' parts (the warp
    // together, part by part).
    auto for_candidates = [&](auto&& visit) {
        for (int l = lane; l < n_lists; l += 32) {
            if (!(cv[(int64_t)l * kTL + kTL - 1] > U)) continue;
            for (int i = 0; i < kTL; ++i) {
                const int64_t e = (int64_t)l * kTL + i;
                if (!(cv[e] <= U)) break;
                visit((int64_t)ci[e]);
            }
        }
        if (all_complete) return;
        for (int l = 0; l < n_lists; ++l) {
            if (cv[(int64_t)l * kTL + kTL - 1] > U) continue;
            const int64_t c = l / kParts, part = l % kParts;
            const int64_t b0 = c * chunk_tiles, b1 = min(Tp, b0 + chunk_tiles);
            for (int64_t t = lane; t < (b1 - b0) * 32; t += 32) {
                const int64_t j = (b0 + t / 32) * 128 + part * 32 + (t & 31);
                if (j < n) visit(j);
            }
        }
    };
    // FP32 keys of the candidates: their k-th smallest
    float topf[kTL];
#pragma unroll
    for (int i = 0; i < kTL; ++i) topf[i] = INFINITY;
    float worstf = INFINITY;
    int n_cached = 0;                            // this lane's candidates, kept for the last pass
    bool spilled = false;
    for_candidates([&](int64_t j) {
        const float* y = X + j * ld;
        const float f = vec4 ? fp32_sqdist_rows4(xq, y, d) : fp32_sqdist_rows(xq, y, d);
        topk_insert(topf, k, FAR ? -f : f, worstf);
        if (n_cached < kCache) {
            c_f[wib][n_cached][lane] = f;
            c_j[wib][n_cached][lane] = (int)j;
            ++n_cached;
        } else {
            spilled = true;
        }
    });
    const float t32 = warp_kth(topf, k, lane);
    const float b_hi = __fadd_ru(__fdiv_ru(__fmul_ru(__fadd_ru(t32, tiny), eta_hi), eta_lo), tiny);
    const float b_lo = __fsub_rd(__fdiv_rd(__fmul_rd(__fsub_rd(-t32, tiny), eta_lo), eta_hi), tiny);
    double topd[kTL];
#pragma unroll
    for (int i = 0; i < kTL; ++i) topd[i] = INFINITY;
    double worstd = INFINITY;
    auto decide = [&](int64_t j, float f) {
        if (FAR ? !(f >= b_lo) : !(f <= b_hi)) return;
        const float* y = X + j * ld;
        const double e2 = vec4 ? exact_sqdist_rows4(xq, y, d) : exact_sqdist_rows(xq, y, d);
        topk_insert(topd, k, FAR ? -e2 : e2, worstd);
    };
    if (__any_sync(0xffffffffu, spilled)) {      // some lane's candidates did not fit: all again
        for_candidates([&](int64_t j) {
            const float* y = X + j * ld;
            decide(j, vec4 ? fp32_sqdist_rows4(xq, y, d) : fp32_sqdist_rows(xq, y, d));
        });
    } else {
        for (int t = 0; t < n_cached; ++t) decide(c_j[wib][t][lane], c_f[wib][t][lane]);
    }
    const double kth = warp_kth(topd, k, lane);
    if (lane == 0) out[qi] = __dsqrt_rn(FAR ? -kth : kth);
}

// Layout of the tensor-core screen's operand rows: points 0 .. n-1 in
// order (tiles 0 .. Tp-1), then the queries (tiles Tp ..); one centre.
__global__ void knn_layout_kernel(int64_t n, int64_t Tp, const int32_t* __restrict__ queries, int64_t q, int64_t T,
                                  int32_t* __restrict__ row_pt, int32_t* __restrict__ tile_n,
                                  int32_t* __restrict__ tile_cent)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t Rp = Tp * 128;
    if (i < T * 128) {
        int32_t pt = 0;
        if (i < Rp) pt = i < n ? (int32_t)i : 0;
        else if (i - Rp < q) pt = queries[i - Rp];
        row_pt[i] = pt;
    }
    if (i < T) {
        const int64_t left = i < Tp ? n - i * 128 : q - (i - Tp) * 128;
        tile_n[i] = (int32_t)(left < 128 ? left : 128);
        tile_cent[i] = 0;
    }
}

// Centre of the screen's operands: the mean of up to 4096 evenly spaced rows
// (any centre gives exact results; one near the data keeps |a| small).
// Partial sums of 32-row groups (block: 32 columns x 8 row groups), then a
// fixed-order sum per column.
constexpr int kCentRows = 4096, kCentGroup = 32;

__global__ void sample_sum_kernel(const float* __restrict__ X, int64_t n, int d, int64_t ld, int dp,
                                  double* __restrict__ part)
{
    const int col = blockIdx.x * 32 + threadIdx.x;
    const int grp = blockIdx.y * 8 + threadIdx.y;
    const int64_t m = n < kCentRows ? n : kCentRows;
    double sum = 0.0;
    if (col < d)
        for (int64_t i = (int64_t)grp * kCentGroup; i < m && i < (int64_t)(grp + 1) * kCentGroup; ++i)
            sum += (double)X[(i * n / m) * ld + col];
    if (col < dp) part[(int64_t)grp * dp + col] = sum;
}

__global__ void sample_centre_kernel(const double* __restrict__ part, int64_t n, int dp, float* __restrict__ c)
{
    const int col = blockIdx.x * blockDim.x + threadIdx.x;
    if (col >= dp) return;
    const int64_t m = n < kCentRows ? n : kCentRows;
    double sum = 0.0;
    for (int g = 0; g < kCentRows / kCentGroup; ++g) sum += part[(int64_t)g * dp + col];
    c[col] = (float)(sum / (double)m);
}



#define KNN_TRY(expr)                                                                  \
    do {                                                                               \
        const cudaError_t e_ = (expr);                                                 \
        if (e_ != cudaSuccess) {                                                       \
            set_error(std::string("k-distance: ") + cudaGetErrorString(e_));           \
            return e_ == cudaErrorMemoryAllocation ? MAPPER_ENOMEM : MAPPER_ECUDA;     \
        }                                                                              \
    } while (0)

// The tensor-core screen: rows centred on the column means, three BF16
// products per tile pair; per query the 16 smallest (FAR: largest) screened
// values, a bound from the screen's absolute error, the exact FP64 distances
// of the candidates; queries whose 16 values do not settle it go through the
// CUDA-core screen.
template <bool FAR>
int knn_select_tc(const float* X, int64_t n, int32_t d, int64_t ld, const int32_t* queries_dev, int64_t q, int32_t k,
                  double* out_dev, int num_sms, cudaStream_t s)
{
    const int dp = (d + 31) / 32 * 32;
    const int64_t Tp = div_up(n, 128), Tq = div_up(q, 128), T = Tp + Tq, R = T * 128;
    // FP32 re-screen of the candidates (the CUDA-core screen's bound)
    const double eta = 1.5 * (d + 4) * std::ldexp(1.0, -24);
    float eta_hi = (float)(1.0 + eta), eta_lo = (float)(1.0 - eta);
    if ((double)eta_hi < 1.0 + eta) eta_hi = std::nextafter(eta_hi, INFINITY);
    if ((double)eta_lo > 1.0 - eta) eta_lo = std::nextafter(eta_lo, 0.f);
    const float tiny = (float)(3.0 * (d + 2) * std::ldexp(1.0, -149)) + FLT_TRUE_MIN;
    const int sms = num_sms > 0 ? num_sms : 152;
    // point chunks: fewest waves of one-CTA-per-SM tasks times items per
    // task; nearest: lists over at most 4096 points each (longer chunks cut
    // the epilogue's insertions but leave more parts whose list may miss a
    // candidate, which the merge then screens whole), within 2 GB of lists
    const int64_t ct_max = FAR ? Tp + 1 : 128;
    const int64_t c_mem = std::max<int64_t>(1, (int64_t(2) << 30) / std::max<int64_t>(1, q * kParts * kTL * 8));
    int64_t best_c = 0, best_ct = 0;
    double best = 1e300;
    for (int64_t c = 1; c <= std::max<int64_t>(1, std::min<int64_t>(Tp, 8192)); ++c) {
        int64_t ct = div_up(Tp, c);
        ct += ct & 1;
        const int64_t cc = div_up(Tp, ct);
        if (cc > c_mem && best_c) break;
        const double cost = (double)div_up(Tq * cc, sms) * (double)(ct / 2 + 4) + (ct > ct_max ? 1e200 : 0.0);
        if (cost < best) { best = cost; best_c = cc; best_ct = ct; }
    }
    if (Tq * best_c > INT32_MAX) {
        set_error("k-distance: too many queries for one launch");
        return MAPPER_EINVAL;
    }
    Buf cpart, cent, row_pt, tile_n, tile_cent, Ah, Al, rn2, rn, cv, ci, err;
    KNN_TRY(cpart.alloc(sizeof(double) * (kCentRows / kCentGroup) * dp, s));
    KNN_TRY(cent.alloc(sizeof(float) * dp, s));
    KNN_TRY(row_pt.alloc(sizeof(int32_t) * R, s));
    KNN_TRY(tile_n.alloc(sizeof(int32_t) * T, s));
    KNN_TRY(tile_cent.alloc(sizeof(int32_t) * T, s));
    KNN_TRY(Ah.alloc(sizeof(uint16_t) * (size_t)R * dp, s));
    KNN_TRY(Al.alloc(sizeof(uint16_t) * (size_t)R * dp, s));
    KNN_TRY(rn2.alloc(sizeof(float) * R, s));
    KNN_TRY(rn.alloc(sizeof(float) * R, s));
    const size_t nc = (size_t)q * best_c * kParts * kTL;
    KNN_TRY(cv.alloc(sizeof(float) * nc, s));
    KNN_TRY(ci.alloc(sizeof(int32_t) * nc, s));
    KNN_TRY(err.alloc(sizeof(int), s));
    KNN_TRY(cudaMemsetAsync(err.p, 0, sizeof(int), s));
    sample_sum_kernel<<<dim3((unsigned)div_up(dp, 32), kCentRows / kCentGroup / 8), dim3(32, 8), 0, s>>>(
        X, n, d, ld, dp, cpart.as<double>());
    sample_centre_kernel<<<div_up(dp, 128), 128, 0, s>>>(cpart.as<double>(), n, dp, cent.as<float>());
    note_launch();
    knn_layout_kernel<<<(unsigned)div_up(R, 256), 256, 0, s>>>(n, Tp, queries_dev, q, T, row_pt.as<int32_t>(),
                                                               tile_n.as<int32_t>(), tile_cent.as<int32_t>());
    note_launch(2);
    KNN_TRY(cudaGetLastError());
    KNN_TRY(centred_operands(X, ld, d, dp, row_pt.as<int32_t>(), tile_n.as<int32_t>(), tile_cent.as<int32_t>(),
                             cent.as<float>(), T, Ah.p, Al.p, rn2.as<float>(), rn.as<float>(), s));
    // error bound of s = |a|^2 + |b|^2 - 2 acc: the screen's constants, plus
    // 4 units of the rounding of s in each term
    double A1, A2, A3;
    tc_bound(3, dp, 0.0, &A1, &A2, &A3);
    const double v = std::ldexp(1.0, -24);
    const float A1f = std::nextafter((float)(A1 + 4.0 * v), INFINITY);
    const float A2f = std::nextafter((float)(A2 + 4.0 * v), INFINITY);
    const float A3f = std::nextafter((float)A3, INFINITY);
    int rc = tc_knn_screen(Ah.p, Al.p, rn2.as<float>(), rn.as<float>(), tile_n.as<int32_t>(), Tp, q, dp,
                           (int)best_ct, (int)best_c, FAR, A1f, A2f, A3f, cv.as<float>(), ci.as<int32_t>(),
                           err.as<int>(), s);
    if (rc) return rc;
    knn_merge_abs_kernel<FAR><<<(unsigned)div_up(q, 8), 256, 0, s>>>(
        X, d, ld, queries_dev, q, (int)(best_c * kParts), cv.as<float>(), ci.as<int32_t>(), k, rn2.as<float>(),
        rn.as<float>(), Tp * 128, A1f, A2f, A3f, eta_lo, eta_hi, tiny, n, Tp, (int)best_ct,
        d % 4 == 0 && ld % 4 == 0 && ((uintptr_t)X & 15) == 0, out_dev);
    note_launch();
    KNN_TRY(cudaGetLastError());
    int h_err = 0;
    KNN_TRY(cudaMemcpyAsync(&h_err, err.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    KNN_TRY(cudaStreamSynchronize(s));
    if (h_err) {
        set_error("k-distance: the tensor-core screen gave up waiting on a barrier");
        return MAPPER_ETIMEOUT;
    }
    return MAPPER_OK;
}

// k-th smallest (FAR: k-th largest) distance of each query row to the cloud.
template <bool FAR>
int knn_select(const float* X, int64_t n, int32_t d, int64_t ld, const int32_t* queries_dev, int64_t q, int32_t k,
               double* out_dev, int num_sms, cudaStream_t s)
{
    if (q == 0) return MAPPER_OK;
    if (k < 1 || k > kKMax || k > n) {
        set_error("k must be in [1, min(16, n)]");
        return MAPPER_EINVAL;
    }
    // FP32 screen bound of the sum of d squared differences (as the CUDA-core
    // DBSCAN screen): relative eta, subnormal terms below tiny
    const double u = std::ldexp(1.0, -24);
    const double eta = 1.5 * (d + 4) * u;
    float eta_hi = (float)(1.0 + eta), eta_lo = (float)(1.0 - eta);
    if ((double)eta_hi < 1.0 + eta) eta_hi = std::nextafter(eta_hi, INFINITY);
    if ((double)eta_lo > 1.0 - eta) eta_lo = std::nextafter(eta_lo, 0.f);
    const float tiny = (float)(3.0 * (d + 2) * std::ldexp(1.0, -149)) + FLT_TRUE_MIN;
    // pass A: point chunks so that the grid fills the GPU a few times over
    const int64_t qt = div_up(q, kTQ);
    const int64_t want = 8LL * (num_sms > 0 ? num_sms : 152);
    int64_t S = std::max<int64_t>(1, std::min<int64_t>(div_up(want, qt), div_up(n, 8 * kTP)));
    S = std::min<int64_t>(S, 65535);
    const int64_t chunk = div_up(div_up(n, S), kTP) * kTP;
    S = div_up(n, chunk);
    Buf cv, ci, redo, n_redo;
    const size_t nc = (size_t)q * S * kParts * kL;
    cudaError_t e = cv.alloc(sizeof(float) * nc, s);
    if (e == cudaSuccess) e = ci.alloc(sizeof(int32_t) * nc, s);
    if (e == cudaSuccess) e = redo.alloc(sizeof(int32_t) * q, s);
    if (e == cudaSuccess) e = n_redo.alloc(sizeof(unsigned long long), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(n_redo.p, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) { set_error(cudaGetErrorString(e)); return MAPPER_ENOMEM; }
    const bool xvec = ld % 4 == 0 && ((uintptr_t)X & 15) == 0;
    knn_screen_kernel<FAR><<<dim3((unsigned)qt, (unsigned)S), 256, 0, s>>>(X, n, d, ld, xvec, queries_dev, q, chunk,
                                                                           cv.as<float>(), ci.as<int32_t>());
    knn_merge_kernel<FAR><<<(unsigned)div_up(q, 8), 256, 0, s>>>(X, d, ld, queries_dev, q, (int)(S * kParts),
                                                                 cv.as<float>(), ci.as<int32_t>(), k, eta_lo, eta_hi,
                                                                 tiny, out_dev, redo.as<int32_t>(),
                                                                 n_redo.as<unsigned long long>());
    note_launch(2);
    e = cudaGetLastError();
    if (e != cudaSuccess) { set_error(cudaGetErrorString(e)); return MAPPER_ECUDA; }
    unsigned long long h_redo = 0;
    e = cudaMemcpyAsync(&h_redo, n_redo.p, sizeof(h_redo), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) { set_error(cudaGetErrorString(e)); return MAPPER_ECUDA; }
    if (h_redo == 0) return MAPPER_OK;
    // the two streaming passes for the queries whose band reaches the 16th value
    const int64_t qr = (int64_t)h_redo;
    Buf thr;
    e = thr.alloc(sizeof(float) * qr, s);
    if (e != cudaSuccess) { set_error(cudaGetErrorString(e)); return MAPPER_ENOMEM; }
    const unsigned grid = (unsigned)div_up(qr, kQ);
    knn_kernel<0, FAR><<<grid, 32 * kQ, 0, s>>>(X, n, d, ld, queries_dev, redo.as<int32_t>(), qr, k, eta_lo, eta_hi,
                                                tiny, thr.as<float>(), out_dev);
    knn_kernel<1, FAR><<<grid, 32 * kQ, 0, s>>>(X, n, d, ld, queries_dev, redo.as<int32_t>(), qr, k, eta_lo, eta_hi,
                                                tiny, thr.as<float>(), out_dev);
    note_launch(2);
    e = cudaGetLastError();
    if (e != cudaSuccess) { set_error(cudaGetErrorString(e)); return MAPPER_ECUDA; }
    return MAPPER_OK;
}

}  // namespace

int knn_distance(const float* X, int64_t n, int32_t d, int64_t ld, const int32_t* queries_dev, int64_t q,
                 int32_t k, double* out_dev, int num_sms, bool tensor_cores, cudaStream_t s)
{
    if (q == 0) return MAPPER_OK;
    if (k < 1 || k > kKMax || k > n) {
        set_error("k must be in [1, min(16, n)]");
        return MAPPER_EINVAL;
    }
    return tensor_cores && k <= kKnnList ? knn_select_tc<false>(X, n, d, ld, queries_dev, q, k, out_dev, num_sms, s)
                                         : knn_select<false>(X, n, d, ld, queries_dev, q, k, out_dev, num_sms, s);
}

// L-infinity centrality filter f(x) = max_y d(x, y): the L-infinity norm of
// x's row of the pairwise distance matrix (§5 filters by the "L_infinity-norm"
// after computing that matrix), the largest distance of every row to the
// cloud, exact.
int lens_ecc_inf(const float* X, int64_t n, int32_t d, int64_t ld, double* f, int m, int j, int num_sms,
                 bool tensor_cores, cudaStream_t s)
{
    if (n == 0) return MAPPER_OK;
    if (n > INT32_MAX) {
        set_error("L-infinity centrality: more than 2^31 points");
        return MAPPER_EINVAL;
    }
    Buf qs, tmp;
    cudaError_t e = qs.alloc(sizeof(int32_t) * n, s);
    if (e == cudaSuccess) e = tmp.alloc(sizeof(double) * n, s);
    if (e != cudaSuccess) { set_error(cudaGetErrorString(e)); return MAPPER_ENOMEM; }
    iota_kernel<<<(unsigned)div_up(n, 256), 256, 0, s>>>(n, qs.as<int32_t>());
    note_launch();
    const int rc = tensor_cores ? knn_select_tc<true>(X, n, d, ld, qs.as<int32_t>(), n, 1, tmp.as<double>(), num_sms, s)
                                : knn_select<true>(X, n, d, ld, qs.as<int32_t>(), n, 1, tmp.as<double>(), num_sms, s);
    if (rc) return rc;
    e = cudaMemcpy2DAsync(f + j, sizeof(double) * m, tmp.p, sizeof(double), sizeof(double), (size_t)n,
                          cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) { set_error(cudaGetErrorString(e)); return MAPPER_ECUDA; }
    return MAPPER_OK;
}

}  // namespace mgb
