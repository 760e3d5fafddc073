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
// kernel (tc_kernel, MODE 3), whose epilogue forms lower bounds (keys) of the
// squared distances. On large clouds a screen of a sample of the point tiles
// bounds each query's k-th key (tau), a screen of all points keeps every key
// <= tau, and knn_merge_tc_kernel settles the query from those; small clouds
// keep per query row and 32-point part of each chunk the 8 smallest keys
// instead. knn_select_tc and knn_merge_tc_kernel give the arguments.
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

// Merge for the tensor-core screen. Its keys l are lower bounds of the exact
// key (d^2, or -d^2 for FAR), and u = RU(l + W), W = RU(Kw (|a|^2 + |b|^2) +
// A3w), bounds it from above (Kw, A3w cover twice the screen's error bound
// and the rounding of l). The k-th smallest exact key is at most U = the k-th
// smallest u over the candidates, and every point that can reach it has l <= U.
//   LISTS: each list (kTL smallest l of a 32-point part of a chunk) holds
//   every point of its part below its last l; the candidates are the entries
//   below U of the lists whose last l exceeds U, and every point of the parts
//   whose list does not (the warp screens those together).
//   TAU: the lists of a sample of the points; writes U (a bound of the k-th
//   smallest exact key over the sample, so over all points) and stops.
//   FLAT: every point with l <= tau[query] (a TAU bound), unordered; a query
//   whose count exceeds the capacity is listed in ovf for another pass.
// The candidates are then screened again by their FP32 sums (relative error
// eta): with T32 the k-th smallest of those keys, only candidates within B32 =
// (T32 + tiny)(1 + eta) / (1 - eta) + tiny (FAR: the mirror bound) can hold the
// k-th exact key, and those few get the FP64 defining expression. One warp per
// query, lane i takes lists (entries) i, i + 32, ..
constexpr int kTL = kKnnList;
enum MergeSrc { kLists = 0, kTau = 1, kFlat = 2 };

struct MergeArgs {
    const float* X;
    int d;
    int64_t ld;
    const int32_t* queries;
    int64_t q;
    int n_lists;                     // LISTS / TAU: lists per query
    const float* cand_v;
    const int32_t* cand_i;
    int k;
    const float* rn2;                // |row|^2 of the operand rows
    int64_t q_row0;                  // operand row of query 0
    float Kw, A3w;
    float eta_lo, eta_hi, tiny;
    int64_t n, Tp;
    int chunk_tiles;
    bool vec4;
    double* out;                     // LISTS / FLAT: the k-th distance per query
    float* tau;                      // TAU: U per query
    const int* count;                // FLAT: entries per query (may exceed cap)
    int cap;
    const int64_t* off;              // FLAT, if set: query i's entries at off[i] .. off[i + 1]
    int* ovf_n;                      // FLAT: queries over capacity, listed in ovf
    int32_t* ovf;
    unsigned long long* stats;       // nullable: keys kept (FLAT), FP32 candidates, FP64
                                     // candidates, largest key count (FLAT)
    // nullable: the FP64 candidates of a query with at most kF of them go to
    // one list for knn_fp64_kernel (all lanes busy: one warp-wide FP64
    // instruction costs the same however few lanes are active); m_off / m_cnt
    // / m_k per query (m_cnt < 0: settled in the merge)
    int* f64_n;
    int64_t f64_cap;
    int32_t* f64_q;
    int32_t* f64_j;
    int64_t* m_off;
    int32_t* m_cnt;
    int32_t* m_k;
};
constexpr int kF = 8;                // FP64 candidates per query sent to the shared list

// FP32 sum of squared differences of two rows, the warp together: lane l
// takes columns l, l + 32, .. (vec4: 4 l .. 4 l + 3, + 128, ..) in order with
// FMAs, then the 32 partial sums meet in a butterfly. A term passes at most
// ceil(d / 128) 4 + 5 roundings (d + 5 for any d), which the merge's eta covers.
__device__ __forceinline__ float warp_sqdist_f32(const float* __restrict__ x, const float* __restrict__ y, int d,
                                                 bool vec4, int lane)
{
    float s = 0.f;
    if (vec4) {
        for (int k = lane * 4; k < d; k += 128) {
            const float4 p = *reinterpret_cast<const float4*>(x + k), r = __ldg(reinterpret_cast<const float4*>(y + k));
            float t = p.x - r.x;
            s = fmaf(t, t, s);
            t = p.y - r.y;
            s = fmaf(t, t, s);
            t = p.z - r.z;
            s = fmaf(t, t, s);
            t = p.w - r.w;
            s = fmaf(t, t, s);
        }
    } else {
        for (int k = lane; k < d; k += 32) {
            const float t = x[k] - __ldg(y + k);
            s = fmaf(t, t, s);
        }
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    return s;
}

template <bool FAR, int SRC>
__global__ void __launch_bounds__(256) knn_merge_tc_kernel(const MergeArgs a)
{
    constexpr int kMC = 256;                     // FP32 keys cached and FP64 candidates listed per warp
    __shared__ int s_j[8][kMC];
    __shared__ float s_f[8][kMC];
    __shared__ int s_p[8][64];                   // candidates gathering into a batch
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int64_t qi = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (qi >= a.q) return;                       // whole warp
    const int k = a.k;
    int64_t e_base = qi * (int64_t)(SRC == kFlat ? a.cap : a.n_lists * kTL), e_cap = a.cap;
    if (SRC == kFlat && a.off) {
        e_base = a.off[qi];
        e_cap = a.off[qi + 1] - e_base;
    }
    const float* cv = a.cand_v + e_base;
    const int32_t* ci = a.cand_i + e_base;
    int n_ent = 0;                               // FLAT: entries of this query
    if constexpr (SRC == kFlat) {
        const int c = a.count[qi];
        if (a.stats && lane == 0) {
            atomicAdd(a.stats, (unsigned long long)c);
            atomicMax(a.stats + 3, (unsigned long long)c);
        }
        if (c > e_cap) {
            if (lane == 0) a.ovf[atomicAdd(a.ovf_n, 1)] = (int32_t)qi;
            return;
        }
        n_ent = c;
    }
    const float na2 = a.rn2[a.q_row0 + qi];
    auto ub = [&](float lo, int j) { return __fadd_ru(lo, __fmaf_ru(a.Kw, __fadd_ru(na2, a.rn2[j]), a.A3w)); };
    float top[kTL];
#pragma unroll
    for (int i = 0; i < kTL; ++i) top[i] = INFINITY;
    float worst = INFINITY, mlast = INFINITY;
    if constexpr (SRC == kFlat) {
        for (int e = lane; e < n_ent; e += 32) topk_insert(top, k, ub(cv[e], ci[e]), worst);
    } else {
        for (int l = lane; l < a.n_lists; l += 32) {
            const int64_t e0 = (int64_t)l * kTL;
            mlast = fminf(mlast, cv[e0 + kTL - 1]);
            for (int i = 0; i < kTL; ++i) {
                const float lo = cv[e0 + i];
                if (!(lo < worst)) break;            // ascending list; u >= l
                topk_insert(top, k, ub(lo, ci[e0 + i]), worst);
            }
        }
    }
    const float U = warp_kth(top, k, lane);
    if constexpr (SRC == kTau) {
        if (lane == 0) a.tau[qi] = U;
        return;
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) mlast = fminf(mlast, __shfl_xor_sync(0xffffffffu, mlast, o));
    const bool all_complete = SRC == kFlat || U < mlast;
    const float* xq = a.X + (int64_t)a.queries[qi] * a.ld;
    // The candidates as one stream, the same order on every call, in batches
    // of up to 32: batch(j, valid) runs on the whole warp, lane l holding
    // candidate base + l. FLAT: the entries up to U; LISTS: entries up to U
    // of the complete lists, then every point of the parts whose list is
    // incomplete. Sparse candidates gather in a per-warp buffer first.
    auto stream = [&](auto&& batch) {
        int np = 0;                              // pending candidates in s_p
        auto push = [&](bool c, int j) {
            const unsigned bal = __ballot_sync(0xffffffffu, c);
            if (c) s_p[wib][np + __popc(bal & ((1u << lane) - 1u))] = j;
            np += __popc(bal);
            __syncwarp();
            if (np >= 32) {
                batch(s_p[wib][lane], true);
                const int rest = np - 32;
                const int moved = lane < rest ? s_p[wib][32 + lane] : 0;
                __syncwarp();
                if (lane < rest) s_p[wib][lane] = moved;
                np = rest;
                __syncwarp();
            }
        };
        if constexpr (SRC == kFlat) {
            for (int e0 = 0; e0 < n_ent; e0 += 32) {
                const int e = e0 + lane;
                const bool c = e < n_ent && cv[e] <= U;
                push(c, c ? ci[e] : 0);
            }
        } else {
            for (int l0 = 0; l0 < a.n_lists; l0 += 32) {
                const int l = l0 + lane;
                const bool complete = l < a.n_lists && cv[(int64_t)l * kTL + kTL - 1] > U;
                for (int i = 0; i < kTL; ++i) {
                    const bool c = complete && cv[(int64_t)l * kTL + i] <= U;
                    push(c, c ? ci[(int64_t)l * kTL + i] : 0);
                }
            }
            if (!all_complete) {
                for (int l = 0; l < a.n_lists; ++l) {
                    if (cv[(int64_t)l * kTL + kTL - 1] > U) continue;
                    const int64_t c = l / kParts, part = l % kParts;
                    const int64_t b0 = c * a.chunk_tiles, b1 = min(a.Tp, b0 + a.chunk_tiles);
                    for (int64_t t0 = 0; t0 < (b1 - b0) * 32; t0 += 32) {
                        const int64_t j = (b0 + t0 / 32) * 128 + part * 32 + lane;
                        push(j < a.n, (int)j);
                    }
                }
            }
        }
        __syncwarp();
        if (np > 0) batch(lane < np ? s_p[wib][lane] : 0, lane < np);
        __syncwarp();
    };
    // FP32 keys g (d^2, FAR -d^2) of the candidates, one per lane (the
    // sequential FMA sum); g and the exact key e lie within
    //   e in [klo(g), khi(g)],  d^2 in [RD(RD(f - tiny) / eta_hi), RU(RU(f + tiny) / eta_lo)].
    // Gk = the k-th smallest g; T_lo = klo(Gk) <= D* <= T_hi = khi(Gk) for the
    // k-th smallest exact key D* (klo, khi increase with g). Candidates with
    // khi(g) < T_lo are below D* (at most k - 1 of them: nb), those with
    // klo(g) > T_hi above it; D* is the (k - nb)-th smallest exact key of the
    // rest, the few that get the FP64 defining expression. The first kMC
    // keys are kept for the later passes.
    const int d = a.d;
    const float tiny = a.tiny, eta_hi = a.eta_hi, eta_lo = a.eta_lo;
    auto d2_lo = [&](float f) { return __fdiv_rd(__fsub_rd(f, tiny), eta_hi); };
    auto d2_hi = [&](float f) { return __fdiv_ru(__fadd_ru(f, tiny), eta_lo); };
    auto klo = [&](float g) { return FAR ? -d2_hi(-g) : d2_lo(g); };
    auto khi = [&](float g) { return FAR ? -d2_lo(-g) : d2_hi(g); };
    int base = 0;                                // candidates before the batch
    auto key32 = [&](int j, bool valid, bool first) {
        const int c = base + lane;
        float f;
        if (!first && c < kMC) {
            f = s_f[wib][c];
        } else {
            const float* y = a.X + (int64_t)(valid ? j : 0) * a.ld;
            f = a.vec4 ? fp32_sqdist_rows4(xq, y, d) : fp32_sqdist_rows(xq, y, d);
            if (first && valid && c < kMC) s_f[wib][c] = f;
        }
        return FAR ? -f : f;
    };
    float topf[kTL];
#pragma unroll
    for (int i = 0; i < kTL; ++i) topf[i] = INFINITY;
    float worstf = INFINITY;
    stream([&](int j, bool valid) {
        const float g = key32(j, valid, true);
        if (valid) topk_insert(topf, k, g, worstf);
        base += __popc(__ballot_sync(0xffffffffu, valid));
    });
    const int nc = base;
    const float Gk = warp_kth(topf, k, lane);
    const float T_lo = klo(Gk), T_hi = khi(Gk);
    double topd[kTL];
#pragma unroll
    for (int i = 0; i < kTL; ++i) topd[i] = INFINITY;
    double worstd = INFINITY;
    int nb = 0, n64 = 0;
    for (int round = 0;; ++round) {
        // middle candidates round kMC .. + kMC go to s_j
        int m = 0;
        base = 0;
        stream([&](int j, bool valid) {
            const float g = key32(j, valid, false);
            const bool below = valid && khi(g) < T_lo;
            const bool mid = valid && !below && !(klo(g) > T_hi);
            if (round == 0) nb += __popc(__ballot_sync(0xffffffffu, below));
            const unsigned bm = __ballot_sync(0xffffffffu, mid);
            const int pos = m + __popc(bm & ((1u << lane) - 1u)) - round * kMC;
            if (mid && pos >= 0 && pos < kMC) s_j[wib][pos] = j;
            m += __popc(bm);
            base += __popc(__ballot_sync(0xffffffffu, valid));
        });
        __syncwarp();
        if (round == 0 && a.f64_n && m <= kF) {
            // the few FP64 candidates join the shared list
            int pos = 0;
            if (lane == 0) pos = atomicAdd(a.f64_n, m);
            pos = __shfl_sync(0xffffffffu, pos, 0);
            if (pos + m <= a.f64_cap) {
                if (lane < m) {
                    a.f64_q[pos + lane] = (int32_t)qi;
                    a.f64_j[pos + lane] = s_j[wib][lane];
                }
                if (lane == 0) {
                    a.m_off[qi] = pos;
                    a.m_cnt[qi] = m;
                    a.m_k[qi] = k - nb;
                }
                if (a.stats) {
                    if (lane == 0) {
                        atomicAdd(a.stats + 1, (unsigned long long)nc);
                        atomicAdd(a.stats + 2, (unsigned long long)m);
                    }
                }
                return;
            }
            if (lane < m && pos + lane < a.f64_cap) a.f64_q[pos + lane] = -1;    // unused slots
        }
        const int hi = min(m, (round + 1) * kMC) - round * kMC;
        for (int t = lane; t < hi; t += 32) {
            const float* y = a.X + (int64_t)s_j[wib][t] * a.ld;
            const double e2 = a.vec4 ? exact_sqdist_rows4(xq, y, d) : exact_sqdist_rows(xq, y, d);
            topk_insert(topd, k - nb, FAR ? -e2 : e2, worstd);
            ++n64;
        }
        __syncwarp();
        if (m <= (round + 1) * kMC) break;
    }
    const double kth = warp_kth(topd, k - nb, lane);
    if (lane == 0) a.out[qi] = __dsqrt_rn(FAR ? -kth : kth);
    if (a.stats) {
        const int e64 = __reduce_add_sync(0xffffffffu, n64);
        if (lane == 0) {
            atomicAdd(a.stats + 1, (unsigned long long)nc);
            atomicAdd(a.stats + 2, (unsigned long long)e64);
        }
    }
}

// FP64 defining expression of the listed (query, point) candidates, one per
// thread: v[i] = d^2(X[queries[f64_q[i]]], X[f64_j[i]]).
__global__ void knn_fp64_kernel(const float* __restrict__ X, int d, int64_t ld, bool vec4,
                                const int32_t* __restrict__ queries, const int* __restrict__ f64_n, int64_t cap,
                                const int32_t* __restrict__ f64_q, const int32_t* __restrict__ f64_j,
                                double* __restrict__ v)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= min((int64_t)*f64_n, cap) || f64_q[i] < 0) return;
    const float* x = X + (int64_t)queries[f64_q[i]] * ld;
    const float* y = X + (int64_t)f64_j[i] * ld;
    v[i] = vec4 ? exact_sqdist_rows4(x, y, d) : exact_sqdist_rows(x, y, d);
}

// The queries whose FP64 candidates went to the list: the m_k-th smallest
// exact key (d^2; FAR -d^2) of its m_cnt <= kF values.
template <bool FAR>
__global__ void knn_f64_select_kernel(int64_t q, const int64_t* __restrict__ m_off, const int32_t* __restrict__ m_cnt,
                                      const int32_t* __restrict__ m_k, const double* __restrict__ v,
                                      double* __restrict__ out)
{
    const int64_t qi = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (qi >= q || m_cnt[qi] < 0) return;
    double top[kF];
#pragma unroll
    for (int i = 0; i < kF; ++i) top[i] = INFINITY;
    double worst = INFINITY;
    const int m = m_cnt[qi], kk = m_k[qi];
    for (int i = 0; i < m; ++i) {
        const double e2 = v[m_off[qi] + i];
        topk_insert(top, kk, FAR ? -e2 : e2, worst);
    }
    double kth = top[0];
#pragma unroll
    for (int i = 0; i < kF; ++i)
        if (i == kk - 1) kth = top[i];
    out[qi] = __dsqrt_rn(FAR ? -kth : kth);
}

// out[ovf[i]] = sub[i]
__global__ void knn_scatter_kernel(const int32_t* __restrict__ ovf, const int* __restrict__ n_ovf,
                                   const double* __restrict__ sub, double* __restrict__ out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < *n_ovf) out[ovf[i]] = sub[i];
}

// For the queries over capacity: cnt[i] = count[ovf[i]], tau2[i] = tau[ovf[i]]
__global__ void knn_ovf_gather_kernel(const int32_t* __restrict__ ovf, const int* __restrict__ n_ovf,
                                      const int* __restrict__ count, const float* __restrict__ tau,
                                      int32_t* __restrict__ cnt, float* __restrict__ tau2)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < *n_ovf) {
        cnt[i] = count[ovf[i]];
        tau2[i] = tau[ovf[i]];
    }
}

// Operand rows dst0 + i (i < rows, a multiple of 128) := rows src0 + ovf[i]
// (i < n_ovf) or zero rows: BF16 hi and lo (dp columns) and |row|^2. One
// warp per row, 16-byte copies.
__global__ void knn_copy_rows_kernel(uint16_t* __restrict__ Ah, uint16_t* __restrict__ Al, float* __restrict__ rn2,
                                     int dp, int64_t src0, const int32_t* __restrict__ ovf,
                                     const int* __restrict__ n_ovf, int64_t dst0, int64_t rows)
{
    const int lane = threadIdx.x & 31;
    const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (i >= rows) return;
    const bool live = i < *n_ovf;
    const int64_t src = live ? src0 + ovf[i] : 0, dst = dst0 + i;
    const uint4 z = make_uint4(0u, 0u, 0u, 0u);
    for (int c = lane * 8; c < dp; c += 256) {
        const uint4 h = live ? *reinterpret_cast<const uint4*>(Ah + src * dp + c) : z;
        const uint4 l = live ? *reinterpret_cast<const uint4*>(Al + src * dp + c) : z;
        *reinterpret_cast<uint4*>(Ah + dst * dp + c) = h;
        *reinterpret_cast<uint4*>(Al + dst * dp + c) = l;
    }
    if (lane == 0) rn2[dst] = live ? rn2[src] : 0.f;
}

// sub[i] = queries[ovf[i]]
__global__ void knn_gather_kernel(const int32_t* __restrict__ ovf, const int* __restrict__ n_ovf,
                                  const int32_t* __restrict__ queries, int32_t* __restrict__ sub)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < *n_ovf) sub[i] = queries[ovf[i]];
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
// products per tile pair. Large clouds: a first screen of a strided sample
// of the point tiles (lists) gives every query a bound tau of its k-th
// smallest key (the k-th smallest upper bound over the sample); the second
// screen over all points keeps every key <= tau, unsorted, and the merge
// settles the query from those (exact FP64 for the few near the k-th). A
// query with more keys below tau than the capacity goes through the list
// screen alone. Small clouds: the list screen over all points, whose merge
// screens whole parts when a list is incomplete.
constexpr int64_t kSampleMinTiles = 512;   // point tiles for the sampled path
constexpr int64_t kSampleTiles = 256;      // about this many sample tiles

template <bool FAR>
int knn_select_tc(const float* X, int64_t n, int32_t d, int64_t ld, const int32_t* queries_dev, int64_t q, int32_t k,
                  double* out_dev, int num_sms, cudaStream_t s, bool sampled = true, int64_t* info = nullptr,
                  bool screen_finite = false)
{
    const int dp = (d + 31) / 32 * 32;
    const int64_t Tp = div_up(n, 128), Tq = div_up(q, 128), T = Tp + Tq, R = T * 128;
    // FP32 re-screen of the candidates: relative error at most (D + 2) 2^-24
    // (1 + 2^-20) for D <= d + 5 roundings of a term (sequential, or the
    // merge's warp butterfly), plus at most 2^-150 for each rounding in the
    // subnormal range; the margin of eta also covers the (d + 2) 2^-53 by
    // which the FP64 defining expression may differ from d^2
    const double eta = 1.5 * (d + 8) * std::ldexp(1.0, -24);
    float eta_hi = (float)(1.0 + eta), eta_lo = (float)(1.0 - eta);
    if ((double)eta_hi < 1.0 + eta) eta_hi = std::nextafter(eta_hi, INFINITY);
    if ((double)eta_lo > 1.0 - eta) eta_lo = std::nextafter(eta_lo, 0.f);
    const float tiny = (float)(3.0 * (d + 8) * std::ldexp(1.0, -149)) + FLT_TRUE_MIN;
    const int sms = num_sms > 0 ? num_sms : 152;
    // point chunks of a screen over `tiles` tiles: fewest waves of
    // one-CTA-per-SM tasks times items per task, chunks of at most ct_max
    // tiles and (lists) at most 2 GB of lists. Nearest, lists: at most 128
    // tiles per chunk (longer chunks cut the epilogue's insertions but leave
    // more parts whose list may miss a candidate, which the merge then
    // screens whole).
    auto pick_chunks = [&](int64_t tiles, int64_t ct_max, bool lists, int64_t* ct_out, int64_t* c_out,
                           int64_t Tq = -1) {
        if (Tq < 0) Tq = div_up(q, 128);
        const int64_t c_mem =
            lists ? std::max<int64_t>(1, (int64_t(2) << 30) / std::max<int64_t>(1, q * kParts * kTL * 8)) : INT64_MAX;
        int64_t best_c = 0, best_ct = 0;
        double best = 1e300;
        for (int64_t c = 1; c <= std::max<int64_t>(1, std::min<int64_t>(tiles, 8192)); ++c) {
            int64_t ct = div_up(tiles, c);
            ct += ct & 1;
            const int64_t cc = div_up(tiles, ct);
            if (cc > c_mem && best_c) break;
            const double cost = (double)div_up(Tq * cc, sms) * (double)(ct / 2 + 4) + (ct > ct_max ? 1e200 : 0.0);
            if (cost < best) { best = cost; best_c = cc; best_ct = ct; }
        }
        *ct_out = best_ct;
        *c_out = best_c;
    };
    const bool use_sample = sampled && Tp >= kSampleMinTiles;
    // sampled: room behind the query tiles for the rows of the queries over
    // capacity (the second append screen)
    const int64_t R2 = use_sample ? R + Tq * 128 : R;
    Buf cpart, cent, row_pt, tile_n, tile_cent, Ah, Al, rn2, rn, cv, ci, err, tau, cnt, ovf;
    KNN_TRY(cpart.alloc(sizeof(double) * (kCentRows / kCentGroup) * dp, s));
    KNN_TRY(cent.alloc(sizeof(float) * dp, s));
    KNN_TRY(row_pt.alloc(sizeof(int32_t) * R, s));
    KNN_TRY(tile_n.alloc(sizeof(int32_t) * T, s));
    KNN_TRY(tile_cent.alloc(sizeof(int32_t) * T, s));
    KNN_TRY(Ah.alloc(sizeof(uint16_t) * (size_t)R2 * dp, s));
    KNN_TRY(Al.alloc(sizeof(uint16_t) * (size_t)R2 * dp, s));
    KNN_TRY(rn2.alloc(sizeof(float) * R2, s));
    KNN_TRY(rn.alloc(sizeof(float) * R, s));
    KNN_TRY(err.alloc(sizeof(int) * 2, s));      // [0]: a wait gave up; [1]: queries over capacity
    KNN_TRY(cudaMemsetAsync(err.p, 0, sizeof(int) * 2, s));
    Buf st;
    KNN_TRY(st.alloc(sizeof(unsigned long long) * 4, s));
    KNN_TRY(cudaMemsetAsync(st.p, 0, sizeof(unsigned long long) * 4, s));
    sample_sum_kernel<<<dim3((unsigned)div_up(dp, 32), kCentRows / kCentGroup / 8), dim3(32, 8), 0, s>>>(
        X, n, d, ld, dp, cpart.as<double>());
    sample_centre_kernel<<<div_up(dp, 128), 128, 0, s>>>(cpart.as<double>(), n, dp, cent.as<float>());
    note_launch();
    knn_layout_kernel<<<(unsigned)div_up(R, 256), 256, 0, s>>>(n, Tp, queries_dev, q, T, row_pt.as<int32_t>(),
                                                               tile_n.as<int32_t>(), tile_cent.as<int32_t>());
    note_launch(2);
    KNN_TRY(cudaGetLastError());
    KNN_TRY(centred_operands(X, ld, d, dp, row_pt.as<int32_t>(), tile_n.as<int32_t>(), tile_cent.as<int32_t>(),
                             cent.as<float>(), T, Ah.p, Al.p, rn2.as<float>(), rn.as<float>(), s,
                             screen_finite ? err.as<int>() : nullptr));
    if (screen_finite) {
        int h_bad = 0;
        KNN_TRY(cudaMemcpyAsync(&h_bad, err.p, sizeof(int), cudaMemcpyDeviceToHost, s));
        KNN_TRY(cudaStreamSynchronize(s));
        if (h_bad) {
            set_error("k-distance: a row holds NaN or Inf, or a norm beyond FP32");
            return MAPPER_ENONFINITE;
        }
    }
    // |s - d^2| <= E = A1f |a||b| + A2f (|a|^2 + |b|^2) + A3f for s = |a|^2 + |b|^2 -
    // 2 acc (the screen's constants plus 4 units of the rounding of s per
    // term); |a||b| <= (|a|^2 + |b|^2) (1 + 2^-12) / 2 for the rounded-up norms,
    // so E <= K (|a|^2 + |b|^2) + A3f. The screen's keys (m, c2) are lower
    // bounds of d^2 (FAR: -d^2) within 2^-20 (|a|^2 + |b|^2) of s -+ E; the
    // merge's upper bounds add W = Kw (|a|^2 + |b|^2) + A3w to a key.
    double A1, A2, A3;
    tc_bound(3, dp, 0.0, &A1, &A2, &A3);
    const double v = std::ldexp(1.0, -24);
    const float A1f = std::nextafter((float)(A1 + 4.0 * v), INFINITY);
    const float A2f = std::nextafter((float)(A2 + 4.0 * v), INFINITY);
    const float A3f = std::nextafter((float)A3, INFINITY);
    auto round_up = [](double x) {
        float f = (float)x;
        if ((double)f < x) f = std::nextafter(f, INFINITY);
        return f;
    };
    const float K = round_up(0.5 * (double)A1f * (1.0 + std::ldexp(1.0, -12)) + (double)A2f);
    float m;
    if (FAR) {
        m = -round_up(1.0 + (double)K);
    } else {
        m = (float)(1.0 - (double)K);
        if ((double)m > 1.0 - (double)K) m = std::nextafter(m, -INFINITY);
    }
    const float Kw = round_up(2.0 * (double)K + std::ldexp(1.0, -20));
    const float A3w = round_up(2.0 * (double)A3f * (1.0 + std::ldexp(1.0, -20)) + std::ldexp(1.0, -147));
    KnnScreen ks{};
    ks.Ah = Ah.p;
    ks.Al = Al.p;
    ks.rn2 = rn2.as<float>();
    ks.tile_n = tile_n.as<int32_t>();
    ks.rows = R2;
    ks.q_tile0 = Tp;
    ks.q = q;
    ks.dp = dp;
    ks.m = m;
    ks.c2 = FAR ? 2.f : -2.f;
    ks.A3f = A3f;
    ks.err = err.as<int>();
    MergeArgs ma{};
    ma.X = X;
    ma.d = d;
    ma.ld = ld;
    ma.queries = queries_dev;
    ma.q = q;
    ma.k = k;
    ma.rn2 = rn2.as<float>();
    ma.q_row0 = Tp * 128;
    ma.Kw = Kw;
    ma.A3w = A3w;
    ma.eta_lo = eta_lo;
    ma.eta_hi = eta_hi;
    ma.tiny = tiny;
    ma.n = n;
    ma.Tp = Tp;
    ma.vec4 = d % 4 == 0 && ld % 4 == 0 && ((uintptr_t)X & 15) == 0;
    ma.out = out_dev;
    ma.stats = st.as<unsigned long long>();
    // list screen over `tiles` screened tiles (operand tile b * stride)
    auto list_screen = [&](int64_t tiles, int64_t stride, int64_t ct_max) -> int {
        int64_t ct = 0, c = 0;
        pick_chunks(tiles, ct_max, true, &ct, &c);
        if (Tq * c > INT32_MAX) {
            set_error("k-distance: too many queries for one launch");
            return MAPPER_EINVAL;
        }
        const size_t nc = (size_t)q * c * kParts * kTL;
        KNN_TRY(cv.alloc(sizeof(float) * nc, s));
        KNN_TRY(ci.alloc(sizeof(int32_t) * nc, s));
        ks.n_tiles = tiles;
        ks.tile_stride = stride;
        ks.chunk_tiles = (int)ct;
        ks.chunks = (int)c;
        ks.tau = nullptr;
        ks.cand_v = cv.as<float>();
        ks.cand_i = ci.as<int32_t>();
        ma.n_lists = (int)(c * kParts);
        ma.chunk_tiles = (int)ct;
        ma.cand_v = cv.as<float>();
        ma.cand_i = ci.as<int32_t>();
        return tc_knn_screen(ks, s);
    };
    const unsigned merge_grid = (unsigned)div_up(q, 8);
    // the shared FP64 list of the first merge: up to 2 entries per query on
    // average (queries beyond it settle their own)
    Buf f64n, f64q, f64j, f64v, moff, mcnt, mk;
    const int64_t f64_cap = 2 * q + 64;
    KNN_TRY(f64n.alloc(sizeof(int), s));
    KNN_TRY(f64q.alloc(sizeof(int32_t) * f64_cap, s));
    KNN_TRY(f64j.alloc(sizeof(int32_t) * f64_cap, s));
    KNN_TRY(f64v.alloc(sizeof(double) * f64_cap, s));
    KNN_TRY(moff.alloc(sizeof(int64_t) * q, s));
    KNN_TRY(mcnt.alloc(sizeof(int32_t) * q, s));
    KNN_TRY(mk.alloc(sizeof(int32_t) * q, s));
    KNN_TRY(cudaMemsetAsync(f64n.p, 0, sizeof(int), s));
    KNN_TRY(cudaMemsetAsync(mcnt.p, 0xFF, sizeof(int32_t) * q, s));
    ma.f64_n = f64n.as<int>();
    ma.f64_cap = f64_cap;
    ma.f64_q = f64q.as<int32_t>();
    ma.f64_j = f64j.as<int32_t>();
    ma.m_off = moff.as<int64_t>();
    ma.m_cnt = mcnt.as<int32_t>();
    ma.m_k = mk.as<int32_t>();
    auto settle_f64 = [&]() -> int {
        knn_fp64_kernel<<<(unsigned)div_up(f64_cap, 256), 256, 0, s>>>(X, d, ld, ma.vec4, queries_dev, f64n.as<int>(),
                                                                       f64_cap, f64q.as<int32_t>(),
                                                                       f64j.as<int32_t>(), f64v.as<double>());
        knn_f64_select_kernel<FAR><<<(unsigned)div_up(q, 256), 256, 0, s>>>(
            q, moff.as<int64_t>(), mcnt.as<int32_t>(), mk.as<int32_t>(), f64v.as<double>(), out_dev);
        note_launch(2);
        KNN_TRY(cudaGetLastError());
        return MAPPER_OK;
    };
    int64_t cap = 0;
    if (!use_sample) {
        int rc = list_screen(Tp, 1, FAR ? Tp + 1 : 128);
        if (rc) return rc;
        knn_merge_tc_kernel<FAR, kLists><<<merge_grid, 256, 0, s>>>(ma);
        note_launch();
        KNN_TRY(cudaGetLastError());
        if ((rc = settle_f64())) return rc;
    } else {
        const int64_t stride = Tp / kSampleTiles;
        const int64_t ns = div_up(Tp, stride);
        // (only U of the lists is used: chunks of any length)
        int rc = list_screen(ns, stride, ns + 1);
        if (rc) return rc;
        KNN_TRY(tau.alloc(sizeof(float) * q, s));
        ma.tau = tau.as<float>();
        knn_merge_tc_kernel<FAR, kTau><<<merge_grid, 256, 0, s>>>(ma);
        note_launch();
        KNN_TRY(cudaGetLastError());
        cv.release();
        ci.release();
        // expected keys below tau: about stride k; room for 16 times that,
        // within 1 GB of entries
        cap = 256;
        while (cap < 16 * stride * k && cap < 8192) cap *= 2;
        cap = std::max<int64_t>(64, std::min<int64_t>(cap, (int64_t(1) << 30) / std::max<int64_t>(1, q * 8)));
        KNN_TRY(cv.alloc(sizeof(float) * (size_t)q * cap, s));
        KNN_TRY(ci.alloc(sizeof(int32_t) * (size_t)q * cap, s));
        KNN_TRY(cnt.alloc(sizeof(int) * q, s));
        KNN_TRY(ovf.alloc(sizeof(int32_t) * q, s));
        KNN_TRY(cudaMemsetAsync(cnt.p, 0, sizeof(int) * q, s));
        int64_t ct = 0, c = 0;
        pick_chunks(Tp, Tp + 1, false, &ct, &c);
        if (Tq * c > INT32_MAX) {
            set_error("k-distance: too many queries for one launch");
            return MAPPER_EINVAL;
        }
        ks.n_tiles = Tp;
        ks.tile_stride = 1;
        ks.chunk_tiles = (int)ct;
        ks.chunks = (int)c;
        ks.tau = tau.as<float>();
        ks.cap = (int)cap;
        ks.count = cnt.as<int>();
        ks.cand_v = cv.as<float>();
        ks.cand_i = ci.as<int32_t>();
        rc = tc_knn_screen(ks, s);
        if (rc) return rc;
        ma.cand_v = cv.as<float>();
        ma.cand_i = ci.as<int32_t>();
        ma.count = cnt.as<int>();
        ma.cap = (int)cap;
        ma.ovf_n = err.as<int>() + 1;
        ma.ovf = ovf.as<int32_t>();
        knn_merge_tc_kernel<FAR, kFlat><<<merge_grid, 256, 0, s>>>(ma);
        note_launch();
        KNN_TRY(cudaGetLastError());
        if ((rc = settle_f64())) return rc;
        ma.f64_n = nullptr;                      // the second merge settles its own
    }
    int h_err[2] = {0, 0};
    unsigned long long h_st[4] = {0, 0, 0, 0};
    KNN_TRY(cudaMemcpyAsync(h_err, err.p, sizeof(int) * 2, cudaMemcpyDeviceToHost, s));
    KNN_TRY(cudaMemcpyAsync(h_st, st.p, sizeof(h_st), cudaMemcpyDeviceToHost, s));
    KNN_TRY(cudaStreamSynchronize(s));
    if (h_err[0]) {
        set_error("k-distance: the tensor-core screen gave up waiting on a barrier");
        return MAPPER_ETIMEOUT;
    }
    if (info) {
        info[0] = use_sample ? 2 : 1;
        info[1] = h_err[1];
        info[2] = cap;
        info[3] = use_sample ? Tp / kSampleTiles : 0;
        info[4] = (int64_t)h_st[0];
        info[5] = (int64_t)h_st[3];
        info[6] = (int64_t)h_st[1];
        info[7] = (int64_t)h_st[2];
    }
    if (h_err[1] > 0) {
        // queries with more keys below tau than the capacity: exact room for
        // each (its count), its operand row copied behind the query tiles,
        // and a second append screen of those queries; the list screen when
        // the room would pass 2^28 entries
        const int64_t nq = h_err[1];
        int* n_ovf = err.as<int>() + 1;
        Buf sub_q, sub_out;
        KNN_TRY(sub_q.alloc(sizeof(int32_t) * nq, s));
        KNN_TRY(sub_out.alloc(sizeof(double) * nq, s));
        knn_gather_kernel<<<(unsigned)div_up(nq, 256), 256, 0, s>>>(ovf.as<int32_t>(), n_ovf, queries_dev,
                                                                     sub_q.as<int32_t>());
        note_launch();
        KNN_TRY(cudaGetLastError());
        Buf scnt, off2, tau2;
        KNN_TRY(scnt.alloc(sizeof(int32_t) * nq, s));
        KNN_TRY(off2.alloc(sizeof(int64_t) * (nq + 1), s));
        KNN_TRY(tau2.alloc(sizeof(float) * nq, s));
        knn_ovf_gather_kernel<<<(unsigned)div_up(nq, 256), 256, 0, s>>>(ovf.as<int32_t>(), n_ovf, cnt.as<int>(),
                                                                         tau.as<float>(), scnt.as<int32_t>(),
                                                                         tau2.as<float>());
        note_launch();
        KNN_TRY(cudaGetLastError());
        KNN_TRY(exclusive_scan_i32_to_i64(scnt.as<int32_t>(), off2.as<int64_t>(), nq, s));
        int64_t total = 0;
        KNN_TRY(cudaMemcpyAsync(&total, off2.as<int64_t>() + nq, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        KNN_TRY(cudaStreamSynchronize(s));
        if (total <= (int64_t(1) << 28)) {
            const int64_t Tq2 = div_up(nq, 128);
            knn_copy_rows_kernel<<<(unsigned)div_up(Tq2 * 128 * 32, 256), 256, 0, s>>>(
                static_cast<uint16_t*>(Ah.p), static_cast<uint16_t*>(Al.p), rn2.as<float>(), dp, Tp * 128,
                ovf.as<int32_t>(), n_ovf, R, Tq2 * 128);
            note_launch();
            KNN_TRY(cudaGetLastError());
            Buf cnt2, cv2, ci2, err2, ovf2;
            KNN_TRY(cnt2.alloc(sizeof(int) * nq, s));
            KNN_TRY(cv2.alloc(sizeof(float) * std::max<int64_t>(1, total), s));
            KNN_TRY(ci2.alloc(sizeof(int32_t) * std::max<int64_t>(1, total), s));
            KNN_TRY(err2.alloc(sizeof(int), s));
            KNN_TRY(ovf2.alloc(sizeof(int32_t) * nq, s));
            KNN_TRY(cudaMemsetAsync(cnt2.p, 0, sizeof(int) * nq, s));
            KNN_TRY(cudaMemsetAsync(err2.p, 0, sizeof(int), s));
            int64_t ct = 0, c = 0;
            pick_chunks(Tp, Tp + 1, false, &ct, &c, Tq2);
            ks.q = nq;
            ks.q_tile0 = Tp + Tq;
            ks.n_tiles = Tp;
            ks.tile_stride = 1;
            ks.chunk_tiles = (int)ct;
            ks.chunks = (int)c;
            ks.tau = tau2.as<float>();
            ks.cap = 0;
            ks.off = off2.as<int64_t>();
            ks.count = cnt2.as<int>();
            ks.cand_v = cv2.as<float>();
            ks.cand_i = ci2.as<int32_t>();
            int rc = tc_knn_screen(ks, s);
            if (rc) return rc;
            ma.q = nq;
            ma.queries = sub_q.as<int32_t>();
            ma.q_row0 = R;
            ma.cand_v = cv2.as<float>();
            ma.cand_i = ci2.as<int32_t>();
            ma.count = cnt2.as<int>();
            ma.cap = 0;
            ma.off = off2.as<int64_t>();
            ma.ovf_n = err2.as<int>();
            ma.ovf = ovf2.as<int32_t>();
            ma.out = sub_out.as<double>();
            knn_merge_tc_kernel<FAR, kFlat><<<(unsigned)div_up(nq, 8), 256, 0, s>>>(ma);
            note_launch();
            KNN_TRY(cudaGetLastError());
            knn_scatter_kernel<<<(unsigned)div_up(nq, 256), 256, 0, s>>>(ovf.as<int32_t>(), n_ovf,
                                                                          sub_out.as<double>(), out_dev);
            note_launch();
            KNN_TRY(cudaGetLastError());
            int h2[2] = {0, 0};
            KNN_TRY(cudaMemcpyAsync(h2, err.p, sizeof(int), cudaMemcpyDeviceToHost, s));
            KNN_TRY(cudaMemcpyAsync(h2 + 1, err2.p, sizeof(int), cudaMemcpyDeviceToHost, s));
            KNN_TRY(cudaMemcpyAsync(h_st, st.p, sizeof(h_st), cudaMemcpyDeviceToHost, s));
            KNN_TRY(cudaStreamSynchronize(s));
            if (h2[0]) {
                set_error("k-distance: the tensor-core screen gave up waiting on a barrier");
                return MAPPER_ETIMEOUT;
            }
            if (h2[1]) {                          // the same keys as in the first screen
                set_error("k-distance: second screen found more keys than the first");
                return MAPPER_EINTERNAL;
            }
            if (info) {
                info[6] = (int64_t)h_st[1];
                info[7] = (int64_t)h_st[2];
            }
        } else {
            int64_t sub_info[8] = {0, 0, 0, 0, 0, 0, 0, 0};
            const int rc = knn_select_tc<FAR>(X, n, d, ld, sub_q.as<int32_t>(), nq, k, sub_out.as<double>(),
                                              num_sms, s, false, sub_info);
            if (rc) return rc;
            if (info) {
                info[6] += sub_info[6];
                info[7] += sub_info[7];
            }
            knn_scatter_kernel<<<(unsigned)div_up(nq, 256), 256, 0, s>>>(ovf.as<int32_t>(), n_ovf,
                                                                          sub_out.as<double>(), out_dev);
            note_launch();
            KNN_TRY(cudaGetLastError());
        }
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

bool knn_on_tensor_cores(int32_t k, bool tensor_cores) { return tensor_cores && k <= kKnnList; }

int knn_distance(const float* X, int64_t n, int32_t d, int64_t ld, const int32_t* queries_dev, int64_t q,
                 int32_t k, double* out_dev, int num_sms, bool tensor_cores, cudaStream_t s, int64_t* info,
                 bool sample, bool screen_finite)
{
    if (info)
        for (int i = 0; i < 8; ++i) info[i] = 0;
    if (q == 0) return MAPPER_OK;
    if (k < 1 || k > kKMax || k > n) {
        set_error("k must be in [1, min(16, n)]");
        return MAPPER_EINVAL;
    }
    return tensor_cores && k <= kKnnList
               ? knn_select_tc<false>(X, n, d, ld, queries_dev, q, k, out_dev, num_sms, s, sample, info, screen_finite)
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
