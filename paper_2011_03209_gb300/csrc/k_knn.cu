// k_knn.cu -- k-th nearest-neighbour distances ("Mapper Interactive" §5,
// "Visualizing Class Separation via Neuron Activations": a module plots the
// distribution of the distances to the k-th nearest neighbours, k = 5, to
// choose eps for DBSCAN).
//
// For each query point p, the k-th smallest distance d(p, y) over all points
// y of the cloud, p itself included (distance 0): p is a core point of
// DBSCAN(eps, k) on the whole cloud iff that distance is <= eps. The result is
// the FP64 distance of the defining expression (double sum of squared
// differences, k ascending, then sqrt), found in two streaming passes:
//   A. FP32 squared distances (FMA sum of squared differences, relative error
//      at most eta = 1.5 (d + 4) 2^-24 plus a subnormal term); each lane keeps
//      its k smallest, the warp merges them: T = the k-th smallest FP32 value.
//   B. every point with FP32 value <= B = (T + tiny)(1 + eta) / (1 - eta) +
//      tiny (rounded up) gets its exact FP64 squared distance; the k smallest
//      of those are the k smallest overall: the k points behind T are within
//      (T + tiny) / (1 - eta) exactly, so the true k-th D* is too, and a point
//      with true value <= D* has an FP32 value <= (1 + eta) D* + tiny <= B.
// One warp per query, 16 queries per CTA, 32 points per shared-memory tile
// (one per lane, rows padded against bank conflicts).
#include <cfloat>
#include <cmath>

#include "../../include/mapper.h"
#include "common.cuh"

namespace mgb {

namespace {

constexpr int kQ = 16;            // queries per CTA (one warp each)
constexpr int kP = 32;            // points per tile (one per lane)
constexpr int kKMax = 16;         // largest k

template <class T>
__device__ __forceinline__ void topk_insert(T (&top)[kKMax], int k, T v, T& worst)
{
    if (!(v < worst)) return;
#pragma unroll
    for (int i = 0; i < kKMax; ++i) {
        if (i < k && v < top[i]) {
            const T t = top[i];
            top[i] = v;
            v = t;
        }
    }
#pragma unroll
    for (int i = 0; i < kKMax; ++i)
        if (i == k - 1) worst = top[i];
}

// k-th smallest of the warp's lane lists (each ascending, k entries)
template <class T>
__device__ __forceinline__ T warp_kth(T (&top)[kKMax], int k, int lane)
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
            for (int i = 0; i + 1 < kKMax; ++i) top[i] = top[i + 1];
            top[kKMax - 1] = (T)INFINITY;
        }
        v = m;
    }
    return v;
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

template <int PASS>
__global__ void __launch_bounds__(32 * kQ, 1) knn_kernel(const float* __restrict__ X, int64_t n, int d, int64_t ld,
                                                          int dp, const int32_t* __restrict__ queries, int64_t q,
                                                          int k, float eta_lo, float eta_hi, float tiny,
                                                          float* __restrict__ thr, double* __restrict__ out)
{
    extern __shared__ float sm[];
    float* qrow = sm;                            // [kQ][dp]
    float* prow = sm + kQ * dp;                  // [kP][dp + 1]
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t qi = (int64_t)blockIdx.x * kQ + w;
    const bool live = qi < q;
    const int64_t qp = live ? queries[qi] : 0;
    for (int c = lane; c < dp; c += 32) qrow[w * dp + c] = (live && c < d) ? X[qp * ld + c] : 0.f;
    float bound = 0.f;
    if (PASS == 1 && live) {
        // B = (T + tiny)(1 + eta) / (1 - eta) + tiny, each step rounded up
        const float t = thr[qi];
        bound = __fadd_ru(__fdiv_ru(__fmul_ru(__fadd_ru(t, tiny), eta_hi), eta_lo), tiny);
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
    const float* qv = qrow + w * dp;
    for (int64_t j0 = 0; j0 < n; j0 += kP) {
        __syncthreads();
        for (int e = threadIdx.x; e < kP * dp; e += blockDim.x) {
            const int r = e / dp, c = e - r * dp;
            const int64_t j = j0 + r;
            prow[r * (dp + 1) + c] = (j < n && c < d) ? X[j * ld + c] : 0.f;
        }
        __syncthreads();
        const int64_t j = j0 + lane;
        if (!live || j >= n) continue;
        const float* pv = prow + lane * (dp + 1);
        float s = 0.f;
        for (int c = 0; c < d; ++c) {
            const float t = qv[c] - pv[c];
            s = fmaf(t, t, s);
        }
        if (PASS == 0) {
            topk_insert(topf, k, s, worstf);
        } else if (s <= bound) {
            const double e2 = exact_sqdist_rows(X + qp * ld, X + j * ld, d);
            topk_insert(topd, k, e2, worstd);
        }
    }
    if (!live) return;                           // whole warp: qi is per warp
    if (PASS == 0) {
        const float t = warp_kth(topf, k, lane);
        if (lane == 0) thr[qi] = t;
    } else {
        const double t = warp_kth(topd, k, lane);
        if (lane == 0) out[qi] = __dsqrt_rn(t);
    }
}

}  // namespace

int knn_distance(const float* X, int64_t n, int32_t d, int64_t ld, const int32_t* queries_dev, int64_t q,
                 int32_t k, double* out_dev, cudaStream_t s)
{
    if (q == 0) return MAPPER_OK;
    if (k < 1 || k > kKMax || k > n) {
        set_error("k must be in [1, min(16, n)]");
        return MAPPER_EINVAL;
    }
    const int dp = (d + 31) / 32 * 32;
    const size_t smem = sizeof(float) * ((size_t)kQ * dp + (size_t)kP * (dp + 1));
    if (smem > 227 * 1024) {
        set_error("k-distance: rows wider than 1184 columns");
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
    Buf thr;
    cudaError_t e = thr.alloc(sizeof(float) * q, s);
    if (e != cudaSuccess) { set_error(cudaGetErrorString(e)); return MAPPER_ENOMEM; }
    const unsigned grid = (unsigned)div_up(q, kQ);
    e = cudaFuncSetAttribute(knn_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(knn_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) { set_error(cudaGetErrorString(e)); return MAPPER_ECUDA; }
    knn_kernel<0><<<grid, 32 * kQ, smem, s>>>(X, n, d, ld, dp, queries_dev, q, k, eta_lo, eta_hi, tiny,
                                               thr.as<float>(), out_dev);
    knn_kernel<1><<<grid, 32 * kQ, smem, s>>>(X, n, d, ld, dp, queries_dev, q, k, eta_lo, eta_hi, tiny,
                                               thr.as<float>(), out_dev);
    note_launch(2);
    e = cudaGetLastError();
    if (e != cudaSuccess) { set_error(cudaGetErrorString(e)); return MAPPER_ECUDA; }
    return MAPPER_OK;
}

}  // namespace mgb
