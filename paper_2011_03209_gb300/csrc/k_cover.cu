// k_cover.cu -- interval / rectangle cover of f(X) and its pull-back
// ("Mapper Interactive" §3: a cover V = {V_k} of f(X) by n intervals of
// uniform size with overlap fraction p; for a 2D filter the cover elements
// are rectangles; the points of f^{-1}(V_k) are clustered separately).
//
// Interval layout (the paper gives no formula; this is the library's
// reading): L = (hi-lo)/(n-(n-1)p), s = L(1-p), a_k = lo + k s,
// b_k = a_k + L; a_0 = lo, b_{n-1} = hi, b_k = max(b_k, a_{k+1}); L = 1 when
// hi == lo. Each operation is one explicitly rounded IEEE double operation,
// so bounds and memberships are reproducible bit for bit. Membership is
// closed (a_k <= f <= b_k). Both a_k and b_k are nondecreasing in k, so the
// elements holding a value f form the index range [first k with b_k >= f,
// last k with a_k <= f], found by binary search.
#include "common.cuh"

namespace mgb {

namespace {

__global__ void range_partial_kernel(const double* __restrict__ f, int64_t n, int m,
                                     double* __restrict__ part)
{
    const int j = blockIdx.y;
    double lo = INFINITY, hi = -INFINITY;
    bool bad = false;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x) {
        const double v = f[p * m + j];
        bad |= !isfinite(v);
        lo = fmin(lo, v);
        hi = fmax(hi, v);
    }
    for (int o = 16; o; o >>= 1) {
        lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    __shared__ double slo[32], shi[32];
    __shared__ int sbad;
    if (threadIdx.x == 0) sbad = 0;
    __syncthreads();
    if (bad) sbad = 1;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) { slo[warp] = lo; shi[warp] = hi; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) { lo = fmin(lo, slo[w]); hi = fmax(hi, shi[w]); }
        double* o = part + ((int64_t)j * gridDim.x + blockIdx.x) * 3;
        o[0] = lo; o[1] = hi; o[2] = sbad ? 1.0 : 0.0;
    }
}

// One CTA per lens dimension reduces the partials (strided over threads).
__global__ void range_final_kernel(const double* __restrict__ part, int nb, int m,
                                   double* __restrict__ lohi, int* __restrict__ nonfinite)
{
    const int j = blockIdx.x;
    double lo = INFINITY, hi = -INFINITY;
    bool bad = false;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) {
        const double* o = part + ((int64_t)j * nb + b) * 3;
        lo = fmin(lo, o[0]);
        hi = fmax(hi, o[1]);
        bad |= o[2] != 0.0;
    }
    for (int o = 16; o; o >>= 1) {
        lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    __shared__ double slo[32], shi[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) { slo[warp] = lo; shi[warp] = hi; }
    bad = __syncthreads_or(bad);
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) { lo = fmin(lo, slo[w]); hi = fmax(hi, shi[w]); }
        lohi[2 * j] = lo;
        lohi[2 * j + 1] = hi;
        if (bad && nonfinite) atomicOr(nonfinite, 1);
    }
}

// Balanced cover (§3: intervals holding equal numbers of points), read as
// the uniform cover of the filter's ranks: filter values sorted through an
// order-preserving map of doubles to 64-bit keys; element k of dimension j
// is [v_ceil(ra_k), v_min(floor(rb_k), n-1)] for the uniform rank intervals
// [ra_k, rb_k] over [0, n-1], and empty (a = +inf) when it starts past the
// last rank, so both bound arrays stay nondecreasing (the membership search
// relies on it).
__global__ void order_keys_kernel(const double* __restrict__ f, int64_t n, int m, int j, uint64_t* __restrict__ keys)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint64_t b = (uint64_t)__double_as_longlong(f[i * m + j]);
    keys[i] = (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}

__global__ void pick_bounds_kernel(const uint64_t* __restrict__ keys, int64_t n, int32_t nk,
                                   const double* __restrict__ rank_a, const double* __restrict__ rank_b,
                                   double* __restrict__ a, double* __restrict__ b)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nk) return;
    const double lo = ceil(rank_a[k]);
    double hi = floor(rank_b[k]);
    if (hi > (double)(n - 1)) hi = (double)(n - 1);
    auto value = [&](int64_t r) {
        const uint64_t key = keys[r];
        const uint64_t bits = (key >> 63) ? (key & 0x7fffffffffffffffull) : ~key;
        return __longlong_as_double((long long)bits);
    };
    b[k] = value((int64_t)hi);
    a[k] = lo > (double)(n - 1) ? INFINITY : value((int64_t)lo);
}

// bounds layout: dim 0: a[n0], b[n0]; dim 1: a[n1], b[n1]
__global__ void bounds_kernel(const double* __restrict__ lohi, int m, int32_t n0, int32_t n1,
                              double p0, double p1, double* __restrict__ bounds)
{
    for (int j = 0; j < m; ++j) {
        const int32_t nk = j == 0 ? n0 : n1;
        const double p = j == 0 ? p0 : p1;
        double* a = bounds + (j == 0 ? 0 : 2 * (int64_t)n0);
        double* b = a + nk;
        const double lo = lohi[2 * j], hi = lohi[2 * j + 1];
        const double span = __dsub_rn(hi, lo);
        const double denom = __dsub_rn((double)nk, __dmul_rn((double)(nk - 1), p));
        const double L = (span == 0.0) ? 1.0 : __ddiv_rn(span, denom);
        const double s = __dmul_rn(L, __dsub_rn(1.0, p));
        for (int32_t k = threadIdx.x; k < nk; k += blockDim.x) {
            double ak = __dadd_rn(lo, __dmul_rn((double)k, s));
            if (k == 0) ak = lo;
            double bk = (k == nk - 1) ? hi : __dadd_rn(__dadd_rn(lo, __dmul_rn((double)k, s)), L);
            if (k + 1 < nk) {
                const double an = __dadd_rn(lo, __dmul_rn((double)(k + 1), s));
                if (bk < an) bk = an;
            }
            a[k] = ak;
            b[k] = bk;
        }
    }
}

// index range of the intervals holding f: [first k with b_k >= f, last k with a_k <= f]
__device__ __forceinline__ void interval_range(const double* a, const double* b, int32_t nk,
                                               double f, int32_t* k_lo, int32_t* k_hi)
{
    int32_t l = 0, r = nk;                   // first k with b_k >= f
    while (l < r) {
        const int32_t mid = (l + r) >> 1;
        if (b[mid] >= f) r = mid; else l = mid + 1;
    }
    *k_lo = l;
    l = 0; r = nk;                           // first k with a_k > f
    while (l < r) {
        const int32_t mid = (l + r) >> 1;
        if (a[mid] > f) r = mid; else l = mid + 1;
    }
    *k_hi = l - 1;
}

__global__ void cover_count_kernel(const double* __restrict__ f, int64_t n, int m,
                                   const double* __restrict__ bounds, int32_t n0, int32_t n1,
                                   int32_t* __restrict__ cnt)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    int32_t l0, h0;
    interval_range(bounds, bounds + n0, n0, f[p * m], &l0, &h0);
    int64_t c = h0 >= l0 ? (h0 - l0 + 1) : 0;
    if (m == 2) {
        int32_t l1, h1;
        const double* a1 = bounds + 2 * (int64_t)n0;
        interval_range(a1, a1 + n1, n1, f[p * m + 1], &l1, &h1);
        c *= h1 >= l1 ? (h1 - l1 + 1) : 0;
    }
    cnt[p] = (int32_t)c;
}

__global__ void cover_emit_kernel(const double* __restrict__ f, int64_t n, int m,
                                  const double* __restrict__ bounds, int32_t n0, int32_t n1,
                                  const int64_t* __restrict__ pos, uint64_t* __restrict__ keys)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    int32_t l0, h0, l1 = 0, h1 = 0;
    interval_range(bounds, bounds + n0, n0, f[p * m], &l0, &h0);
    if (m == 2) {
        const double* a1 = bounds + 2 * (int64_t)n0;
        interval_range(a1, a1 + n1, n1, f[p * m + 1], &l1, &h1);
    }
    const int32_t nn1 = (m == 2) ? n1 : 1;
    int64_t o = pos[p];
    for (int32_t i = l0; i <= h0; ++i)
        for (int32_t k = l1; k <= h1; ++k) {
            const uint64_t e = (uint64_t)((int64_t)i * nn1 + k);
            keys[o++] = (e << 32) | (uint64_t)(uint32_t)p;
        }
}

__global__ void split_keys_kernel(const uint64_t* __restrict__ keys, int64_t M,
                                  int32_t* __restrict__ slot_point, int32_t* __restrict__ slot_elem)
{
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= M) return;
    const uint64_t k = keys[s];
    slot_point[s] = (int32_t)(uint32_t)k;
    slot_elem[s] = (int32_t)(k >> 32);
}

}  // namespace

// The cover of one element holding every point: slot i is point i.
__global__ void whole_cloud_slots_kernel(int64_t n, int32_t* __restrict__ slot_point, int32_t* __restrict__ slot_elem)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    slot_point[i] = (int32_t)i;
    slot_elem[i] = 0;
}

cudaError_t whole_cloud_slots(int64_t n, int32_t* slot_point, int32_t* slot_elem, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    { whole_cloud_slots_kernel<<<div_up(n, 256), 256, 0, s>>>(n, slot_point, slot_elem); note_launch(); }
    return cudaGetLastError();
}

cudaError_t split_keys(const uint64_t* keys, int64_t M, int32_t* slot_point, int32_t* slot_elem,
                       cudaStream_t s)
{
    if (M == 0) return cudaSuccess;
    { split_keys_kernel<<<div_up(M, 256), 256, 0, s>>>(keys, M, slot_point, slot_elem); note_launch(); }
    return cudaGetLastError();
}

cudaError_t lens_range_flag(const double* f, int64_t n, int m, double* lohi, int* nonfinite,
                            cudaStream_t s)
{
    const int nb = (int)std::min<int64_t>(512, std::max<int64_t>(1, div_up(n, 256)));
    Buf part;
    MGB_TRY(part.alloc(sizeof(double) * 3 * nb * m, s));
    { range_partial_kernel<<<dim3(nb, m), 256, 0, s>>>(f, n, m, part.as<double>()); note_launch(); }
    { range_final_kernel<<<m, 256, 0, s>>>(part.as<double>(), nb, m, lohi, nonfinite); note_launch(); }
    return cudaGetLastError();
}

cudaError_t interval_bounds(const double* lohi, int m, const int32_t* n_int_host,
                            const double* p_host, double* bounds, cudaStream_t s)
{
    { bounds_kernel<<<1, 256, 0, s>>>(lohi, m, n_int_host[0], m == 2 ? n_int_host[1] : 1,
                                    p_host[0], m == 2 ? p_host[1] : 0.0, bounds); note_launch(); }
    return cudaGetLastError();
}

cudaError_t balanced_bounds(const double* f, int64_t n, int m, const int32_t* n_int_host, const double* p_host,
                            double* bounds, cudaStream_t s)
{
    const int32_t n0 = n_int_host[0], n1 = m == 2 ? n_int_host[1] : 1;
    Buf rank_lohi, rank_bounds, keys, tmp;
    MGB_TRY(rank_lohi.alloc(sizeof(double) * 4, s));
    MGB_TRY(rank_bounds.alloc(sizeof(double) * 2 * ((size_t)n0 + (m == 2 ? n1 : 0)), s));
    MGB_TRY(keys.alloc(sizeof(uint64_t) * n, s));
    MGB_TRY(tmp.alloc(sizeof(uint64_t) * n, s));
    static thread_local double h_lohi[4];
    h_lohi[0] = 0.0;
    h_lohi[1] = (double)(n - 1);
    h_lohi[2] = 0.0;
    h_lohi[3] = (double)(n - 1);
    MGB_TRY(cudaMemcpyAsync(rank_lohi.p, h_lohi, sizeof(double) * 4, cudaMemcpyHostToDevice, s));
    MGB_TRY(interval_bounds(rank_lohi.as<double>(), m, n_int_host, p_host, rank_bounds.as<double>(), s));
    for (int j = 0; j < m; ++j) {
        const int32_t nk = j == 0 ? n0 : n1;
        const int64_t off = j == 0 ? 0 : 2 * (int64_t)n0;
        { order_keys_kernel<<<div_up(n, 256), 256, 0, s>>>(f, n, m, j, keys.as<uint64_t>()); note_launch(); }
        MGB_TRY(cudaGetLastError());
        MGB_TRY(radix_sort_u64(keys.as<uint64_t>(), tmp.as<uint64_t>(), n, 0, 64, s));
        const double* ra = rank_bounds.as<double>() + off;
        { pick_bounds_kernel<<<div_up(nk, 256), 256, 0, s>>>(keys.as<uint64_t>(), n, nk, ra, ra + nk,
                                                            bounds + off, bounds + off + nk); note_launch(); }
        MGB_TRY(cudaGetLastError());
    }
    MGB_TRY(cudaStreamSynchronize(s));              // h_lohi read before it is rewritten
    return cudaSuccess;
}

cudaError_t cover_count(const double* f, int64_t n, int m, const double* bounds, int32_t n0,
                        int32_t n1, int32_t* cnt, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    { cover_count_kernel<<<div_up(n, 256), 256, 0, s>>>(f, n, m, bounds, n0, n1, cnt); note_launch(); }
    return cudaGetLastError();
}

cudaError_t cover_emit(const double* f, int64_t n, int m, const double* bounds, int32_t n0,
                       int32_t n1, const int64_t* pos, uint64_t* keys, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    { cover_emit_kernel<<<div_up(n, 256), 256, 0, s>>>(f, n, m, bounds, n0, n1, pos, keys); note_launch(); }
    return cudaGetLastError();
}

}  // namespace mgb
