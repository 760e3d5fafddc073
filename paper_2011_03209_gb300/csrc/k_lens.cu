// k_lens.cu -- filter (lens) kernels, "Mapper Interactive" §3 (filter
// function f: X -> R or R^2) and §4.1 (L2 norm, a chosen column; PCA;
// eccentricity), §5 (L-infinity norm). The density filter is a count pass of
// the DBSCAN kernels (capi.cu).
//
// The projection lens sums in double, k ascending, with explicitly rounded
// operations (never fused), so it is the exact IEEE result of the defining
// expression; the L2 lens rounds the exact sum of squares once. Rows are staged
// through shared memory so the loads stay coalesced while every thread walks
// its own row in order.
#include <cuda_bf16.h>

#include "common.cuh"

namespace mgb {

namespace {

constexpr int kRows = 128;    // rows per CTA (one thread per row)
constexpr int kChunk = 32;    // columns staged per step

// One CTA = 128 rows. Each warp loads whole 32-column row segments
// (coalesced); then each thread consumes its row's segment in order.
// MODE 0: sum x^2 then sqrt (L2). MODE 1: sum (x - mu) v (projection).
// MODE 2: sum (x - mu)^2 (squared distance to the mean).
template <int MODE>
__global__ void __launch_bounds__(kRows) lens_rows_kernel(const float* __restrict__ X, int64_t n,
                                                          int32_t d, int64_t ld,
                                                          const double* __restrict__ mu,
                                                          const double* __restrict__ v,
                                                          double* __restrict__ f, int m, int j)
{
    __shared__ float tile[kRows][kChunk + 1];
    __shared__ double smu[kChunk], sv[kChunk];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t row0 = (int64_t)blockIdx.x * kRows;
    double acc = 0.0;
    for (int32_t k0 = 0; k0 < d; k0 += kChunk) {
        const int kc = min(kChunk, d - k0);
#pragma unroll 4
        for (int r = warp; r < kRows; r += kRows / 32) {
            const int64_t row = row0 + r;
            float x = 0.f;
            if (row < n && lane < kc) x = __ldg(X + row * ld + k0 + lane);
            tile[r][lane] = x;
        }
        if (MODE >= 1 && tid < kc) {
            smu[tid] = mu[k0 + tid];
            if (MODE == 1) sv[tid] = v[k0 + tid];
        }
        __syncthreads();
        for (int k = 0; k < kc; ++k) {
            const double x = (double)tile[tid][k];
            if (MODE == 0) {
                // x * x is exact in double (24-bit significands), so one
                // fused rounding equals the separate multiply and add
                acc = __fma_rn(x, x, acc);
            } else if (MODE == 1) {
                const double t = __dsub_rn(x, smu[k]);
                acc = __dadd_rn(acc, __dmul_rn(t, sv[k]));
            } else {
                const double t = __dsub_rn(x, smu[k]);
                acc = __fma_rn(t, t, acc);
            }
        }
        __syncthreads();
    }
    const int64_t row = row0 + tid;
    if (row < n) f[row * m + j] = (MODE == 0) ? __dsqrt_rn(acc) : acc;
}

// L2 lens from the exact sum of squares. A float x = m 2^(e-150) (m < 2^24)
// squares to m^2 2^(2e-300) exactly; the row's squares are added as integers
// and the exact sum is rounded to double once, then a correctly rounded sqrt.
// Per lane and 256-column chunk, with el the lane's largest exponent:
//   e >= el - 6:       (m << (e - el + 6))^2 into a 64-bit sum (unit 2^(2el-312))
//   el - 13 <= e < ..: (m << (e - el + 13))^2 into a second one (2^(2el-326))
// (one multiply-add each, at most 8 terms below 2^60); rarer small values
// and subnormals go to a 128-bit fixed-point sum whose unit is 2^(2emax-364)
// (emax: the row's largest exponent), where the two 64-bit sums also land at
// the end of each chunk. Bits of that sum below its unit are dropped: a
// relative change of at most d 2^-110, so the result is the exact sum rounded
// once up to that, within (d - 1) 2^-53 relative of a sequential double sum.
// A row holding a NaN (an Inf) gets NaN (Inf); d <= 32768 keeps the 128-bit
// sum below 2^127. One warp per row, 256 columns in registers at a time.
__device__ __forceinline__ void add128(unsigned long long& hi, unsigned long long& lo, unsigned long long bh,
                                       unsigned long long bl)
{
    const unsigned long long t = lo + bl;
    hi += bh + (t < lo ? 1ull : 0ull);
    lo = t;
}

// (hi, lo) += v 2^f, bits below 2^0 dropped (f < 64)
__device__ __forceinline__ void add128_shifted(unsigned long long& hi, unsigned long long& lo, unsigned long long v,
                                               int f)
{
    if (v == 0ull) return;
    if (f > 0) add128(hi, lo, v >> (64 - f), v << f);
    else if (f == 0) add128(hi, lo, 0ull, v);
    else if (f > -64) add128(hi, lo, 0ull, v >> -f);
}

__device__ __forceinline__ unsigned long long mad_wide(uint32_t a, unsigned long long acc)
{
    unsigned long long r;
    asm("mad.wide.u32 %0, %1, %1, %2;" : "=l"(r) : "r"(a), "l"(acc));
    return r;
}

constexpr int kL2Per = 8;                     // values per lane per 256-column chunk

// lane l takes columns k0 + 8 l .. k0 + 8 l + 7 of the chunk (two 16-byte
// loads when the row allows; the exact sum does not depend on the order)
__device__ __forceinline__ void l2_load(const float* __restrict__ x, int k0, int d, int lane, unsigned* v, bool vec)
{
    const int k = k0 + kL2Per * lane;
    if (vec && k + kL2Per <= d) {
        const uint4 a = __ldg(reinterpret_cast<const uint4*>(x + k));
        const uint4 b = __ldg(reinterpret_cast<const uint4*>(x + k + 4));
        v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
        v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
        return;
    }
#pragma unroll
    for (int i = 0; i < kL2Per; ++i) v[i] = k + i < d ? __float_as_uint(__ldg(x + k + i)) : 0u;
}

// sqrt of (hi 2^64 + lo) 2^(2 emax - 364): the 128-bit value rounded once
// to double (its top 64 bits, a sticky bit for the rest), then sqrt
__device__ __forceinline__ double l2_finish(unsigned long long hi, unsigned long long lo, int emax, unsigned special)
{
    double val = 0.0;
    if (hi != 0ull || lo != 0ull) {
        const int lz = hi ? __clzll((long long)hi) : 64 + __clzll((long long)lo);
        unsigned long long top, rest;
        if (lz < 64) {
            top = lz ? (hi << lz) | (lo >> (64 - lz)) : hi;
            rest = lz ? lo << lz : lo;
        } else {
            top = lo << (lz - 64);
            rest = 0ull;
        }
        if (rest) top |= 1ull;
        val = ldexp(__ull2double_rn(top), 64 - lz + 2 * emax - 300 - 64);
    }
    if (special) val = (special & 2u) ? __longlong_as_double(0x7FF8000000000000ll)
                                      : __longlong_as_double(0x7FF0000000000000ll);
    return __dsqrt_rn(val);
}

// the largest biased exponent of the lane's values (254 for Inf/NaN, which
// are flagged separately), at least 1
__device__ __forceinline__ int lane_emax(const unsigned* v, int* raw)
{
    int el = 1;
#pragma unroll
    for (int t = 0; t < kL2Per; ++t) el = max(el, (int)((v[t] >> 23) & 0xFFu));
    *raw = el;
    return min(el, 254);
}

// A warp sums 32 rows in turn (all lanes on one row), lane i keeps row i's
// sum, and the 32 double conversions and square roots then run side by side.
// SPLIT: the same pass also writes the rows for the pivot assignment, x - c
// rounded to BF16 (pitch dp, zero padded) and |x - c|^2 in FP32.
template <bool SPLIT>
__global__ void __launch_bounds__(256) lens_l2_exact_kernel(const float* __restrict__ X, int64_t n, int32_t d,
                                                            int64_t ld, double* __restrict__ f, int m, int j,
                                                            const float* __restrict__ c, int dp,
                                                            __nv_bfloat16* __restrict__ xh, float* __restrict__ xn2)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarp = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const bool one_chunk = d <= 32 * kL2Per;
    const bool vec = ld % 4 == 0 && ((uintptr_t)X & 15) == 0;
    for (int64_t r0 = warp * 32; r0 < n; r0 += nwarp * 32) {
        unsigned long long my_hi = 0ull, my_lo = 0ull;
        int my_emax = 1;
        unsigned my_special = 0u;
        const int rows = n - r0 < 32 ? (int)(n - r0) : 32;
        for (int i = 0; i < rows; ++i) {
            const float* x = X + (r0 + i) * ld;
            unsigned v[kL2Per];
            int emax = 1, raw_max = 0;
            for (int k0 = 0; k0 < d; k0 += 32 * kL2Per) {
                l2_load(x, k0, d, lane, v, vec);
                int raw;
                emax = max(emax, lane_emax(v, &raw));
                raw_max = max(raw_max, raw);
            }
            emax = __reduce_max_sync(0xffffffffu, emax);
            unsigned special = 0u;                                 // 1: an Inf, 2: a NaN
            if (__any_sync(0xffffffffu, raw_max == 255)) {
                for (int k0 = 0; k0 < d; k0 += 32 * kL2Per) {
                    l2_load(x, k0, d, lane, v, vec);
#pragma unroll
                    for (int t = 0; t < kL2Per; ++t)
                        if (((v[t] >> 23) & 0xFFu) == 0xFFu) special |= (v[t] & 0x7FFFFFu) ? 2u : 1u;
                }
                special = __reduce_or_sync(0xffffffffu, special);
            }
            unsigned long long hi = 0ull, lo = 0ull;
            float n2 = 0.f;
            for (int k0 = 0; k0 < d && !special; k0 += 32 * kL2Per) {
                if (!one_chunk) l2_load(x, k0, d, lane, v, vec);
                int raw;
                const int el = lane_emax(v, &raw);
                unsigned long long s1 = 0ull, s2 = 0ull;
#pragma unroll
                for (int t = 0; t < kL2Per; ++t) {
                    const int e = (int)((v[t] >> 23) & 0xFFu);
                    const int sh1 = e - el + 6;
                    if (e != 0 && sh1 >= 0) {
                        s1 = mad_wide(((v[t] | 0x800000u) & 0xFFFFFFu) << sh1, s1);
                    } else if (e != 0 && sh1 >= -7) {
                        s2 = mad_wide(((v[t] | 0x800000u) & 0xFFFFFFu) << (sh1 + 7), s2);
                    } else if (v[t] & 0x7FFFFFFFu) {
                        // small or subnormal: (m^2 << 64) >> 2 (emax - e) into the 128-bit sum
                        const unsigned mm = e ? ((v[t] | 0x800000u) & 0xFFFFFFu) : (v[t] & 0x7FFFFFu);
                        const int sh = 2 * (emax - (e ? e : 1));
                        const unsigned long long sq = (unsigned long long)mm * mm;
                        if (sh < 64) add128(hi, lo, sq >> sh, sh ? sq << (64 - sh) : 0ull);
                        else if (sh < 112) add128(hi, lo, 0ull, sq >> (sh - 64));
                    }
                }
                add128_shifted(hi, lo, s1, 52 - 2 * (emax - el));
                add128_shifted(hi, lo, s2, 38 - 2 * (emax - el));
                if constexpr (SPLIT) {
                    const int col0 = k0 + kL2Per * lane;
                    float a[kL2Per];
#pragma unroll
                    for (int t = 0; t < kL2Per; ++t) {
                        a[t] = col0 + t < d ? __uint_as_float(v[t]) - c[col0 + t] : 0.f;
                        n2 = fmaf(a[t], a[t], n2);
                    }
                    __nv_bfloat16* dst = xh + (r0 + i) * dp + col0;
                    if (col0 + kL2Per <= dp) {
                        uint32_t w[4];
#pragma unroll
                        for (int t = 0; t < kL2Per; t += 2) {
                            const __nv_bfloat162 h = __floats2bfloat162_rn(a[t], a[t + 1]);
                            w[t >> 1] = *reinterpret_cast<const uint32_t*>(&h);
                        }
                        *reinterpret_cast<uint4*>(dst) = make_uint4(w[0], w[1], w[2], w[3]);
                    } else {
                        for (int t = 0; t < kL2Per && col0 + t < dp; ++t) dst[t] = __float2bfloat16_rn(a[t]);
                    }
                }
            }
            if constexpr (SPLIT) {
#pragma unroll
                for (int o = 16; o; o >>= 1) n2 += __shfl_xor_sync(0xffffffffu, n2, o);
                if (lane == 0) xn2[r0 + i] = n2;
            }
#pragma unroll
            for (int o = 16; o; o >>= 1) {
                const unsigned long long oh = __shfl_xor_sync(0xffffffffu, hi, o);
                const unsigned long long ol = __shfl_xor_sync(0xffffffffu, lo, o);
                add128(hi, lo, oh, ol);
            }
            if (lane == i) {
                my_hi = hi;
                my_lo = lo;
                my_emax = emax;
                my_special = special;
            }
        }
        if (lane < rows) f[(r0 + lane) * m + j] = l2_finish(my_hi, my_lo, my_emax, my_special);
    }
}

// Mean of f[r * m + j] over the rows: per-block sums (rows strided over the
// threads, then a shuffle and shared-memory tree), then one block adds the
// block sums in a fixed order (the same result run to run).
constexpr int kMeanBlocks = 512;

__global__ void __launch_bounds__(256) col_lens_partial_kernel(const double* __restrict__ f, int64_t n, int m,
                                                               int j, double* __restrict__ part)
{
    __shared__ double ws[8];
    double s = 0.0;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x)
        s += f[r * m + j];
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < 8; ++w) t += ws[w];
        part[blockIdx.x] = t;
    }
}

// f = sqrt(q + V), V = (sum of the block sums) / n
__global__ void __launch_bounds__(256) ecc_finish_kernel(double* __restrict__ f, int64_t n, int m, int j,
                                                         const double* __restrict__ part, int nb)
{
    __shared__ double V;
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int b = 0; b < nb; ++b) t += part[b];
        V = t / (double)n;
    }
    __syncthreads();
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x)
        f[r * m + j] = __dsqrt_rn(__dadd_rn(f[r * m + j], V));
}

__global__ void lens_coord_kernel(const float* __restrict__ X, int64_t n, int64_t ld, int32_t col,
                                  double* __restrict__ f, int m, int j)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p < n) f[p * m + j] = (double)X[p * ld + col];
}

// L-infinity norm max_k |x_k|: one warp per row, lanes over columns, a
// NaN-propagating maximum (exact: no arithmetic, FP32 values widen exactly).
__global__ void __launch_bounds__(256) lens_linf_kernel(const float* __restrict__ X, int64_t n, int32_t d,
                                                        int64_t ld, double* __restrict__ f, int m, int j)
{
    const int lane = threadIdx.x & 31;
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t r = w0; r < n; r += nw) {
        const float* x = X + r * ld;
        float mx = 0.f;
        for (int k = lane; k < d; k += 32) {
            const float v = fabsf(__ldg(x + k));
            if (v > mx || v != v) mx = v;
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            const float v = __shfl_xor_sync(0xffffffffu, mx, o);
            if (v > mx || v != v) mx = v;
        }
        if (lane == 0) f[r * m + j] = (double)mx;
    }
}

// One warp per row (grid-stride), lanes over columns, 16-byte loads when
// the rows allow them.
__global__ void __launch_bounds__(256) finite_kernel(const float* __restrict__ X, int64_t n, int32_t d, int64_t ld,
                                                     bool vec, int* flag)
{
    const int lane = threadIdx.x & 31;
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    bool bad = false;
    for (int64_t r = w0; r < n; r += nw) {
        const float* x = X + r * ld;
        if (vec) {
            const int d4 = d >> 2;
            for (int c = lane; c < d4; c += 32) {
                const float4 v = __ldg(reinterpret_cast<const float4*>(x) + c);
                bad |= !(isfinite(v.x) && isfinite(v.y) && isfinite(v.z) && isfinite(v.w));
            }
            for (int c = 4 * d4 + lane; c < d; c += 32) bad |= !isfinite(__ldg(x + c));
        } else {
            for (int c = lane; c < d; c += 32) bad |= !isfinite(__ldg(x + c));
        }
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(flag, 1);
}

// --------------------------------------------------------------------- PCA
// Column means: partial FP64 sums per row block, then a fixed-order reduce
// (deterministic run to run).
constexpr int kMeanRows = 4096;

__global__ void col_partial_sum_kernel(const float* __restrict__ X, int64_t n, int32_t d,
                                       int64_t ld, double* __restrict__ part)
{
    const int64_t r0 = (int64_t)blockIdx.x * kMeanRows;
    const int64_t r1 = min(n, r0 + kMeanRows);
    for (int c = threadIdx.x; c < d; c += blockDim.x) {
        double s = 0.0;
        for (int64_t r = r0; r < r1; ++r) s += (double)X[r * ld + c];
        part[(int64_t)blockIdx.x * d + c] = s;
    }
}

__global__ void col_mean_kernel(const double* __restrict__ part, int nblk, int32_t d, int64_t n,
                                double* __restrict__ mu)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= d) return;
    double s = 0.0;
    for (int b = 0; b < nblk; ++b) s += part[(int64_t)b * d + c];
    mu[c] = s / (double)n;
}

// FP32 covariance tiles: block (ti, tj, chunk) accumulates the 64 x 64 tile
// (ti, tj), tj >= ti, of sum_p (x_p - mu)(x_p - mu)^T over its row chunk.
constexpr int kCovT = 64;
constexpr int kCovRows = 2048;

__global__ void __launch_bounds__(256) cov_partial_kernel(const float* __restrict__ X, int64_t n,
                                                          int32_t d, int64_t ld,
                                                          const double* __restrict__ mu,
                                                          float* __restrict__ part, int ntile)
{
    int ti = 0, tj = 0, t = blockIdx.x;       // decode upper-triangle tile index
    for (ti = 0; ti < ntile; ++ti) {
        const int row_len = ntile - ti;
        if (t < row_len) { tj = ti + t; break; }
        t -= row_len;
    }
    const int chunk = blockIdx.y;
    __shared__ float sa[32][kCovT + 1], sb[32][kCovT + 1];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    float acc[4][4] = {};
    const int64_t r0 = (int64_t)chunk * kCovRows, r1 = min(n, r0 + kCovRows);
    const int ca = ti * kCovT, cb = tj * kCovT;
    for (int64_t rb = r0; rb < r1; rb += 32) {
        for (int e = threadIdx.x; e < 32 * kCovT; e += 256) {
            const int rr = e / kCovT, cc = e % kCovT;
            const int64_t r = rb + rr;
            float xa = 0.f, xb = 0.f;
            if (r < r1) {
                if (ca + cc < d) xa = (float)((double)X[r * ld + ca + cc] - mu[ca + cc]);
                if (cb + cc < d) xb = (float)((double)X[r * ld + cb + cc] - mu[cb + cc]);
            }
            sa[rr][cc] = xa;
            sb[rr][cc] = xb;
        }
        __syncthreads();
#pragma unroll 8
        for (int rr = 0; rr < 32; ++rr) {
            float a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) { a[i] = sa[rr][ty * 4 + i]; b[i] = sb[rr][tx * 4 + i]; }
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int k = 0; k < 4; ++k) acc[i][k] = fmaf(a[i], b[k], acc[i][k]);
        }
        __syncthreads();
    }
    float* out = part + ((int64_t)chunk * gridDim.x + blockIdx.x) * kCovT * kCovT;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int k = 0; k < 4; ++k) out[(ty * 4 + i) * kCovT + tx * 4 + k] = acc[i][k];
}

__global__ void cov_reduce_kernel(const float* __restrict__ part, int nchunk, int ntile, int32_t d,
                                  int64_t n, double* __restrict__ C)
{
    const int tile = blockIdx.x;
    int ti = 0, tj = 0, t = tile;
    for (ti = 0; ti < ntile; ++ti) {
        const int row_len = ntile - ti;
        if (t < row_len) { tj = ti + t; break; }
        t -= row_len;
    }
    const int ntiles = gridDim.x;
    for (int e = threadIdx.x; e < kCovT * kCovT; e += blockDim.x) {
        const int i = ti * kCovT + e / kCovT, k = tj * kCovT + e % kCovT;
        if (i >= d || k >= d) continue;
        double s = 0.0;
        for (int c = 0; c < nchunk; ++c) s += (double)part[((int64_t)c * ntiles + tile) * kCovT * kCovT + e];
        s /= (double)n;
        C[(int64_t)i * d + k] = s;
        C[(int64_t)k * d + i] = s;
    }
}

// Power iteration for the top-K eigenvectors of C (d x d, FP64), one CTA.
// Each axis is orthogonalised against the earlier ones every step (deflation
// by projection), iterated until ||v_new - v|| < 1e-7 or 2000 steps, then
// signed so its entry of largest magnitude is positive (ties: lowest index).
__global__ void __launch_bounds__(1024) power_iter_kernel(const double* __restrict__ C, int32_t d,
                                                          int K, double* __restrict__ axes,
                                                          int* status)
{
    extern __shared__ double sm[];
    double* v = sm;           // d
    double* w = sm + d;       // d
    __shared__ double red[32];
    __shared__ double s_norm, s_diff;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarp = blockDim.x >> 5;
    int not_conv = 0;
    for (int c = 0; c < K; ++c) {
        for (int k = tid; k < d; k += blockDim.x) v[k] = 1.0 + 0.25 * (double)((k * 7919) % 13);
        __syncthreads();
        for (int it = 0; it < 2000; ++it) {
            // w = C v
            for (int r = warp; r < d; r += nwarp) {
                double s = 0.0;
                for (int k = lane; k < d; k += 32) s += C[(int64_t)r * d + k] * v[k];
                for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
                if (lane == 0) w[r] = s;
            }
            __syncthreads();
            // orthogonalise against earlier axes
            for (int q = 0; q < c; ++q) {
                double s = 0.0;
                for (int k = tid; k < d; k += blockDim.x) s += axes[q * d + k] * w[k];
                for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
                if (lane == 0) red[warp] = s;
                __syncthreads();
                if (tid == 0) { double t = 0; for (int i = 0; i < nwarp; ++i) t += red[i]; s_norm = t; }
                __syncthreads();
                const double proj = s_norm;
                for (int k = tid; k < d; k += blockDim.x) w[k] -= proj * axes[q * d + k];
                __syncthreads();
            }
            double s = 0.0;
            for (int k = tid; k < d; k += blockDim.x) s += w[k] * w[k];
            for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if (lane == 0) red[warp] = s;
            __syncthreads();
            if (tid == 0) { double t = 0; for (int i = 0; i < nwarp; ++i) t += red[i]; s_norm = sqrt(t); }
            __syncthreads();
            const double inv = s_norm > 0.0 ? 1.0 / s_norm : 0.0;
            double dd = 0.0;
            for (int k = tid; k < d; k += blockDim.x) {
                const double nv = w[k] * inv;
                dd += (nv - v[k]) * (nv - v[k]);
                v[k] = nv;
            }
            for (int o = 16; o; o >>= 1) dd += __shfl_xor_sync(0xffffffffu, dd, o);
            if (lane == 0) red[warp] = dd;
            __syncthreads();
            if (tid == 0) { double t = 0; for (int i = 0; i < nwarp; ++i) t += red[i]; s_diff = t; }
            __syncthreads();
            if (s_diff < 1e-14) break;           // ||dv|| < 1e-7
            if (it == 1999) not_conv = 1;
        }
        // sign rule
        if (tid == 0) {
            int arg = 0;
            for (int k = 1; k < d; ++k)
                if (fabs(v[k]) > fabs(v[arg])) arg = k;
            s_norm = v[arg] < 0.0 ? -1.0 : 1.0;
        }
        __syncthreads();
        for (int k = tid; k < d; k += blockDim.x) axes[c * d + k] = s_norm * v[k];
        __syncthreads();
    }
    if (tid == 0) *status = not_conv;
}

}  // namespace

cudaError_t lens_l2_split(const float* X, int64_t n, int32_t d, int64_t ld, double* f, int m, int j,
                          const float* c, int dp, void* xh, float* xn2, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    if (d > 32768) return cudaErrorInvalidValue;
    const int blocks = (int)std::min<int64_t>(div_up(n, 8 * 32), 152 * 8);
    lens_l2_exact_kernel<true><<<blocks, 256, 0, s>>>(X, n, d, ld, f, m, j, c, dp,
                                                      static_cast<__nv_bfloat16*>(xh), xn2);
    note_launch();
    return cudaGetLastError();
}

cudaError_t lens_l2(const float* X, int64_t n, int32_t d, int64_t ld, double* f, int m, int j,
                    cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    if (d <= 32768) {
        const int blocks = (int)std::min<int64_t>(div_up(n, 8 * 32), 152 * 8);
        lens_l2_exact_kernel<false><<<blocks, 256, 0, s>>>(X, n, d, ld, f, m, j, nullptr, 0, nullptr, nullptr);
    } else {
        lens_rows_kernel<0><<<div_up(n, kRows), kRows, 0, s>>>(X, n, d, ld, nullptr, nullptr, f, m, j);
    }
    note_launch();
    return cudaGetLastError();
}

cudaError_t lens_project(const float* X, int64_t n, int32_t d, int64_t ld, const double* mu,
                         const double* v, double* f, int m, int j, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    { lens_rows_kernel<1><<<div_up(n, kRows), kRows, 0, s>>>(X, n, d, ld, mu, v, f, m, j); note_launch(); }
    return cudaGetLastError();
}

cudaError_t column_means(const float* X, int64_t n, int32_t d, int64_t ld, double* mu, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    const int nblk = div_up(n, kMeanRows);
    Buf part;
    MGB_TRY(part.alloc(sizeof(double) * (size_t)nblk * d, s));
    { col_partial_sum_kernel<<<nblk, 256, 0, s>>>(X, n, d, ld, part.as<double>()); note_launch(); }
    { col_mean_kernel<<<div_up(d, 256), 256, 0, s>>>(part.as<double>(), nblk, d, n, mu); note_launch(); }
    return cudaGetLastError();
}

// Eccentricity with exponent 2 (§3 and §4.1 name eccentricity among the
// common filters): the mean squared distance from x to the cloud equals
// |x - mu|^2 + mean_y |y - mu|^2 (mu the column means), so f(x) =
// sqrt(|x - mu|^2 + V) in FP64 without any pair of points: column means by
// fixed-order block sums, |x - mu|^2 summed k ascending, V their mean.
cudaError_t lens_ecc2(const float* X, int64_t n, int32_t d, int64_t ld, double* f, int m, int j, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    const int nblk = div_up(n, kMeanRows);
    Buf part, mu, vpart;
    MGB_TRY(part.alloc(sizeof(double) * (size_t)nblk * d, s));
    MGB_TRY(mu.alloc(sizeof(double) * d, s));
    MGB_TRY(vpart.alloc(sizeof(double) * kMeanBlocks, s));
    { col_partial_sum_kernel<<<nblk, 256, 0, s>>>(X, n, d, ld, part.as<double>()); note_launch(); }
    { col_mean_kernel<<<div_up(d, 256), 256, 0, s>>>(part.as<double>(), nblk, d, n, mu.as<double>()); note_launch(); }
    { lens_rows_kernel<2><<<div_up(n, kRows), kRows, 0, s>>>(X, n, d, ld, mu.as<double>(), nullptr, f, m, j);
      note_launch(); }
    { col_lens_partial_kernel<<<kMeanBlocks, 256, 0, s>>>(f, n, m, j, vpart.as<double>()); note_launch(); }
    { ecc_finish_kernel<<<std::min(div_up(n, 256), 152 * 8), 256, 0, s>>>(f, n, m, j, vpart.as<double>(), kMeanBlocks);
      note_launch(); }
    return cudaGetLastError();
}

// L-infinity norm filter (§5: the breast-cancer graphs filter by the
// "L_infinity-norm"), read as the norm of the point: f(x) = max_k |x_k|.
cudaError_t lens_linf(const float* X, int64_t n, int32_t d, int64_t ld, double* f, int m, int j, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    const int blocks = (int)std::min<int64_t>(div_up(n, 8), 152 * 8);
    { lens_linf_kernel<<<blocks, 256, 0, s>>>(X, n, d, ld, f, m, j); note_launch(); }
    return cudaGetLastError();
}

cudaError_t lens_coord(const float* X, int64_t n, int64_t ld, int32_t col, double* f, int m,
                       int j, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    { lens_coord_kernel<<<div_up(n, 256), 256, 0, s>>>(X, n, ld, col, f, m, j); note_launch(); }
    return cudaGetLastError();
}

cudaError_t check_finite(const float* X, int64_t n, int32_t d, int64_t ld, int* flag,
                         cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    const int blocks = (int)std::min<int64_t>(152 * 8, div_up(n, 8));
    const bool vec = ld % 4 == 0 && ((uintptr_t)X & 15) == 0;
    { finite_kernel<<<blocks, 256, 0, s>>>(X, n, d, ld, vec, flag); note_launch(); }
    return cudaGetLastError();
}

cudaError_t pca_axes(const float* X, int64_t n, int32_t d, int64_t ld, int K, double* mu,
                     double* axes, int* status, cudaStream_t s)
{
    const int nblk = div_up(n, kMeanRows);
    Buf part;
    MGB_TRY(part.alloc(sizeof(double) * (size_t)nblk * d, s));
    { col_partial_sum_kernel<<<nblk, 256, 0, s>>>(X, n, d, ld, part.as<double>()); note_launch(); }
    { col_mean_kernel<<<div_up(d, 256), 256, 0, s>>>(part.as<double>(), nblk, d, n, mu); note_launch(); }
    MGB_TRY(cudaGetLastError());

    const int ntile = div_up(d, kCovT);
    const int ntri = ntile * (ntile + 1) / 2;
    const int nchunk = div_up(n, kCovRows);
    Buf cpart, C;
    MGB_TRY(cpart.alloc(sizeof(float) * (size_t)nchunk * ntri * kCovT * kCovT, s));
    MGB_TRY(C.alloc(sizeof(double) * (size_t)d * d, s));
    { cov_partial_kernel<<<dim3(ntri, nchunk), 256, 0, s>>>(X, n, d, ld, mu, cpart.as<float>(), ntile); note_launch(); }
    { cov_reduce_kernel<<<ntri, 256, 0, s>>>(cpart.as<float>(), nchunk, ntile, d, n, C.as<double>()); note_launch(); }
    MGB_TRY(cudaGetLastError());
    const size_t smem = sizeof(double) * 2 * (size_t)d;
    if (smem > 48 * 1024)
        MGB_TRY(cudaFuncSetAttribute(power_iter_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem));
    { power_iter_kernel<<<1, 1024, smem, s>>>(C.as<double>(), d, K, axes, status); note_launch(); }
    return cudaGetLastError();
}

}  // namespace mgb
