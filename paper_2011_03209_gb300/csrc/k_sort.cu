// k_sort.cu -- exclusive scans and a stable LSD radix sort of 64-bit keys.
//
// These are the data-movement primitives behind cover bucketing (sort of
// (element, point) keys), node emission (sort of (node, point) keys) and the
// nerve (sort-unique of (node, node) keys). The sort is stable, so sorting a
// key on its high field only keeps the low field's incoming order.
#include "common.cuh"

namespace mgb {

namespace {

// ---------------------------------------------------------------- scan
constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ __forceinline__ int64_t block_exclusive_scan(int64_t v, int64_t* total)
{
    __shared__ int64_t warp_sums[kScanThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int64_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int64_t w = lane < kScanThreads / 32 ? warp_sums[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < kScanThreads / 32) warp_sums[lane] = w;
    }
    __syncthreads();
    const int64_t before = warp ? warp_sums[warp - 1] : 0;
    *total = warp_sums[kScanThreads / 32 - 1];
    __syncthreads();
    return before + x - v;
}

template <class T>
__global__ void __launch_bounds__(kScanThreads) scan_reduce_kernel(const T* __restrict__ in, int64_t n,
                                                                   int64_t* __restrict__ sums)
{
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    int64_t s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        const int64_t idx = base + (int64_t)threadIdx.x * kScanItems + i;
        if (idx < n) s += (int64_t)in[idx];
    }
    int64_t total;
    block_exclusive_scan(s, &total);
    if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

template <class T>
__global__ void __launch_bounds__(kScanThreads) scan_apply_kernel(const T* __restrict__ in, int64_t n,
                                                                  const int64_t* __restrict__ offs,
                                                                  int64_t* __restrict__ out,
                                                                  bool write_total)
{
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    int64_t v[kScanItems];
    int64_t s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        const int64_t idx = base + (int64_t)threadIdx.x * kScanItems + i;
        v[i] = idx < n ? (int64_t)in[idx] : 0;
        s += v[i];
    }
    int64_t total;
    int64_t run = block_exclusive_scan(s, &total) + (offs ? offs[blockIdx.x] : 0);
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        const int64_t idx = base + (int64_t)threadIdx.x * kScanItems + i;
        if (idx < n) out[idx] = run;
        run += v[i];
    }
    if (write_total && blockIdx.x == gridDim.x - 1 && threadIdx.x == kScanThreads - 1) out[n] = run;
}

// Exclusive scan of up to kScanOneMax values in one CTA (one launch, no
// scratch): thread t sums its contiguous run of the input, the CTA scans the
// run sums, then each thread writes its run's prefixes.
constexpr int kScanOneThreads = 1024;
constexpr int64_t kScanOneMax = 1 << 15;

template <class T>
__global__ void __launch_bounds__(kScanOneThreads) scan_one_kernel(const T* __restrict__ in, int64_t n,
                                                                   int64_t* __restrict__ out)
{
    __shared__ int64_t warp_sums[kScanOneThreads / 32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t per = (n + kScanOneThreads - 1) / kScanOneThreads;
    const int64_t b = (int64_t)tid * per, e = min(n, b + per);
    int64_t v = 0;
    for (int64_t i = b; i < e; ++i) v += (int64_t)in[i];
    int64_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int64_t w = warp_sums[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        warp_sums[lane] = w;
    }
    __syncthreads();
    int64_t run = (warp ? warp_sums[warp - 1] : 0) + x - v;
    for (int64_t i = b; i < e; ++i) {
        out[i] = run;
        run += (int64_t)in[i];
    }
    if (tid == kScanOneThreads - 1) out[n] = warp_sums[kScanOneThreads / 32 - 1];
}

template <class T>
cudaError_t exclusive_scan_impl(const T* in, int64_t* out, int64_t n, cudaStream_t s)
{
    // out[0..n) = exclusive prefix sums, out[n] = total
    if (n == 0) return cudaMemsetAsync(out, 0, sizeof(int64_t), s);
    const int64_t nb = div_up(n, kScanTile);
    if (nb == 1) {
        { scan_apply_kernel<T><<<1, kScanThreads, 0, s>>>(in, n, nullptr, out, true); note_launch(); }
        return cudaGetLastError();
    }
    if (n <= kScanOneMax) {
        { scan_one_kernel<T><<<1, kScanOneThreads, 0, s>>>(in, n, out); note_launch(); }
        return cudaGetLastError();
    }
    Buf sums, offs;
    MGB_TRY(sums.alloc(sizeof(int64_t) * nb, s));
    MGB_TRY(offs.alloc(sizeof(int64_t) * (nb + 1), s));
    { scan_reduce_kernel<T><<<(unsigned)nb, kScanThreads, 0, s>>>(in, n, sums.as<int64_t>()); note_launch(); }
    MGB_TRY(cudaGetLastError());
    MGB_TRY(exclusive_scan_impl<int64_t>(sums.as<int64_t>(), offs.as<int64_t>(), nb, s));
    { scan_apply_kernel<T><<<(unsigned)nb, kScanThreads, 0, s>>>(in, n, offs.as<int64_t>(), out, true); note_launch(); }
    return cudaGetLastError();
}

// ---------------------------------------------------------------- radix sort
constexpr int kRsThreads = 256;
constexpr int kRsWarps = kRsThreads / 32;
constexpr int kRsItems = 16;                         // rounds per warp
constexpr int kRsTile = kRsThreads * kRsItems;       // 4096 keys per block
constexpr int kRsBins = 256;

__device__ __forceinline__ int digit_of(uint64_t k, int shift, uint32_t mask)
{
    return (int)((k >> shift) & mask);
}

// hist[digit * nblocks + block]
__global__ void __launch_bounds__(kRsThreads) radix_hist_kernel(const uint64_t* __restrict__ keys,
                                                                int64_t n, int shift, uint32_t mask,
                                                                int64_t* __restrict__ hist)
{
    __shared__ int cnt[kRsBins];
    for (int b = threadIdx.x; b < kRsBins; b += kRsThreads) cnt[b] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kRsTile;
    for (int i = threadIdx.x; i < kRsTile; i += kRsThreads) {
        const int64_t idx = base + i;
        if (idx < n) atomicAdd(&cnt[digit_of(keys[idx], shift, mask)], 1);
    }
    __syncthreads();
    for (int b = threadIdx.x; b < kRsBins; b += kRsThreads)
        hist[(int64_t)b * gridDim.x + blockIdx.x] = cnt[b];
}

// Each warp ranks a contiguous run of 32 * kRsItems keys, round by round
// (lane order inside a round), so ranks follow input order: the sort is
// stable. Warp offsets per digit are then combined across the block.
__global__ void __launch_bounds__(kRsThreads) radix_scatter_kernel(const uint64_t* __restrict__ in,
                                                                   uint64_t* __restrict__ out,
                                                                   int64_t n, int shift, uint32_t mask,
                                                                   const int64_t* __restrict__ offs)
{
    __shared__ int wcnt[kRsWarps][kRsBins];
    __shared__ int64_t boff[kRsBins];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int b = lane; b < kRsBins; b += 32) wcnt[warp][b] = 0;
    for (int b = threadIdx.x; b < kRsBins; b += kRsThreads) boff[b] = offs[(int64_t)b * gridDim.x + blockIdx.x];
    __syncwarp();
    const unsigned lt = (1u << lane) - 1u;
    const int64_t wbase = (int64_t)blockIdx.x * kRsTile + (int64_t)warp * 32 * kRsItems;
    uint64_t key[kRsItems];
    int rank[kRsItems];
#pragma unroll
    for (int r = 0; r < kRsItems; ++r) {
        const int64_t idx = wbase + r * 32 + lane;
        const bool valid = idx < n;
        key[r] = valid ? in[idx] : 0ull;
        const int dg = valid ? digit_of(key[r], shift, mask) : kRsBins + lane;
        const unsigned peers = __match_any_sync(0xffffffffu, dg);
        const int before = valid ? wcnt[warp][dg] : 0;
        rank[r] = before + __popc(peers & lt);
        __syncwarp();
        if (valid && (peers & lt) == 0) wcnt[warp][dg] = before + __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    // exclusive prefix over warps per digit (in place)
    for (int b = threadIdx.x; b < kRsBins; b += kRsThreads) {
        int run = 0;
        for (int w = 0; w < kRsWarps; ++w) {
            const int c = wcnt[w][b];
            wcnt[w][b] = run;
            run += c;
        }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kRsItems; ++r) {
        const int64_t idx = wbase + r * 32 + lane;
        if (idx < n) {
            const int dg = digit_of(key[r], shift, mask);
            out[boff[dg] + wcnt[warp][dg] + rank[r]] = key[r];
        }
    }
}

}  // namespace

cudaError_t exclusive_scan_i32_to_i64(const int32_t* in, int64_t* out, int64_t n, cudaStream_t s)
{
    return exclusive_scan_impl<int32_t>(in, out, n, s);
}

cudaError_t exclusive_scan_i64(const int64_t* in, int64_t* out, int64_t n, cudaStream_t s)
{
    return exclusive_scan_impl<int64_t>(in, out, n, s);
}

cudaError_t radix_sort_u64(uint64_t* keys, uint64_t* tmp, int64_t n, int lo_bit, int hi_bit,
                           cudaStream_t s)
{
    if (n <= 1 || hi_bit <= lo_bit) return cudaSuccess;
    const int64_t nb = div_up(n, kRsTile);
    Buf hist, offs;
    MGB_TRY(hist.alloc(sizeof(int64_t) * kRsBins * nb, s));
    MGB_TRY(offs.alloc(sizeof(int64_t) * (kRsBins * nb + 1), s));
    uint64_t* src = keys;
    uint64_t* dst = tmp;
    for (int shift = lo_bit; shift < hi_bit; shift += 8) {
        const int bits = hi_bit - shift < 8 ? hi_bit - shift : 8;
        const uint32_t mask = (1u << bits) - 1u;
        { radix_hist_kernel<<<(unsigned)nb, kRsThreads, 0, s>>>(src, n, shift, mask, hist.as<int64_t>()); note_launch(); }
        MGB_TRY(cudaGetLastError());
        MGB_TRY(exclusive_scan_i64(hist.as<int64_t>(), offs.as<int64_t>(), kRsBins * nb, s));
        { radix_scatter_kernel<<<(unsigned)nb, kRsThreads, 0, s>>>(src, dst, n, shift, mask,
                                                                  offs.as<int64_t>()); note_launch(); }
        MGB_TRY(cudaGetLastError());
        uint64_t* t = src; src = dst; dst = t;
    }
    if (src != keys)
        MGB_TRY(cudaMemcpyAsync(keys, src, sizeof(uint64_t) * n, cudaMemcpyDeviceToDevice, s));
    return cudaSuccess;
}

}  // namespace mgb
