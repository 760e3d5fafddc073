// common.cuh -- internal declarations shared by the library's translation
// units (never installed; the public ABI is include/mapper.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

namespace mgb {

// ------------------------------------------------------------ error plumbing
// Every internal step returns a cudaError_t; the C ABI layer turns it into a
// mapper_status and records a message for mapper_last_error().
void set_error(const std::string& msg);

// Kernels launched by the calling thread since the counter was last reset
// (every launch site adds to it; reported per call in mapper_stats).
extern thread_local int64_t g_launches;
inline void note_launch(int k = 1) { g_launches += k; }

#define MGB_TRY(expr)                                                       \
    do {                                                                    \
        cudaError_t e__ = (expr);                                           \
        if (e__ != cudaSuccess) return e__;                                 \
    } while (0)

inline int div_up(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

// Index checks of the checked build (compiled with -DMAPPER_BOUNDS_CHECK):
// an index outside [0, n) adds one to *oob (when oob is set) and the guarded
// access is skipped; the host turns a nonzero count into MAPPER_EINTERNAL.
// In the normal build the checks compile to nothing.
#ifdef MAPPER_BOUNDS_CHECK
__device__ __forceinline__ bool mgb_in_range(int64_t i, int64_t n, unsigned long long* oob)
{
    if (i >= 0 && i < n) return true;
    if (oob) atomicAdd(oob, 1ull);
    return false;
}
#define MGB_IN_RANGE(i, n, oob) ::mgb::mgb_in_range((int64_t)(i), (int64_t)(n), (oob))
#else
#define MGB_IN_RANGE(i, n, oob) true
#endif

// ------------------------------------------------------- stream-ordered memory
// Scratch and result arrays come from the device's stream-ordered pool
// (cudaMallocAsync); `Buf` frees on destruction on the same stream.
struct Buf {
    void* p = nullptr;
    size_t bytes = 0;
    cudaStream_t s = nullptr;
    Buf() = default;
    Buf(const Buf&) = delete;
    Buf& operator=(const Buf&) = delete;
    Buf(Buf&& o) noexcept { *this = static_cast<Buf&&>(o); }
    Buf& operator=(Buf&& o) noexcept {
        if (this != &o) { release(); p = o.p; bytes = o.bytes; s = o.s; o.p = nullptr; o.bytes = 0; }
        return *this;
    }
    ~Buf() { release(); }
    cudaError_t alloc(size_t nbytes, cudaStream_t stream) {
        release();
        s = stream;
        bytes = nbytes;
        if (nbytes == 0) nbytes = 16;
        return cudaMallocAsync(&p, nbytes, stream);
    }
    void release() {
        if (p) cudaFreeAsync(p, s);
        p = nullptr;
        bytes = 0;
    }
    template <class T> T* as() const { return static_cast<T*>(p); }
};

// ------------------------------------------------------------------ kernels
// lens (k_lens.cu)
cudaError_t lens_l2(const float* X, int64_t n, int32_t d, int64_t ld, double* f, int m, int j,
                    cudaStream_t s);
cudaError_t lens_ecc2(const float* X, int64_t n, int32_t d, int64_t ld, double* f, int m, int j,
                      cudaStream_t s);
// k-th nearest-neighbour distances of q query rows (device indices) over all
// n rows, the row itself first; out: q doubles on the device. Returns a
// mapper_status (k in [1, min(16, n)]).
// tensor_cores: screen on the tensor cores (else the FP32 CUDA-core screen);
// sample: large clouds take the sampled-threshold screen (else the list
// screen alone). info (nullable, 8 entries): the path taken (0 CUDA cores,
// 1 tensor-core lists, 2 sampled threshold), the queries over capacity, the
// capacity per query, the sample's tile stride (0 where not sampled), the
// keys below the thresholds, the largest such count of a query, and the
// candidates given FP32 sums and FP64 distances by the merges.
// screen_finite: the tensor-core path checks the rows for NaN / Inf while
// it builds its operands (no separate pass) and returns MAPPER_ENONFINITE,
// computing nothing, if a row's |row - c|^2 is not finite; the caller then
// decides exactly.
int knn_distance(const float* X, int64_t n, int32_t d, int64_t ld, const int32_t* queries_dev, int64_t q,
                 int32_t k, double* out_dev, int num_sms, bool tensor_cores, cudaStream_t s,
                 int64_t* info = nullptr, bool sample = true, bool screen_finite = false);
// Whether knn_distance takes the tensor-core path for these arguments.
bool knn_on_tensor_cores(int32_t k, bool tensor_cores);
// L-infinity centrality f(x) = max_y |x - y| into f[p * m + j]; a mapper_status.
int lens_ecc_inf(const float* X, int64_t n, int32_t d, int64_t ld, double* f, int m, int j, int num_sms,
                 bool tensor_cores, cudaStream_t s);
// lens_l2 that also writes, for the pivot assignment, the rows x - c rounded to
// BF16 (xh: n rows of pitch dp, columns d .. dp zero) and |x - c|^2 in FP32
// (xn2); d <= 32768 (else cudaErrorInvalidValue).
cudaError_t lens_l2_split(const float* X, int64_t n, int32_t d, int64_t ld, double* f, int m, int j,
                          const float* c, int dp, void* xh, float* xn2, cudaStream_t s);
cudaError_t lens_coord(const float* X, int64_t n, int64_t ld, int32_t col, double* f, int m,
                       int j, cudaStream_t s);
cudaError_t lens_linf(const float* X, int64_t n, int32_t d, int64_t ld, double* f, int m, int j,
                      cudaStream_t s);
cudaError_t lens_project(const float* X, int64_t n, int32_t d, int64_t ld, const double* mu,
                         const double* v, double* f, int m, int j, cudaStream_t s);
// Column means of X (FP64, fixed-order block sums): mu[d] on the device.
cudaError_t column_means(const float* X, int64_t n, int32_t d, int64_t ld, double* mu, cudaStream_t s);
// Principal axes: mu (d doubles) and K axes (K*d doubles), device outputs.
cudaError_t pca_axes(const float* X, int64_t n, int32_t d, int64_t ld, int K, double* mu,
                     double* axes, int* status, cudaStream_t s);
// Non-finite scan: sets *flag to 1 if any X entry is NaN/Inf.
cudaError_t check_finite(const float* X, int64_t n, int32_t d, int64_t ld, int* flag,
                         cudaStream_t s);

// cover (k_cover.cu)
// bounds: per lens dim j, a_j[n_int_j], b_j[n_int_j] (device, packed one
// after the other); lohi: 2*m doubles (min, max per dim).
cudaError_t lens_range_flag(const double* f, int64_t n, int m, double* lohi, int* nonfinite,
                            cudaStream_t s);
cudaError_t interval_bounds(const double* lohi, int m, const int32_t* n_int_host,
                            const double* p_host, double* bounds, cudaStream_t s);
// interval bounds of the balanced cover (same layout as interval_bounds)
cudaError_t balanced_bounds(const double* f, int64_t n, int m, const int32_t* n_int_host, const double* p_host,
                            double* bounds, cudaStream_t s);
// number of memberships per point (cnt[n]) and the emitted element keys
cudaError_t cover_count(const double* f, int64_t n, int m, const double* bounds,
                        int32_t n0, int32_t n1, int32_t* cnt, cudaStream_t s);
cudaError_t cover_emit(const double* f, int64_t n, int m, const double* bounds, int32_t n0,
                       int32_t n1, const int64_t* pos, uint64_t* keys, cudaStream_t s);

// scan / sort / compaction (k_sort.cu)
cudaError_t exclusive_scan_i32_to_i64(const int32_t* in, int64_t* out, int64_t n,
                                      cudaStream_t s);   // out has n+1 entries
cudaError_t exclusive_scan_i64(const int64_t* in, int64_t* out, int64_t n, cudaStream_t s);
// Stable LSD radix sort of 64-bit keys on bits [lo_bit, hi_bit). In place
// (keys) with a scratch buffer of the same size.
cudaError_t radix_sort_u64(uint64_t* keys, uint64_t* tmp, int64_t n, int lo_bit, int hi_bit,
                           cudaStream_t s);

// slots of a cover with one element holding every point (slot i = point i)
cudaError_t whole_cloud_slots(int64_t n, int32_t* slot_point, int32_t* slot_elem, cudaStream_t s);

// split sorted (element << 32 | point) keys into slot_point / slot_elem
cudaError_t split_keys(const uint64_t* keys, int64_t M, int32_t* slot_point, int32_t* slot_elem,
                       cudaStream_t s);

}  // namespace mgb
