// k_noalloc.cu -- DBSCAN of one point set with no device allocation.
//
// mapper_cluster takes its scratch (gathered rows, neighbour counts,
// union-find parents, border roots) from the stream-ordered pool with
// cudaMallocAsync. Some callers cannot allocate device memory at all: a host
// framework that owns every device allocation through a fixed memory plan
// and forbids its plug-ins from allocating, or a latency-critical caller that
// must never let an allocation synchronise the device or fail half way. For
// them, mapper_dbscan_noalloc runs the same three screening passes on scratch
// held in one file-scope device array of fixed size (about 8.6 MB, held by
// every GPU that loads the library until the process exits).
//
// Use: the array's device address is looked up with cudaGetSymbolAddress
// the first time a call runs in a CUDA context (normally the device's primary
// context) and cached under that context's unique id, so a context that is
// destroyed and created again (cudaDeviceReset, a released primary context)
// gets a fresh lookup; a context whose id cannot be read is looked up on
// every call. The first call in a context should come before any stream
// capture. Every call reuses the same array, so two calls that overlap on
// the GPU (on two streams, or from two threads) race on it; calls must be
// ordered by the caller.
#include <cuda.h>

#include <climits>
#include <cmath>
#include <map>
#include <mutex>
#include <string>

#include "../../include/mapper.h"
#include "dbscan.cuh"

namespace mgb {

namespace {

constexpr int64_t kNaPoints = MAPPER_NOALLOC_MAX_POINTS;
constexpr int kNaDim = MAPPER_NOALLOC_MAX_DIM;     // also the largest row pitch (multiple of 32)

// byte offsets inside the array (each a multiple of 256)
constexpr size_t kNaRowsOff = 0;                                      // kNaPoints x kNaDim float
constexpr size_t kNaCountOff = kNaRowsOff + sizeof(float) * kNaPoints * kNaDim;
constexpr size_t kNaParentOff = kNaCountOff + sizeof(int32_t) * kNaPoints;
constexpr size_t kNaRootOff = kNaParentOff + sizeof(int32_t) * kNaPoints;
constexpr size_t kNaBorderOff = kNaRootOff + sizeof(int32_t) * kNaPoints;
constexpr size_t kNaCoreOff = kNaBorderOff + sizeof(unsigned long long) * kNaPoints;
constexpr size_t kNaMetaOff = kNaCoreOff + kNaPoints;                // offsets, stats, flag
constexpr size_t kNaBytes = kNaMetaOff + 256;
static_assert(kNaCoreOff % 256 == 0 && kNaMetaOff % 256 == 0, "scratch layout alignment");

struct NaMeta {
    int64_t elem_off[2];
    int64_t pair_off[2];
    unsigned long long stats[kStatCount];
    int nonfinite;
};
static_assert(sizeof(NaMeta) <= 256, "meta block");

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNaBytes];

std::mutex g_na_mutex;
std::map<unsigned long long, void*> g_na_addr;     // context id -> the array's address there

typedef CUresult (*PfnCtxGetCurrent)(CUcontext*);
typedef CUresult (*PfnCtxGetId)(CUcontext, unsigned long long*);

// Unique id of the calling thread's current CUDA context (ids are never
// reused within a process); false if it cannot be read.
bool current_context_id(unsigned long long* id)
{
    static PfnCtxGetCurrent get_current = nullptr;
    static PfnCtxGetId get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        cudaDriverEntryPointQueryResult q;
        void* p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<PfnCtxGetCurrent>(p);
        p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<PfnCtxGetId>(p);
    });
    CUcontext ctx = nullptr;
    if (!get_current || !get_id || get_current(&ctx) != CUDA_SUCCESS || !ctx) return false;
    return get_id(ctx, id) == CUDA_SUCCESS;
}

// Device address of the array in the current context (looked up once per
// context, or on every call when the context's id cannot be read).
cudaError_t scratch_address(unsigned char** out)
{
    unsigned long long id = 0;
    const bool keyed = current_context_id(&id);
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (keyed) {
        auto it = g_na_addr.find(id);
        if (it != g_na_addr.end()) {
            *out = static_cast<unsigned char*>(it->second);
            return cudaSuccess;
        }
    }
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    if (keyed) g_na_addr[id] = p;
    *out = static_cast<unsigned char*>(p);
    return cudaSuccess;
}

// True if p is device (or managed) memory of `device`.
cudaError_t on_device(const void* p, int device, bool* ok)
{
    cudaPointerAttributes attr{};
    const cudaError_t e = cudaPointerGetAttributes(&attr, p);
    if (e != cudaSuccess) return e;
    *ok = (attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged) && attr.device == device;
    return cudaSuccess;
}

// Clears what must start at zero, writes the single element's offsets and
// copies the rows (zero padded to the pitch), flagging non-finite values.
__global__ void na_setup_kernel(const float* __restrict__ X, int64_t n, int d, int64_t ld, int dp,
                                float* __restrict__ G, int32_t* __restrict__ count, NaMeta* meta)
{
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    if (tid == 0) {
        const int64_t T = (n + 127) / 128;
        meta->elem_off[0] = 0;
        meta->elem_off[1] = n;
        meta->pair_off[0] = 0;
        meta->pair_off[1] = T * (T + 1) / 2;
        for (int i = 0; i < kStatCount; ++i) meta->stats[i] = 0ull;
        meta->nonfinite = 0;
    }
    for (int64_t s = tid; s < n; s += stride) count[s] = 0;
    bool bad = false;
    for (int64_t i = tid; i < n * dp; i += stride) {
        const int64_t r = i / dp;
        const int k = (int)(i - r * dp);
        float v = 0.f;
        if (k < d) {
            v = X[r * ld + k];
            bad |= !isfinite(v);
        }
        G[i] = v;
    }
    if (bad) atomicOr(&meta->nonfinite, 1);
}

// label = canonical id (row of the cluster's smallest core point) or -1
__global__ void na_labels_kernel(const uint8_t* __restrict__ core, const int32_t* __restrict__ root,
                                 const unsigned long long* __restrict__ border, int64_t n,
                                 int64_t* __restrict__ label, uint8_t* __restrict__ core_out)
{
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    int64_t l = -1;
    if (core[s]) l = root[s];
    else if (border[s] != ~0ull) l = (int64_t)(border[s] & 0xffffffffull);
    if (label) label[s] = l;
    if (core_out) core_out[s] = core[s];
}

}  // namespace

}  // namespace mgb

using namespace mgb;

extern "C" int mapper_dbscan_noalloc(const float* X_dev, int64_t n, int32_t d, int64_t ld,
                                     double eps, int32_t min_pts, int64_t* label_dev,
                                     uint8_t* core_dev, void* cuda_stream)
{
    if (!X_dev || !label_dev) { set_error("X_dev and label_dev must not be null"); return MAPPER_EINVAL; }
    if (n < 1 || n > kNaPoints) {
        set_error("mapper_dbscan_noalloc: n must be in [1, MAPPER_NOALLOC_MAX_POINTS = 8192]");
        return MAPPER_EINVAL;
    }
    if (d < 1 || d > kNaDim) {
        set_error("mapper_dbscan_noalloc: d must be in [1, MAPPER_NOALLOC_MAX_DIM = 256]");
        return MAPPER_EINVAL;
    }
    if (ld < d) { set_error("ld must be >= d"); return MAPPER_EINVAL; }
    if (!(eps > 0.0) || !std::isfinite(eps)) { set_error("eps must be finite and > 0"); return MAPPER_EINVAL; }
    if (min_pts < 1) { set_error("min_pts must be >= 1"); return MAPPER_EINVAL; }

    int device = 0;
    cudaError_t e = cudaGetDevice(&device);
    const void* ptrs[3] = {X_dev, label_dev, core_dev};
    const char* names[3] = {"X_dev", "label_dev", "core_dev"};
    for (int i = 0; i < 3 && e == cudaSuccess; ++i) {
        if (!ptrs[i]) continue;
        bool ok = false;
        e = on_device(ptrs[i], device, &ok);
        if (e == cudaSuccess && !ok) {
            set_error(std::string("mapper_dbscan_noalloc: ") + names[i] + " is not device memory of the current device");
            return MAPPER_EINVAL;
        }
    }
    if (e != cudaSuccess) {
        set_error(std::string("mapper_dbscan_noalloc: ") + cudaGetErrorString(e));
        return MAPPER_ECUDA;
    }
    unsigned char* base = nullptr;
    if ((e = scratch_address(&base)) != cudaSuccess) {
        set_error(std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        return MAPPER_ECUDA;
    }
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    const int dp = (d + 31) / 32 * 32;
    float* G = reinterpret_cast<float*>(base + kNaRowsOff);
    int32_t* count = reinterpret_cast<int32_t*>(base + kNaCountOff);
    int32_t* parent = reinterpret_cast<int32_t*>(base + kNaParentOff);
    int32_t* root = reinterpret_cast<int32_t*>(base + kNaRootOff);
    unsigned long long* border = reinterpret_cast<unsigned long long*>(base + kNaBorderOff);
    uint8_t* core = base + kNaCoreOff;
    NaMeta* meta = reinterpret_cast<NaMeta*>(base + kNaMetaOff);

    const int64_t T = (n + 127) / 128;
    const int64_t n_pairs = T * (T + 1) / 2;
    na_setup_kernel<<<304, 256, 0, s>>>(X_dev, n, d, ld, dp, G, count, meta);
    note_launch();

    PassArgs a{};
    a.G = G;
    a.dp = dp;
    a.d = d;
    a.elem_off = meta->elem_off;
    a.pair_off = meta->pair_off;
    a.E = 1;
    a.eps2 = eps * eps;
    a.tie_thr = 1e-12 * a.eps2;
    fp32_thresholds(a.eps2, d, &a.lo_thr, &a.hi_thr);
    a.count = count;
    a.core = core;
    a.parent = parent;
    a.root = root;
    a.border = border;
    a.stats = meta->stats;

    const char* where = "setup";
    if ((e = cudaGetLastError()) == cudaSuccess && (where = "pass 1", e = simt_pass(1, a, n_pairs, s)) == cudaSuccess &&
        (where = "core", e = core_flags(count, n, min_pts, core, parent, border, meta->stats, s)) == cudaSuccess &&
        (where = "pass 2", e = simt_pass(2, a, n_pairs, s)) == cudaSuccess &&
        (where = "flatten", e = flatten(parent, core, n, root, s)) == cudaSuccess &&
        (where = "pass 3", e = simt_pass(3, a, n_pairs, s)) == cudaSuccess) {
        where = "labels";
        na_labels_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(core, root, border, n, label_dev, core_dev);
        note_launch();
        e = cudaGetLastError();
    }
    int nonfinite = 0;
    if (e == cudaSuccess) {
        where = "read flag";
        e = cudaMemcpyAsync(&nonfinite, &meta->nonfinite, sizeof(int), cudaMemcpyDeviceToHost, s);
    }
    if (e == cudaSuccess) {
        where = "sync";
        e = cudaStreamSynchronize(s);
    }
    if (e != cudaSuccess) {
        set_error(std::string("mapper_dbscan_noalloc ") + where + ": " + cudaGetErrorString(e));
        // kernels queued before the failure still use the shared array: let
        // them finish so that a retry (on any stream) does not race with them
        cudaStreamSynchronize(s);
        return MAPPER_ECUDA;
    }
    if (nonfinite) { set_error("X holds NaN or Inf"); return MAPPER_ENONFINITE; }
    return MAPPER_OK;
}
