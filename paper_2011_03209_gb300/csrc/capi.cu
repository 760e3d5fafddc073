// capi.cu -- the C ABI (include/mapper.h) and the host side of the pipeline:
// argument checks, handle ownership, stream-ordered scratch, size read-backs,
// and the order of the kernel launches of each step.
#include <algorithm>
#include <cfloat>
#include <cstdio>
#include <cstdlib>
#include <climits>
#include <cmath>
#include <cstring>
#include <map>
#include <memory>
#include <string>
#include <vector>

#include "../../include/mapper.h"
#include "dbscan.cuh"
#include "tc.cuh"

namespace mgb {

thread_local std::string g_last_error;
thread_local int64_t g_launches = 0;
void set_error(const std::string& msg) { g_last_error = msg; }

}  // namespace mgb

using namespace mgb;

namespace {

constexpr uint32_t kMagic = 0x4d415052u;   // "MAPR"
enum : uint32_t { kKindCover = 1, kKindClusters = 2, kKindGraph = 3, kKindForest = 4 };

struct HandleHdr {
    uint32_t magic;
    uint32_t kind;
};

// Owns (or borrows) the stream; every result array holds a reference so the
// stream outlives the stream-ordered frees of the arrays.
struct StreamHolder {
    cudaStream_t s = nullptr;
    bool owned = false;
    ~StreamHolder() { if (owned && s) cudaStreamDestroy(s); }
};
using StreamRef = std::shared_ptr<StreamHolder>;

struct CoverData {
    StreamRef stream;          // first member: destroyed last
    int m = 1;
    int32_t n_int[2] = {1, 1};
    double overlap[2] = {0, 0};
    int64_t n = 0, E = 0, M = 0;
    Buf keys;                  // sorted (element << 32 | point), M
    Buf elem_off;              // E + 1 int64
    Buf slot_point, slot_elem; // M int32 each
    std::vector<int64_t> h_elem_off;
};

struct ClusterData {
    StreamRef stream;
    std::shared_ptr<CoverData> cover;
    Buf core, lab, is_root, is_member, slot_label;    // per cover slot
    mapper_stats stats{};
};

}  // namespace

struct mapper_ctx {
    int device = 0;
    StreamRef stream;
    size_t budget = 0;
    bool timing = false;
    int num_sms = 152;
    std::map<uint64_t, int> pass1_tile_n;      // autotuner: (row pitch, products) -> N
    int pass1_forced = 0;                      // 128 or 256: fixed by the caller
    int cross_mode = 0;                        // cross-segment pairs: 0 auto, 1 tensor cores, 2 CUDA cores
    int knn_mode = 0;                          // k-distance screen: 0 auto (tensor cores), 1 tensor, 2 CUDA cores,
                                               // 3 tensor-core lists only
    int64_t knn_info[8] = {0, 0, 0, 0, 0, 0, 0, 0};  // the last k-distance call's path (mapper_knn_info)
    int64_t band_cap = 0;                      // band-queue entries (0: sized from the tile pairs)
    int screen_mode = 0;                       // MAPPER_BF16 count pass: 0 one or two phases from a sample,
                                               // 1 two phases, 2 three products, 3 two phases deferring
                                               // every mixed block
};

struct mapper_cover_t {
    HandleHdr h{kMagic, kKindCover};
    std::shared_ptr<CoverData> c;
    bool view = false;
};

struct mapper_clusters_t {
    HandleHdr h{kMagic, kKindClusters};
    std::shared_ptr<ClusterData> c;
    bool view = false;
};

struct mapper_forest_t {
    HandleHdr h{kMagic, kKindForest};
    StreamRef stream;
    std::shared_ptr<CoverData> cover;
    ForestOut f;
    double eps = 0.0;
    mapper_stats stats{};
};

struct mapper_graph_t {
    HandleHdr h{kMagic, kKindGraph};
    StreamRef stream;
    std::shared_ptr<ClusterData> clusters;
    Buf node_off, node_members, node_elem, edges, lens, pca;
    int64_t N = 0, Gm = 0, Eg = 0, n = 0, m = 1, n_pca = 0;
    mapper_stats stats{};
    mapper_cover_t cover_view;
    mapper_clusters_t clusters_view;
};

namespace {

int fail(int status, const std::string& msg)
{
    set_error(msg);
    return status;
}

int cuda_fail(cudaError_t e, const char* where)
{
    return fail(e == cudaErrorMemoryAllocation ? MAPPER_ENOMEM : MAPPER_ECUDA,
                std::string(where) + ": " + cudaGetErrorString(e));
}

#define CK(expr, where)                                                    \
    do {                                                                   \
        cudaError_t e_ = (expr);                                           \
        if (e_ != cudaSuccess) return cuda_fail(e_, where);                \
    } while (0)

int bits_for(int64_t n)      // bits to hold values 0 .. n-1
{
    int b = 1;
    while (b < 63 && (int64_t(1) << b) < n) ++b;
    return b;
}

struct Timer {
    bool on;
    cudaStream_t s;
    cudaEvent_t ev[8]{};
    int n = 0;
    Timer(bool on_, cudaStream_t s_) : on(on_), s(s_) {}
    ~Timer() { for (int i = 0; i < n; ++i) cudaEventDestroy(ev[i]); }
    void mark() {
        if (!on || n >= 8) return;
        cudaEventCreate(&ev[n]);
        cudaEventRecord(ev[n], s);
        ++n;
    }
    double ms(int a, int b) const {
        if (!on || b >= n) return 0.0;
        float t = 0.f;
        cudaEventSynchronize(ev[b]);
        cudaEventElapsedTime(&t, ev[a], ev[b]);
        return t;
    }
};

int check_ctx(mapper_ctx* ctx)
{
    if (!ctx) return fail(MAPPER_EINVAL, "null context");
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    return MAPPER_OK;
}

int check_x(const float* X, int64_t n, int32_t d, int64_t ld)
{
    if (!X) return fail(MAPPER_EINVAL, "X is null");
    if (n < 1 || n > INT32_MAX) return fail(MAPPER_EINVAL, "n must be in [1, 2^31)");
    if (d < 1) return fail(MAPPER_EINVAL, "d must be >= 1");
    if (ld < d) return fail(MAPPER_EINVAL, "ld must be >= d");
    return MAPPER_OK;
}

// ------------------------------------------------------------------- lens
int run_density(mapper_ctx* ctx, const float* X, int64_t n, int32_t d, int64_t ld, double r, int32_t precision,
                double* f, int m, int j);

int run_lens(mapper_ctx* ctx, const float* X, int64_t n, int32_t d, int64_t ld, int32_t m,
             const int32_t* kinds, const int32_t* args, const double* lens_param, int32_t precision,
             double* lens_dev, Buf* pca_dev, int64_t* n_pca, PivotSet* split = nullptr)
{
    cudaStream_t s = ctx->stream->s;
    int K = 0;
    for (int j = 0; j < m; ++j) {
        if (kinds[j] == MAPPER_LENS_DENSITY &&
            (!lens_param || !(lens_param[j] > 0.0) || !std::isfinite(lens_param[j])))
            return fail(MAPPER_EINVAL, "density lens radius must be finite and > 0");
        if (kinds[j] == MAPPER_LENS_COORD && (args[j] < 0 || args[j] >= d))
            return fail(MAPPER_EINVAL, "coordinate lens column out of range");
        if (kinds[j] == MAPPER_LENS_PCA) {
            if (args[j] < 0 || args[j] >= d) return fail(MAPPER_EINVAL, "PCA axis out of range");
            K = std::max(K, args[j] + 1);
        }
        if (kinds[j] < 0 || kinds[j] > MAPPER_LENS_ECC_INF) return fail(MAPPER_EINVAL, "unknown lens kind");
    }
    *n_pca = 0;
    Buf status;
    if (K) {
        CK(pca_dev->alloc(sizeof(double) * (size_t)d * (K + 1), s), "alloc pca");
        CK(status.alloc(sizeof(int), s), "alloc");
        CK(pca_axes(X, n, d, ld, K, pca_dev->as<double>(), pca_dev->as<double>() + d,
                    status.as<int>(), s), "pca");
        *n_pca = (int64_t)d * (K + 1);
    }
    for (int j = 0; j < m; ++j) {
        if (kinds[j] == MAPPER_LENS_L2 && split) {
            // the first L2 lens also writes the points' split for the pivot assignment
            const int dp = (d + 31) / 32 * 32;
            CK(lens_l2_split(X, n, d, ld, lens_dev, m, j, split->c.as<float>(), dp, split->xh.p,
                             split->xn2.as<float>(), s), "lens_l2");
            split = nullptr;
        } else if (kinds[j] == MAPPER_LENS_L2) CK(lens_l2(X, n, d, ld, lens_dev, m, j, s), "lens_l2");
        else if (kinds[j] == MAPPER_LENS_COORD)
            CK(lens_coord(X, n, ld, args[j], lens_dev, m, j, s), "lens_coord");
        else if (kinds[j] == MAPPER_LENS_ECC)
            CK(lens_ecc2(X, n, d, ld, lens_dev, m, j, s), "lens_ecc2");
        else if (kinds[j] == MAPPER_LENS_LINF)
            CK(lens_linf(X, n, d, ld, lens_dev, m, j, s), "lens_linf");
        else if (kinds[j] == MAPPER_LENS_DENSITY) {
            const int rc = run_density(ctx, X, n, d, ld, lens_param[j], precision, lens_dev, m, j);
            if (rc) return rc;
        } else if (kinds[j] == MAPPER_LENS_ECC_INF) {
            const int rc = lens_ecc_inf(X, n, d, ld, lens_dev, m, j, ctx->num_sms, precision != MAPPER_FP32, s);
            if (rc) return rc;
        } else
            CK(lens_project(X, n, d, ld, pca_dev->as<double>(),
                            pca_dev->as<double>() + (size_t)d * (1 + args[j]), lens_dev, m, j, s),
               "lens_project");
    }
    return MAPPER_OK;
}

// ------------------------------------------------------------------ cover
int run_cover(mapper_ctx* ctx, const double* lens, int64_t n, int32_t m, const int32_t* n_int,
              const double* overlap, std::shared_ptr<CoverData>* out, int* nonfinite_dev, bool balanced = false)
{
    if (m < 1 || m > 2) return fail(MAPPER_EINVAL, "m must be 1 or 2");
    for (int j = 0; j < m; ++j) {
        if (n_int[j] < 1) return fail(MAPPER_EINVAL, "n_intervals must be >= 1");
        if (!(overlap[j] >= 0.0 && overlap[j] < 1.0)) return fail(MAPPER_EINVAL, "overlap must be in [0, 1)");
    }
    const int64_t E = (int64_t)n_int[0] * (m == 2 ? n_int[1] : 1);
    if (E > (int64_t(1) << 30)) return fail(MAPPER_EINVAL, "too many cover elements");
    cudaStream_t s = ctx->stream->s;
    auto c = std::make_shared<CoverData>();
    c->stream = ctx->stream;
    c->m = m;
    c->n = n;
    c->E = E;
    for (int j = 0; j < m; ++j) { c->n_int[j] = n_int[j]; c->overlap[j] = overlap[j]; }

    Buf lohi, bounds, cnt, pos, flag;
    CK(lohi.alloc(sizeof(double) * 2 * m, s), "alloc");
    CK(bounds.alloc(sizeof(double) * 2 * ((size_t)n_int[0] + (m == 2 ? n_int[1] : 0)), s), "alloc");
    CK(cnt.alloc(sizeof(int32_t) * n, s), "alloc");
    CK(pos.alloc(sizeof(int64_t) * (n + 1), s), "alloc");
    int* nf = nonfinite_dev;
    if (!nf) {
        CK(flag.alloc(sizeof(int), s), "alloc");
        CK(cudaMemsetAsync(flag.p, 0, sizeof(int), s), "memset");
        nf = flag.as<int>();
    }
    CK(lens_range_flag(lens, n, m, lohi.as<double>(), nf, s), "lens_range");
    if (balanced) CK(balanced_bounds(lens, n, m, n_int, overlap, bounds.as<double>(), s), "balanced bounds");
    else CK(interval_bounds(lohi.as<double>(), m, n_int, overlap, bounds.as<double>(), s), "bounds");
    CK(cover_count(lens, n, m, bounds.as<double>(), n_int[0], m == 2 ? n_int[1] : 1,
                   cnt.as<int32_t>(), s), "cover_count");
    CK(exclusive_scan_i32_to_i64(cnt.as<int32_t>(), pos.as<int64_t>(), n, s), "scan");
    int64_t M = 0;
    int h_nf = 0;
    CK(cudaMemcpyAsync(&M, pos.as<int64_t>() + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s), "copy");
    CK(cudaMemcpyAsync(&h_nf, nf, sizeof(int), cudaMemcpyDeviceToHost, s), "copy");
    CK(cudaStreamSynchronize(s), "sync");
    if (h_nf) return fail(MAPPER_ENONFINITE, "lens or X holds NaN or Inf");
    if (M > INT32_MAX) return fail(MAPPER_ENOMEM, "more than 2^31 cover memberships");
    c->M = M;
    Buf tmp;
    CK(c->keys.alloc(sizeof(uint64_t) * M, s), "alloc keys");
    CK(tmp.alloc(sizeof(uint64_t) * M, s), "alloc");
    CK(cover_emit(lens, n, m, bounds.as<double>(), n_int[0], m == 2 ? n_int[1] : 1,
                  pos.as<int64_t>(), c->keys.as<uint64_t>(), s), "cover_emit");
    CK(radix_sort_u64(c->keys.as<uint64_t>(), tmp.as<uint64_t>(), M, 32, 32 + bits_for(E), s), "sort");
    CK(c->elem_off.alloc(sizeof(int64_t) * (E + 1), s), "alloc");
    CK(element_offsets(c->keys.as<uint64_t>(), M, E, c->elem_off.as<int64_t>(), s), "elem_off");
    CK(c->slot_point.alloc(sizeof(int32_t) * M, s), "alloc");
    CK(c->slot_elem.alloc(sizeof(int32_t) * M, s), "alloc");
    CK(split_keys(c->keys.as<uint64_t>(), M, c->slot_point.as<int32_t>(), c->slot_elem.as<int32_t>(), s),
       "split");
    c->h_elem_off.resize(E + 1);
    CK(cudaMemcpyAsync(c->h_elem_off.data(), c->elem_off.p, sizeof(int64_t) * (E + 1),
                       cudaMemcpyDeviceToHost, s), "copy");
    CK(cudaStreamSynchronize(s), "sync");
    *out = c;
    return MAPPER_OK;
}

// Count-pass phases, decided per call (pass-1 screen 0): the first phase
// (one BF16 product, or three FP8 ones, deferring every 32 x 32 block whose
// rows' extremes leave a row undecided) runs on every stride-th pair of the
// tensor-core list into scratch outputs; with f the fraction of those pairs
// that defer a block, two phases cost about T1 + f T3 and one phase T3 (T1,
// T3: the one- and three-product passes over the list; T1 ~ 0.6 T3 at d =
// 256), so a call takes one phase when f exceeds kDeferMax. Lists shorter
// than kSampleMinPairs keep two phases.
constexpr double kDeferMax = 0.35;
constexpr int64_t kSampleMinPairs = 8192;
// Within a two-phase pass (MAPPER_BF16), the sample also decides per bin of
// the tile-pair statistic (pair_bins): a pair skipping the first phase saves
// its one-product screen (~0.55 T3/pair) and costs a three-product screen
// (T3/pair) when it would not have deferred, so bins whose sampled pairs
// deferred a block at least kDirectRate of the time (with at least
// kDirectSamples sampled pairs) go straight to three products.
// The same rates then choose one phase or two: two when the estimate
// sum over sampled pairs of (1 if its bin goes straight, else kPhase1Cost +
// its bin's deferred fraction), in T3 units per pair, is below kTwoPhaseGain
// per pair (one phase costs 1).
constexpr double kDirectRate = 0.5;
constexpr unsigned long long kDirectSamples = 16;
constexpr double kPhase1Cost = 0.55;
constexpr double kTwoPhaseGain = 0.97;

int sample_deferral(const mapper_ctx* ctx, const PassArgs& a, const TcArgs& first, int64_t n_pairs, int64_t R,
                    int cap, cudaStream_t s, double* frac, const uint8_t* bins = nullptr,
                    unsigned long long* h_bins = nullptr)
{
    (void)ctx;
    const int64_t n_s = std::min<int64_t>(std::max<int64_t>(n_pairs / 64, 2048), n_pairs);
    const int64_t stride = n_pairs / n_s;
    Buf sp, cnt, nbr, hit, q, qn, st, err, mask;
    CK(sp.alloc(sizeof(int2) * n_s, s), "alloc");
    CK(cnt.alloc(sizeof(int32_t) * R, s), "alloc");
    if (cap) CK(nbr.alloc(sizeof(int32_t) * (size_t)R * cap, s), "alloc");
    CK(hit.alloc(n_s, s), "alloc");
    CK(q.alloc(sizeof(uint2) * 1024, s), "alloc");
    CK(qn.alloc(sizeof(unsigned long long), s), "alloc");
    CK(st.alloc(sizeof(unsigned long long) * kStatCount, s), "alloc");
    CK(err.alloc(sizeof(int), s), "alloc");
    CK(mask.alloc(sizeof(uint32_t) * n_s, s), "alloc");
    CK(cudaMemsetAsync(cnt.p, 0, sizeof(int32_t) * R, s), "memset");
    if (cap) CK(cudaMemsetAsync(nbr.p, 0xff, sizeof(int32_t) * (size_t)R * cap, s), "memset");
    CK(cudaMemsetAsync(hit.p, 0, n_s, s), "memset");
    CK(cudaMemsetAsync(qn.p, 0, sizeof(unsigned long long), s), "memset");
    CK(cudaMemsetAsync(st.p, 0, sizeof(unsigned long long) * kStatCount, s), "memset");
    CK(cudaMemsetAsync(err.p, 0, sizeof(int), s), "memset");
    CK(cudaMemsetAsync(mask.p, 0, sizeof(uint32_t) * n_s, s), "memset");
    int rc = tc_sample_pairs(a.pairs, stride, n_s, sp.as<int2>(), s);
    if (rc) return rc;
    PassArgs as = a;
    as.pairs = sp.as<int2>();
    as.count = cnt.as<int32_t>();
    as.nbr = nbr.as<int32_t>();
    as.pair_hit = hit.as<uint8_t>();
    as.stats = st.as<unsigned long long>();
    TcArgs ts = first;
    // several radii: every radius writes the same scratch outputs
    for (int e = 0; e < ts.n_radii; ++e)
        ts.radii[e] = RadiusOut{cnt.as<int32_t>(), nbr.as<int32_t>(), hit.as<uint8_t>(), q.as<uint2>(),
                                qn.as<unsigned long long>(), st.as<unsigned long long>(), ts.radii[e].eps2};
    if (!ts.f8) ts.ns = 1;
    ts.defer = true;
    ts.defer_mixed = true;
    ts.redo_mask = mask.as<uint32_t>();
    ts.sub_mask = nullptr;
    ts.sub_q = nullptr;
    ts.queue = q.as<uint2>();
    ts.queue_n = qn.as<unsigned long long>();
    ts.queue_cap = 1024;
    ts.err = err.as<int>();
    ts.groups = nullptr;
    ts.groups_dev = nullptr;
    ts.n_dev = nullptr;
    ts.ev_begin = ts.ev_end = nullptr;
    if ((rc = tc_pass(ts.n_radii > 0 ? 5 : 1, as, ts, n_s, s))) return rc;
    unsigned long long h_redo = 0;
    int h_err = 0;
    Buf bc;
    if (bins && h_bins) {
        CK(bc.alloc(sizeof(unsigned long long) * 2 * kPairBins, s), "alloc");
        CK(sample_bins(mask.as<uint32_t>(), n_s, bins, stride, bc.as<unsigned long long>(), s), "sample bins");
        CK(cudaMemcpyAsync(h_bins, bc.p, sizeof(unsigned long long) * 2 * kPairBins, cudaMemcpyDeviceToHost, s),
           "copy");
    }
    CK(cudaMemcpyAsync(&h_redo, st.as<unsigned long long>() + kStatRedo, sizeof(h_redo), cudaMemcpyDeviceToHost, s),
       "copy");
    CK(cudaMemcpyAsync(&h_err, err.p, sizeof(int), cudaMemcpyDeviceToHost, s), "copy");
    CK(cudaStreamSynchronize(s), "sync");
    if (h_err) return fail(MAPPER_ETIMEOUT, "a tensor-core pass gave up waiting on a barrier (phase sample)");
    *frac = (double)h_redo / (double)n_s;
    return MAPPER_OK;
}

// Pass-1 autotuner. The tensor-core count kernel runs its tile pairs as work
// items of one pair (an M = 128, N = 128 product) or of two pairs sharing
// tile A (N = 256, tile A loaded once); which is faster depends on the row
// pitch (MMA work per pair against the fixed epilogue work) and the number of
// products. The first call for a (pitch, products, screen format, one radius
// or several) key times both shapes on a prefix of its own pair list, into
// scratch outputs, and the context keeps the faster; lists too short to time
// take N = 256 without caching.
int tune_pass1(mapper_ctx* ctx, const PassArgs& a, const TcArgs& t, int64_t n_pairs, int64_t R, int cap,
               cudaStream_t s, int* tile_n)
{
    if (ctx->pass1_forced) {
        *tile_n = ctx->pass1_forced;
        return MAPPER_OK;
    }
    const uint64_t key = ((uint64_t)a.dp << 8) | ((uint64_t)(t.n_radii > 1) << 5) | ((uint64_t)t.f8 << 4) |
                         (uint64_t)t.ns;
    auto it = ctx->pass1_tile_n.find(key);
    if (it != ctx->pass1_tile_n.end()) {
        *tile_n = it->second;
        return MAPPER_OK;
    }
    *tile_n = 256;
    const int64_t n_t = std::min<int64_t>(n_pairs, (int64_t)ctx->num_sms * 32);
    if (n_t < (int64_t)ctx->num_sms * 8) return MAPPER_OK;
    const unsigned long long qcap = 1ull << 20;
    Buf cnt, nbr, hit, q, qn, st, err, grp, gpos, mask;
    CK(cnt.alloc(sizeof(int32_t) * R, s), "alloc");
    if (t.defer) CK(mask.alloc(sizeof(uint32_t) * n_t, s), "alloc");
    if (cap) CK(nbr.alloc(sizeof(int32_t) * (size_t)R * cap, s), "alloc");
    CK(hit.alloc(n_t, s), "alloc");
    CK(q.alloc(sizeof(uint2) * qcap, s), "alloc");
    CK(qn.alloc(sizeof(unsigned long long), s), "alloc");
    CK(st.alloc(sizeof(unsigned long long) * kStatCount, s), "alloc");
    CK(err.alloc(sizeof(int), s), "alloc");
    CK(cudaMemsetAsync(err.p, 0, sizeof(int), s), "memset");
    PassArgs as = a;
    as.count = cnt.as<int32_t>();
    as.nbr = nbr.as<int32_t>();
    as.pair_hit = hit.as<uint8_t>();
    as.stats = st.as<unsigned long long>();
    TcArgs ts = t;
    ts.queue = q.as<uint2>();
    ts.queue_n = qn.as<unsigned long long>();
    ts.queue_cap = qcap;
    // several radii: the kernel over several radii is timed, every radius
    // writing the same scratch outputs
    for (int e = 0; e < ts.n_radii; ++e)
        ts.radii[e] = RadiusOut{cnt.as<int32_t>(), nbr.as<int32_t>(), hit.as<uint8_t>(), q.as<uint2>(),
                                qn.as<unsigned long long>(), st.as<unsigned long long>(), ts.radii[e].eps2};
    ts.err = err.as<int>();
    ts.groups = nullptr;
    ts.groups_dev = nullptr;
    ts.n_dev = nullptr;
    ts.redo_mask = mask.as<uint32_t>();
    ts.sub_mask = nullptr;
    ts.sub_q = nullptr;
    // each shape twice, alternating; the faster of each counts
    constexpr int kRuns = 4;
    cudaEvent_t ev[2 * kRuns] = {};
    struct Guard {
        cudaEvent_t* e;
        ~Guard() { for (int i = 0; i < 2 * kRuns; ++i) if (e[i]) cudaEventDestroy(e[i]); }
    } guard{ev};
    for (int i = 0; i < 2 * kRuns; ++i) CK(cudaEventCreate(&ev[i]), "event");
    for (int run = 0; run < kRuns; ++run) {
        const int v = run & 1;
        CK(cudaMemsetAsync(cnt.p, 0, sizeof(int32_t) * R, s), "memset");
        if (cap) CK(cudaMemsetAsync(nbr.p, 0xff, sizeof(int32_t) * (size_t)R * cap, s), "memset");
        CK(cudaMemsetAsync(hit.p, 0, n_t, s), "memset");
        CK(cudaMemsetAsync(st.p, 0, sizeof(unsigned long long) * kStatCount, s), "memset");
        if (t.defer) CK(cudaMemsetAsync(mask.p, 0, sizeof(uint32_t) * n_t, s), "memset");
        TcArgs tv = ts;
        tv.ev_begin = ev[2 * run];
        tv.ev_end = ev[2 * run + 1];
        if (v == 1) {
            int rc = tc_groups(a.pairs, n_t, &grp, &gpos, s);
            if (rc) return rc;
            tv.groups = grp.as<int2>();
            tv.n_groups = n_t;
            tv.groups_dev = reinterpret_cast<const unsigned long long*>(gpos.as<int64_t>() + n_t);
        }
        int rc = tc_pass(ts.n_radii > 0 ? 5 : 1, as, tv, n_t, s);
        if (rc) return rc;
    }
    int h_err = 0;
    CK(cudaMemcpyAsync(&h_err, err.p, sizeof(int), cudaMemcpyDeviceToHost, s), "copy");
    CK(cudaStreamSynchronize(s), "sync");
    if (h_err) return fail(MAPPER_ETIMEOUT, "a tensor-core pass gave up waiting on a barrier (autotuning)");
    float ms[2] = {INFINITY, INFINITY};
    for (int run = 0; run < kRuns; ++run) {
        float m = 0.f;
        CK(cudaEventElapsedTime(&m, ev[2 * run], ev[2 * run + 1]), "event time");
        ms[run & 1] = std::min(ms[run & 1], m);
    }
    *tile_n = ms[1] <= ms[0] ? 256 : 128;
    ctx->pass1_tile_n[key] = *tile_n;
    return MAPPER_OK;
}

// ---------------------------------------------------------------- cluster
// Per-element DBSCAN: tiles ordered by pivot group (k_tiles.cu), tile pairs
// classified by bounding spheres, then the passes over the three lists:
// all-in pairs need no distance, mixed pairs of one group go to the
// tensor-core screen (BF16) and all others to the CUDA-core FP32 screen.
// `layout` (optional): a tile layout of this cover built beforehand with
// operands for this precision, shared by several radii (a sweep).
// Where a counts-only run (the density filter) writes its neighbour counts:
// f[point * m + j].
struct CountsOut {
    double* f;
    int m, j;
};

// The same for n_radii radii eps[0] < eps[1] < .. of one cover (at most
// kMaxRadii; one radius unless the screen runs on BF16 tensor cores): one tile
// layout and one classification (pairs all out at the largest radius dropped,
// all in at the smallest counted without distances), one count pass over the
// mixed pairs for every radius (mode 5 of tc_pass), then the unions, border
// rows and labels of each radius. outs[e] receives radius e's clusters.
int run_cluster_radii(mapper_ctx* ctx, const float* X, int64_t n, int32_t d, int64_t ld,
                      const std::shared_ptr<CoverData>& cov, int n_radii, const double* eps_list, int32_t min_pts,
                      int32_t precision, std::shared_ptr<ClusterData>* outs, int* nonfinite_dev,
                      TileLayout* layout = nullptr, const CountsOut* counts_out = nullptr,
                      const PivotSet* pivots = nullptr)
{
    if (n_radii < 1 || n_radii > kMaxRadii) return fail(MAPPER_EINVAL, "bad number of radii");
    for (int e = 0; e < n_radii; ++e) {
        if (!(eps_list[e] > 0.0) || !std::isfinite(eps_list[e])) return fail(MAPPER_EINVAL, "eps must be finite and > 0");
        if (e > 0 && !(eps_list[e] > eps_list[e - 1])) return fail(MAPPER_EINTERNAL, "radii not ascending");
    }
    if (min_pts < 1) return fail(MAPPER_EINVAL, "min_pts must be >= 1");
    if (precision != MAPPER_FP32 && precision != MAPPER_BF16 && precision != MAPPER_BF16X1 &&
        precision != MAPPER_FP8)
        return fail(MAPPER_EINVAL, "unknown precision");
    if (cov->n != n) return fail(MAPPER_EINVAL, "cover was built for another point count");
    const int K = n_radii;
    if (K > 1 && (precision == MAPPER_FP32 || precision == MAPPER_FP8 || counts_out))
        return fail(MAPPER_EINTERNAL, "several radii need the BF16 tensor-core screen");
    const double eps_min = eps_list[0], eps_max = eps_list[K - 1];
    cudaStream_t s = ctx->stream->s;
    const int64_t M = cov->M, E = cov->E;
    const int dp = (d + 31) / 32 * 32;
    const bool use_tc = precision != MAPPER_FP32;
    const int cap = (!counts_out && min_pts >= 2 && min_pts - 1 <= 64) ? min_pts - 1 : 0;
    const double rows_est = (double)M + 128.0 * (double)E;
    const double est = rows_est * dp * (use_tc ? (precision == MAPPER_FP8 ? 10.0 : 8.0) : 4.0) +
                       K * rows_est * (40.0 + 4.0 * cap);
    if (ctx->budget && est > (double)ctx->budget)
        return fail(MAPPER_ENOMEM, "estimated scratch exceeds the context's HBM budget");

    mapper_stats st{};                                            // shared by the radii
    st.n_points = n;
    st.n_elements = E;
    st.n_members = M;
    double s2 = 0.0;
    for (int64_t e = 0; e < E; ++e) {
        const double ne = (double)(cov->h_elem_off[e + 1] - cov->h_elem_off[e]);
        s2 += ne * ne;
    }
    st.sum_ni2 = s2;

    // per radius: outputs, counters and the pass arguments
    struct Radius {
        Buf stats, count, nbr, core, parent, root, border, hit_tc, hit_simt, queue, queue_n;
        PassArgs a, a_in, a_tc, a_simt;
    };
    std::vector<Radius> rs(K);
    Buf shared_stats, flag;                                       // K > 1: the count pass's own counters
    for (int e = 0; e < K; ++e) {
        CK(rs[e].stats.alloc(sizeof(unsigned long long) * kStatCount, s), "alloc");
        CK(cudaMemsetAsync(rs[e].stats.p, 0, sizeof(unsigned long long) * kStatCount, s), "memset");
    }
    if (K > 1) {
        CK(shared_stats.alloc(sizeof(unsigned long long) * kStatCount, s), "alloc");
        CK(cudaMemsetAsync(shared_stats.p, 0, sizeof(unsigned long long) * kStatCount, s), "memset");
    }
    int* nf = nonfinite_dev;
    if (!nf) {
        CK(flag.alloc(sizeof(int), s), "alloc");
        CK(cudaMemsetAsync(flag.p, 0, sizeof(int), s), "memset");
        nf = flag.as<int>();
    }

    Timer pt(ctx->timing, s);
    pt.mark();                                                    // 0
    TileLayout own;
    int rc = MAPPER_OK;
    if (!layout) {
        rc = build_tiles(X, n, d, ld, dp, cov->slot_point.as<int32_t>(), cov->slot_elem.as<int32_t>(), M, E,
                         4.0 * eps_max, use_tc, ctx->num_sms, &own, nf, s, pivots);
        if (rc) return rc;
        layout = &own;
    }
    // FP8 screen: E4M3 operands with per-tile scales beside the BF16 ones (the
    // union pass and the second phase of the count pass stay in BF16)
    const bool f8 = precision == MAPPER_FP8;
    if (f8 && (rc = fp8_operands(layout, X, ld, d, dp, s))) return rc;
    const TileLayout& L = *layout;
    PairLists PL;
    if ((rc = classify_pairs(L, X, ld, d, dp, E, eps_max, use_tc, &PL, s, eps_min))) return rc;
    const int64_t R = L.R;
    st.tile_pairs = PL.n_candidates;
    st.tile_pairs_out = PL.n_out;
    st.tile_pairs_in = PL.n[kListAllIn];
    st.tile_pairs_tc = PL.n[kListTC];
    st.tile_pairs_simt = PL.n[kListSimt];
    st.n_groups = L.n_groups;
    if (PL.n[kListSimt] > INT32_MAX || PL.n[kListTC] > INT32_MAX || PL.n[kListAllIn] > INT32_MAX)
        return fail(MAPPER_ENOMEM, "too many tile pairs for one launch");

    // Mixed tile pairs across two segments of one element have no common
    // centre; when they are many (a cover element holding scattered points,
    // whose tiles have wide spheres), they run on the tensor cores too, with
    // a second operand set centred per element, instead of on CUDA cores.
    const bool cross_tc = use_tc && PL.n[kListSimt] > 0 && ctx->cross_mode != 2 &&
                          (ctx->cross_mode == 1 || PL.n[kListSimt] * 32 >= R);
    const unsigned long long queue_cap =
        ctx->band_cap > 0 ? (unsigned long long)ctx->band_cap
                          : (unsigned long long)std::min<int64_t>(
                                int64_t(1) << 25, std::max<int64_t>(int64_t(1) << 20, 128 * PL.n[kListTC]));
    for (int e = 0; e < K; ++e) {
        Radius& rd = rs[e];
        CK(rd.count.alloc(sizeof(int32_t) * R, s), "alloc");
        CK(rd.core.alloc(R, s), "alloc");
        CK(rd.parent.alloc(sizeof(int32_t) * R, s), "alloc");
        CK(rd.root.alloc(sizeof(int32_t) * R, s), "alloc");
        CK(rd.border.alloc(sizeof(unsigned long long) * R, s), "alloc");
        if (cap) {
            // every writer fills the slots below cap it reserves; -1 marks any left
            CK(rd.nbr.alloc(sizeof(int32_t) * (size_t)R * cap, s), "alloc");
            CK(cudaMemsetAsync(rd.nbr.p, 0xff, sizeof(int32_t) * (size_t)R * cap, s), "memset");
        }
        CK(cudaMemsetAsync(rd.count.p, 0, sizeof(int32_t) * R, s), "memset");
        PassArgs& a = rd.a;
        a = PassArgs{};
        a.G = L.G.as<float>();
        a.X = X;
        a.ld = ld;
        a.xvec = ld % 4 == 0 && ((uintptr_t)X & 15) == 0;
        a.dp = dp;
        a.d = d;
        a.tile_n = L.tile_n.as<int32_t>();
        a.eps2 = eps_list[e] * eps_list[e];
        a.tie_thr = 1e-12 * a.eps2;
        fp32_thresholds(a.eps2, d, &a.lo_thr, &a.hi_thr);
        a.row_pt = L.row_pt.as<int32_t>();
        a.count = rd.count.as<int32_t>();
        a.nbr = rd.nbr.as<int32_t>();
        a.cap = cap;
        a.core = rd.core.as<uint8_t>();
        a.parent = rd.parent.as<int32_t>();
        a.root = rd.root.as<int32_t>();
        a.border = rd.border.as<unsigned long long>();
        a.stats = rd.stats.as<unsigned long long>();
        a.n_rows = R;
        a.n_tiles = L.T;
    }
    // tensor-core pairs in (a, b) order: pairs sharing tile A form the
    // groups of the pass-1 kernel, and consecutive groups, which run on
    // neighbouring SMs at the same time, share tiles in L2
    for (int li : {(int)kListTC, (int)kListSimt}) {
        if (PL.n[li] <= 1 || (li == kListSimt && !cross_tc)) continue;
        Buf tmp;
        CK(tmp.alloc(sizeof(uint64_t) * PL.n[li], s), "alloc");
        uint64_t* keys = PL.list[li].as<uint64_t>();
        const int tb = bits_for(L.T);
        CK(radix_sort_u64(keys, tmp.as<uint64_t>(), PL.n[li], 32, 32 + tb, s), "sort pairs");
        CK(radix_sort_u64(keys, tmp.as<uint64_t>(), PL.n[li], 0, tb, s), "sort pairs");
    }
    // pass 1 flags the screened tile pairs holding a neighbour pair; only
    // those can matter to the union pass
    for (int e = 0; e < K; ++e) {
        Radius& rd = rs[e];
        CK(rd.hit_tc.alloc(std::max<int64_t>(PL.n[kListTC], 1), s), "alloc");
        CK(rd.hit_simt.alloc(std::max<int64_t>(PL.n[kListSimt], 1), s), "alloc");
        CK(cudaMemsetAsync(rd.hit_tc.p, 0, std::max<int64_t>(PL.n[kListTC], 1), s), "memset");
        CK(cudaMemsetAsync(rd.hit_simt.p, 0, std::max<int64_t>(PL.n[kListSimt], 1), s), "memset");
        rd.a_in = rd.a_tc = rd.a_simt = rd.a;
        rd.a_in.pairs = PL.list[kListAllIn].as<int2>();
        rd.a_tc.pairs = PL.list[kListTC].as<int2>();
        rd.a_tc.pair_hit = rd.hit_tc.as<uint8_t>();
        rd.a_simt.pairs = PL.list[kListSimt].as<int2>();
        rd.a_simt.pair_hit = rd.hit_simt.as<uint8_t>();
        if (use_tc) {
            CK(rd.queue.alloc(sizeof(uint2) * queue_cap, s), "alloc band queue");
            CK(rd.queue_n.alloc(sizeof(unsigned long long), s), "alloc");
        }
    }
    // the count pass's arguments: the largest radius's (its counters: the
    // shared ones when there are several radii)
    PassArgs a_tc = rs[K - 1].a_tc, a_simt = rs[K - 1].a_simt;
    if (K > 1) a_tc.stats = a_simt.stats = shared_stats.as<unsigned long long>();
    TcArgs t{};
    Buf tc_err;
    if (use_tc) {
        t.Ah = L.Ah.p;
        t.Al = L.Al.p;
        t.rn2 = L.rn2.as<float>();
        t.rn = L.rn.as<float>();
        t.rl = L.rl.as<float>();
        t.tmax = L.tmax.as<float4>();
        t.tn2min = L.tn2min.as<float>();
        t.R = R;
        t.ns = precision == MAPPER_BF16X1 ? 1 : 3;
        t.num_sms = ctx->num_sms;
        t.queue_cap = queue_cap;
        CK(tc_err.alloc(sizeof(int), s), "alloc");
        CK(cudaMemsetAsync(tc_err.p, 0, sizeof(int), s), "memset");
        t.queue = rs[K - 1].queue.as<uint2>();
        t.queue_n = rs[K - 1].queue_n.as<unsigned long long>();
        t.err = tc_err.as<int>();
    }

    TcArgs tx{};                                                  // the cross-segment operands
    Buf xAh, xAl, xrn2, xrn, xrl, xtmax, xtn2min;
    if (cross_tc) {
        if ((rc = cross_operands(L, X, ld, d, dp, E, &xAh, &xAl, &xrn2, &xrn, &xrl, &xtmax, &xtn2min, s))) return rc;
        tx = t;
        tx.Ah = xAh.p;
        tx.Al = xAl.p;
        tx.rn2 = xrn2.as<float>();
        tx.rn = xrn.as<float>();
        tx.rl = xrl.as<float>();
        tx.tmax = xtmax.as<float4>();
        tx.tn2min = xtn2min.as<float>();
    }
    st.tile_pairs_cross = cross_tc ? PL.n[kListSimt] : 0;
    // the radii of a count pass over several (mode 5): per radius its
    // outputs and the hit flags of one pair list from pair `off` on (none in
    // a second phase)
    auto with_radii = [&](TcArgs v, bool simt_list, bool hits, int64_t off = 0) {
        if (K == 1) return v;
        v.n_radii = K;
        for (int e = 0; e < K; ++e) {
            Radius& rd = rs[e];
            v.radii[e] = RadiusOut{rd.a.count, rd.a.nbr,
                                   hits ? (simt_list ? rd.a_simt.pair_hit : rd.a_tc.pair_hit) + off : nullptr,
                                   rd.queue.as<uint2>(), rd.queue_n.as<unsigned long long>(),
                                   rd.stats.as<unsigned long long>(), rd.a.eps2};
        }
        return v;
    };
    const int count_mode = K > 1 ? 5 : 1;
    // Count pass in two phases (MAPPER_BF16: one BF16 product first; MAPPER_FP8:
    // three FP8 products first): the 32 x 32 sub-blocks with a pair inside the
    // first screen's band run again with three BF16 products
    // (hi.hi + hi.lo + lo.hi); the others are final after the first
    bool two_phase = use_tc && t.ns == 3 && ctx->screen_mode != 2;
    TcArgs t8 = t;                                                // the FP8 operands of the first phase
    if (f8) {
        t8.f8 = true;
        t8.Ah = L.Fh.p;
        t8.Al = L.Fl.p;
        t8.rl = L.frl.as<float>();
        t8.tmax = L.ftmax.as<float4>();
    }
    // default screen: two phases or one, from a sample of the first phase
    const bool defer_mixed = ctx->screen_mode == 3 || ctx->screen_mode == 0;
    st.pass1_sample_deferred = -1.0;
    int64_t n_direct = 0;                                         // TC-list pairs straight to three products
    if (two_phase && ctx->screen_mode == 0 && PL.n[kListTC] >= kSampleMinPairs) {
        double f = 0.0;
        const int64_t n = PL.n[kListTC];
        const bool per_bin = !f8;
        Buf bins;
        unsigned long long h_bins[2 * kPairBins] = {};
        if (per_bin) {
            CK(bins.alloc(n, s), "alloc");
            CK(pair_bins(L, PL.list[kListTC].as<int2>(), n, dp, eps_max, bins.as<uint8_t>(), s), "pair bins");
        }
        if ((rc = sample_deferral(ctx, a_tc, with_radii(f8 ? t8 : t, false, true), n, R, cap, s, &f,
                                  per_bin ? bins.as<uint8_t>() : nullptr, per_bin ? h_bins : nullptr)))
            return rc;
        st.pass1_sample_deferred = f;
        uint8_t chosen[kPairBins] = {};
        bool any = false;
        if (per_bin) {
            double est_one = 0.0, est_two = 0.0;
            for (int b = 0; b < kPairBins; ++b) {
                const double c = (double)h_bins[2 * b];
                if (c == 0.0) continue;
                const double p = (double)h_bins[2 * b + 1] / c;
                chosen[b] = h_bins[2 * b] >= kDirectSamples && p >= kDirectRate;
                est_one += c;
                est_two += chosen[b] ? c : c * (kPhase1Cost + p);
            }
            two_phase = est_two < kTwoPhaseGain * est_one;
            for (int b = 0; two_phase && b < kPairBins; ++b) any |= chosen[b] != 0;
        } else if (f > kDeferMax) {
            two_phase = false;
        }
        if (any) {
            // the chosen bins' pairs first (list order kept within each part)
            Buf dchosen, part, pos;
            CK(dchosen.alloc(kPairBins, s), "alloc");
            CK(part.alloc(sizeof(int2) * n, s), "alloc");
            CK(cudaMemcpyAsync(dchosen.p, chosen, kPairBins, cudaMemcpyHostToDevice, s), "copy");
            CK(partition_pairs(PL.list[kListTC].as<int2>(), bins.as<uint8_t>(), dchosen.as<uint8_t>(), n,
                               part.as<int2>(), &pos, s), "partition");
            CK(cudaMemcpyAsync(PL.list[kListTC].p, part.p, sizeof(int2) * n, cudaMemcpyDeviceToDevice, s), "copy");
            CK(cudaMemcpyAsync(&n_direct, pos.as<int64_t>() + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s), "copy");
            CK(cudaStreamSynchronize(s), "sync");
        }
    }
    st.tile_pairs_direct = n_direct;
    st.pass1_phases = use_tc ? (two_phase ? 2 : 1) : 0;
    Buf redo, redo_mask, redo_q;
    if (two_phase) {
        const int64_t rcap = std::max<int64_t>(std::max(PL.n[kListTC], cross_tc ? PL.n[kListSimt] : 0), 1);
        CK(redo.alloc(sizeof(int2) * rcap, s), "alloc");
        CK(redo_mask.alloc(sizeof(uint32_t) * rcap, s), "alloc");
        CK(redo_q.alloc(sizeof(int32_t) * rcap, s), "alloc");
    }
    int tile_n = 0;
    // the first (or only) screen: FP8 products when chosen, except a
    // one-phase pass the sample picked (three BF16 products then)
    const bool first_f8 = f8 && (two_phase || ctx->screen_mode != 0);
    TcArgs t_tune = first_f8 ? t8 : t, tx_tune = tx;
    if (two_phase && !f8) t_tune.ns = 1;
    if (two_phase) tx_tune.ns = 1;
    t_tune.defer = tx_tune.defer = two_phase;                    // timed as the first phase runs
    t_tune.defer_mixed = tx_tune.defer_mixed = defer_mixed;
    // timed on the pairs the first screen will take (after those sent straight)
    PassArgs a_first = a_tc;
    a_first.pairs += n_direct;
    if (use_tc && PL.n[kListTC] > n_direct &&
        (rc = tune_pass1(ctx, a_first, with_radii(t_tune, false, true), PL.n[kListTC] - n_direct, R, cap, s,
                         &tile_n)))
        return rc;
    if (use_tc && PL.n[kListTC] == 0 && cross_tc &&
        (rc = tune_pass1(ctx, a_simt, with_radii(tx_tune, true, true), PL.n[kListSimt], R, cap, s, &tile_n)))
        return rc;
    // the pairs sent straight to three products: the shape tuned for three products
    int tile_n_direct = tile_n;
    if (n_direct > 0 && (rc = tune_pass1(ctx, a_tc, with_radii(t, false, true), n_direct, R, cap, s, &tile_n_direct)))
        return rc;
    pt.mark();                                                    // 1
    for (int e = 0; e < K; ++e) CK(allin_pass(1, rs[e].a_in, PL.n[kListAllIn], s), "pass 1 all-in");
    cudaEvent_t tev[2] = {nullptr, nullptr};
    if (ctx->timing) {
        CK(cudaEventCreate(&tev[0]), "event");
        CK(cudaEventCreate(&tev[1]), "event");
    }
    struct EvGuard {
        cudaEvent_t* e;
        ~EvGuard() { for (int i = 0; i < 2; ++i) if (e[i]) cudaEventDestroy(e[i]); }
    } tev_guard{tev};
    Buf groups, group_pos, xgroups, xgroup_pos;
    // pass 1 on the tensor cores of one pair list (its events bracket the
    // count kernels: both lists' launches when the cross list runs there)
    auto tc_count = [&](const PassArgs& pa, const TcArgs& base, const TcArgs& first_screen, int64_t np, Buf& gr,
                        Buf& gp, bool first, bool last, bool simt_list, bool two, int64_t off, int tn) -> int {
        TcArgs t1 = with_radii(first_screen, simt_list, true, off);
        t1.ev_begin = first ? tev[0] : nullptr;
        t1.ev_end = last && !two ? tev[1] : nullptr;
        if (tn == 256) {
            int r2;
            if ((r2 = tc_groups(pa.pairs, np, &gr, &gp, s))) return r2;
            t1.groups = gr.as<int2>();
            t1.n_groups = np;
            t1.groups_dev = reinterpret_cast<const unsigned long long*>(gp.as<int64_t>() + np);
        }
        if (!two) return tc_pass(count_mode, pa, t1, np, s);
        if (!t1.f8) t1.ns = 1;
        t1.defer = true;
        t1.defer_mixed = defer_mixed;
        t1.redo_mask = redo_mask.as<uint32_t>();
        CK(cudaMemsetAsync(redo_mask.p, 0, sizeof(uint32_t) * np, s), "memset");
        int r2;
        if ((r2 = tc_pass(count_mode, pa, t1, np, s))) return r2;
        // second phase: the tile pairs with deferred sub-blocks in list order,
        // grouped by tile A as in the first, counting only those sub-blocks
        // (their number stays on the device)
        Buf rpos, rgr, rgp;
        if ((r2 = tc_redo_list(pa.pairs, redo_mask.as<uint32_t>(), np, redo.as<int2>(), redo_q.as<int32_t>(), &rpos,
                               s, pa.stats + kStatRedoBlocks)))
            return r2;
        const unsigned long long* n_redo = reinterpret_cast<const unsigned long long*>(rpos.as<int64_t>() + np);
        PassArgs p2 = pa;
        p2.pairs = redo.as<int2>();
        p2.pair_hit = nullptr;
        TcArgs t2 = with_radii(base, simt_list, false);
        t2.groups = nullptr;
        t2.n_groups = 0;
        t2.groups_dev = nullptr;
        t2.n_dev = n_redo;
        if (tn == 256) {
            if ((r2 = tc_groups_dev(redo.as<int2>(), np, n_redo, &rgr, &rgp, s))) return r2;
            t2.groups = rgr.as<int2>();
            t2.n_groups = np;
            t2.groups_dev = reinterpret_cast<const unsigned long long*>(rgp.as<int64_t>() + np);
        }
        t2.sub_mask = redo_mask.as<uint32_t>();
        t2.sub_q = redo_q.as<int32_t>();
        t2.ev_begin = nullptr;
        t2.ev_end = last ? tev[1] : nullptr;
        return tc_pass(count_mode, p2, t2, np, s);
    };
    if (use_tc) {
        const bool x_last = cross_tc && PL.n[kListSimt] > 0;
        const int64_t n_rest = PL.n[kListTC] - n_direct;
        Buf dgroups, dgroup_pos;
        // the pairs sent straight to three products, then the rest in the chosen phases
        if (n_direct > 0 &&
            (rc = tc_count(a_tc, t, t, n_direct, dgroups, dgroup_pos, true, n_rest == 0 && !x_last, false, false, 0,
                           tile_n_direct)))
            return rc;
        PassArgs a_rest = a_tc;
        a_rest.pairs += n_direct;
        a_rest.pair_hit += n_direct;
        if (n_rest > 0 && (rc = tc_count(a_rest, t, first_f8 ? t8 : t, n_rest, groups, group_pos, n_direct == 0,
                                         !x_last, false, two_phase, n_direct, tile_n)))
            return rc;
        if (x_last && (rc = tc_count(a_simt, tx, tx, PL.n[kListSimt], xgroups, xgroup_pos, PL.n[kListTC] == 0, true,
                                     true, two_phase, 0, tile_n)))
            return rc;
    }
    else CK(simt_pass(1, rs[0].a_tc, PL.n[kListTC], s), "pass 1 tc list");
    if (!use_tc && tev[0]) CK(cudaEventRecord(tev[0], s), "event");
    if (!cross_tc)
        for (int e = 0; e < K; ++e) CK(simt_pass(1, rs[e].a_simt, PL.n[kListSimt], s), "pass 1");
    if (!use_tc && tev[1]) CK(cudaEventRecord(tev[1], s), "event");
    pt.mark();                                                    // 2
    int h_err = 0;
    if (counts_out) {
        // the counts are final after pass 1 (band pairs re-decided)
        const PassArgs& a = rs[0].a;
        CK(counts_to_lens(L.row_slot.as<int32_t>(), a.row_pt, a.count, R, counts_out->f, counts_out->m,
                          counts_out->j, s), "counts");
        int h_nf = 0;
        unsigned long long h_oob = 0;
        CK(cudaMemcpyAsync(&h_nf, nf, sizeof(int), cudaMemcpyDeviceToHost, s), "copy");
        CK(cudaMemcpyAsync(&h_oob, a.stats + kStatOob, sizeof(h_oob), cudaMemcpyDeviceToHost, s), "copy");
        if (use_tc) CK(cudaMemcpyAsync(&h_err, tc_err.p, sizeof(int), cudaMemcpyDeviceToHost, s), "copy");
        CK(cudaStreamSynchronize(s), "sync");
        if (h_nf) return fail(MAPPER_ENONFINITE, "X holds NaN or Inf");
        if (h_err) return fail(MAPPER_ETIMEOUT, "a tensor-core pass gave up waiting on a barrier");
        if (h_oob) return fail(MAPPER_EINTERNAL, "a device-side index check failed");
        auto c = std::make_shared<ClusterData>();
        c->stream = ctx->stream;
        c->cover = cov;
        c->stats = st;
        outs[0] = c;
        return MAPPER_OK;
    }
    unsigned long long h_shared[kStatCount] = {};
    if (K > 1) CK(cudaMemcpyAsync(h_shared, shared_stats.p, sizeof(h_shared), cudaMemcpyDeviceToHost, s), "copy");
    float ms_count = 0.f;
    bool have_ms_count = false;
    for (int e = 0; e < K; ++e) {
        Radius& rd = rs[e];
        const PassArgs& a = rd.a;
        auto c = std::make_shared<ClusterData>();
        c->stream = ctx->stream;
        c->cover = cov;
        c->stats = st;
        Timer pr(ctx->timing, s);
        CK(core_flags(a.count, R, min_pts, rd.core.as<uint8_t>(), a.parent, a.border, a.stats, s), "core");
        pr.mark();                                                // 0
        CK(list_unions(a.count, a.nbr, cap, a.core, a.parent, a.row_pt, R, s, a.stats + kStatOob), "list unions");
        CK(allin_pass(2, rd.a_in, PL.n[kListAllIn], s), "pass 2 all-in");
        // Unions in rounds of growing tile distance b - a (tiles of one pivot
        // region are adjacent), after the unions along the neighbour lists: a
        // pair is kept only if its core rows are not all joined yet (from the
        // second round on when there are no lists), and pairs whose two sides are
        // each already one component only need one neighbour pair.
        auto union_rounds = [&](const PassArgs& base, const TcArgs& tbase, int64_t n, bool tc) -> int {
            if (n == 0) return MAPPER_OK;
            // every count stays on the device: each launch covers the list's
            // capacity n and reads its length there, so the rounds need no host
            // round trip
            static const int kBounds[] = {-1, 1, 4, 16, 64, INT_MAX};
            Buf hits, sel, kept, cnt, troots;
            CK(troots.alloc(sizeof(int2) * std::max<int64_t>(L.T, 1), s), "alloc");
            CK(hits.alloc(sizeof(int2) * n, s), "alloc");
            CK(sel.alloc(sizeof(int2) * n, s), "alloc");
            CK(kept.alloc(sizeof(int2) * n, s), "alloc");
            CK(cnt.alloc(sizeof(unsigned long long) * 3, s), "alloc");
            unsigned long long* c_hit = cnt.as<unsigned long long>();
            unsigned long long* c_sel = c_hit + 1;
            unsigned long long* c_kept = c_hit + 2;
            CK(cudaMemsetAsync(c_hit, 0, sizeof(unsigned long long), s), "memset");
            CK(select_hit(base.pairs, base.pair_hit, n, hits.as<int2>(), c_hit, s), "select");
            CK(add_counter(base.stats + kStatUnion, c_hit, s), "count");
            for (int k = 0; k + 1 < (int)(sizeof(kBounds) / sizeof(kBounds[0])); ++k) {
                CK(cudaMemsetAsync(c_sel, 0, sizeof(unsigned long long) * 2, s), "memset");
                CK(select_delta(hits.as<int2>(), n, c_hit, kBounds[k], kBounds[k + 1], sel.as<int2>(), c_sel, s),
                   "select");
                const int2* list = sel.as<int2>();
                const unsigned long long* c_list = c_sel;
                if (k > 0 || cap) {
                    CK(filter_joined(base, L.T, troots.as<int2>(), sel.as<int2>(), n, c_sel, kept.as<int2>(), c_kept,
                                     s), "filter");
                    list = kept.as<int2>();
                    c_list = c_kept;
                }
                PassArgs ar = base;
                ar.pairs = list;
                ar.n_dev = c_list;
                ar.pair_hit = nullptr;
                int r2;
                if (tc) {
                    TcArgs t2 = tbase;
                    t2.n_dev = c_list;
                    if ((r2 = tc_pass(2, ar, t2, n, s))) return r2;
                } else {
                    CK(simt_pass(2, ar, n, s), "pass 2");
                }
            }
            return MAPPER_OK;
        };
        if (use_tc) {
            if ((rc = union_rounds(rd.a_tc, t, PL.n[kListTC], true))) return rc;
            if ((rc = union_rounds(rd.a_simt, tx, PL.n[kListSimt], cross_tc))) return rc;
        } else {
            if ((rc = union_rounds(rd.a_simt, t, PL.n[kListSimt], false))) return rc;
        }
        pr.mark();                                                // 1
        CK(flatten(a.parent, a.core, R, rd.root.as<int32_t>(), s), "flatten");
        if (cap) {
            CK(border_from_lists(a.count, a.nbr, cap, a.core, a.root, a.row_pt, R, a.border, s, a.stats + kStatOob),
               "border");
        } else if (min_pts > 1) {
            CK(allin_pass(3, rd.a_in, PL.n[kListAllIn], s), "pass 3 all-in");
            CK(simt_pass(3, rd.a_tc, PL.n[kListTC], s), "pass 3 tc list");
            CK(simt_pass(3, rd.a_simt, PL.n[kListSimt], s), "pass 3");
        }
        pr.mark();                                                // 2

        CK(c->core.alloc(M, s), "alloc");
        CK(c->lab.alloc(sizeof(int32_t) * M, s), "alloc");
        CK(c->is_root.alloc(sizeof(int32_t) * M, s), "alloc");
        CK(c->is_member.alloc(sizeof(int32_t) * M, s), "alloc");
        CK(c->slot_label.alloc(sizeof(int64_t) * M, s), "alloc");
        CK(rows_to_slots(L.row_slot.as<int32_t>(), a.row_pt, a.core, a.root, a.border, R, c->lab.as<int32_t>(),
                         c->is_root.as<int32_t>(), c->is_member.as<int32_t>(), c->slot_label.as<int64_t>(),
                         c->core.as<uint8_t>(), s), "labels");

        unsigned long long h_stats[kStatCount];
        int h_nf = 0;
        CK(cudaMemcpyAsync(h_stats, a.stats, sizeof(h_stats), cudaMemcpyDeviceToHost, s), "copy");
        CK(cudaMemcpyAsync(&h_nf, nf, sizeof(int), cudaMemcpyDeviceToHost, s), "copy");
        if (use_tc) CK(cudaMemcpyAsync(&h_err, tc_err.p, sizeof(int), cudaMemcpyDeviceToHost, s), "copy");
        CK(cudaStreamSynchronize(s), "sync");
        if (h_nf) return fail(MAPPER_ENONFINITE, "X holds NaN or Inf");
        if (h_err) return fail(MAPPER_ETIMEOUT, "a tensor-core pass gave up waiting on a barrier");
        // the count pass's counters (kept apart when there are several radii)
        for (int k : {(int)kStatScreened, (int)kStatTcPairs, (int)kStatRedo, (int)kStatRedoBlocks,
                      (int)kStatRedoParts, (int)kStatOob})
            h_stats[k] += h_shared[k];
        if (h_stats[kStatOob])
            return fail(MAPPER_EINTERNAL, "a device-side index check failed (" + std::to_string(h_stats[kStatOob]) +
                                              " indices out of range)");
        mapper_stats& sr = c->stats;
        sr.band_pairs = (int64_t)h_stats[kStatBand];
        sr.near_ties = (int64_t)h_stats[kStatTies];
        sr.pairs_screened = (int64_t)h_stats[kStatScreened];
        sr.n_core = (int64_t)h_stats[kStatCore];
        sr.union_skipped = (int64_t)h_stats[kStatSkipped];
        sr.fp64_pairs = (int64_t)h_stats[kStatFp64];
        sr.union_pairs = (int64_t)h_stats[kStatUnion];
        sr.pass1_tile_n = tile_n;
        sr.n_rows = R;
        sr.tile_pairs_screen1 = two_phase ? PL.n[kListTC] - n_direct + (cross_tc ? PL.n[kListSimt] : 0) : 0;
        sr.tile_pairs_redo = (int64_t)h_stats[kStatRedo];
        sr.redo_blocks = (int64_t)h_stats[kStatRedoBlocks];
        sr.redo_parts = (int64_t)h_stats[kStatRedoParts];
        if (tev[0] && (PL.n[use_tc ? kListTC : kListSimt] > 0 || cross_tc)) {
            if (!have_ms_count) CK(cudaEventElapsedTime(&ms_count, tev[0], tev[1]), "event time");
            have_ms_count = true;
            sr.ms_count_kernel = ms_count;
        }
        sr.count_kernel_pairs = (int64_t)h_stats[use_tc ? kStatTcPairs : kStatSimtPairs];
        if (pt.n >= 3 && pr.n >= 3) {
            sr.ms_tiles = pt.ms(0, 1);
            sr.ms_pass[0] = pt.ms(1, 2);
            sr.ms_pass[1] = pr.ms(0, 1);
            sr.ms_pass[2] = pr.ms(1, 2);
        }
        outs[e] = c;
    }
    return MAPPER_OK;
}

int run_cluster(mapper_ctx* ctx, const float* X, int64_t n, int32_t d, int64_t ld,
                const std::shared_ptr<CoverData>& cov, double eps, int32_t min_pts, int32_t precision,
                std::shared_ptr<ClusterData>* out, int* nonfinite_dev, TileLayout* layout = nullptr,
                const CountsOut* counts_out = nullptr, const PivotSet* pivots = nullptr)
{
    return run_cluster_radii(ctx, X, n, d, ld, cov, 1, &eps, min_pts, precision, out, nonfinite_dev, layout,
                             counts_out, pivots);
}

// Density filter (§4.1 names density among the derived filters; no estimator
// is given): the number of points within distance r of each point, itself
// included, i.e. pass 1 of DBSCAN(r, .) on one cover element holding the
// whole cloud. Exact: the counts are those of the FP64 definition.
int run_density(mapper_ctx* ctx, const float* X, int64_t n, int32_t d, int64_t ld, double r, int32_t precision,
                double* f, int m, int j)
{
    if (n > INT32_MAX) return fail(MAPPER_EINVAL, "density lens: more than 2^31 points");
    cudaStream_t s = ctx->stream->s;
    auto c = std::make_shared<CoverData>();
    c->stream = ctx->stream;
    c->m = 1;
    c->n = n;
    c->E = 1;
    c->M = n;
    CK(c->slot_point.alloc(sizeof(int32_t) * n, s), "alloc");
    CK(c->slot_elem.alloc(sizeof(int32_t) * n, s), "alloc");
    CK(whole_cloud_slots(n, c->slot_point.as<int32_t>(), c->slot_elem.as<int32_t>(), s), "slots");
    c->h_elem_off = {0, n};
    std::shared_ptr<ClusterData> cl;
    const CountsOut co{f, m, j};
    return run_cluster(ctx, X, n, d, ld, c, r, 1, precision, &cl, nullptr, nullptr, &co);
}

// ------------------------------------------------------------------ nerve
int nerve_edges(mapper_ctx* ctx, uint64_t* keys2, int64_t Gm, int64_t n_points, int64_t N, mapper_graph_t* g);

int run_nerve(mapper_ctx* ctx, const std::shared_ptr<ClusterData>& cl, mapper_graph_t* g)
{
    cudaStream_t s = ctx->stream->s;
    const auto& cov = cl->cover;
    const int64_t M = cov->M;
    Buf nid, mpos;
    CK(nid.alloc(sizeof(int64_t) * (M + 1), s), "alloc");
    CK(mpos.alloc(sizeof(int64_t) * (M + 1), s), "alloc");
    CK(exclusive_scan_i32_to_i64(cl->is_root.as<int32_t>(), nid.as<int64_t>(), M, s), "scan");
    CK(exclusive_scan_i32_to_i64(cl->is_member.as<int32_t>(), mpos.as<int64_t>(), M, s), "scan");
    int64_t h[2];
    CK(cudaMemcpyAsync(&h[0], nid.as<int64_t>() + M, sizeof(int64_t), cudaMemcpyDeviceToHost, s), "copy");
    CK(cudaMemcpyAsync(&h[1], mpos.as<int64_t>() + M, sizeof(int64_t), cudaMemcpyDeviceToHost, s), "copy");
    CK(cudaStreamSynchronize(s), "sync");
    const int64_t N = h[0], Gm = h[1];
    g->N = N;
    g->Gm = Gm;
    Buf keys, tmp, keys2;
    CK(keys.alloc(sizeof(uint64_t) * Gm, s), "alloc");
    CK(tmp.alloc(sizeof(uint64_t) * Gm, s), "alloc");
    CK(keys2.alloc(sizeof(uint64_t) * Gm, s), "alloc");
    CK(g->node_elem.alloc(sizeof(int32_t) * N, s), "alloc");
    CK(g->node_off.alloc(sizeof(int64_t) * (N + 1), s), "alloc");
    CK(g->node_members.alloc(sizeof(int32_t) * Gm, s), "alloc");
    CK(member_keys(cl->lab.as<int32_t>(), nid.as<int64_t>(), mpos.as<int64_t>(),
                   cov->slot_point.as<int32_t>(), cov->slot_elem.as<int32_t>(), M,
                   keys.as<uint64_t>(), g->node_elem.as<int32_t>(), s), "member keys");
    CK(radix_sort_u64(keys.as<uint64_t>(), tmp.as<uint64_t>(), Gm, 32, 32 + bits_for(N), s), "sort");
    CK(node_offsets(keys.as<uint64_t>(), Gm, g->node_off.as<int64_t>(), g->node_members.as<int32_t>(),
                    keys2.as<uint64_t>(), s), "node offsets");
    CK(cudaMemcpyAsync(g->node_off.as<int64_t>() + N, &g->Gm, sizeof(int64_t), cudaMemcpyHostToDevice, s),
       "copy");
    int rc = nerve_edges(ctx, keys2.as<uint64_t>(), Gm, cov->n, N, g);
    if (rc) return rc;
    g->stats = cl->stats;
    g->stats.n_nodes = N;
    g->stats.n_edges = g->Eg;
    return MAPPER_OK;
}

// Nerve edges from the memberships (point << 32 | node) of N nodes (the keys
// are sorted in place): group by point, emit each point's node pairs, sort,
// unique. Sets g->edges and g->Eg.
int nerve_edges(mapper_ctx* ctx, uint64_t* keys2, int64_t Gm, int64_t n_points, int64_t N, mapper_graph_t* g)
{
    cudaStream_t s = ctx->stream->s;
    Buf tmp;
    CK(tmp.alloc(sizeof(uint64_t) * std::max<int64_t>(Gm, 1), s), "alloc");
    CK(radix_sort_u64(keys2, tmp.as<uint64_t>(), Gm, 32, 32 + bits_for(n_points), s), "sort");
    Buf cnt, ppos;
    CK(cnt.alloc(sizeof(int64_t) * Gm, s), "alloc");
    CK(ppos.alloc(sizeof(int64_t) * (Gm + 1), s), "alloc");
    CK(run_pairs(keys2, Gm, cnt.as<int64_t>(), s), "run pairs");
    CK(exclusive_scan_i64(cnt.as<int64_t>(), ppos.as<int64_t>(), Gm, s), "scan");
    int64_t P = 0;
    CK(cudaMemcpyAsync(&P, ppos.as<int64_t>() + Gm, sizeof(int64_t), cudaMemcpyDeviceToHost, s), "copy");
    CK(cudaStreamSynchronize(s), "sync");
    Buf pairs, ptmp, flag, upos;
    CK(pairs.alloc(sizeof(uint64_t) * P, s), "alloc");
    CK(ptmp.alloc(sizeof(uint64_t) * P, s), "alloc");
    CK(emit_pairs(keys2, Gm, ppos.as<int64_t>(), pairs.as<uint64_t>(), s), "emit pairs");
    const int nb = bits_for(N);
    CK(radix_sort_u64(pairs.as<uint64_t>(), ptmp.as<uint64_t>(), P, 0, nb, s), "sort");
    CK(radix_sort_u64(pairs.as<uint64_t>(), ptmp.as<uint64_t>(), P, 32, 32 + nb, s), "sort");
    CK(flag.alloc(sizeof(int32_t) * P, s), "alloc");
    CK(upos.alloc(sizeof(int64_t) * (P + 1), s), "alloc");
    CK(unique_flags(pairs.as<uint64_t>(), P, flag.as<int32_t>(), s), "unique");
    CK(exclusive_scan_i32_to_i64(flag.as<int32_t>(), upos.as<int64_t>(), P, s), "scan");
    int64_t Eg = 0;
    CK(cudaMemcpyAsync(&Eg, upos.as<int64_t>() + P, sizeof(int64_t), cudaMemcpyDeviceToHost, s), "copy");
    CK(cudaStreamSynchronize(s), "sync");
    g->Eg = Eg;
    CK(g->edges.alloc(sizeof(int32_t) * 2 * Eg, s), "alloc");
    CK(unique_emit(pairs.as<uint64_t>(), flag.as<int32_t>(), upos.as<int64_t>(), P,
                   g->edges.as<int32_t>(), s), "unique emit");
    CK(cudaStreamSynchronize(s), "sync");
    return MAPPER_OK;
}

int copy_out(void* dst, const void* src, size_t bytes, int on_device, cudaStream_t s)
{
    if (!dst || bytes == 0) return MAPPER_OK;
    CK(cudaMemcpyAsync(dst, src, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s),
       "copy out");
    CK(cudaStreamSynchronize(s), "sync");
    return MAPPER_OK;
}

bool is_host_pointer(const void* p)
{
    cudaPointerAttributes attr;
    if (cudaPointerGetAttributes(&attr, p) != cudaSuccess) {
        cudaGetLastError();
        return true;
    }
    return attr.type == cudaMemoryTypeHost || attr.type == cudaMemoryTypeUnregistered;
}

template <class T>
T* handle_as(const void* h, uint32_t kind)
{
    if (!h) return nullptr;
    const HandleHdr* hh = static_cast<const HandleHdr*>(h);
    if (hh->magic != kMagic || hh->kind != kind) return nullptr;
    return const_cast<T*>(static_cast<const T*>(h));
}

}  // namespace

// =================================================================== C ABI
extern "C" {

int mapper_abi_version(void) { return MAPPER_ABI_VERSION; }

const char* mapper_last_error(void) { return g_last_error.c_str(); }

const char* mapper_strerror(int status)
{
    switch (status) {
    case MAPPER_OK: return "ok";
    case MAPPER_EINVAL: return "invalid argument";
    case MAPPER_ENOMEM: return "out of device memory or over budget";
    case MAPPER_ECUDA: return "CUDA error";
    case MAPPER_ETIMEOUT: return "device wait timed out";
    case MAPPER_ENONFINITE: return "input holds NaN or Inf";
    case MAPPER_EINTERNAL: return "internal consistency check failed";
    case MAPPER_ENOTIMPL: return "not implemented";
    case MAPPER_ECANCELED: return "request dropped by server shutdown";
    default: return "unknown status";
    }
}

namespace {

// Persistent autotuner choices: a text file named by MAPPER_TUNE_CACHE, a
// header line with the device name and SM count, then one "key tile_n" line
// per tuned (row pitch, format, products) key. Read when a context is
// created on the same kind of device; the context's choices are merged in
// and the file replaced (write to a temporary, then rename) when it is
// destroyed. Without the variable nothing is read or written.
std::string tune_cache_header(int device)
{
    cudaDeviceProp prop{};
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) return std::string();
    return std::string("mapper-tune-v1 ") + prop.name + " sms=" + std::to_string(prop.multiProcessorCount);
}

void tune_cache_load(mapper_ctx* ctx)
{
    const char* path = std::getenv("MAPPER_TUNE_CACHE");
    if (!path || !*path) return;
    std::FILE* f = std::fopen(path, "r");
    if (!f) return;
    char line[512];
    const std::string want = tune_cache_header(ctx->device);
    bool ok = std::fgets(line, sizeof(line), f) && !want.empty() && want == std::string(line).substr(0, want.size());
    unsigned long long key = 0;
    int tile_n = 0;
    while (ok && std::fscanf(f, "%llu %d", &key, &tile_n) == 2)
        if (tile_n == 128 || tile_n == 256) ctx->pass1_tile_n[key] = tile_n;
    std::fclose(f);
}

void tune_cache_save(const mapper_ctx* ctx)
{
    const char* path = std::getenv("MAPPER_TUNE_CACHE");
    if (!path || !*path || ctx->pass1_tile_n.empty()) return;
    const std::string head = tune_cache_header(ctx->device);
    if (head.empty()) return;
    std::map<uint64_t, int> all;
    if (std::FILE* f = std::fopen(path, "r")) {                // keep other contexts' keys
        char line[512];
        unsigned long long key = 0;
        int tile_n = 0;
        if (std::fgets(line, sizeof(line), f) && head == std::string(line).substr(0, head.size()))
            while (std::fscanf(f, "%llu %d", &key, &tile_n) == 2) all[key] = tile_n;
        std::fclose(f);
    }
    for (const auto& kv : ctx->pass1_tile_n) all[kv.first] = kv.second;
    const std::string tmp = std::string(path) + ".tmp" + std::to_string((unsigned long long)(uintptr_t)ctx);
    std::FILE* f = std::fopen(tmp.c_str(), "w");
    if (!f) return;
    std::fprintf(f, "%s\n", head.c_str());
    for (const auto& kv : all) std::fprintf(f, "%llu %d\n", (unsigned long long)kv.first, kv.second);
    const bool written = std::fclose(f) == 0;
    if (written) std::rename(tmp.c_str(), path);
    else std::remove(tmp.c_str());
}

}  // namespace

int mapper_create(mapper_ctx** out, int device, size_t hbm_budget_bytes, void* cuda_stream)
{
    if (!out) return fail(MAPPER_EINVAL, "out is null");
    *out = nullptr;
    int ndev = 0;
    CK(cudaGetDeviceCount(&ndev), "cudaGetDeviceCount");
    if (device < 0 || device >= ndev) return fail(MAPPER_EINVAL, "no such device");
    CK(cudaSetDevice(device), "cudaSetDevice");
    auto ctx = std::make_unique<mapper_ctx>();
    ctx->device = device;
    ctx->budget = hbm_budget_bytes;
    ctx->stream = std::make_shared<StreamHolder>();
    if (cuda_stream) {
        ctx->stream->s = static_cast<cudaStream_t>(cuda_stream);
    } else {
        CK(cudaStreamCreateWithFlags(&ctx->stream->s, cudaStreamNonBlocking), "cudaStreamCreate");
        ctx->stream->owned = true;
    }
    CK(cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device), "attr");

    // keep freed scratch in the pool between calls
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
        uint64_t thr = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    tune_cache_load(ctx.get());
    *out = ctx.release();
    return MAPPER_OK;
}

void mapper_destroy(mapper_ctx* ctx)
{
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    if (ctx->stream && ctx->stream->s) cudaStreamSynchronize(ctx->stream->s);
    tune_cache_save(ctx);
    delete ctx;
}

int mapper_set_stream(mapper_ctx* ctx, void* cuda_stream)
{
    if (!ctx) return fail(MAPPER_EINVAL, "null context");
    auto h = std::make_shared<StreamHolder>();
    if (cuda_stream) {
        h->s = static_cast<cudaStream_t>(cuda_stream);
    } else {
        CK(cudaSetDevice(ctx->device), "cudaSetDevice");
        CK(cudaStreamCreateWithFlags(&h->s, cudaStreamNonBlocking), "cudaStreamCreate");
        h->owned = true;
    }
    ctx->stream = h;
    return MAPPER_OK;
}

int mapper_set_timing(mapper_ctx* ctx, int enabled)
{
    if (!ctx) return fail(MAPPER_EINVAL, "null context");
    ctx->timing = enabled != 0;
    return MAPPER_OK;
}

int mapper_selftest_wait(mapper_ctx* ctx)
{
    int rc = check_ctx(ctx);
    if (rc) return rc;
    return tc_wait_selftest(ctx->stream->s);
}

int mapper_selftest_mma_error(mapper_ctx* ctx, int32_t dp, int32_t products, int32_t format, uint64_t seed,
                              double* observed, double* modelled)
{
    int rc = check_ctx(ctx);
    if (rc) return rc;
    if (!observed || !modelled) return fail(MAPPER_EINVAL, "null output");
    return tc_mma_probe(products, format, dp, seed, ctx->num_sms, observed, modelled, ctx->stream->s);
}

int mapper_set_knn_screen(mapper_ctx* ctx, int mode)
{
    if (!ctx) return fail(MAPPER_EINVAL, "null context");
    if (mode < 0 || mode > 3) return fail(MAPPER_EINVAL, "mode must be 0, 1, 2 or 3");
    ctx->knn_mode = mode;
    return MAPPER_OK;
}

int mapper_knn_info(const mapper_ctx* ctx, int64_t* info)
{
    if (!ctx || !info) return fail(MAPPER_EINVAL, "null argument");
    for (int i = 0; i < 8; ++i) info[i] = ctx->knn_info[i];
    return MAPPER_OK;
}

int mapper_set_cross_screen(mapper_ctx* ctx, int mode)
{
    if (!ctx) return fail(MAPPER_EINVAL, "null context");
    if (mode < 0 || mode > 2) return fail(MAPPER_EINVAL, "mode must be 0, 1 or 2");
    ctx->cross_mode = mode;
    return MAPPER_OK;
}

int mapper_set_pass1_screen(mapper_ctx* ctx, int mode)
{
    if (!ctx) return fail(MAPPER_EINVAL, "null context");
    if (mode < 0 || mode > 3) return fail(MAPPER_EINVAL, "pass-1 screen must be 0, 1, 2 or 3");
    ctx->screen_mode = mode;
    return MAPPER_OK;
}

int mapper_set_band_queue_cap(mapper_ctx* ctx, int64_t entries)
{
    if (!ctx) return fail(MAPPER_EINVAL, "null context");
    if (entries < 0 || entries > (int64_t(1) << 30)) return fail(MAPPER_EINVAL, "band queue entries must be in [0, 2^30]");
    ctx->band_cap = entries;
    return MAPPER_OK;
}

int mapper_set_pass1_tile_n(mapper_ctx* ctx, int tile_n)
{
    if (!ctx) return fail(MAPPER_EINVAL, "null context");
    if (tile_n != 0 && tile_n != 128 && tile_n != 256) return fail(MAPPER_EINVAL, "tile_n must be 0, 128 or 256");
    ctx->pass1_forced = tile_n;
    return MAPPER_OK;
}

int mapper_lens(mapper_ctx* ctx, const float* X_dev, int64_t n, int32_t d, int64_t ld, int32_t m,
                const int32_t* kinds, const int32_t* args, double* lens_dev, double* pca_out)
{
    return mapper_lens_ex(ctx, X_dev, n, d, ld, m, kinds, args, nullptr, MAPPER_BF16, lens_dev, pca_out);
}

int mapper_lens_ex(mapper_ctx* ctx, const float* X_dev, int64_t n, int32_t d, int64_t ld, int32_t m,
                   const int32_t* kinds, const int32_t* args, const double* lens_param, int32_t precision,
                   double* lens_dev, double* pca_out)
{
    int rc = check_ctx(ctx);
    if (rc) return rc;
    if ((rc = check_x(X_dev, n, d, ld))) return rc;
    if (m < 1 || m > 2 || !kinds || !args || !lens_dev) return fail(MAPPER_EINVAL, "bad lens arguments");
    cudaStream_t s = ctx->stream->s;
    Buf flag, pca;
    CK(flag.alloc(sizeof(int), s), "alloc");
    CK(cudaMemsetAsync(flag.p, 0, sizeof(int), s), "memset");
    CK(check_finite(X_dev, n, d, ld, flag.as<int>(), s), "finite");
    int64_t n_pca = 0;
    if ((rc = run_lens(ctx, X_dev, n, d, ld, m, kinds, args, lens_param, precision, lens_dev, &pca, &n_pca)))
        return rc;
    int h_nf = 0;
    CK(cudaMemcpyAsync(&h_nf, flag.p, sizeof(int), cudaMemcpyDeviceToHost, s), "copy");
    if (pca_out && n_pca)
        CK(cudaMemcpyAsync(pca_out, pca.p, sizeof(double) * n_pca, cudaMemcpyDeviceToHost, s), "copy");
    CK(cudaStreamSynchronize(s), "sync");
    if (h_nf) return fail(MAPPER_ENONFINITE, "X holds NaN or Inf");
    return MAPPER_OK;
}

static int cover_call(mapper_ctx* ctx, const double* lens_dev, int64_t n, int32_t m,
                      const int32_t* n_intervals, const double* overlap, int balanced, mapper_cover_t** out)
{
    int rc = check_ctx(ctx);
    if (rc) return rc;
    if (!out || !lens_dev || !n_intervals || !overlap) return fail(MAPPER_EINVAL, "null argument");
    *out = nullptr;
    if (n < 1 || n > INT32_MAX) return fail(MAPPER_EINVAL, "n must be in [1, 2^31)");
    std::shared_ptr<CoverData> c;
    if ((rc = run_cover(ctx, lens_dev, n, m, n_intervals, overlap, &c, nullptr, balanced != 0))) return rc;
    auto h = new mapper_cover_t;
    h->c = c;
    *out = h;
    return MAPPER_OK;
}

int mapper_cover(mapper_ctx* ctx, const double* lens_dev, int64_t n, int32_t m,
                 const int32_t* n_intervals, const double* overlap, mapper_cover_t** out)
{
    return cover_call(ctx, lens_dev, n, m, n_intervals, overlap, 0, out);
}

int mapper_cover_balanced(mapper_ctx* ctx, const double* lens_dev, int64_t n, int32_t m,
                          const int32_t* n_intervals, const double* overlap, mapper_cover_t** out)
{
    return cover_call(ctx, lens_dev, n, m, n_intervals, overlap, 1, out);
}

int mapper_cover_sizes(const mapper_cover_t* cover, int64_t* n_elements, int64_t* n_members)
{
    auto* h = handle_as<mapper_cover_t>(cover, kKindCover);
    if (!h) return fail(MAPPER_EINVAL, "not a cover handle");
    if (n_elements) *n_elements = h->c->E;
    if (n_members) *n_members = h->c->M;
    return MAPPER_OK;
}

int mapper_cover_copy(const mapper_cover_t* cover, int64_t* elem_offsets, int32_t* elem_points,
                      int on_device)
{
    auto* h = handle_as<mapper_cover_t>(cover, kKindCover);
    if (!h) return fail(MAPPER_EINVAL, "not a cover handle");
    cudaStream_t s = h->c->stream->s;
    int rc = copy_out(elem_offsets, h->c->elem_off.p, sizeof(int64_t) * (h->c->E + 1), on_device, s);
    if (rc) return rc;
    return copy_out(elem_points, h->c->slot_point.p, sizeof(int32_t) * h->c->M, on_device, s);
}

int mapper_cluster(mapper_ctx* ctx, const float* X_dev, int64_t n, int32_t d, int64_t ld,
                   const mapper_cover_t* cover, double eps, int32_t min_pts, int32_t precision,
                   mapper_clusters_t** out)
{
    int rc = check_ctx(ctx);
    if (rc) return rc;
    if ((rc = check_x(X_dev, n, d, ld))) return rc;
    auto* cv = handle_as<mapper_cover_t>(cover, kKindCover);
    if (!cv || !out) return fail(MAPPER_EINVAL, "bad cover handle or out");
    *out = nullptr;
    std::shared_ptr<ClusterData> c;
    if ((rc = run_cluster(ctx, X_dev, n, d, ld, cv->c, eps, min_pts, precision, &c, nullptr))) return rc;
    auto h = new mapper_clusters_t;
    h->c = c;
    *out = h;
    return MAPPER_OK;
}

int mapper_clusters_copy(const mapper_clusters_t* clusters, int64_t* label, uint8_t* core, int on_device)
{
    auto* h = handle_as<mapper_clusters_t>(clusters, kKindClusters);
    if (!h) return fail(MAPPER_EINVAL, "not a clusters handle");
    cudaStream_t s = h->c->stream->s;
    const int64_t M = h->c->cover->M;
    int rc = copy_out(label, h->c->slot_label.p, sizeof(int64_t) * M, on_device, s);
    if (rc) return rc;
    return copy_out(core, h->c->core.p, M, on_device, s);
}

int mapper_single_linkage(mapper_ctx* ctx, const float* X_dev, int64_t n, int32_t d, int64_t ld,
                          const mapper_cover_t* cover, double eps, mapper_forest_t** out)
{
    int rc = check_ctx(ctx);
    if (rc) return rc;
    if ((rc = check_x(X_dev, n, d, ld))) return rc;
    auto* cv = handle_as<mapper_cover_t>(cover, kKindCover);
    if (!cv || !out) return fail(MAPPER_EINVAL, "bad cover handle or out");
    *out = nullptr;
    if (!(eps > 0.0) || !std::isfinite(eps)) return fail(MAPPER_EINVAL, "eps must be finite and > 0");
    const auto& cov = cv->c;
    if (cov->n != n) return fail(MAPPER_EINVAL, "cover was built for another point count");
    cudaStream_t s = ctx->stream->s;
    const int dp = (d + 31) / 32 * 32;
    Buf flag;
    CK(flag.alloc(sizeof(int), s), "alloc");
    CK(cudaMemsetAsync(flag.p, 0, sizeof(int), s), "memset");
    // tile layout (FP32 rows gathered) and the element tile pairs that may hold a pair within eps
    TileLayout L;
    if ((rc = build_tiles(X_dev, n, d, ld, dp, cov->slot_point.as<int32_t>(), cov->slot_elem.as<int32_t>(), cov->M,
                          cov->E, 4.0 * eps, false, ctx->num_sms, &L, flag.as<int>(), s)))
        return rc;
    PairLists PL;
    if ((rc = classify_pairs(L, X_dev, ld, d, dp, cov->E, eps, false, &PL, s))) return rc;
    const int64_t np = PL.n[kListAllIn] + PL.n[kListTC] + PL.n[kListSimt];
    if (np > INT32_MAX) return fail(MAPPER_ENOMEM, "too many tile pairs for one launch");
    Buf pairs;
    CK(pairs.alloc(sizeof(int2) * std::max<int64_t>(np, 1), s), "alloc");
    int64_t at = 0;
    for (int li : {(int)kListAllIn, (int)kListTC, (int)kListSimt}) {
        if (PL.n[li] == 0) continue;
        CK(cudaMemcpyAsync(pairs.as<int2>() + at, PL.list[li].p, sizeof(int2) * PL.n[li], cudaMemcpyDeviceToDevice, s),
           "copy");
        at += PL.n[li];
    }
    PassArgs a{};
    a.G = L.G.as<float>();
    a.X = X_dev;
    a.ld = ld;
    a.xvec = ld % 4 == 0 && ((uintptr_t)X_dev & 15) == 0;
    a.dp = dp;
    a.d = d;
    a.tile_n = L.tile_n.as<int32_t>();
    a.eps2 = eps * eps;
    fp32_thresholds(a.eps2, d, &a.lo_thr, &a.hi_thr);
    a.row_pt = L.row_pt.as<int32_t>();
    a.pairs = pairs.as<int2>();
    a.n_rows = L.R;
    a.n_tiles = L.T;
    auto h = std::make_unique<mapper_forest_t>();
    h->stream = ctx->stream;
    h->cover = cov;
    h->eps = eps;
    if ((rc = msf_forest(a, L.row_slot.as<int32_t>(), cov->slot_point.as<int32_t>(), cov->slot_elem.as<int32_t>(),
                         cov->M, L.R, L.T, np, &h->f, s)))
        return rc;
    int h_nf = 0;
    CK(cudaMemcpyAsync(&h_nf, flag.p, sizeof(int), cudaMemcpyDeviceToHost, s), "copy");
    CK(cudaStreamSynchronize(s), "sync");
    if (h_nf) return fail(MAPPER_ENONFINITE, "X holds NaN or Inf");
    h->stats.n_points = n;
    h->stats.n_elements = cov->E;
    h->stats.n_members = cov->M;
    h->stats.tile_pairs = PL.n_candidates;
    h->stats.tile_pairs_out = PL.n_out;
    h->stats.tile_pairs_in = PL.n[kListAllIn];
    h->stats.n_edges = h->f.n;
    h->stats.n_rows = L.R;
    *out = h.release();
    return MAPPER_OK;
}

int mapper_forest_sizes(const mapper_forest_t* forest, int64_t* n_edges)
{
    auto* h = handle_as<mapper_forest_t>(forest, kKindForest);
    if (!h || !n_edges) return fail(MAPPER_EINVAL, "bad forest handle or output");
    *n_edges = h->f.n;
    return MAPPER_OK;
}

int mapper_forest_copy(const mapper_forest_t* forest, int32_t* elem, int32_t* u, int32_t* v, double* d2,
                       int on_device)
{
    auto* h = handle_as<mapper_forest_t>(forest, kKindForest);
    if (!h) return fail(MAPPER_EINVAL, "bad forest handle");
    cudaStream_t s = h->stream->s;
    const size_t n = (size_t)h->f.n;
    int rc;
    if (elem && (rc = copy_out(elem, h->f.elem.p, sizeof(int32_t) * n, on_device, s))) return rc;
    if (u && (rc = copy_out(u, h->f.u.p, sizeof(int32_t) * n, on_device, s))) return rc;
    if (v && (rc = copy_out(v, h->f.v.p, sizeof(int32_t) * n, on_device, s))) return rc;
    if (d2 && (rc = copy_out(d2, h->f.d2.p, sizeof(double) * n, on_device, s))) return rc;
    CK(cudaStreamSynchronize(s), "sync");
    return MAPPER_OK;
}

int mapper_forest_cut(mapper_ctx* ctx, const mapper_forest_t* forest, double h, mapper_clusters_t** out)
{
    int rc = check_ctx(ctx);
    if (rc) return rc;
    auto* f = handle_as<mapper_forest_t>(forest, kKindForest);
    if (!f || !out) return fail(MAPPER_EINVAL, "bad forest handle or out");
    *out = nullptr;
    if (!(h > 0.0) || !(h <= f->eps)) return fail(MAPPER_EINVAL, "the height must be in (0, eps]");
    cudaStream_t s = ctx->stream->s;
    const int64_t M = f->cover->M;
    auto c = std::make_shared<ClusterData>();
    c->stream = ctx->stream;
    c->cover = f->cover;
    CK(c->core.alloc(std::max<int64_t>(M, 1), s), "alloc");
    CK(c->lab.alloc(sizeof(int32_t) * std::max<int64_t>(M, 1), s), "alloc");
    CK(c->is_root.alloc(sizeof(int32_t) * std::max<int64_t>(M, 1), s), "alloc");
    CK(c->is_member.alloc(sizeof(int32_t) * std::max<int64_t>(M, 1), s), "alloc");
    CK(c->slot_label.alloc(sizeof(int64_t) * std::max<int64_t>(M, 1), s), "alloc");
    if ((rc = msf_cut(f->f, f->cover->slot_point.as<int32_t>(), M, h, c->lab.as<int32_t>(), c->is_root.as<int32_t>(),
                      c->is_member.as<int32_t>(), c->slot_label.as<int64_t>(), c->core.as<uint8_t>(), s)))
        return rc;
    CK(cudaStreamSynchronize(s), "sync");
    c->stats = f->stats;
    c->stats.n_core = M;
    auto hnd = new mapper_clusters_t;
    hnd->c = c;
    *out = hnd;
    return MAPPER_OK;
}

int mapper_nerve(mapper_ctx* ctx, const mapper_clusters_t* clusters, mapper_graph_t** out)
{
    int rc = check_ctx(ctx);
    if (rc) return rc;
    auto* cl = handle_as<mapper_clusters_t>(clusters, kKindClusters);
    if (!cl || !out) return fail(MAPPER_EINVAL, "bad clusters handle or out");
    *out = nullptr;
    auto g = std::make_unique<mapper_graph_t>();
    g->stream = ctx->stream;
    g->clusters = cl->c;
    g->n = cl->c->cover->n;
    g->m = cl->c->cover->m;
    if ((rc = run_nerve(ctx, cl->c, g.get()))) return rc;
    g->cover_view.c = cl->c->cover;
    g->cover_view.view = true;
    g->clusters_view.c = cl->c;
    g->clusters_view.view = true;
    *out = g.release();
    return MAPPER_OK;
}

int mapper_cover_subset(mapper_ctx* ctx, const mapper_cover_t* cover, const int32_t* elements, int32_t k,
                        mapper_cover_t** out)
{
    int rc = check_ctx(ctx);
    if (rc) return rc;
    auto* h = handle_as<mapper_cover_t>(cover, kKindCover);
    if (!h || !out || (k > 0 && !elements) || k < 0) return fail(MAPPER_EINVAL, "bad cover subset arguments");
    *out = nullptr;
    const auto& src = *h->c;
    std::vector<char> seen(src.E, 0);
    auto c = std::make_shared<CoverData>();
    c->stream = ctx->stream;
    c->m = src.m;
    c->n_int[0] = src.n_int[0];
    c->n_int[1] = src.n_int[1];
    c->overlap[0] = src.overlap[0];
    c->overlap[1] = src.overlap[1];
    c->n = src.n;
    c->E = k;
    c->h_elem_off.assign(1, 0);
    for (int32_t j = 0; j < k; ++j) {
        const int32_t e = elements[j];
        if (e < 0 || e >= src.E || seen[e]) return fail(MAPPER_EINVAL, "element index out of range or repeated");
        seen[e] = 1;
        c->h_elem_off.push_back(c->h_elem_off.back() + (src.h_elem_off[e + 1] - src.h_elem_off[e]));
    }
    c->M = c->h_elem_off.back();
    cudaStream_t s = ctx->stream->s;
    CK(c->elem_off.alloc(sizeof(int64_t) * (k + 1), s), "alloc");
    CK(c->slot_point.alloc(sizeof(int32_t) * std::max<int64_t>(c->M, 1), s), "alloc");
    CK(c->slot_elem.alloc(sizeof(int32_t) * std::max<int64_t>(c->M, 1), s), "alloc");
    CK(cudaMemcpyAsync(c->elem_off.p, c->h_elem_off.data(), sizeof(int64_t) * (k + 1), cudaMemcpyHostToDevice, s),
       "copy");
    for (int32_t j = 0; j < k; ++j) {
        const int32_t e = elements[j];
        const int64_t len = src.h_elem_off[e + 1] - src.h_elem_off[e];
        if (len)
            CK(cudaMemcpyAsync(c->slot_point.as<int32_t>() + c->h_elem_off[j],
                               src.slot_point.as<int32_t>() + src.h_elem_off[e], sizeof(int32_t) * len,
                               cudaMemcpyDeviceToDevice, s), "copy");
    }
    CK(fill_slot_elem(c->elem_off.as<int64_t>(), k, c->M, c->slot_elem.as<int32_t>(), s), "slot elements");
    CK(cudaStreamSynchronize(s), "sync");                 // h_elem_off copied before it goes out of scope
    auto o = new mapper_cover_t;
    o->c = c;
    *out = o;
    return MAPPER_OK;
}

int mapper_nerve_from_nodes(mapper_ctx* ctx, int64_t n_points, int64_t n_nodes, const int64_t* node_offsets,
                            const int32_t* node_members, const int32_t* node_elem, mapper_graph_t** out)
{
    int rc = check_ctx(ctx);
    if (rc) return rc;
    if (!out || n_points < 1 || n_points > INT32_MAX || n_nodes < 0 || !node_offsets ||
        (n_nodes > 0 && (!node_members || !node_elem)))
        return fail(MAPPER_EINVAL, "bad node arguments");
    *out = nullptr;
    cudaStream_t s = ctx->stream->s;
    auto g = std::make_unique<mapper_graph_t>();
    g->stream = ctx->stream;
    g->n = n_points;
    g->N = n_nodes;
    const bool host = is_host_pointer(node_offsets);
    const cudaMemcpyKind kind = host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    CK(g->node_off.alloc(sizeof(int64_t) * (n_nodes + 1), s), "alloc");
    CK(cudaMemcpyAsync(g->node_off.p, node_offsets, sizeof(int64_t) * (n_nodes + 1), kind, s), "copy");
    int64_t Gm = 0;
    CK(cudaMemcpyAsync(&Gm, g->node_off.as<int64_t>() + n_nodes, sizeof(int64_t), cudaMemcpyDeviceToHost, s),
       "copy");
    CK(cudaStreamSynchronize(s), "sync");
    if (Gm < 0 || Gm > INT32_MAX) return fail(MAPPER_EINVAL, "bad node offsets");
    g->Gm = Gm;
    CK(g->node_members.alloc(sizeof(int32_t) * std::max<int64_t>(Gm, 1), s), "alloc");
    CK(g->node_elem.alloc(sizeof(int32_t) * std::max<int64_t>(n_nodes, 1), s), "alloc");
    if (Gm) CK(cudaMemcpyAsync(g->node_members.p, node_members, sizeof(int32_t) * Gm, kind, s), "copy");
    if (n_nodes) CK(cudaMemcpyAsync(g->node_elem.p, node_elem, sizeof(int32_t) * n_nodes, kind, s), "copy");
    Buf keys2;
    CK(keys2.alloc(sizeof(uint64_t) * std::max<int64_t>(Gm, 1), s), "alloc");
    CK(node_member_keys(g->node_off.as<int64_t>(), n_nodes, Gm, g->node_members.as<int32_t>(),
                        keys2.as<uint64_t>(), s), "member keys");
    if ((rc = nerve_edges(ctx, keys2.as<uint64_t>(), Gm, n_points, n_nodes, g.get()))) return rc;
    g->stats.n_points = n_points;
    g->stats.n_nodes = n_nodes;
    g->stats.n_edges = g->Eg;
    *out = g.release();
    return MAPPER_OK;
}

int mapper_knn_distance(mapper_ctx* ctx, const float* X_dev, int64_t n, int32_t d, int64_t ld,
                        const int32_t* queries, int64_t q, int32_t k, double* out)
{
    int rc = check_ctx(ctx);
    if (rc) return rc;
    if ((rc = check_x(X_dev, n, d, ld))) return rc;
    if (q < 0 || (q > 0 && (!queries || !out))) return fail(MAPPER_EINVAL, "bad query arguments");
    if (q == 0) return MAPPER_OK;
    if (is_host_pointer(X_dev)) return fail(MAPPER_EINVAL, "X must be in device memory");
    cudaStream_t s = ctx->stream->s;
    std::vector<int32_t> hq((size_t)q);
    const bool q_host = is_host_pointer(queries);
    CK(cudaMemcpyAsync(hq.data(), queries, sizeof(int32_t) * q,
                       q_host ? cudaMemcpyHostToHost : cudaMemcpyDeviceToHost, s), "copy");
    Buf qd, od, flag;
    // X is checked for NaN / Inf: on the tensor-core path while its operands
    // are built (a flagged row is then decided by the exact check below)
    auto finite_or_fail = [&]() -> int {
        CK(flag.alloc(sizeof(int), s), "alloc");
        CK(cudaMemsetAsync(flag.p, 0, sizeof(int), s), "memset");
        CK(check_finite(X_dev, n, d, ld, flag.as<int>(), s), "finite");
        int h_nf = 0;
        CK(cudaMemcpyAsync(&h_nf, flag.p, sizeof(int), cudaMemcpyDeviceToHost, s), "copy");
        CK(cudaStreamSynchronize(s), "sync");
        if (h_nf) return fail(MAPPER_ENONFINITE, "X holds NaN or Inf");
        return MAPPER_OK;
    };
    const bool tc = knn_on_tensor_cores(k, ctx->knn_mode != 2) && k >= 1 && k <= n;
    if (!tc && (rc = finite_or_fail())) return rc;
    for (int64_t i = 0; i < q; ++i)
        if (hq[i] < 0 || hq[i] >= n) return fail(MAPPER_EINVAL, "query index out of range");
    CK(qd.alloc(sizeof(int32_t) * q, s), "alloc");
    CK(od.alloc(sizeof(double) * q, s), "alloc");
    CK(cudaMemcpyAsync(qd.p, hq.data(), sizeof(int32_t) * q, cudaMemcpyHostToDevice, s), "copy");
    rc = knn_distance(X_dev, n, d, ld, qd.as<int32_t>(), q, k, od.as<double>(), ctx->num_sms, ctx->knn_mode != 2, s,
                      ctx->knn_info, ctx->knn_mode != 3, tc);
    if (rc == MAPPER_ENONFINITE && tc) {
        // a NaN or Inf, or finite rows whose norms pass FP32: the CUDA-core screen
        if ((rc = finite_or_fail())) return rc;
        rc = knn_distance(X_dev, n, d, ld, qd.as<int32_t>(), q, k, od.as<double>(), ctx->num_sms, false, s,
                          ctx->knn_info);
    }
    if (rc) return rc;
    return copy_out(out, od.p, sizeof(double) * q, !is_host_pointer(out), s);
}

// Host rows to the device (xdev, n x d). When every lens of p is row-local
// (L2, coordinate, L-infinity norm), the rows go in kLensChunks chunks on a
// copy stream and each chunk's lens values are computed on the context's
// stream as soon as it lands, so the lens hides under the copy; *lens_done
// tells the caller. Otherwise one copy on the context's stream.
constexpr int kLensChunks = 8;

int copy_rows_with_lens(mapper_ctx* ctx, const float* X, int64_t n, int32_t d, int64_t ld, const mapper_params* p,
                        float* xdev, double* lens, bool* lens_done, const PivotSet* split)
{
    cudaStream_t s = ctx->stream->s;
    *lens_done = false;
    bool row_local = n >= 64 * kLensChunks;
    for (int j = 0; j < p->m; ++j) {
        const int k = p->lens_kind[j];
        row_local &= k == MAPPER_LENS_L2 || k == MAPPER_LENS_LINF ||
                     (k == MAPPER_LENS_COORD && p->lens_arg[j] >= 0 && p->lens_arg[j] < d);
    }
    auto copy = [&](int64_t r0, int64_t rows, cudaStream_t st) -> cudaError_t {
        if (ld == d)
            return cudaMemcpyAsync(xdev + r0 * d, X + r0 * ld, sizeof(float) * (size_t)rows * d,
                                   cudaMemcpyHostToDevice, st);
        return cudaMemcpy2DAsync(xdev + r0 * d, sizeof(float) * d, X + r0 * ld, sizeof(float) * ld,
                                 sizeof(float) * d, rows, cudaMemcpyHostToDevice, st);
    };
    if (!row_local) {
        CK(copy(0, n, s), "copy X");
        return MAPPER_OK;
    }
    cudaStream_t cs = nullptr;
    cudaEvent_t ev[kLensChunks + 1] = {};
    struct Guard {
        cudaStream_t* cs;
        cudaEvent_t* ev;
        ~Guard()
        {
            for (int i = 0; i <= kLensChunks; ++i) if (ev[i]) cudaEventDestroy(ev[i]);
            if (*cs) cudaStreamDestroy(*cs);
        }
    } guard{&cs, ev};
    CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking), "stream");
    for (int i = 0; i <= kLensChunks; ++i) CK(cudaEventCreateWithFlags(&ev[i], cudaEventDisableTiming), "event");
    // the copies start once xdev is allocated (stream order of s)
    CK(cudaEventRecord(ev[kLensChunks], s), "event");
    CK(cudaStreamWaitEvent(cs, ev[kLensChunks], 0), "wait");
    const int64_t chunk = (n + kLensChunks - 1) / kLensChunks;
    for (int c = 0; c < kLensChunks; ++c) {
        const int64_t r0 = c * chunk, rows = std::min<int64_t>(chunk, n - r0);
        if (rows <= 0) break;
        CK(copy(r0, rows, cs), "copy X");
        CK(cudaEventRecord(ev[c], cs), "event");
        CK(cudaStreamWaitEvent(s, ev[c], 0), "wait");
        bool split_done = false;
        for (int j = 0; j < p->m; ++j) {
            const int k = p->lens_kind[j];
            const float* xr = xdev + r0 * d;
            double* f = lens + r0 * p->m;
            if (k == MAPPER_LENS_L2 && split && !split_done) {
                const int dp = (d + 31) / 32 * 32;
                CK(lens_l2_split(xr, rows, d, d, f, p->m, j, split->c.as<float>(), dp,
                                 static_cast<uint16_t*>(split->xh.p) + r0 * dp, split->xn2.as<float>() + r0, s),
                   "lens_l2");
                split_done = true;
            } else if (k == MAPPER_LENS_L2) CK(lens_l2(xr, rows, d, d, f, p->m, j, s), "lens_l2");
            else if (k == MAPPER_LENS_LINF) CK(lens_linf(xr, rows, d, d, f, p->m, j, s), "lens_linf");
            else CK(lens_coord(xr, rows, d, p->lens_arg[j], f, p->m, j, s), "lens_coord");
        }
    }
    *lens_done = true;
    return MAPPER_OK;
}

int mapper_graph(mapper_ctx* ctx, const float* X, int64_t n, int32_t d, int64_t ld,
                 const mapper_params* p, mapper_graph_t** out)
{
    int rc = check_ctx(ctx);
    if (rc) return rc;
    if ((rc = check_x(X, n, d, ld))) return rc;
    if (!p || !out) return fail(MAPPER_EINVAL, "null params or out");
    *out = nullptr;
    if (p->m < 1 || p->m > 2) return fail(MAPPER_EINVAL, "m must be 1 or 2");
    cudaStream_t s = ctx->stream->s;
    Timer tm(ctx->timing, s);
    tm.mark();
    const int64_t launches0 = g_launches;

    auto g = std::make_unique<mapper_graph_t>();
    g->stream = ctx->stream;
    g->n = n;
    g->m = p->m;
    Buf flag;
    CK(flag.alloc(sizeof(int), s), "alloc");
    CK(cudaMemsetAsync(flag.p, 0, sizeof(int), s), "memset");
    CK(g->lens.alloc(sizeof(double) * (size_t)n * p->m, s), "alloc lens");
    Buf xdev;
    const float* Xd = X;
    int64_t ldd = ld;
    bool lens_done = false;
    // tensor-core graphs with an L2 lens: the lens pass also writes the
    // points' split for the pivot assignment of the tile layout
    bool has_l2 = false;
    for (int j = 0; j < p->m; ++j) has_l2 |= p->lens_kind[j] == MAPPER_LENS_L2;
    const bool fuse_split = has_l2 && p->precision != MAPPER_FP32 && d <= 32768;
    PivotSet piv;
    const int dp = (d + 31) / 32 * 32;
    if (fuse_split) {
        CK(pivot_alloc(n, dp, &piv, s), "alloc pivots");
        if ((rc = pivot_prepare(X, n, d, ld, dp, is_host_pointer(X), &piv, s))) return rc;
    }
    if (is_host_pointer(X)) {
        CK(xdev.alloc(sizeof(float) * (size_t)n * d, s), "alloc X");
        Xd = xdev.as<float>();
        ldd = d;
        if ((rc = copy_rows_with_lens(ctx, X, n, d, ld, p, xdev.as<float>(), g->lens.as<double>(), &lens_done,
                                      fuse_split ? &piv : nullptr)))
            return rc;
    }
    bool split_written = fuse_split && lens_done;
    if (!lens_done) {
        if ((rc = run_lens(ctx, Xd, n, d, ldd, p->m, p->lens_kind, p->lens_arg, p->lens_param, p->precision,
                           g->lens.as<double>(), &g->pca, &g->n_pca, fuse_split ? &piv : nullptr)))
            return rc;
        split_written = fuse_split;
    }
    tm.mark();
    std::shared_ptr<CoverData> cov;
    if (p->cover_kind != MAPPER_COVER_UNIFORM && p->cover_kind != MAPPER_COVER_BALANCED)
        return fail(MAPPER_EINVAL, "unknown cover kind");
    if ((rc = run_cover(ctx, g->lens.as<double>(), n, p->m, p->n_intervals, p->overlap, &cov,
                        flag.as<int>(), p->cover_kind == MAPPER_COVER_BALANCED))) return rc;
    tm.mark();
    std::shared_ptr<ClusterData> cl;
    // the pivot assignment on the points split by the lens pass
    if (split_written && (rc = pivot_assign(Xd, n, d, ldd, dp, true, ctx->num_sms, &piv, s))) return rc;
    if ((rc = run_cluster(ctx, Xd, n, d, ldd, cov, p->eps, p->min_pts, p->precision, &cl, flag.as<int>(), nullptr,
                          nullptr, split_written ? &piv : nullptr)))
        return rc;
    tm.mark();
    g->clusters = cl;
    if ((rc = run_nerve(ctx, cl, g.get()))) return rc;
    tm.mark();
    if (ctx->timing) {
        g->stats.ms_lens = tm.ms(0, 1);
        g->stats.ms_cover = tm.ms(1, 2);
        g->stats.ms_cluster = tm.ms(2, 3);
        g->stats.ms_nerve = tm.ms(3, 4);
        g->stats.ms_total = tm.ms(0, 4);
        cl->stats.ms_lens = g->stats.ms_lens;
        cl->stats.ms_cover = g->stats.ms_cover;
        cl->stats.ms_cluster = g->stats.ms_cluster;
    }
    g->stats.n_launches = g_launches - launches0;
    g->cover_view.c = cov;
    g->cover_view.view = true;
    g->clusters_view.c = cl;
    g->clusters_view.view = true;
    *out = g.release();
    return MAPPER_OK;
}

int mapper_graph_footprint(int64_t n, int32_t d, const mapper_params* p, size_t* bytes)
{
    if (!p || !bytes) return fail(MAPPER_EINVAL, "null argument");
    if (n < 1 || d < 1 || p->m < 1 || p->m > 2) return fail(MAPPER_EINVAL, "bad sizes or filter dimension");
    double mult = 1.0, E = 1.0;
    for (int j = 0; j < p->m; ++j) {
        if (p->n_intervals[j] < 1 || !(p->overlap[j] >= 0.0 && p->overlap[j] < 1.0))
            return fail(MAPPER_EINVAL, "bad cover parameters");
        // a point lies in at most floor(1/(1-p)) + 1 intervals, one more on exact ties
        mult *= std::min<double>(p->n_intervals[j], std::floor(1.0 / (1.0 - p->overlap[j])) + 2.0);
        E *= p->n_intervals[j];
    }
    const double dp = (double)((d + 31) / 32 * 32);
    const bool tc = p->precision != MAPPER_FP32;
    // scratch of one clustering of M memberships in E elements
    auto cluster_bytes = [&](double M, double E, int cap) {
        const double rows = 1.1 * M + 128.0 * E;
        double b = rows * dp * (tc ? 12.0 : 4.0);                // FP32 rows (+ BF16 hi, lo, twice)
        if (p->precision == MAPPER_FP8) b += rows * dp * 2.0;   // FP8 hi, lo
        b += tc ? (double)n * dp * 4.0 : 0.0;                     // pivot assignment operands
        b += rows * (29.0 + 4.0 * cap) + M * 40.0;
        b += 3.0 * 8.0 * rows * rows / (128.0 * 128.0) / std::max(1.0, E);   // tile-pair lists
        return b;
    };
    const int cap = (p->min_pts >= 2 && p->min_pts - 1 <= 64) ? p->min_pts - 1 : 0;
    double b = cluster_bytes((double)n * mult, E, cap);
    for (int j = 0; j < p->m; ++j)                            // a density lens: one element of n points
        if (p->lens_kind[j] == MAPPER_LENS_DENSITY) b = std::max(b, cluster_bytes((double)n, 1.0, 0));
    b += (double)n * 24.0 * p->m;
    *bytes = (size_t)(b * 1.1) + (size_t)(64u << 20);
    return MAPPER_OK;
}

int mapper_graph_sweep(mapper_ctx* ctx, const float* X, int64_t n, int32_t d, int64_t ld, const mapper_params* p,
                       int32_t n_sweep, const double* eps, const double* overlap, mapper_graph_t** out)
{
    int rc = check_ctx(ctx);
    if (rc) return rc;
    if ((rc = check_x(X, n, d, ld))) return rc;
    if (!p || !out || !eps || !overlap || n_sweep < 1) return fail(MAPPER_EINVAL, "bad sweep arguments");
    if (p->cover_kind != MAPPER_COVER_UNIFORM && p->cover_kind != MAPPER_COVER_BALANCED)
        return fail(MAPPER_EINVAL, "unknown cover kind");
    if (p->m < 1 || p->m > 2) return fail(MAPPER_EINVAL, "m must be 1 or 2");
    for (int i = 0; i < n_sweep; ++i) out[i] = nullptr;
    cudaStream_t s = ctx->stream->s;
    const int64_t launches0 = g_launches;
    Buf xdev;
    const float* Xd = X;
    int64_t ldd = ld;
    if (is_host_pointer(X)) {
        CK(xdev.alloc(sizeof(float) * (size_t)n * d, s), "alloc X");
        if (ld == d)
            CK(cudaMemcpyAsync(xdev.p, X, sizeof(float) * (size_t)n * d, cudaMemcpyHostToDevice, s), "copy X");
        else
            CK(cudaMemcpy2DAsync(xdev.p, sizeof(float) * d, X, sizeof(float) * ld, sizeof(float) * d, n,
                                 cudaMemcpyHostToDevice, s), "copy X");
        Xd = xdev.as<float>();
        ldd = d;
    }
    Buf lens, pca, flag;
    int64_t n_pca = 0;
    CK(flag.alloc(sizeof(int), s), "alloc");
    CK(cudaMemsetAsync(flag.p, 0, sizeof(int), s), "memset");
    CK(lens.alloc(sizeof(double) * (size_t)n * p->m, s), "alloc lens");
    if ((rc = run_lens(ctx, Xd, n, d, ldd, p->m, p->lens_kind, p->lens_arg, p->lens_param, p->precision,
                       lens.as<double>(), &pca, &n_pca)))
        return rc;
    std::vector<std::unique_ptr<mapper_graph_t>> graphs(n_sweep);
    std::vector<char> done(n_sweep, 0);
    const int dp = (d + 31) / 32 * 32;
    const bool use_tc = p->precision != MAPPER_FP32;
    PivotSet piv;                              // one pivot assignment for every tile layout
    CK(pivot_alloc(n, dp, &piv, s), "alloc pivots");
    if ((rc = pivot_assign(Xd, n, d, ldd, dp, use_tc, ctx->num_sms, &piv, s))) return rc;
    // one cover and one tile layout per distinct overlap, shared by its radii
    for (int i = 0; i < n_sweep; ++i) {
        if (done[i]) continue;
        double ov[2] = {overlap[i], overlap[i]};
        std::shared_ptr<CoverData> cov;
        if ((rc = run_cover(ctx, lens.as<double>(), n, p->m, p->n_intervals, ov, &cov, flag.as<int>(),
                            p->cover_kind == MAPPER_COVER_BALANCED)))
            return rc;
        double eps_max = 0.0;
        for (int j = i; j < n_sweep; ++j)
            if (overlap[j] == overlap[i]) eps_max = std::max(eps_max, eps[j]);
        if (!(eps_max > 0.0) || !std::isfinite(eps_max)) return fail(MAPPER_EINVAL, "eps must be finite and > 0");
        TileLayout L;
        if ((rc = build_tiles(Xd, n, d, ldd, dp, cov->slot_point.as<int32_t>(), cov->slot_elem.as<int32_t>(), cov->M,
                              cov->E, 4.0 * eps_max, use_tc, ctx->num_sms, &L, flag.as<int>(), s, &piv)))
            return rc;
        // the overlap's distinct radii, ascending; on the BF16 tensor-core
        // screen up to kMaxRadii of them share one count pass
        std::vector<double> radii;
        for (int j = i; j < n_sweep; ++j)
            if (overlap[j] == overlap[i]) radii.push_back(eps[j]);
        for (double r : radii)
            if (!(r > 0.0) || !std::isfinite(r)) return fail(MAPPER_EINVAL, "eps must be finite and > 0");
        std::sort(radii.begin(), radii.end());
        radii.erase(std::unique(radii.begin(), radii.end()), radii.end());
        const int per_pass = (p->precision == MAPPER_BF16 || p->precision == MAPPER_BF16X1) ? kMaxRadii : 1;
        std::vector<std::shared_ptr<ClusterData>> by_radius(radii.size());
        for (size_t r0 = 0; r0 < radii.size(); r0 += per_pass) {
            const int k = (int)std::min<size_t>(per_pass, radii.size() - r0);
            if ((rc = run_cluster_radii(ctx, Xd, n, d, ldd, cov, k, radii.data() + r0, p->min_pts, p->precision,
                                        by_radius.data() + r0, flag.as<int>(), &L)))
                return rc;
        }
        for (int j = i; j < n_sweep; ++j) {
            if (done[j] || overlap[j] != overlap[i]) continue;
            const std::shared_ptr<ClusterData>& cl =
                by_radius[std::lower_bound(radii.begin(), radii.end(), eps[j]) - radii.begin()];
            auto g = std::make_unique<mapper_graph_t>();
            g->stream = ctx->stream;
            g->n = n;
            g->m = p->m;
            g->clusters = cl;
            CK(g->lens.alloc(sizeof(double) * (size_t)n * p->m, s), "alloc lens");
            CK(cudaMemcpyAsync(g->lens.p, lens.p, sizeof(double) * (size_t)n * p->m, cudaMemcpyDeviceToDevice, s),
               "copy lens");
            if (n_pca) {
                CK(g->pca.alloc(sizeof(double) * n_pca, s), "alloc");
                CK(cudaMemcpyAsync(g->pca.p, pca.p, sizeof(double) * n_pca, cudaMemcpyDeviceToDevice, s), "copy");
                g->n_pca = n_pca;
            }
            if ((rc = run_nerve(ctx, cl, g.get()))) return rc;
            g->cover_view.c = cov;
            g->cover_view.view = true;
            g->clusters_view.c = cl;
            g->clusters_view.view = true;
            graphs[j] = std::move(g);
            done[j] = 1;
        }
    }
    const int64_t launches = g_launches - launches0;
    for (int i = 0; i < n_sweep; ++i) {
        graphs[i]->stats.n_launches = launches / n_sweep;
        out[i] = graphs[i].release();
    }
    return MAPPER_OK;
}

int mapper_graph_sizes(const mapper_graph_t* g, int64_t* n_nodes, int64_t* n_members, int64_t* n_edges)
{
    auto* h = handle_as<mapper_graph_t>(g, kKindGraph);
    if (!h) return fail(MAPPER_EINVAL, "not a graph handle");
    if (n_nodes) *n_nodes = h->N;
    if (n_members) *n_members = h->Gm;
    if (n_edges) *n_edges = h->Eg;
    return MAPPER_OK;
}

int mapper_graph_copy(const mapper_graph_t* g, int64_t* node_offsets, int32_t* node_members,
                      int32_t* node_elem, int32_t* edges, int on_device)
{
    auto* h = handle_as<mapper_graph_t>(g, kKindGraph);
    if (!h) return fail(MAPPER_EINVAL, "not a graph handle");
    cudaStream_t s = h->stream->s;
    int rc;
    if ((rc = copy_out(node_offsets, h->node_off.p, sizeof(int64_t) * (h->N + 1), on_device, s))) return rc;
    if ((rc = copy_out(node_members, h->node_members.p, sizeof(int32_t) * h->Gm, on_device, s))) return rc;
    if ((rc = copy_out(node_elem, h->node_elem.p, sizeof(int32_t) * h->N, on_device, s))) return rc;
    return copy_out(edges, h->edges.p, sizeof(int32_t) * 2 * h->Eg, on_device, s);
}

int mapper_graph_lens(const mapper_graph_t* g, double* lens, double* pca, int64_t* n_pca, int on_device)
{
    auto* h = handle_as<mapper_graph_t>(g, kKindGraph);
    if (!h) return fail(MAPPER_EINVAL, "not a graph handle");
    if (n_pca) *n_pca = h->n_pca;
    cudaStream_t s = h->stream->s;
    if (lens && !h->lens.p) return fail(MAPPER_EINVAL, "graph was built from a given cover; no lens stored");
    int rc = copy_out(lens, h->lens.p, sizeof(double) * h->n * h->m, on_device, s);
    if (rc) return rc;
    return copy_out(pca, h->pca.p, sizeof(double) * h->n_pca, on_device, s);
}

const mapper_cover_t* mapper_graph_cover(const mapper_graph_t* g)
{
    auto* h = handle_as<mapper_graph_t>(g, kKindGraph);
    return h && h->cover_view.c ? &h->cover_view : nullptr;
}

const mapper_clusters_t* mapper_graph_clusters(const mapper_graph_t* g)
{
    auto* h = handle_as<mapper_graph_t>(g, kKindGraph);
    return h && h->clusters_view.c ? &h->clusters_view : nullptr;
}

int mapper_stats_get(const void* handle, mapper_stats* out)
{
    if (!out) return fail(MAPPER_EINVAL, "out is null");
    if (auto* g = handle_as<mapper_graph_t>(handle, kKindGraph)) { *out = g->stats; return MAPPER_OK; }
    if (auto* c = handle_as<mapper_clusters_t>(handle, kKindClusters)) { *out = c->c->stats; return MAPPER_OK; }
    if (auto* f = handle_as<mapper_forest_t>(handle, kKindForest)) { *out = f->stats; return MAPPER_OK; }
    return fail(MAPPER_EINVAL, "not a graph, clusters or forest handle");
}

void mapper_free(void* handle)
{
    if (!handle) return;
    const HandleHdr* hh = static_cast<const HandleHdr*>(handle);
    if (hh->magic != kMagic) return;
    if (hh->kind == kKindCover) {
        auto* h = static_cast<mapper_cover_t*>(handle);
        if (h->view) return;
        delete h;
    } else if (hh->kind == kKindClusters) {
        auto* h = static_cast<mapper_clusters_t*>(handle);
        if (h->view) return;
        delete h;
    } else if (hh->kind == kKindGraph) {
        delete static_cast<mapper_graph_t*>(handle);
    } else if (hh->kind == kKindForest) {
        delete static_cast<mapper_forest_t*>(handle);
    }
}

}  // extern "C"
