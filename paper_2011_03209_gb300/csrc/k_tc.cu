// k_tc.cu -- tcgen05 tensor-core screen for the per-element DBSCAN passes
// ("Mapper Interactive" §3 DBSCAN per cover element; §4.3 names the
// all-pairs distances the bottleneck).
//
// For a tile pair (A, B) of one segment, rows are centred on the segment's
// FP64 centroid c: a = x - c, b = y - c, so d^2(x, y) = |a|^2 + |b|^2 - 2 a.b.
// a and b are split into BF16 parts a = hi + lo (+ tiny), and the cross term
// comes from tcgen05.mma (kind::f16, BF16 in, FP32 accumulate in TMEM):
//   NS = 3: hi.hi + hi.lo + lo.hi      NS = 1: hi.hi only.
// The screen value s = (|a|^2 + |b|^2) - 2 acc is certified against eps^2 by
// a rigorous bound E(a, b) = A1 |a||b| + A2 (|a|^2 + |b|^2) + A3 (see
// tc_bound below); pairs with |s - eps^2| <= E are queued and re-decided in
// FP64 by the defining expression, so every decision equals FP64.
//
// Kernel layout (one CTA per SM, persistent over a static share of the tile
// pairs): warp 0 issues TMA loads of 64-column K blocks (128-byte swizzle)
// into a ring of smem stages; warp 1 issues the MMAs into one of two TMEM
// accumulators (128 x 128 FP32 each); 16 warps read the accumulator back
// with tcgen05.ld (four warps per TMEM lane quadrant, each thread one row and
// 32 columns) and run the pass epilogue, branch-free per pair:
//   pass 1: neighbour counts of rows and columns (and neighbour lists),
//   pass 2: unions of core-core neighbour pairs.
// Every mbarrier wait is bounded in time; a wait that runs out sets an error
// flag, stops all roles, waits (bounded) for its own copies and MMAs, frees
// TMEM and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <cfloat>
#include <climits>
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "../../include/mapper.h"
#include "tc.cuh"

namespace mgb {

namespace {

constexpr int kT = kTile;
constexpr int kKB = 64;                       // BF16 columns per K block (128-byte rows)
constexpr int kBlk = kT * kKB * 2;            // bytes of one 128 x 64 BF16 block
constexpr int kEpiWarps = 16;                 // epilogue warps: 4 per TMEM lane quadrant
constexpr int kEpiThreads = 32 * kEpiWarps;
constexpr int kChunks = 128 / (kEpiWarps / 4) / 32;   // 32-column chunks per epilogue thread
constexpr int kThreads = 64 + kEpiThreads;    // producer, MMA, epilogue warps
constexpr unsigned long long kWaitNs = 4000000000ull;   // 4 s per wait at most

struct TcParams {
    PassArgs A;
    const float* rn2;
    const float* rn;
    const float* rl;                          // |a - hi| per row (rounded up), or nullptr
    int64_t n_pairs;
    const int2* groups;                       // W = 2: (pair, pair or -1) sharing tile A
    int64_t n_groups;
    const unsigned long long* n_dev;          // if set: work items on the device (<= n_pairs or n_groups)
    int nkb;                                  // K blocks per row
    double A1, A2, A3;                        // bound constants
    float A1f, A2f, A3f;                      // ... rounded up to FP32
    float K0f, K1f, K2f;                      // bound from the residual norms (rl set), rounded up
    float K4f, K5f;                           // FP8: subnormal-floor terms of the bound
    float eps2_lo, eps2_hi;                   // eps^2 rounded down / up to FP32
    uint2* queue;                             // band pairs: (row a, row b | flags << 30)
    unsigned long long* queue_n;
    unsigned long long queue_cap;
    int* err;                                 // 1: a wait timed out
    // pass 1, one-product screen of the two-phase count pass: a sub-block with
    // any pair in the band is not counted here but marked in redo_mask (and
    // its pair flagged in pair_hit) for a three-product pass
    int defer;                                // 1: defer blocks with a band pair; 2: every mixed block
    uint32_t* redo_mask;                      // first phase: deferred sub-blocks per pair (bit quad * 4 + part)
    const uint32_t* sub_mask;                 // second phase: sub-blocks to count per pair: sub_mask[sub_q[q]]
    const int32_t* sub_q;
    const float4* tmax;                       // count pass: per tile largest |b|^2, |b|, |b - hi|
    const float* tn2min;                      // count pass: per tile smallest |b|^2 (valid rows)
    // k-distance screen (MODE 3): CTA t = (query tile t / kq_chunks, chunk t % kq_chunks)
    // against screened point tiles chunk * kq_ct .. + kq_ct of kq_tp; screened
    // tile b is operand tile b * kq_stride, query tile u operand tile kq_qt0 + u
    int64_t kq_tp, kq_q, kq_stride, kq_qt0;
    int kq_ct, kq_chunks;
    float kq_m, kq_c2;                        // key = RD(RD(|a|^2 m - A3f) + RD(c2 acc + RD(|b|^2 m)))
    const float* kq_tau;                      // append mode: keep every key <= tau[query]; else lists
    int kq_cap;                               // append mode: entries per query
    const int64_t* kq_off;                    // append mode, if set: query i's entries at off[i] .. off[i + 1]
    int* kq_cnt;                              // append mode: keys found per query (may exceed kq_cap)
    float* kq_v;                              // lists: [((query * chunks + chunk) * 4 + part) * kKnnL]
    int32_t* kq_i;                            // append: [query * kq_cap + slot]
    float* dump;                              // MODE 4 (accumulation probe): [item][128][128] accumulators
    // MODE 5 (count pass over several radii, ascending): per radius its
    // outputs and eps^2 (double; FP32 rounded down / up)
    struct Radius {
        int32_t* count;
        int32_t* nbr;
        uint8_t* pair_hit;
        uint2* queue;
        unsigned long long* queue_n;
        unsigned long long* stats;
        double eps2, tie_thr;
        float eps2_lo, eps2_hi;
    } rad[kMaxRadii];
    int n_rad;
};

// ------------------------------------------------------------------ PTX
__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ unsigned long long gtime()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_test(uint64_t* bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(su32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait: false (and *abort set) if the phase did not complete in time
// or another role already gave up.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort)
{
    if (mbar_test(bar, parity)) return true;
    const unsigned long long t0 = gtime();
    for (uint32_t it = 1;; ++it) {
        if (mbar_test(bar, parity)) return true;
        if ((it & 255u) == 0) {
            if (*abort) return false;
            if (gtime() - t0 > kWaitNs) {
                *abort = 1;
                return false;
            }
        }
    }
}

__device__ __forceinline__ void tma_load(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
            "r"(su32(dst)),
        "l"(map), "r"(x), "r"(y), "r"(su32(bar))
        : "memory");
}

// K-major operand, 128-byte swizzle: 8-row groups 1024 bytes apart; the
// start address moves 32 bytes per 16-column MMA step inside the atom.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr)
{
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// kind::f16, A = B = BF16, D = F32, both K-major, M = 128, N = 128
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kT >> 3) << 17) |
                            ((uint32_t)(kT >> 4) << 24);
// ... N = 256: tile A against two B tiles stacked in shared memory
constexpr uint32_t kIdesc2 = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(2 * kT >> 3) << 17) |
                             ((uint32_t)(kT >> 4) << 24);

// kind::f8f6f4, A = B = E4M3 (format 0), D = F32, both K-major: K = 32 per
// instruction, the same 32 bytes of a row as K = 16 of BF16
constexpr uint32_t kIdescF8 = (1u << 4) | ((uint32_t)(kT >> 3) << 17) | ((uint32_t)(kT >> 4) << 24);
constexpr uint32_t kIdescF8x2 = (1u << 4) | ((uint32_t)(2 * kT >> 3) << 17) | ((uint32_t)(kT >> 4) << 24);

__device__ __forceinline__ void mma_f8_id(uint32_t tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          uint32_t acc)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}" ::"r"(
            tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_bf16_id(uint32_t tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                            uint32_t acc)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(
            tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint64_t* bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(bar))
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v)
{
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,"
        "%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
          "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v)
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float* v)
{
    uint32_t r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

// u = fl(m u + n) for two columns at once (packed FMA, each lane correctly
// rounded as fmaf).
__device__ __forceinline__ void fma2_inplace(float& u0, float& u1, float m, float n0, float n1)
{
    unsigned long long x, c, mm, r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(x) : "f"(u0), "f"(u1));
    asm("mov.b64 %0, {%1, %2};" : "=l"(c) : "f"(n0), "f"(n1));
    asm("mov.b64 %0, {%1, %1};" : "=l"(mm) : "f"(m));
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(x), "l"(mm), "l"(c));
    asm("mov.b64 {%0, %1}, %2;" : "=f"(u0), "=f"(u1) : "l"(r));
}

__device__ __forceinline__ float fmax3(float a, float b, float c)
{
    float r;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}

__device__ __forceinline__ float fmin3(float a, float b, float c)
{
    float r;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}

__device__ __forceinline__ void epi_sync() { asm volatile("bar.sync 1, %0;" ::"n"(kEpiThreads) : "memory"); }

// Barrier of the epilogue threads that also ORs a flag over them, so all
// take the same branch afterwards.
__device__ __forceinline__ bool epi_sync_or(bool v)
{
    uint32_t r;
    asm volatile(
        "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.or.pred q, 1, %2, p;\n selp.u32 %0, 1, 0, q;\n}"
        : "=r"(r)
        : "r"((uint32_t)v), "n"(kEpiThreads)
        : "memory");
    return r != 0;
}

// ------------------------------------------------------- union-find, FP64
__device__ __forceinline__ int key_of(const int32_t* row_pt, int row) { return row_pt ? __ldg(row_pt + row) : row; }

__device__ __forceinline__ int gfind(int32_t* parent, int x)
{
    volatile int32_t* par = parent;
    int p = par[x];
    while (p != x) {
        const int gp = par[p];
        if (gp != p) par[x] = gp;
        x = p;
        p = par[x];
    }
    return x;
}

__device__ __forceinline__ void gunion(int32_t* parent, const int32_t* row_pt, int a, int b)
{
    while (true) {
        a = gfind(parent, a);
        b = gfind(parent, b);
        if (a == b) return;
        if (key_of(row_pt, a) < key_of(row_pt, b)) { const int t = a; a = b; b = t; }
        if (atomicCAS(&parent[a], a, b) == a) return;
    }
}

// Shared-memory union-find over the 256 rows of a tile pair (local index as
// key; parents always smaller), for sparse pairs.
__device__ __forceinline__ int lfind(volatile int* par, int x)
{
    int p = par[x];
    while (p != x) {
        const int gp = par[p];
        if (gp != p) par[x] = gp;
        x = p;
        p = par[x];
    }
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

__device__ __forceinline__ double exact_sqdist(const float* __restrict__ x, const float* __restrict__ y, int d)
{
    double s = 0.0;
    for (int k = 0; k < d; ++k) {
        const double t = __dsub_rn((double)x[k], (double)y[k]);
        s = __dadd_rn(s, __dmul_rn(t, t));
    }
    return s;
}

// Queue flags (bits 30-31 of the second row): pass 1: bit 0 = also count for
// row b, bit 1 = count the pair as a near tie candidate.
enum : uint32_t { kQBoth = 1u, kQTie = 2u };

// Queue a band pair, or decide it here when the queue is full.
__device__ __forceinline__ bool push_band(const TcParams& P, int ra, int rb, uint32_t flags, bool* decided)
{
    const unsigned long long at = atomicAdd(P.queue_n, 1ull);
    if (at < P.queue_cap) {
        P.queue[at] = make_uint2((uint32_t)ra, (uint32_t)rb | (flags << 30));
        *decided = false;
        return false;
    }
    const PassArgs& A = P.A;
    const double d2 = exact_sqdist(pass_row(A, ra), pass_row(A, rb), A.d);
    atomicAdd(&A.stats[kStatBand], 1ull);
    if ((flags & kQTie) && fabs(d2 - A.eps2) <= A.tie_thr) atomicAdd(&A.stats[kStatTies], 1ull);
    *decided = true;
    return d2 <= A.eps2;
}

// The same for radius e of a count pass over several radii.
__device__ __forceinline__ bool push_band_radius(const TcParams& P, uint2* queue, unsigned long long* queue_n,
                                                 unsigned long long* stats, double eps2, double tie_thr, int ra,
                                                 int rb, uint32_t flags, bool* decided)
{
    const unsigned long long at = atomicAdd(queue_n, 1ull);
    if (at < P.queue_cap) {
        queue[at] = make_uint2((uint32_t)ra, (uint32_t)rb | (flags << 30));
        *decided = false;
        return false;
    }
    const PassArgs& A = P.A;
    const double d2 = exact_sqdist(pass_row(A, ra), pass_row(A, rb), A.d);
    atomicAdd(&stats[kStatBand], 1ull);
    if ((flags & kQTie) && fabs(d2 - eps2) <= tie_thr) atomicAdd(&stats[kStatTies], 1ull);
    *decided = true;
    return d2 <= eps2;
}

// ------------------------------------------------------------------ kernel
// Per-pair epilogue data is double-buffered (index: pair counter & 1): a
// pair's buffer is written before the barrier that follows the accumulator
// wait and read after it, so the next pair can be staged meanwhile.
struct SmemTail {
    uint64_t full[4], empty[4], acc_full[2], acc_empty[2], fin;
    uint32_t tmem_base;
    int abort;
    int consumed;                              // stage fills consumed by the MMA warp
    int s_mm[2][2];                            // union pass: min / max root of the core rows
    uint32_t colcore[2][4];                    // union pass: core columns, bit per column
    float red[2][12];                          // max |b|^2, |b| and |b - hi| of the columns, per warp
    __align__(16) float nbn[2][kT];            // -|b|^2 of the pair's columns
    __align__(16) float nbr[2][kT];            // k-distance pass: |b| (rounded up) of the pair's columns
    __align__(16) float wn[kEpiWarps][32];     // count pass: -|b|^2 of each warp's 32 columns
    uint32_t colmask[4][kT];                   // union pass: neighbour bits per column (by row quadrant)
    uint32_t rowmask[kT / 32][kT];             // neighbour bits per row (by 32-column chunk)
    int par[2][2 * kT];                        // union pass: local union-find / component
    int groot[2][2 * kT];                      // union pass: global root of each core row
    int edges[2];                              // union pass: certain core-core pairs
    unsigned char core[2][2 * kT];             // union pass: core flags of A rows, B rows
};

// Connected components of a tile pair's core-core neighbour graph, on one
// warp. Nodes: A rows 0..127 and (off-diagonal pairs) B rows 128..255; edges:
// S.rowmask[c][r] (columns c*32.. of row r) and S.colmask[q][j] (rows
// q*32.. of column j), both already restricted to core-core pairs. Writes
// S.par[buf][x] = the first node of x's component (for every node).
__device__ __forceinline__ void bfs_components(SmemTail& S, int buf, bool diag, int lane)
{
    const unsigned char* core = S.core[buf];
    int* rep = S.par[buf];
    uint32_t vis_r[4], vis_c[4];
#pragma unroll
    for (int w = 0; w < 4; ++w) {
        vis_r[w] = ~__ballot_sync(0xffffffffu, core[w * 32 + lane] != 0);
        vis_c[w] = diag ? 0xffffffffu : ~__ballot_sync(0xffffffffu, core[kT + w * 32 + lane] != 0);
    }
    for (int x = lane; x < 2 * kT; x += 32) rep[x] = x;
    __syncwarp();
    while (true) {
        int w0 = 0;
        while (w0 < 4 && vis_r[w0] == 0xffffffffu) ++w0;
        if (w0 == 4) break;
        const int r0 = w0 * 32 + __ffs(~vis_r[w0]) - 1;
        uint32_t comp_r[4] = {0u, 0u, 0u, 0u}, comp_c[4] = {0u, 0u, 0u, 0u}, front[4] = {0u, 0u, 0u, 0u};
        front[w0] = 1u << (r0 & 31);
        comp_r[w0] = front[w0];
        vis_r[w0] |= front[w0];
        for (int step = 0; step < 2 * kT; ++step) {
            // neighbours of the frontier rows: columns (or, diagonal pair, rows)
            uint32_t acc[4] = {0u, 0u, 0u, 0u};
#pragma unroll
            for (int w = 0; w < 4; ++w)
                if ((front[w] >> lane) & 1u) {
#pragma unroll
                    for (int c = 0; c < 4; ++c) acc[c] |= S.rowmask[c][w * 32 + lane];
                }
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[c] = __reduce_or_sync(0xffffffffu, acc[c]);
            bool grew = false;
            if (diag) {
#pragma unroll
                for (int w = 0; w < 4; ++w) {
                    front[w] = acc[w] & ~vis_r[w];
                    vis_r[w] |= front[w];
                    comp_r[w] |= front[w];
                    grew |= front[w] != 0u;
                }
            } else {
                uint32_t newc[4];
#pragma unroll
                for (int w = 0; w < 4; ++w) {
                    newc[w] = acc[w] & ~vis_c[w];
                    vis_c[w] |= newc[w];
                    comp_c[w] |= newc[w];
                }
                // rows adjacent to the new columns
                uint32_t accr[4] = {0u, 0u, 0u, 0u};
#pragma unroll
                for (int w = 0; w < 4; ++w)
                    if ((newc[w] >> lane) & 1u) {
#pragma unroll
                        for (int q = 0; q < 4; ++q) accr[q] |= q == 0 ? S.colmask[0][w * 32 + lane]
                                                              : q == 1 ? S.colmask[1][w * 32 + lane]
                                                              : q == 2 ? S.colmask[2][w * 32 + lane]
                                                                       : S.colmask[3][w * 32 + lane];
                    }
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    accr[q] = __reduce_or_sync(0xffffffffu, accr[q]);
                    front[q] = accr[q] & ~vis_r[q];
                    vis_r[q] |= front[q];
                    comp_r[q] |= front[q];
                    grew |= front[q] != 0u;
                }
            }
            if (!grew) break;
        }
        // every node of the component points at r0
#pragma unroll
        for (int w = 0; w < 4; ++w) {
            if ((comp_r[w] >> lane) & 1u) rep[w * 32 + lane] = r0;
            if ((comp_c[w] >> lane) & 1u) rep[kT + w * 32 + lane] = r0;
        }
        __syncwarp();
    }
}

// k-distance lists: insert (v, j) into an ascending list (v below its last).
constexpr int kKnnL = kKnnList;
__device__ __forceinline__ void knn_insert(float (&lv)[kKnnL], int (&li)[kKnnL], float v, int j)
{
#pragma unroll
    for (int i = kKnnL - 1; i > 0; --i) {
        const bool sh = v < lv[i - 1];
        const bool here = !sh && v < lv[i];
        lv[i] = sh ? lv[i - 1] : (here ? v : lv[i]);
        li[i] = sh ? li[i - 1] : (here ? j : li[i]);
    }
    if (v < lv[0]) { lv[0] = v; li[0] = j; }
}

template <int NS, int W>
struct TcShape {
    // blocks per stage: W = 1: Ah, Bh (, Al, Bl); W = 2: Ah (, Al), Bh0, Bh1 (, Bl0, Bl1)
    static constexpr int kOps = W == 1 ? (NS == 1 ? 2 : 4) : (NS == 1 ? 3 : 6);
    static constexpr int kStages = W == 1 ? (NS == 1 ? 4 : 3) : (NS == 1 ? 4 : 2);
    static constexpr int kStageBytes = kOps * kBlk;
    static constexpr int kAccCols = W * kT;               // TMEM columns of one accumulator
};

// W = 1: one tile pair per work item. W = 2: a group of one or two tile
// pairs sharing tile A, computed as one N = 256 product (both B tiles
// stacked), which halves the A loads; the epilogue takes its pairs in turn.
template <int NS, int MODE, int W, int F>
__global__ void __launch_bounds__(kThreads, 1) tc_kernel(const __grid_constant__ CUtensorMap mAh,
                                                         const __grid_constant__ CUtensorMap mAl,
                                                         const TcParams P)
{
    constexpr int kOps = TcShape<NS, W>::kOps;
    constexpr int kStages = TcShape<NS, W>::kStages;
    constexpr int kStageBytes = TcShape<NS, W>::kStageBytes;
    constexpr int kAccCols = TcShape<NS, W>::kAccCols;
    const int64_t n_cap = W == 1 ? P.n_pairs : P.n_groups;
    const int64_t n_items = MODE == 3 ? 0 : (P.n_dev ? min(n_cap, (int64_t)*P.n_dev) : n_cap);
    auto group_at = [&](int64_t g) -> int2 { return W == 1 ? make_int2((int)g, -1) : P.groups[g]; };
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    SmemTail& S = *reinterpret_cast<SmemTail*>(smem + kStages * kStageBytes);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const PassArgs& A = P.A;
    volatile int* abort = &S.abort;
    // work items of this CTA: g_begin, g_begin + g_step, .. < g_end. MODE 3: the
    // tile pairs (b, b + 1) of its chunk in order; else every gridDim-th group
    const int64_t kq_ch = MODE == 3 ? blockIdx.x % P.kq_chunks : 0;
    const int64_t kq_qt = MODE == 3 ? blockIdx.x / P.kq_chunks : 0;
    const int64_t kq_bhi = MODE == 3 ? min(P.kq_tp, (kq_ch + 1) * P.kq_ct) : 0;
    const int64_t g_begin = MODE == 3 ? 0 : blockIdx.x;
    const int64_t g_step = MODE == 3 ? 1 : gridDim.x;
    const int64_t g_end = MODE == 3 ? (kq_bhi > kq_ch * P.kq_ct ? (kq_bhi - kq_ch * P.kq_ct + 1) / 2 : 0) : n_items;
    // the k-th work item of this CTA. Count pass: runs of kRun consecutive
    // items (consecutive groups of the list mostly share tile A, whose blocks
    // then stay in the stages), the CTAs' runs interleaved so that the CTAs
    // working at one time stay close in the list (tiles shared through L2)
    constexpr bool kCountPass = MODE == 1 || MODE == 5;
    constexpr int kRun = kCountPass ? 4 : 1;
    auto item_at = [&](int64_t k) -> int64_t {
        if (MODE == 3) return k;
        return ((k / kRun) * (int64_t)gridDim.x + blockIdx.x) * kRun + (k % kRun);
    };
    // item_at(k + 1) from g = item_at(k)
    auto next_item = [&](int64_t k, int64_t g) -> int64_t {
        if (kRun == 1) return g + g_step;
        return ((k + 1) % kRun) ? g + 1 : g + ((int64_t)gridDim.x - 1) * kRun + 1;
    };
    // tiles of item g: (A, B0, B1 or -1)
    auto item = [&](int64_t g) -> int3 {
        if (MODE == 3) {
            const int64_t b0 = kq_ch * P.kq_ct + 2 * g;
            return make_int3((int)(P.kq_qt0 + kq_qt), (int)(b0 * P.kq_stride),
                             b0 + 1 < kq_bhi ? (int)((b0 + 1) * P.kq_stride) : -1);
        }
        const int2 grp = group_at(g);
        const int2 tp = A.pairs[grp.x];
        const int tb1 = W == 2 && grp.y >= 0 ? (A.pairs[grp.y].y & kPairTileMask) : -1;
        return make_int3(tp.x, tp.y & kPairTileMask, tb1);
    };

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&S.tmem_base)),
                     "r"(2 * kAccCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 32) {
        for (int i = 0; i < kStages; ++i) {
            mbar_init(&S.full[i], 1);
            mbar_init(&S.empty[i], 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(&S.acc_full[i], 1);
            mbar_init(&S.acc_empty[i], kEpiWarps);
        }
        mbar_init(&S.fin, 1);
        S.abort = 0;
        S.consumed = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = S.tmem_base;

    if (warp == 0) {
        // ---------------------------------------------------- TMA producer
        if (lane == 0) {
            int stage = 0;
            uint32_t phase = 0;
            int issued = 0;
            // count pass: the (tile A, K block) whose A blocks each stage holds;
            // a fill that needs the same ones leaves them in place
            int64_t tag[kCountPass ? kStages : 1];
#pragma unroll
            for (int i = 0; i < (kCountPass ? kStages : 1); ++i) tag[i] = -1;
            constexpr int nA = NS == 3 ? 2 : 1;                 // A blocks per stage (hi, lo)
            for (int64_t k = 0, g = kRun == 1 ? g_begin : item_at(0); g < g_end && !*abort; g = next_item(k, g), ++k) {
                const int3 itm = item(g);
                const int2 tp = make_int2(itm.x, itm.y);
                const bool diag = W == 1 && tp.x == tp.y;
                const int tb1 = itm.z;
                const int nbt = tb1 >= 0 ? 2 : 1;
                const uint32_t bytes = (uint32_t)((W == 1 ? (diag ? kOps / 2 : kOps)
                                                          : (NS == 3 ? 2 + 2 * nbt : 1 + nbt)) * kBlk);
                for (int kb = 0; kb < P.nkb; ++kb) {
                    if (!mbar_wait(&S.empty[stage], phase ^ 1, abort)) break;
                    unsigned char* st = smem + stage * kStageBytes;
                    bool keepA = false;
                    if constexpr (kCountPass) {
                        const int64_t want = (int64_t)tp.x * 4096 + kb;
                        keepA = tag[stage] == want;
                        tag[stage] = want;
                    }
                    mbar_expect_tx(&S.full[stage], keepA ? bytes - (uint32_t)(nA * kBlk) : bytes);
                    if (W == 1) {
                        if (!keepA) tma_load(st, &mAh, kb * kKB, tp.x * kT, &S.full[stage]);
                        if (!diag) tma_load(st + kBlk, &mAh, kb * kKB, tp.y * kT, &S.full[stage]);
                        if (NS == 3) {
                            if (!keepA) tma_load(st + 2 * kBlk, &mAl, kb * kKB, tp.x * kT, &S.full[stage]);
                            if (!diag) tma_load(st + 3 * kBlk, &mAl, kb * kKB, tp.y * kT, &S.full[stage]);
                        }
                    } else {
                        constexpr int bo = NS == 3 ? 2 : 1;      // first B block
                        if (!keepA) tma_load(st, &mAh, kb * kKB, tp.x * kT, &S.full[stage]);
                        tma_load(st + bo * kBlk, &mAh, kb * kKB, tp.y * kT, &S.full[stage]);
                        if (nbt == 2) tma_load(st + (bo + 1) * kBlk, &mAh, kb * kKB, tb1 * kT, &S.full[stage]);
                        if (NS == 3) {
                            if (!keepA) tma_load(st + kBlk, &mAl, kb * kKB, tp.x * kT, &S.full[stage]);
                            tma_load(st + 4 * kBlk, &mAl, kb * kKB, tp.y * kT, &S.full[stage]);
                            if (nbt == 2) tma_load(st + 5 * kBlk, &mAl, kb * kKB, tb1 * kT, &S.full[stage]);
                        }
                    }
                    ++issued;
                    if (++stage == kStages) { stage = 0; phase ^= 1; }
                }
            }
            // on abort: let the copies already issued land before the CTA exits
            if (*abort) {
                __threadfence_block();
                int consumed = *(volatile int*)&S.consumed;
                int st = consumed % kStages;
                uint32_t ph = (uint32_t)((consumed / kStages) & 1);
                volatile int dummy = 0;
                for (int f = consumed; f < issued; ++f) {
                    mbar_wait(&S.full[st], ph, &dummy);
                    if (++st == kStages) { st = 0; ph ^= 1; }
                }
            }
        }
    } else if (warp == 1) {
        // ---------------------------------------------------- MMA issuer
        if (lane == 0) {
            int stage = 0;
            uint32_t phase = 0;
            int it = 0;
            for (int64_t k = 0, g = kRun == 1 ? g_begin : item_at(0); g < g_end && !*abort;
                 g = next_item(k, g), ++k, ++it) {
                const int3 itm = item(g);
                const bool diag = W == 1 && itm.x == itm.y;
                const uint32_t idesc = F ? (W == 2 && itm.z >= 0 ? kIdescF8x2 : kIdescF8)
                                         : (W == 2 && itm.z >= 0 ? kIdesc2 : kIdesc);
                const int buf = it & 1;
                const uint32_t acc_phase = (uint32_t)((it >> 1) & 1);
                if (!mbar_wait(&S.acc_empty[buf], acc_phase ^ 1, abort)) break;
                tc_fence_after();
                const uint32_t d_tmem = tmem + (uint32_t)(buf * kAccCols);
                bool ok = true;
                for (int kb = 0; kb < P.nkb; ++kb) {
                    if (!mbar_wait(&S.full[stage], phase, abort)) { ok = false; break; }
                    tc_fence_after();
                    const uint32_t base = su32(smem + stage * kStageBytes);
                    uint32_t ah, bh, al, bl;
                    if (W == 1) {
                        ah = base; bh = diag ? base : base + kBlk;
                        al = base + 2 * kBlk; bl = diag ? al : base + 3 * kBlk;
                    } else {
                        ah = base; al = base + kBlk;
                        bh = base + (NS == 3 ? 2 : 1) * kBlk; bl = base + 4 * kBlk;
                    }
#pragma unroll
                    for (int j = 0; j < kKB / 16; ++j) {
                        const uint32_t acc0 = (kb | j) ? 1u : 0u;
                        if constexpr (F) {
                            mma_f8_id(d_tmem, smem_desc(ah + 32 * j), smem_desc(bh + 32 * j), idesc, acc0);
                            if (NS == 3) {
                                mma_f8_id(d_tmem, smem_desc(ah + 32 * j), smem_desc(bl + 32 * j), idesc, 1u);
                                mma_f8_id(d_tmem, smem_desc(al + 32 * j), smem_desc(bh + 32 * j), idesc, 1u);
                            }
                        } else {
                            mma_bf16_id(d_tmem, smem_desc(ah + 32 * j), smem_desc(bh + 32 * j), idesc, acc0);
                            if (NS == 3) {
                                mma_bf16_id(d_tmem, smem_desc(ah + 32 * j), smem_desc(bl + 32 * j), idesc, 1u);
                                mma_bf16_id(d_tmem, smem_desc(al + 32 * j), smem_desc(bh + 32 * j), idesc, 1u);
                            }
                        }
                    }
                    mma_commit(&S.empty[stage]);
                    *(volatile int*)&S.consumed = S.consumed + 1;
                    if (++stage == kStages) { stage = 0; phase ^= 1; }
                }
                if (!ok) break;
                mma_commit(&S.acc_full[buf]);
            }
            // all MMAs issued by this thread have completed once `fin` flips
            mma_commit(&S.fin);
            volatile int dummy = 0;
            mbar_wait(&S.fin, 0, &dummy);
        }
    } else if constexpr (MODE == 4) {
        // ------------------------------ epilogue: accumulators to memory (probe)
        const int quad = warp & 3, part = (warp - 2) >> 2, r = quad * 32 + lane;
        int git = 0;
        for (int64_t g = blockIdx.x; g < n_items; g += gridDim.x, ++git) {
            const int tbuf = git & 1;
            const bool bad = !mbar_wait(&S.acc_full[tbuf], (uint32_t)((git >> 1) & 1), abort) || *abort;
            if (epi_sync_or(bad)) break;
            tc_fence_after();
            float v[32];
            tmem_ld32(tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(tbuf * kAccCols + part * 32), v);
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&S.acc_empty[tbuf]);
            float* out = P.dump + ((int64_t)g * kT + r) * kT + part * 32;
#pragma unroll
            for (int i = 0; i < 32; ++i) out[i] = v[i];
        }
    } else if constexpr (MODE == 3) {
        // ------------------------------------- epilogue: k smallest distances
        // Warp w holds TMEM lane quadrant (w & 3) = query rows 32 (w & 3) ..
        // +31 (a row per lane) and the 32-column part (w - 2) >> 2 of every
        // point tile, and works alone (no barrier across warps). For query
        // row a and point b, key = RD(R + t) with R = RD(|a|^2 m - A3) and t =
        // RD(c2 acc + C_b), C_b = RD(|b|^2 m), is a lower bound of d^2 (FAR:
        // of -d^2; the host picks m, c2). A row keeps the keys below its
        // limit T: list mode, the kKnnL smallest per part of the chunk (T =
        // the list's last entry); append mode, every key <= tau[query] (T =
        // the next float above tau). key < T implies t < RU(T - R) = thr, so
        // values with t >= thr are dropped on the FMA result alone, 16 at a
        // time.
        const int ew = warp - 2;
        const int quad = warp & 3;
        const int part = ew >> 2;
        const int r = quad * 32 + lane;
        const int64_t qi = kq_qt * kT + r;
        const bool valid_r = qi < P.kq_q;
        const bool append = P.kq_tau != nullptr;
        const float c2 = P.kq_c2, m = P.kq_m;
        const float R = __fmaf_rd(P.rn2[(P.kq_qt0 + kq_qt) * kT + r], m, -P.A3f);
        float lim = INFINITY;                                 // append: largest key kept
        if (append && valid_r) lim = P.kq_tau[qi];
        const float t_app = lim < INFINITY ? nextafterf(lim, INFINITY) : INFINITY;
        float lv[kKnnL];
        int li[kKnnL];
#pragma unroll
        for (int i = 0; i < kKnnL; ++i) { lv[i] = INFINITY; li[i] = -1; }
        float thr = valid_r ? __fsub_ru(append ? t_app : INFINITY, R) : -INFINITY;
        float* cst = S.wn[ew];                                // C_b of the warp's 32 columns
        int git = 0;
        bool stop = false;
        for (int64_t g = g_begin; g < g_end; g += g_step, ++git) {
            const int3 itm = item(g);
            const int nbt = itm.z >= 0 ? 2 : 1;
            const int tbuf = git & 1;
            // the columns' C_b, loaded before the accumulator wait
            float cj[2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int tb = h ? (itm.z >= 0 ? itm.z : itm.y) : itm.y;
                const int jc = part * 32 + lane;
                cj[h] = jc < A.tile_n[tb] ? __fmul_rd(P.rn2[(int64_t)tb * kT + jc], m) : INFINITY;
            }
            const bool bad = !mbar_wait(&S.acc_full[tbuf], (uint32_t)((git >> 1) & 1), abort) || *abort;
            if (__any_sync(0xffffffffu, bad)) { stop = true; break; }
            tc_fence_after();
            for (int h = 0; h < nbt; ++h) {
                const int64_t sb = (int64_t)(h ? itm.z : itm.y) * kT;
                __syncwarp();                                 // the previous tile's reads are done
                cst[lane] = cj[h];
                __syncwarp();
#pragma unroll 1
                for (int c16 = 0; c16 < 2; ++c16) {
                    float v[16];
                    tmem_ld16(tmem + ((uint32_t)(quad * 32) << 16) +
                                  (uint32_t)(tbuf * kAccCols + h * kT + part * 32 + c16 * 16), v);
                    if (c16 == 1 && h == nbt - 1) {
                        tc_fence_before();
                        __syncwarp();
                        if (lane == 0) mbar_arrive(&S.acc_empty[tbuf]);
                    }
                    const float4* c4 = reinterpret_cast<const float4*>(cst + c16 * 16);
                    float t[16];
#pragma unroll
                    for (int i4 = 0; i4 < 4; ++i4) {
                        const float4 cc = c4[i4];
                        t[4 * i4 + 0] = __fmaf_rd(c2, v[4 * i4 + 0], cc.x);
                        t[4 * i4 + 1] = __fmaf_rd(c2, v[4 * i4 + 1], cc.y);
                        t[4 * i4 + 2] = __fmaf_rd(c2, v[4 * i4 + 2], cc.z);
                        t[4 * i4 + 3] = __fmaf_rd(c2, v[4 * i4 + 3], cc.w);
                    }
                    float tmin = fmin3(t[0], t[1], t[2]);
#pragma unroll
                    for (int i = 3; i + 1 < 16; i += 2) tmin = fmin3(tmin, t[i], t[i + 1]);
                    tmin = fminf(tmin, t[15]);
                    if (!__any_sync(0xffffffffu, tmin < thr)) continue;
                    const int j0 = (int)sb + part * 32 + c16 * 16;
#pragma unroll
                    for (int i = 0; i < 16; ++i) {
                        if (!(t[i] < thr)) continue;
                        const float key = __fadd_rd(R, t[i]);
                        if (append) {
                            if (key < t_app) {
                                const int slot = atomicAdd(&P.kq_cnt[qi], 1);
                                const int64_t base = P.kq_off ? P.kq_off[qi] : qi * P.kq_cap;
                                if (slot < (P.kq_off ? P.kq_off[qi + 1] - base : (int64_t)P.kq_cap)) {
                                    P.kq_v[base + slot] = key;
                                    P.kq_i[base + slot] = j0 + i;
                                }
                            }
                        } else if (key < lv[kKnnL - 1]) {
                            knn_insert(lv, li, key, j0 + i);
                            thr = __fsub_ru(lv[kKnnL - 1], R);
                        }
                    }
                }
            }
        }
        if (!stop && valid_r && !append) {
            const int64_t base = ((qi * P.kq_chunks + kq_ch) * 4 + part) * kKnnL;
#pragma unroll
            for (int i = 0; i < kKnnL; ++i) {
                P.kq_v[base + i] = lv[i];
                P.kq_i[base + i] = li[i];
            }
        }
    } else if constexpr (kCountPass) {
        // ------------------------------------------ epilogue: count pass
        // Each epilogue warp works alone on one 32 x 32 sub-block of every
        // tile pair: TMEM lane quadrant quad = A rows 32 quad .. +31 (a row per
        // lane) and B columns 32 part .. +31; no barrier across warps. Per
        // pair: screen values u = fl(2 acc - |b|^2) against per-row limits
        // (all out / all in at once from the row's extremes), then the row
        // counts (and lists) from the lane's bits and the column counts from
        // a 32 x 32 bit transpose; band pairs go to the FP64 recheck, or, in
        // the first phase of the two-phase pass, defer the whole sub-block to
        // the three-product pass. Each item's group and tile pairs are loaded
        // while the previous item is processed, its row and column data before
        // the accumulator wait.
        const int ew = warp - 2;                              // 0 .. 15
        const int quad = warp & 3;
        const int part = ew >> 2;
        const int sub = quad * 4 + part;
        const int r = quad * 32 + lane;
        float* wn = S.wn[ew];
        struct Item {
            int q[2], tb[2], nb[2], pre_col[2];               // per pair (B side)
            float ncol2[2], bn2[2], bn[2], bl[2], bmin2[2];
            float sb[2];                                      // FP8: the B tiles' scales
            int ta, na, pre_row;                              // A side (shared by the pairs)
            float na2, nra, rla, sa;
            int nbt;
            bool mine[2];
        };
        // the item's group and tile pairs (the first loads of its chain), then the rest
        struct Head {
            int2 grp, tp[2];
        };
        auto load_head = [&](int64_t g, Head& hd) {
            hd.grp = group_at(g);
            hd.tp[0] = A.pairs[hd.grp.x];
            hd.tp[1] = hd.grp.y >= 0 ? A.pairs[hd.grp.y] : hd.tp[0];
        };
        auto load_item = [&](const Head& hd, Item& it) {
            const int2 grp = hd.grp;
            it.nbt = grp.y >= 0 ? 2 : 1;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                if (h >= it.nbt) break;
                it.q[h] = h ? grp.y : grp.x;
                it.mine[h] = P.sub_mask ? ((P.sub_mask[P.sub_q[it.q[h]]] >> sub) & 1u) != 0u : true;
                int2 tp = hd.tp[h];
                if (!MGB_IN_RANGE(tp.x, A.n_tiles, A.stats + kStatOob) ||
                    !MGB_IN_RANGE(tp.y & kPairTileMask, A.n_tiles, A.stats + kStatOob)) {
                    tp = make_int2(0, 0);                     // checked build: counted, then skipped
                    it.mine[h] = false;
                }
                it.tb[h] = tp.y & kPairTileMask;
                if (h == 0) {
                    it.ta = tp.x;
                    it.na = A.tile_n[tp.x];
                    const int64_t row = (int64_t)tp.x * kT + r;
                    it.na2 = P.rn2[row];
                    it.nra = P.rn[row];
                    it.rla = P.rl ? P.rl[row] : 0.f;
                    if constexpr (MODE == 5) {
                        // bit e: radius e's list of this row is full (its count can only grow)
                        int full = A.cap > 0 ? 0 : 0xF;
#pragma unroll
                        for (int e = 0; e < kMaxRadii; ++e)
                            if (A.cap > 0 && e < P.n_rad && P.rad[e].count[row] >= A.cap) full |= 1 << e;
                        it.pre_row = full;
                    } else {
                        it.pre_row = MODE == 1 && A.cap > 0 ? A.count[row] : INT_MAX;
                    }
                    it.sa = F ? P.tmax[tp.x].w : 1.f;
                }
                it.nb[h] = A.tile_n[it.tb[h]];
                const int64_t col = (int64_t)it.tb[h] * kT + part * 32 + lane;
                it.ncol2[h] = -P.rn2[col];
                const float4 tm = P.tmax[it.tb[h]];
                it.bn2[h] = tm.x;
                it.bn[h] = tm.y;
                it.bl[h] = tm.z;
                it.sb[h] = tm.w;
                it.bmin2[h] = P.tn2min[it.tb[h]];
                if constexpr (MODE == 5) {
                    // (W = 2: rows only; the columns' reads would not fit the registers)
                    int full = A.cap > 0 ? 0 : 0xF;
                    if constexpr (W == 1) {
#pragma unroll
                        for (int e = 0; e < kMaxRadii; ++e)
                            if (A.cap > 0 && it.mine[h] && tp.x != it.tb[h] && e < P.n_rad &&
                                P.rad[e].count[col] >= A.cap)
                                full |= 1 << e;
                    }
                    it.pre_col[h] = full;
                } else {
                    it.pre_col[h] = MODE == 1 && A.cap > 0 && it.mine[h] && tp.x != it.tb[h] ? A.count[col] : INT_MAX;
                }
            }
        };
        int64_t screened = 0;
        int git = 0;
        Item cur;
        Head head;
        int64_t g = item_at(0), g_next = 0;
        if (g < n_items) load_head(g, head);
        for (int64_t k = 0; g < n_items; ++k, ++git, g = g_next) {
            g_next = next_item(k, g);
            load_item(head, cur);
            if (g_next < n_items) load_head(g_next, head);
            const int tbuf = git & 1;
            const bool bad = !mbar_wait(&S.acc_full[tbuf], (uint32_t)((git >> 1) & 1), abort) || *abort;
            if (__any_sync(0xffffffffu, bad)) break;
            tc_fence_after();
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                if (h >= cur.nbt) break;
                const int q = cur.q[h];
                const bool diag = cur.ta == cur.tb[h];
                const int64_t sa = (int64_t)cur.ta * kT, sb = (int64_t)cur.tb[h] * kT;
                const int64_t row = sa + r, col = sb + part * 32 + lane;
                float u[32];
                tmem_ld32(tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(tbuf * kAccCols + h * kT + part * 32), u);
                if (h == cur.nbt - 1) {
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&S.acc_empty[tbuf]);
                }
                if (!P.sub_mask && ew == 0 && lane == 0)
                    screened += diag ? (int64_t)cur.na * (cur.na + 1) / 2 : (int64_t)cur.na * cur.nb[h];
                if (!cur.mine[h]) continue;
                // per-row limits: in iff u >= k_in, out iff u < k_out (FP32, outward rounding)
                float E;
                if (P.rl) {
                    const float cross = __fadd_ru(__fmul_ru(cur.rla, cur.bn[h]), __fmul_ru(cur.nra, cur.bl[h]));
                    E = __fmaf_ru(P.K2f, __fmul_ru(cur.rla, cur.bl[h]),
                                  __fmaf_ru(P.K1f, cross,
                                            __fmaf_ru(P.K0f, __fmul_ru(cur.nra, cur.bn[h]),
                                                      __fmaf_ru(P.A2f, __fadd_ru(cur.na2, cur.bn2[h]), P.A3f))));
                } else {
                    E = __fmaf_ru(P.A1f, __fmul_ru(cur.nra, cur.bn[h]),
                                  __fmaf_ru(P.A2f, __fadd_ru(cur.na2, cur.bn2[h]), P.A3f));
                }
                float two = 2.f;
                if constexpr (F) {
                    // E4M3 subnormal floor of the scaled rows: K4 (s_b |a| + s_a |b|) + K5 s_a s_b
                    const float ss = cur.sa * cur.sb[h];              // exact (powers of two)
                    E = __fmaf_ru(P.K4f, __fadd_ru(__fmul_ru(cur.sb[h], cur.nra), __fmul_ru(cur.sa, cur.bn[h])),
                                  __fmaf_ru(P.K5f, ss, E));
                    two = 2.f * ss;
                }
                if constexpr (MODE == 5) {
                    // Several radii, ascending, each with the limits of the
                    // one-radius pass below. A row all out at a radius is all
                    // out at every smaller one; the screen values are formed
                    // once and compared with each radius's limits.
                    const int nr = P.n_rad;
                    const bool pad = r >= cur.na;             // padding rows hold no pair
                    auto k_in_of = [&](float lo) { return __fadd_ru(__fsub_ru(cur.na2, lo), E); };
                    auto k_out_of = [&](float hi) { return __fsub_rd(__fsub_rd(cur.na2, hi), E); };
                    float vmax = fmax3(u[0], u[1], u[2]);
#pragma unroll
                    for (int i = 3; i + 1 < 32; i += 2) vmax = fmax3(vmax, u[i], u[i + 1]);
                    vmax = fmaxf(vmax, u[31]);
                    const float xmax = __fmaf_ru(two, vmax, -cur.bmin2[h]);
                    int e_lo = nr;                            // radii e_lo .. nr - 1 hold a row not all out
#pragma unroll
                    for (int e = kMaxRadii - 1; e >= 0; --e) {
                        if (e >= nr) continue;
                        const bool out = pad || xmax < k_out_of(P.rad[e].eps2_hi);
                        if (__all_sync(0xffffffffu, out)) break;
                        e_lo = e;
                    }
                    if (e_lo == nr) continue;                 // all out at every radius
                    float vmin = fmin3(u[0], u[1], u[2]);
#pragma unroll
                    for (int i = 3; i + 1 < 32; i += 2) vmin = fmin3(vmin, u[i], u[i + 1]);
                    vmin = fminf(vmin, u[31]);
                    const float xmin = __fmaf_rd(two, vmin, -cur.bn2[h]);
                    bool mixed = false;
#pragma unroll
                    for (int e = 0; e < kMaxRadii; ++e) {
                        if (e < e_lo || e >= nr) continue;
                        const bool out = pad || xmax < k_out_of(P.rad[e].eps2_hi);
                        mixed |= !out && !(xmin >= k_in_of(P.rad[e].eps2_lo));
                    }
                    mixed = __any_sync(0xffffffffu, mixed);
                    auto defer_radii = [&]() {
                        if (lane == 0) {
                            if (atomicOr(&P.redo_mask[q], 1u << sub) == 0u) atomicAdd(&A.stats[kStatRedo], 1ull);
#pragma unroll
                            for (int e = 0; e < kMaxRadii; ++e)
                                if (e < nr && P.rad[e].pair_hit) P.rad[e].pair_hit[q] = 1;
                        }
                    };
                    if (P.defer == 2 && mixed) {
                        defer_radii();
                        continue;
                    }
                    if (mixed) {
                        __syncwarp();                         // the previous pair's wn is read
                        wn[lane] = cur.ncol2[h];
                        __syncwarp();
                        const float4* wn4 = reinterpret_cast<const float4*>(wn);
#pragma unroll
                        for (int i4 = 0; i4 < 8; ++i4) {
                            const float4 nn = wn4[i4];
                            fma2_inplace(u[4 * i4 + 0], u[4 * i4 + 1], two, nn.x, nn.y);
                            fma2_inplace(u[4 * i4 + 2], u[4 * i4 + 3], two, nn.z, nn.w);
                        }
                    }
                    const int left = cur.nb[h] - part * 32;
                    const uint32_t cand = pad ? 0u : (left >= 32 ? 0xffffffffu : (left > 0 ? (1u << left) - 1u : 0u));
                    // in and band bits of one radius
                    auto bits_of = [&](float lo, float hi, uint32_t& inb, uint32_t& band) {
                        const float k_in = k_in_of(lo), k_out = k_out_of(hi);
                        const bool out = pad || xmax < k_out;
                        uint32_t ib = 0u, kb = 0u;
                        if (!out && xmin >= k_in) {
                            ib = kb = 0xffffffffu;
                        } else if (!out) {
#pragma unroll
                            for (int i = 0; i < 32; ++i) {
                                if (u[i] >= k_in) ib |= 1u << i;
                                if (u[i] >= k_out) kb |= 1u << i;
                            }
                        }
                        inb = ib & cand;
                        band = kb & ~ib & cand;
                    };
                    if (P.defer == 1) {
                        bool any_band = false;
#pragma unroll
                        for (int e = 0; e < kMaxRadii; ++e) {
                            if (e < e_lo || e >= nr) continue;
                            uint32_t ib, bd;
                            bits_of(P.rad[e].eps2_lo, P.rad[e].eps2_hi, ib, bd);
                            any_band |= bd != 0u;
                        }
                        if (__any_sync(0xffffffffu, any_band)) {
                            defer_radii();
                            continue;
                        }
                    }
#pragma unroll
                    for (int e = 0; e < kMaxRadii; ++e) {
                        if (e < e_lo || e >= nr) continue;
                        int32_t* const cnt = P.rad[e].count;
                        int32_t* const nbl = P.rad[e].nbr;
                        uint32_t inb, band;
                        bits_of(P.rad[e].eps2_lo, P.rad[e].eps2_hi, inb, band);
                        if (!__any_sync(0xffffffffu, (inb | band) != 0u)) continue;
                        if (lane == 0 && P.rad[e].pair_hit) P.rad[e].pair_hit[q] = 1;
                        uint32_t bq = band;
                        while (bq) {
                            const int i = __ffs(bq) - 1;
                            bq &= bq - 1;
                            const int j = part * 32 + i;
                            const uint32_t fl = (diag ? 0u : kQBoth) | ((!diag || r < j) ? kQTie : 0u);
                            bool decided;
                            const bool in = push_band_radius(P, P.rad[e].queue, P.rad[e].queue_n, P.rad[e].stats,
                                                             P.rad[e].eps2, P.rad[e].tie_thr, (int)row, (int)(sb + j),
                                                             fl, &decided);
                            if (decided && in) inb |= 1u << i;
                        }
                        // counts, and list entries while the list has room (read
                        // before the item: a full list takes no returning atomic)
                        const int k = __popc(inb);
                        if (k) {
                            if ((cur.pre_row >> e) & 1) {
                                atomicAdd(&cnt[row], k);
                            } else {
                                int pos = atomicAdd(&cnt[row], k);
                                uint32_t bm = inb;
                                while (bm && pos < A.cap) {
                                    const int i = __ffs(bm) - 1;
                                    bm &= bm - 1;
                                    nbl[row * A.cap + pos++] = (int32_t)(sb + part * 32 + i);
                                }
                            }
                        }
                        if (!diag && __any_sync(0xffffffffu, inb != 0u)) {
                            uint32_t x = inb;
#pragma unroll
                            for (int sft = 16; sft >= 1; sft >>= 1) {
                                const uint32_t m = sft == 16 ? 0x0000FFFFu : sft == 8 ? 0x00FF00FFu
                                                 : sft == 4 ? 0x0F0F0F0Fu : sft == 2 ? 0x33333333u : 0x55555555u;
                                const uint32_t y = __shfl_xor_sync(0xffffffffu, x, sft);
                                x = (lane & sft) ? (((y >> sft) & m) | (x & ~m)) : ((x & m) | ((y & m) << sft));
                            }
                            const int kc = __popc(x);
                            if (kc) {
                                if ((cur.pre_col[h] >> e) & 1) {
                                    atomicAdd(&cnt[col], kc);
                                } else {
                                    int pos = atomicAdd(&cnt[col], kc);
                                    while (x && pos < A.cap) {
                                        const int i = __ffs(x) - 1;
                                        x &= x - 1;
                                        nbl[col * A.cap + pos++] = (int32_t)(sa + quad * 32 + i);
                                    }
                                }
                            }
                        }
                    }
                    continue;
                }
                const float k_in = __fadd_ru(__fsub_ru(cur.na2, P.eps2_lo), E);
                const float k_out = __fsub_rd(__fsub_rd(cur.na2, P.eps2_hi), E);
                // the row's extremes from the raw accumulator: with x_j = two acc_j -
                // |b_j|^2 (exact), max x <= RU(two max acc - min |b|^2) and min x >=
                // RD(two min acc - max |b|^2); x < k_out certifies out and x >= k_in in
                // (E covers the rounding of the computed screen value too)
                float vmax = fmax3(u[0], u[1], u[2]);
#pragma unroll
                for (int i = 3; i + 1 < 32; i += 2) vmax = fmax3(vmax, u[i], u[i + 1]);
                vmax = fmaxf(vmax, u[31]);
                uint32_t in_bits = 0u, keep_bits = 0u;
                // padding rows hold no pair: out
                const bool all_out = r >= cur.na || __fmaf_ru(two, vmax, -cur.bmin2[h]) < k_out;
                if (__all_sync(0xffffffffu, all_out)) continue;   // nothing in, no band: nothing to do
                bool all_in = false;
                if (!all_out) {
                    float vmin = fmin3(u[0], u[1], u[2]);
#pragma unroll
                    for (int i = 3; i + 1 < 32; i += 2) vmin = fmin3(vmin, u[i], u[i + 1]);
                    vmin = fminf(vmin, u[31]);
                    all_in = __fmaf_rd(two, vmin, -cur.bn2[h]) >= k_in;
                }
                const bool mixed = !all_out && !all_in;
                auto defer_block = [&]() {
                    // first phase: the sub-block goes to the three-product pass, whole
                    if (lane == 0) {
                        if (atomicOr(&P.redo_mask[q], 1u << sub) == 0u) atomicAdd(&A.stats[kStatRedo], 1ull);
                        if (A.pair_hit) A.pair_hit[q] = 1;
                    }
                };
                // first phase, extremes only: a block with a row neither all in
                // nor all out is deferred without looking at its values
                if (P.defer == 2 && __any_sync(0xffffffffu, mixed)) {
                    defer_block();
                    continue;
                }
                if (__any_sync(0xffffffffu, mixed)) {
                    __syncwarp();                             // the previous pair's wn is read
                    wn[lane] = cur.ncol2[h];
                    __syncwarp();
                }
                if (all_in) {
                    in_bits = keep_bits = 0xffffffffu;
                } else if (mixed) {
                    // u = fl(two acc - |b|^2) (two = 2, or 2 s_a s_b for FP8), two
                    // columns per packed FMA (each lane correctly rounded)
                    const float4* wn4 = reinterpret_cast<const float4*>(wn);
#pragma unroll
                    for (int i4 = 0; i4 < 8; ++i4) {
                        const float4 nn = wn4[i4];
                        fma2_inplace(u[4 * i4 + 0], u[4 * i4 + 1], two, nn.x, nn.y);
                        fma2_inplace(u[4 * i4 + 2], u[4 * i4 + 3], two, nn.z, nn.w);
                    }
#pragma unroll
                    for (int i = 0; i < 32; ++i) {
                        if (u[i] >= k_in) in_bits |= 1u << i;
                        if (u[i] >= k_out) keep_bits |= 1u << i;
                    }
                }
                const int left = cur.nb[h] - part * 32;
                const uint32_t cand = r >= cur.na ? 0u
                                                  : (left >= 32 ? 0xffffffffu : (left > 0 ? (1u << left) - 1u : 0u));
                uint32_t inb = in_bits & cand;
                const uint32_t band = keep_bits & ~in_bits & cand;
                if (P.defer && __any_sync(0xffffffffu, band != 0u)) {
                    defer_block();
                    continue;
                }
                if (A.pair_hit && __any_sync(0xffffffffu, (inb | band) != 0u) && lane == 0) A.pair_hit[q] = 1;
                // band pairs: queued for the FP64 recheck; decided here if the queue is full
                uint32_t bq = band;
                while (bq) {
                    const int i = __ffs(bq) - 1;
                    bq &= bq - 1;
                    const int j = part * 32 + i;
                    const uint32_t fl = (diag ? 0u : kQBoth) | ((!diag || r < j) ? kQTie : 0u);
                    bool decided;
                    const bool in = push_band(P, (int)row, (int)(sb + j), fl, &decided);
                    if (decided && in) inb |= 1u << i;
                }
                // row counts (and the first cap neighbours of each row)
                const int k = __popc(inb);
                if (k) {
                    if (cur.pre_row < A.cap) {
                        int pos = atomicAdd(&A.count[row], k);
                        uint32_t bm = inb;
                        while (bm && pos < A.cap) {
                            const int i = __ffs(bm) - 1;
                            bm &= bm - 1;
                            A.nbr[row * A.cap + pos++] = (int32_t)(sb + part * 32 + i);
                        }
                    } else {
                        atomicAdd(&A.count[row], k);
                    }
                }
                // column counts: 32 x 32 bit transpose, lane j gets column part * 32 + j
                if (!diag && __any_sync(0xffffffffu, inb != 0u)) {
                    uint32_t x = inb;
#pragma unroll
                    for (int sft = 16; sft >= 1; sft >>= 1) {
                        const uint32_t m = sft == 16 ? 0x0000FFFFu : sft == 8 ? 0x00FF00FFu : sft == 4 ? 0x0F0F0F0Fu
                                                               : sft == 2 ? 0x33333333u : 0x55555555u;
                        const uint32_t y = __shfl_xor_sync(0xffffffffu, x, sft);
                        x = (lane & sft) ? (((y >> sft) & m) | (x & ~m)) : ((x & m) | ((y & m) << sft));
                    }
                    const int kc = __popc(x);
                    if (kc) {
                        if (cur.pre_col[h] < A.cap) {
                            int pos = atomicAdd(&A.count[col], kc);
                            while (x && pos < A.cap) {
                                const int i = __ffs(x) - 1;
                                x &= x - 1;
                                A.nbr[col * A.cap + pos++] = (int32_t)(sa + quad * 32 + i);
                            }
                        } else {
                            atomicAdd(&A.count[col], kc);
                        }
                    }
                }
            }
        }
        if (screened) {
            atomicAdd(&A.stats[kStatScreened], (unsigned long long)screened);
            atomicAdd(&A.stats[kStatTcPairs], (unsigned long long)screened);
        }
    } else {
        // ---------------------------------------------------- epilogue
        // Union pass. kEpiWarps warps: warp w reads TMEM lane quadrant (w & 3)
        // = A rows 32(w & 3) .. +31 and the 32 kChunks columns of part
        // (w - 2) / 4. Each pair's norms and core flags are loaded one pair
        // ahead.
        const int et = tid - 64;                              // 0 .. kEpiThreads-1
        const int quad = warp & 3;
        const int half = (warp - 2) >> 2;                     // column part
        const int r = quad * 32 + lane;                       // accumulator row = A-tile row
        struct Pre {
            int2 tp;
            bool one_each;                                    // union pass: see kPairOneEach
            int na, nb;
            float na2, nra, rla;                              // row r
            float c2, c1, c3;                                 // column et (et < 128)
            bool core_et;                                     // union pass: row et of A | B
            int count_et;                                     // count pass: count of row / column et
        };
        auto prefetch = [&](int64_t q, Pre& f) {
            f.tp = A.pairs[q];
            f.one_each = (f.tp.y & kPairOneEach) != 0;
            f.tp.y &= kPairTileMask;
            if (!MGB_IN_RANGE(f.tp.x, A.n_tiles, A.stats + kStatOob) ||
                !MGB_IN_RANGE(f.tp.y, A.n_tiles, A.stats + kStatOob))
                f.tp = make_int2(0, 0);                       // checked build: counted (results flagged)
            f.na = A.tile_n[f.tp.x];
            f.nb = A.tile_n[f.tp.y];
            const int64_t sa = (int64_t)f.tp.x * kT, sb = (int64_t)f.tp.y * kT;
            f.na2 = P.rn2[sa + r];
            f.nra = P.rn[sa + r];
            f.rla = P.rl ? P.rl[sa + r] : 0.f;
            if (et < kT) {
                f.c2 = P.rn2[sb + et];
                f.c1 = P.rn[sb + et];
                f.c3 = P.rl ? P.rl[sb + et] : 0.f;
            }
            if (MODE == 2) {
                const bool diag = f.tp.x == f.tp.y;
                f.core_et = et < kT ? (et < f.na && A.core[sa + et])
                                    : (et < 2 * kT && !diag && et - kT < f.nb && A.core[sb + et - kT]);
            } else if (et < 2 * kT) {
                f.count_et = et < kT ? A.count[sa + et] : A.count[sb + et - kT];
            }
        };
        // work items in turn, each one or (W = 2) two pairs: `it` counts pairs
        // (staging buffers), `git` items (TMEM accumulators)
        Pre cur{};
        int64_t g = blockIdx.x;
        int2 grp = g < n_items ? group_at(g) : make_int2(-1, -1);
        int h = 0;                                            // pair of the item
        if (g < n_items) prefetch(grp.x, cur);
        int it = 0, git = 0;
        int64_t screened = 0;
        while (g < n_items) {
            const int64_t q = h ? grp.y : grp.x;
            const bool last_sub = h == 1 || grp.y < 0;
            int64_t g_next = g;
            int h_next = 1;
            int2 grp_next = grp;
            if (last_sub) {
                g_next = g + gridDim.x;
                h_next = 0;
                grp_next = g_next < n_items ? group_at(g_next) : make_int2(-1, -1);
            }
            const int2 tp = cur.tp;
            const bool diag = tp.x == tp.y;
            const bool one_each = MODE == 2 && cur.one_each;
            const int na = cur.na, nb = cur.nb;
            const int64_t sa = (int64_t)tp.x * kT, sb = (int64_t)tp.y * kT;
            const int buf = it & 1;
            const int tbuf = git & 1;
            const uint32_t acc_phase = (uint32_t)((git >> 1) & 1);
            const bool valid_r = r < na;
            const float na2 = cur.na2, nra = cur.nra, rla = cur.rla;
            const int pre_count = cur.count_et;

            // (1) stage this pair's column data (and core rows, roots) in buffer `buf`
            if (et < kT) {
                S.nbn[buf][et] = -cur.c2;
                float m2 = cur.c2, m1 = cur.c1, m3 = cur.c3;
                for (int o = 16; o; o >>= 1) {
                    m2 = fmaxf(m2, __shfl_xor_sync(0xffffffffu, m2, o));
                    m1 = fmaxf(m1, __shfl_xor_sync(0xffffffffu, m1, o));
                    m3 = fmaxf(m3, __shfl_xor_sync(0xffffffffu, m3, o));
                }
                if (lane == 0) {
                    S.red[buf][et >> 5] = m2;
                    S.red[buf][4 + (et >> 5)] = m1;
                    S.red[buf][8 + (et >> 5)] = m3;
                }
            }
            if (MODE == 2 && et < 2 * kT) {
                const bool cc = cur.core_et;
                S.core[buf][et] = cc;
                S.par[buf][et] = et;
                // column core bits: B rows (diagonal pair: A rows)
                const bool colc = diag ? (et < kT && cc) : (et >= kT && cc);
                const uint32_t m = __ballot_sync(0xffffffffu, colc);
                if (lane == 0 && (diag ? et < kT : et >= kT)) S.colcore[buf][(et & (kT - 1)) >> 5] = m;
                if (et == 0) { S.s_mm[buf][0] = INT_MAX; S.s_mm[buf][1] = -1; }
            }
            if (MODE == 2) {
                if (et == 0) S.edges[buf] = 0;
                epi_sync();                                     // s_mm, edges initialised
            }
            if (MODE == 2 && et < 2 * kT && cur.core_et) {
                const int rr = gfind(A.parent, (int)(et < kT ? sa + et : sb + et - kT));
                S.groot[buf][et] = rr;
                atomicMin(&S.s_mm[buf][0], rr);
                atomicMax(&S.s_mm[buf][1], rr);
            }

            // (2) wait for the accumulator; the barrier also publishes (1)
            const bool bad = (h == 0 && !mbar_wait(&S.acc_full[tbuf], acc_phase, abort)) || *abort;
            if (epi_sync_or(bad)) break;
            tc_fence_after();
            if (g_next < n_items) prefetch(h_next ? grp_next.y : grp_next.x, cur);

            // (3) per-row limits: in iff u >= k_in, out iff u < k_out, where
            //     u = fl(2 acc - |b|^2); all FP32 with outward rounding
            const float nb2max = fmaxf(fmaxf(S.red[buf][0], S.red[buf][1]), fmaxf(S.red[buf][2], S.red[buf][3]));
            const float nrbmax = fmaxf(fmaxf(S.red[buf][4], S.red[buf][5]), fmaxf(S.red[buf][6], S.red[buf][7]));
            float E;
            if (P.rl) {
                // from the residual norms: K2 r_a r_b + K1 (r_a |b| + |a| r_b) + K0 |a||b| + A2 (..) + A3
                const float rlbmax = fmaxf(fmaxf(S.red[buf][8], S.red[buf][9]), fmaxf(S.red[buf][10], S.red[buf][11]));
                const float cross = __fadd_ru(__fmul_ru(rla, nrbmax), __fmul_ru(nra, rlbmax));
                E = __fmaf_ru(P.K2f, __fmul_ru(rla, rlbmax),
                              __fmaf_ru(P.K1f, cross,
                                        __fmaf_ru(P.K0f, __fmul_ru(nra, nrbmax),
                                                  __fmaf_ru(P.A2f, __fadd_ru(na2, nb2max), P.A3f))));
            } else {
                E = __fmaf_ru(P.A1f, __fmul_ru(nra, nrbmax), __fmaf_ru(P.A2f, __fadd_ru(na2, nb2max), P.A3f));
            }
            const float k_in = __fadd_ru(__fsub_ru(na2, P.eps2_lo), E);
            const float k_out = __fsub_rd(__fsub_rd(na2, P.eps2_hi), E);
            bool work = true;
            if (MODE == 2) {
                work = S.s_mm[buf][1] >= 0 && S.s_mm[buf][0] != S.s_mm[buf][1];
                if (!work && S.s_mm[buf][1] >= 0 && et == 0) atomicAdd(&A.stats[kStatSkipped], 1ull);
            }
            const bool core_r = MODE == 2 && S.core[buf][r];

            // (4) accumulator rows -> neighbour bits
            uint32_t inb[kChunks], band[kChunks];
#pragma unroll
            for (int c2 = 0; c2 < kChunks; ++c2) {
                const int c = half * kChunks + c2;
                float v[32];
                tmem_ld32(tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(tbuf * kAccCols + h * kT + c * 32), v);
                if (c2 == kChunks - 1 && last_sub) {
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&S.acc_empty[tbuf]);
                }
                uint32_t in_bits = 0u, keep_bits = 0u;
                const float4* nbn4 = reinterpret_cast<const float4*>(S.nbn[buf] + c * 32);
#pragma unroll
                for (int i4 = 0; i4 < 8; ++i4) {
                    const float4 nn = nbn4[i4];
                    const float n4[4] = {nn.x, nn.y, nn.z, nn.w};
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const int i = i4 * 4 + k;
                        const float u = fmaf(2.f, v[i], n4[k]);
                        if (u >= k_in) in_bits |= 1u << i;
                        if (u >= k_out) keep_bits |= 1u << i;
                    }
                }
                // candidate columns: valid (and core-core, upper triangle for unions)
                const int left = nb - c * 32;
                uint32_t cand = !valid_r ? 0u : (left >= 32 ? 0xffffffffu : (left > 0 ? (1u << left) - 1u : 0u));
                uint32_t cand_band = cand;
                if (MODE == 2) {
                    cand = (work && core_r) ? cand & S.colcore[buf][c] : 0u;
                    cand_band = cand;
                    if (diag) {                                       // band pairs once: j > r
                        const int lo = r + 1 - c * 32;
                        cand_band &= lo <= 0 ? 0xffffffffu : (lo >= 32 ? 0u : ~((1u << lo) - 1u));
                    }
                }
                inb[c2] = in_bits & cand;
                band[c2] = keep_bits & ~in_bits & cand_band;
                S.rowmask[c][r] = inb[c2];
                if (MODE == 2 && inb[c2]) atomicAdd(&S.edges[buf], __popc(inb[c2]));
                if (!diag) {
                    // 32 x 32 bit transpose across the warp: lane k gets column c*32+k
                    uint32_t x = inb[c2];
#pragma unroll
                    for (int sft = 16; sft >= 1; sft >>= 1) {
                        const uint32_t m = sft == 16 ? 0x0000FFFFu : sft == 8 ? 0x00FF00FFu : sft == 4 ? 0x0F0F0F0Fu
                                                                   : sft == 2 ? 0x33333333u : 0x55555555u;
                        const uint32_t y = __shfl_xor_sync(0xffffffffu, x, sft);
                        x = (lane & sft) ? (((y >> sft) & m) | (x & ~m)) : ((x & m) | ((y & m) << sft));
                    }
                    S.colmask[quad][c * 32 + lane] = x;
                }
            }

            // (5) band pairs: queued for the FP64 recheck (decided here if the queue is full);
            //     a one-each union pair needs none once any pair is certainly in
            bool any_in = false;
            uint32_t all_in = 0u;
#pragma unroll
            for (int c2 = 0; c2 < kChunks; ++c2) all_in |= inb[c2];
            if (one_each) any_in = epi_sync_or(all_in != 0u);
#pragma unroll
            for (int c2 = 0; c2 < kChunks && !any_in; ++c2) {
                uint32_t b = band[c2];
                while (b) {
                    const int i = __ffs(b) - 1;
                    b &= b - 1;
                    const int j = (half * kChunks + c2) * 32 + i;
                    const uint32_t fl = MODE == 1 ? ((diag ? 0u : kQBoth) | ((!diag || r < j) ? kQTie : 0u)) : 0u;
                    bool decided;
                    const bool in = push_band(P, (int)(sa + r), (int)(sb + j), fl, &decided);
                    if (decided && in) {
                        if (MODE == 1) {
                            int old = atomicAdd(&A.count[sa + r], 1);
                            if (A.cap > 0 && old < A.cap) A.nbr[(sa + r) * A.cap + old] = (int32_t)(sb + j);
                            if (!diag) {
                                old = atomicAdd(&A.count[sb + j], 1);
                                if (A.cap > 0 && old < A.cap) A.nbr[(sb + j) * A.cap + old] = (int32_t)(sa + r);
                            }
                        } else {
                            gunion(A.parent, A.row_pt, (int)(sa + r), (int)(sb + j));
                        }
                    }
                }
            }

            // (6) counts and lists, or unions
            if (MODE == 1) {
                // one thread per row (et < 128) and per column (128 <= et < 256) adds the
                // pair's neighbours to the count; lists are written only while a count may
                // still be below cap (the count read one pair ahead is a lower bound)
                int k = 0;
                uint32_t any_band = 0u;
#pragma unroll
                for (int c2 = 0; c2 < kChunks; ++c2) {
                    k += __popc(inb[c2]);
                    any_band |= band[c2];
                }
                const bool hit = epi_sync_or(k > 0 || any_band != 0u);
                if (et == 0 && hit && A.pair_hit) A.pair_hit[q] = 1;
                const bool is_row = et < kT, is_col = !diag && et >= kT && et < 2 * kT;
                if (is_row || is_col) {
                    const int x = is_row ? et : et - kT;
                    const int64_t row = (is_row ? sa : sb) + x;
                    const int64_t other = is_row ? sb : sa;
                    int tot = 0;
                    if (is_row) {
#pragma unroll
                        for (int w = 0; w < kT / 32; ++w) tot += __popc(S.rowmask[w][x]);
                    } else {
#pragma unroll
                        for (int w = 0; w < 4; ++w) tot += __popc(S.colmask[w][x]);
                    }
                    if (tot > 0) {
                        if (pre_count >= A.cap) {
                            atomicAdd(&A.count[row], tot);          // no list entry can be due
                        } else {
                            const int old = atomicAdd(&A.count[row], tot);
                            int pos = old;
                            for (int w = 0; w < kT / 32 && pos < A.cap; ++w) {
                                uint32_t bm = is_row ? S.rowmask[w][x] : S.colmask[w & 3][x];
                                if (!is_row && w >= 4) bm = 0u;
                                while (bm && pos < A.cap) {
                                    const int i = __ffs(bm) - 1;
                                    bm &= bm - 1;
                                    A.nbr[row * A.cap + pos++] = (int32_t)(other + w * 32 + i);
                                }
                            }
                        }
                    }
                }
                if (et == 0) screened += diag ? (int64_t)na * (na + 1) / 2 : (int64_t)na * nb;
            } else if (one_each) {
                // both sides are single components: join them through any neighbour pair
                if (work && all_in) {
                    int c2 = 0;
                    while (!inb[c2]) ++c2;
                    const int j = (half * kChunks + c2) * 32 + __ffs(inb[c2]) - 1;
                    gunion(A.parent, A.row_pt, (int)(sa + r), (int)(sb + j));
                }
            } else {
                // components of the pair's core-core neighbour graph: dense pairs by a
                // bitset breadth-first search on one warp (each row's and column's
                // mask is OR-ed once), sparse ones by shared-memory unions per pair.
                // Then each core row whose global root (read before) differs from its
                // component head's joins it globally.
                epi_sync();                                   // masks and edge count ready
                const bool dense = S.edges[buf] > 1024;
                if (work && dense && warp == 2) bfs_components(S, buf, diag, lane);
                if (work && !dense) {
#pragma unroll
                    for (int c2 = 0; c2 < kChunks; ++c2) {
                        uint32_t b = inb[c2];
                        while (b) {
                            const int i = __ffs(b) - 1;
                            b &= b - 1;
                            const int j = (half * kChunks + c2) * 32 + i;
                            lunion(S.par[buf], r, diag ? j : kT + j);
                        }
                    }
                }
                epi_sync();
                if (work && et < 2 * kT && S.core[buf][et]) {
                    const int x = et;
                    const int rx = dense ? S.par[buf][x] : lfind(S.par[buf], x);
                    if (rx != x && S.groot[buf][x] != S.groot[buf][rx])
                        gunion(A.parent, A.row_pt, S.groot[buf][x], S.groot[buf][rx]);
                }
            }
            ++it;
            if (last_sub) ++git;
            g = g_next;
            h = h_next;
            grp = grp_next;
        }
        if (MODE == 1 && et == 0 && screened) {
            atomicAdd(&A.stats[kStatScreened], (unsigned long long)screened);
            atomicAdd(&A.stats[kStatTcPairs], (unsigned long long)screened);
        }
    }

    // ---------------------------------------------------------- teardown
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (tid == 0 && S.abort) atomicExch(P.err, 1);
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * kAccCols));
}

// ------------------------------------------------ nearest pivot (layout)
// Point tiles (128 rows) against all pivots (up to 256) in one MMA of
// N = 256: rows and pivots centred on the pivots' mean c and rounded to BF16
// (one product), so |x - p|^2 = |x - c|^2 + |p - c|^2 - 2 acc with error
// ~2^-7 |x - c||p - c|. The nearest pivot only orders points for the tile
// layout (a near tie may go either way); no decision of the method depends
// on it.
constexpr int kPivN = 256;
constexpr int kAsgStages = 4;
constexpr int kAsgStageBytes = kBlk + kPivN * kKB * 2;               // x, pivots

struct AssignParams {
    int64_t n, n_tiles;
    int nkb;
    const float* xn2;                         // |x - c|^2 per point
    const float* pn2;                         // |p - c|^2 per pivot, +inf past the last
    int32_t* piv;
    float* pd2;
    int* err;
};

struct AsgTail {
    uint64_t full[kAsgStages], empty[kAsgStages], acc_full[2], acc_empty[2], fin;
    uint32_t tmem_base;
    int abort;
    float pn2[kPivN];
};

// kind::f16, BF16 in, F32 out, K-major, M = 128, N = 256
constexpr uint32_t kIdescN256 = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kPivN >> 3) << 17) |
                                ((uint32_t)(kT >> 4) << 24);

__device__ __forceinline__ void mma_bf16_n256(uint32_t tmem, uint64_t adesc, uint64_t bdesc, uint32_t acc)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(
            tmem),
        "l"(adesc), "l"(bdesc), "r"(kIdescN256), "r"(acc));
}

__global__ void __launch_bounds__(192, 1) assign_tc_kernel(const __grid_constant__ CUtensorMap mXh,
                                                           const __grid_constant__ CUtensorMap mPh,
                                                           const AssignParams P)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    AsgTail& S = *reinterpret_cast<AsgTail*>(smem + kAsgStages * kAsgStageBytes);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    volatile int* abort = &S.abort;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&S.tmem_base)),
                     "r"(2 * kPivN));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 32) {
        for (int i = 0; i < kAsgStages; ++i) {
            mbar_init(&S.full[i], 1);
            mbar_init(&S.empty[i], 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(&S.acc_full[i], 1);
            mbar_init(&S.acc_empty[i], 4);
        }
        mbar_init(&S.fin, 1);
        S.abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    for (int j = tid; j < kPivN; j += blockDim.x) S.pn2[j] = P.pn2[j];
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = S.tmem_base;

    if (warp == 0) {
        if (lane == 0) {
            int stage = 0;
            uint32_t phase = 0;
            for (int64_t t = blockIdx.x; t < P.n_tiles && !*abort; t += gridDim.x) {
                for (int kb = 0; kb < P.nkb; ++kb) {
                    if (!mbar_wait(&S.empty[stage], phase ^ 1, abort)) break;
                    unsigned char* st = smem + stage * kAsgStageBytes;
                    mbar_expect_tx(&S.full[stage], (uint32_t)kAsgStageBytes);
                    tma_load(st, &mXh, kb * kKB, (int)(t * kT), &S.full[stage]);
                    tma_load(st + kBlk, &mPh, kb * kKB, 0, &S.full[stage]);
                    if (++stage == kAsgStages) { stage = 0; phase ^= 1; }
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            int stage = 0;
            uint32_t phase = 0;
            int it = 0;
            for (int64_t t = blockIdx.x; t < P.n_tiles && !*abort; t += gridDim.x, ++it) {
                const int buf = it & 1;
                if (!mbar_wait(&S.acc_empty[buf], (uint32_t)(((it >> 1) & 1) ^ 1), abort)) break;
                tc_fence_after();
                const uint32_t d_tmem = tmem + (uint32_t)(buf * kPivN);
                bool ok = true;
                for (int kb = 0; kb < P.nkb; ++kb) {
                    if (!mbar_wait(&S.full[stage], phase, abort)) { ok = false; break; }
                    tc_fence_after();
                    const uint32_t base = su32(smem + stage * kAsgStageBytes);
                    const uint32_t xh = base, ph = base + kBlk;
#pragma unroll
                    for (int j = 0; j < kKB / 16; ++j)
                        mma_bf16_n256(d_tmem, smem_desc(xh + 32 * j), smem_desc(ph + 32 * j), (kb | j) ? 1u : 0u);
                    mma_commit(&S.empty[stage]);
                    if (++stage == kAsgStages) { stage = 0; phase ^= 1; }
                }
                if (!ok) break;
                mma_commit(&S.acc_full[buf]);
            }
            mma_commit(&S.fin);
            volatile int dummy = 0;
            mbar_wait(&S.fin, 0, &dummy);
        }
    } else {
        const int quad = warp & 3;
        const int r = quad * 32 + lane;
        int it = 0;
        for (int64_t t = blockIdx.x; t < P.n_tiles; t += gridDim.x, ++it) {
            const int buf = it & 1;
            const bool bad = !mbar_wait(&S.acc_full[buf], (uint32_t)((it >> 1) & 1), abort) || *abort;
            if (__any_sync(0xffffffffu, bad)) break;
            tc_fence_after();
            float best = INFINITY;
            int bidx = 0;
#pragma unroll 1
            for (int c = 0; c < kPivN / 32; ++c) {
                float v[32];
                tmem_ld32(tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(buf * kPivN + c * 32), v);
                if (c == kPivN / 32 - 1) {
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&S.acc_empty[buf]);
                }
#pragma unroll
                for (int i = 0; i < 32; ++i) {
                    const float val = fmaf(-2.f, v[i], S.pn2[c * 32 + i]);
                    if (val < best) { best = val; bidx = c * 32 + i; }
                }
            }
            const int64_t p = t * kT + r;
            if (p < P.n) {
                P.piv[p] = bidx;
                P.pd2[p] = fmaxf(0.f, P.xn2[p] + best);
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (tid == 0 && S.abort) atomicExch(P.err, 1);
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * kPivN));
}

// Rows of `src` (n rows, stride ld, d values) minus c, rounded to BF16
// (rows_out rows of pitch dp, zero padded) with |row - c|^2 in FP32. A lane
// converts 8 consecutive columns (one 16-byte store).
__global__ void split_rows_kernel(const float* __restrict__ src, int64_t n, int d, int64_t ld, int dp,
                                  const float* __restrict__ c, int64_t rows_out, __nv_bfloat16* __restrict__ hi,
                                  float* __restrict__ n2, float pad_n2, bool vec)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarp = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t r = warp; r < rows_out; r += nwarp) {
        float s = 0.f;
        for (int k0 = 0; k0 < dp; k0 += 256) {
            const int k = k0 + lane * 8;
            if (k >= dp) continue;
            float a[8];
            const float* x = src + r * ld + k;
            if (r < n && vec && k + 7 < d) {
                const float4 x0 = *reinterpret_cast<const float4*>(x);
                const float4 x1 = *reinterpret_cast<const float4*>(x + 4);
                a[0] = x0.x; a[1] = x0.y; a[2] = x0.z; a[3] = x0.w;
                a[4] = x1.x; a[5] = x1.y; a[6] = x1.z; a[7] = x1.w;
            } else {
#pragma unroll
                for (int t = 0; t < 8; ++t) a[t] = (r < n && k + t < d) ? x[t] : 0.f;
            }
            uint32_t w[4];
#pragma unroll
            for (int t = 0; t < 8; t += 2) {
                const float a0 = (r < n && k + t < d) ? a[t] - c[k + t] : 0.f;
                const float a1 = (r < n && k + t + 1 < d) ? a[t + 1] - c[k + t + 1] : 0.f;
                const __nv_bfloat162 h = __floats2bfloat162_rn(a0, a1);
                w[t >> 1] = *reinterpret_cast<const uint32_t*>(&h);
                s = fmaf(a0, a0, s);
                s = fmaf(a1, a1, s);
            }
            *reinterpret_cast<uint4*>(hi + r * dp + k) = make_uint4(w[0], w[1], w[2], w[3]);
        }
        for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0 && n2) n2[r] = r < n ? s : pad_n2;
    }
}

__global__ void mean_rows_kernel(const float* __restrict__ rows, int K, int dp, float* __restrict__ c)
{
    for (int k = threadIdx.x; k < dp; k += blockDim.x) {
        float s = 0.f;
        for (int i = 0; i < K; ++i) s += rows[(int64_t)i * dp + k];
        c[k] = s / (float)K;
    }
}

// Band pairs queued by the epilogues, 8 lanes per pair (4 pairs per warp in
// flight), decided in three steps that each keep the FP64 decision:
//   1. FP32: each lane sums dp/8 squared differences with FMA, then a
//      3-level shuffle tree: |s - d^2| <= (2 + dp/8 + 3) 2^-24 d^2 (+ tiny),
//      certified in/out outside that band (thresholds lo32, hi32);
//   2. FP64, same split: |s - d^2| <= (dp/8 + 5) 2^-53 d^2, so outside
//      4e-12 eps^2 of eps^2 it decides like the defining expression;
//   3. else the defining expression itself (k ascending, one rounding per
//      operation) on the group's first lane, which also counts near ties.
template <int MODE>
__global__ void __launch_bounds__(256) recheck_kernel(const PassArgs A, const uint2* __restrict__ queue,
                                                      const unsigned long long* __restrict__ queue_n,
                                                      unsigned long long cap, float lo32, float hi32)
{
    const long long n = (long long)min(*queue_n, cap);
    const int lane = threadIdx.x & 31, sub = lane & 7;
    const long long group = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 3;
    const long long ngroup = ((long long)gridDim.x * blockDim.x) >> 3;
    const long long rounds = (n + ngroup - 1) / ngroup;         // same trip count for the whole warp
    for (long long rd = 0; rd < rounds; ++rd) {
        const long long i = group + rd * ngroup;
        const bool live = i < n;
        uint2 e = make_uint2(0u, 0u);
        if (live) e = queue[i];
        int ra = (int)e.x, rb = (int)(e.y & 0x3FFFFFFFu);
        const uint32_t fl = e.y >> 30;
        if (live && (!MGB_IN_RANGE(ra, A.n_rows, A.stats + kStatOob) || !MGB_IN_RANGE(rb, A.n_rows, A.stats + kStatOob)))
            ra = rb = 0;                                  // checked build: counted (results flagged)
        const float* xa = live ? pass_row(A, ra) : nullptr;
        const float* xb = live ? pass_row(A, rb) : nullptr;
        float s32 = 0.f;
        if (live) {
#pragma unroll 4
            for (int k = sub; k < A.dp / 4; k += 8) {
                const float4 p = pass_ld4(A, xa, k), q = pass_ld4(A, xb, k);
                float t = p.x - q.x;
                s32 = fmaf(t, t, s32);
                t = p.y - q.y;
                s32 = fmaf(t, t, s32);
                t = p.z - q.z;
                s32 = fmaf(t, t, s32);
                t = p.w - q.w;
                s32 = fmaf(t, t, s32);
            }
        }
        s32 += __shfl_xor_sync(0xffffffffu, s32, 1);
        s32 += __shfl_xor_sync(0xffffffffu, s32, 2);
        s32 += __shfl_xor_sync(0xffffffffu, s32, 4);
        int state = !live ? 3 : (s32 <= lo32 ? 1 : (s32 > hi32 ? 0 : 2));   // 2: undecided
        if (__any_sync(0xffffffffu, state == 2)) {
            double s64 = 0.0;
            if (state == 2) {
                for (int k = sub; k < A.dp / 4; k += 8) {
                    const float4 p = pass_ld4(A, xa, k), q = pass_ld4(A, xb, k);
                    double t = (double)p.x - (double)q.x;
                    s64 = fma(t, t, s64);
                    t = (double)p.y - (double)q.y;
                    s64 = fma(t, t, s64);
                    t = (double)p.z - (double)q.z;
                    s64 = fma(t, t, s64);
                    t = (double)p.w - (double)q.w;
                    s64 = fma(t, t, s64);
                }
            }
            s64 += __shfl_xor_sync(0xffffffffu, s64, 1);
            s64 += __shfl_xor_sync(0xffffffffu, s64, 2);
            s64 += __shfl_xor_sync(0xffffffffu, s64, 4);
            if (state == 2) {
                if (fabs(s64 - A.eps2) > 4e-12 * A.eps2) state = s64 <= A.eps2 ? 1 : 0;
                else state = 4;                                        // the defining expression decides
            }
        }
        if (live && sub == 0) {
            bool in = state == 1;
            if (state == 4) {
                const double d2 = exact_sqdist(xa, xb, A.d);
                if (MODE == 1 && (fl & kQTie) && fabs(d2 - A.eps2) <= A.tie_thr)
                    atomicAdd(&A.stats[kStatTies], 1ull);
                atomicAdd(&A.stats[kStatFp64], 1ull);
                in = d2 <= A.eps2;
            }
            if (in) {
                if (MODE == 1) {
                    int old = atomicAdd(&A.count[ra], 1);
                    if (A.cap > 0 && old < A.cap) A.nbr[(int64_t)ra * A.cap + old] = rb;
                    if (fl & kQBoth) {
                        old = atomicAdd(&A.count[rb], 1);
                        if (A.cap > 0 && old < A.cap) A.nbr[(int64_t)rb * A.cap + old] = ra;
                    }
                } else {
                    gunion(A.parent, A.row_pt, ra, rb);
                }
            }
        }
        __syncwarp();
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(&A.stats[kStatBand], (unsigned long long)n);
}

// --------------------------------------------------------------- host side
PFN_cuTensorMapEncodeTiled_v12000 encoder()
{
    static std::once_flag once;
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    std::call_once(once, [] {
        cudaDriverEntryPointQueryResult q;
        void* p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

bool make_map(CUtensorMap* m, const void* ptr, int64_t rows, int dp, int box_rows = kT)
{
    auto enc = encoder();
    if (!enc) return false;
    cuuint64_t dims[2] = {(cuuint64_t)dp, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)dp * 2};
    cuuint32_t box[2] = {kKB, (cuuint32_t)box_rows};
    cuuint32_t es[2] = {1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(ptr), dims, strides, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int NS, int W>
constexpr int smem_bytes()
{
    return TcShape<NS, W>::kStages * TcShape<NS, W>::kStageBytes + (int)sizeof(SmemTail) + 1024;
}
static_assert(smem_bytes<3, 1>() <= 232448 && smem_bytes<1, 1>() <= 232448, "shared memory");
static_assert(smem_bytes<3, 2>() <= 232448 && smem_bytes<1, 2>() <= 232448, "shared memory");

template <int NS, int MODE, int W, int F = 0>
cudaError_t launch(const CUtensorMap& mh, const CUtensorMap& ml, const TcParams& p, int grid, cudaStream_t s)
{
    const int smem = smem_bytes<NS, W>();
    cudaError_t e =
        cudaFuncSetAttribute(tc_kernel<NS, MODE, W, F>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    tc_kernel<NS, MODE, W, F><<<grid, kThreads, smem, s>>>(mh, ml, p);
    return cudaGetLastError();
}

// Groups of the pass-1 pair list (sorted by tile A, then B): each pair at an
// even position within its run of equal A leads a group, with the next pair
// of the run if there is one.
__global__ void group_lead_kernel(const int2* __restrict__ pairs, int64_t n, int32_t* __restrict__ lead)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int a = pairs[i].x;
    int64_t lo = 0, hi = i;                               // first index of the run
    while (lo < hi) {
        const int64_t m = (lo + hi) >> 1;
        if (pairs[m].x < a) lo = m + 1; else hi = m;
    }
    lead[i] = ((i - lo) & 1) == 0;
}

__global__ void group_emit_kernel(const int2* __restrict__ pairs, int64_t n, const int32_t* __restrict__ lead,
                                  const int64_t* __restrict__ pos, int2* __restrict__ groups)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || !lead[i]) return;
    const bool two = i + 1 < n && pairs[i + 1].x == pairs[i].x;
    groups[pos[i]] = make_int2((int)i, two ? (int)(i + 1) : -1);
}

// The same grouping over the first *n_dev entries of a list of capacity n.
__global__ void group_lead_dev_kernel(const int2* __restrict__ pairs, int64_t n,
                                      const unsigned long long* __restrict__ n_dev, int32_t* __restrict__ lead)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if ((unsigned long long)i >= *n_dev) {
        lead[i] = 0;
        return;
    }
    const int a = pairs[i].x;
    int64_t lo = 0, hi = i;
    while (lo < hi) {
        const int64_t m = (lo + hi) >> 1;
        if (pairs[m].x < a) lo = m + 1; else hi = m;
    }
    lead[i] = ((i - lo) & 1) == 0;
}

__global__ void group_emit_dev_kernel(const int2* __restrict__ pairs, int64_t n,
                                      const unsigned long long* __restrict__ n_dev, const int32_t* __restrict__ lead,
                                      const int64_t* __restrict__ pos, int2* __restrict__ groups)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || !lead[i]) return;
    const bool two = (unsigned long long)(i + 1) < *n_dev && pairs[i + 1].x == pairs[i].x;
    groups[pos[i]] = make_int2((int)i, two ? (int)(i + 1) : -1);
}

// flag[q] = 1 if the first phase deferred a sub-block of pair q
__global__ void redo_flag_kernel(const uint32_t* __restrict__ mask, int64_t n, int32_t* __restrict__ flag,
                                 unsigned long long* __restrict__ stats)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t m = i < n ? mask[i] : 0u;
    if (i < n) flag[i] = m != 0u;
    if (stats) {
        // bit quad * 4 + part: blocks, and parts holding one
        const int blocks = __reduce_add_sync(0xffffffffu, __popc(m));
        const int parts = __reduce_add_sync(0xffffffffu, __popc((m | m >> 4 | m >> 8 | m >> 12) & 0xFu));
        if ((threadIdx.x & 31) == 0 && blocks) {
            atomicAdd(stats, (unsigned long long)blocks);
            atomicAdd(stats + 1, (unsigned long long)parts);
        }
    }
}

// every stride-th pair of a list: out[j] = pairs[j * stride], j < n
__global__ void sample_pairs_kernel(const int2* __restrict__ pairs, int64_t stride, int64_t n, int2* __restrict__ out)
{
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j < n) out[j] = pairs[j * stride];
}

// the deferred pairs in list order: redo[pos[q]] = pairs[q], redo_q[pos[q]] = q
__global__ void redo_scatter_kernel(const int2* __restrict__ pairs, const int32_t* __restrict__ flag,
                                    const int64_t* __restrict__ pos, int64_t n, int2* __restrict__ redo,
                                    int32_t* __restrict__ redo_q)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || !flag[i]) return;
    redo[pos[i]] = pairs[i];
    redo_q[pos[i]] = (int32_t)i;
}

}  // namespace

int tc_sample_pairs(const int2* pairs, int64_t stride, int64_t n, int2* out, cudaStream_t s)
{
    if (n == 0) return MAPPER_OK;
    sample_pairs_kernel<<<(unsigned)div_up(n, 256), 256, 0, s>>>(pairs, stride, n, out);
    note_launch();
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error(std::string("tc_sample_pairs: ") + cudaGetErrorString(e));
        return MAPPER_ECUDA;
    }
    return MAPPER_OK;
}

int tc_redo_list(const int2* pairs, const uint32_t* mask, int64_t n, int2* redo, int32_t* redo_q, Buf* pos,
                 cudaStream_t s, unsigned long long* stats)
{
    if (n == 0) return MAPPER_OK;
    Buf flag;
    cudaError_t e = flag.alloc(sizeof(int32_t) * n, s);
    if (e == cudaSuccess) e = pos->alloc(sizeof(int64_t) * (n + 1), s);
    if (e == cudaSuccess) {
        redo_flag_kernel<<<(unsigned)div_up(n, 256), 256, 0, s>>>(mask, n, flag.as<int32_t>(), stats);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = exclusive_scan_i32_to_i64(flag.as<int32_t>(), pos->as<int64_t>(), n, s);
    if (e == cudaSuccess) {
        redo_scatter_kernel<<<(unsigned)div_up(n, 256), 256, 0, s>>>(pairs, flag.as<int32_t>(), pos->as<int64_t>(), n,
                                                                      redo, redo_q);
        e = cudaGetLastError();
    }
    note_launch(2);
    if (e != cudaSuccess) {
        set_error(std::string("tc_redo_list: ") + cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? MAPPER_ENOMEM : MAPPER_ECUDA;
    }
    return MAPPER_OK;
}

int tc_groups_dev(const int2* pairs, int64_t n, const unsigned long long* n_dev, Buf* groups, Buf* pos,
                  cudaStream_t s)
{
    if (n == 0) return MAPPER_OK;
    Buf lead;
    cudaError_t e = lead.alloc(sizeof(int32_t) * n, s);
    if (e == cudaSuccess) e = pos->alloc(sizeof(int64_t) * (n + 1), s);
    if (e == cudaSuccess) e = groups->alloc(sizeof(int2) * (size_t)n, s);
    const unsigned blocks = (unsigned)div_up(n, 256);
    if (e == cudaSuccess) {
        group_lead_dev_kernel<<<blocks, 256, 0, s>>>(pairs, n, n_dev, lead.as<int32_t>());
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = exclusive_scan_i32_to_i64(lead.as<int32_t>(), pos->as<int64_t>(), n, s);
    if (e == cudaSuccess) {
        group_emit_dev_kernel<<<blocks, 256, 0, s>>>(pairs, n, n_dev, lead.as<int32_t>(), pos->as<int64_t>(),
                                                     groups->as<int2>());
        e = cudaGetLastError();
    }
    note_launch(2);
    if (e != cudaSuccess) {
        set_error(std::string("tc_groups_dev: ") + cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? MAPPER_ENOMEM : MAPPER_ECUDA;
    }
    return MAPPER_OK;
}

int assign_pivots_tc(const float* X, int64_t n, int d, int64_t ld, int dp, const float* Pv, int K,
                     int num_sms, int32_t* piv, float* pd2, cudaStream_t s, const PivotSplit* pre)
{
    if (K > kPivN) { set_error("assign_pivots_tc: more than 256 pivots"); return MAPPER_EINVAL; }
    const int64_t n_tiles = (n + kT - 1) / kT, rows = n_tiles * kT;
    Buf c, xh, xn2, ph, pn2, err;
#define AK(expr)                                                                         \
    do {                                                                                 \
        cudaError_t e_ = (expr);                                                         \
        if (e_ != cudaSuccess) {                                                         \
            set_error(std::string("assign_pivots_tc: ") + cudaGetErrorString(e_));       \
            return e_ == cudaErrorMemoryAllocation ? MAPPER_ENOMEM : MAPPER_ECUDA;       \
        }                                                                                \
    } while (0)
    AK(ph.alloc(sizeof(__nv_bfloat16) * (size_t)kPivN * dp, s));
    AK(pn2.alloc(sizeof(float) * kPivN, s));
    AK(err.alloc(sizeof(int), s));
    AK(cudaMemsetAsync(err.p, 0, sizeof(int), s));
    const float* cc = pre ? pre->c : nullptr;
    const void* xhp = pre ? pre->xh : nullptr;
    const float* xn2p = pre ? pre->xn2 : nullptr;
    if (!pre) {
        AK(c.alloc(sizeof(float) * dp, s));
        AK(xh.alloc(sizeof(__nv_bfloat16) * (size_t)rows * dp, s));
        AK(xn2.alloc(sizeof(float) * rows, s));
        mean_rows_kernel<<<1, 256, 0, s>>>(Pv, K, dp, c.as<float>());
        const bool vec = ld % 4 == 0 && ((uintptr_t)X & 15) == 0;
        split_rows_kernel<<<num_sms * 8, 256, 0, s>>>(X, n, d, ld, dp, c.as<float>(), rows,
                                                      xh.as<__nv_bfloat16>(), xn2.as<float>(), 0.f, vec);
        note_launch(2);
        cc = c.as<float>();
        xhp = xh.p;
        xn2p = xn2.as<float>();
    }
    split_rows_kernel<<<8, 256, 0, s>>>(Pv, K, d, dp, dp, cc, kPivN, ph.as<__nv_bfloat16>(), pn2.as<float>(),
                                        INFINITY, true);
    note_launch();
    AK(cudaGetLastError());
    CUtensorMap mxh, mph;
    if (!make_map(&mxh, xhp, rows, dp) || !make_map(&mph, ph.p, kPivN, dp, kPivN)) {
        set_error("cuTensorMapEncodeTiled failed (or is unavailable)");
        return MAPPER_ECUDA;
    }
    AssignParams p{};
    p.n = n;
    p.n_tiles = n_tiles;
    p.nkb = (dp + kKB - 1) / kKB;
    p.xn2 = xn2p;
    p.pn2 = pn2.as<float>();
    p.piv = piv;
    p.pd2 = pd2;
    p.err = err.as<int>();
    const int smem = kAsgStages * kAsgStageBytes + (int)sizeof(AsgTail) + 1024;
    AK(cudaFuncSetAttribute(assign_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    assign_tc_kernel<<<(int)std::min<int64_t>(n_tiles, num_sms), 192, smem, s>>>(mxh, mph, p);
    note_launch();
    AK(cudaGetLastError());
    int h_err = 0;
    AK(cudaMemcpyAsync(&h_err, err.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    AK(cudaStreamSynchronize(s));
#undef AK
    if (h_err) { set_error("pivot assignment gave up waiting on a barrier"); return MAPPER_ETIMEOUT; }
    return MAPPER_OK;
}

// Error bound of the screen value against d^2 = |a|^2 + |b|^2 - 2 a.b, where
// a = x - c and b = y - c exactly (c: the segment's FP32 centre), with
// u = 2^-8 (BF16) and v = 2^-24 (FP32):
//   operand rounding  a32 = fl(x - c), hi = bf16(a32), lo = bf16(a32 - hi):
//                     |a - hi| <= u'|a|, |a - hi - lo| <= rho |a| with
//                     u' = u + 2v, rho = u^2 + 2v;
//                     NS = 1: |hi.hi - a.b| <= (2u' + u'^2) S
//                     NS = 3: dropping lo.lo and the residuals costs
//                             <= (u'^2 + 2 rho + rho^2) S,  S = sum |a_k||b_k|
//   accumulation      m MMA steps of 16 exact products each into the FP32
//                     accumulator: <= (m + 8) 2^-22 (1 + 2u')^2 S (two units
//                     per step, allowing truncation, and a floor of 8 units;
//                     accu_model); S <= |a||b|
//   screen            u = fl(2 acc - |b|^2): <= v (2|acc| + |b|^2)
//   norms             FP32 sums of d squares (lane partials and a shuffle
//                     tree): <= (dp/32 + 16) v per norm, relative
// A1 = 1.25 (2 (operand + accumulation) + 4v); A2 = 2 (dp/32 + 16) v + 4v;
// A3 covers subnormal terms. |a| and |b| enter through upper bounds.
// Accumulation term of the bound, relative to the sum of the products'
// magnitudes: 2^-22 per MMA step (16 products of K each) plus a floor of 8
// such units (the hardware's error does not shrink with the step count: at
// one K block it is already ~2^-22, measured by mapper_selftest_mma_error),
// times (1 + 2u')^2 for the magnitudes of the BF16 parts.
double accu_model(int ns, int dp)
{
    const double up = std::ldexp(1.0, -8) + 2.0 * std::ldexp(1.0, -24);
    const int steps = ns * ((dp + kKB - 1) / kKB) * (kKB / 16);
    return (steps + 8) * std::ldexp(1.0, -22) * (1.0 + 2.0 * up) * (1.0 + 2.0 * up);
}

double accu_model_f8(int ns, int dp)
{
    const int steps = ns * ((dp + 127) / 128) * 4;
    return (steps + 8) * std::ldexp(1.0, -22) * 1.3;
}

void tc_bound(int ns, int dp, double eps2, double* A1, double* A2, double* A3)
{
    const double u = std::ldexp(1.0, -8), v = std::ldexp(1.0, -24);
    const double up = u + 2.0 * v, rho = u * u + 2.0 * v;
    const double oper = ns == 1 ? (2.0 * up + up * up) : (up * up + 2.0 * rho + rho * rho);
    const double accu = accu_model(ns, dp);
    *A1 = 1.25 * (2.0 * (oper + accu) + 4.0 * v);
    *A2 = 2.0 * (dp / 32 + 16) * v + 4.0 * v;
    *A3 = std::ldexp(1.0, -40) * eps2 + 1e-30;
}

// The same bound from the residual norms r = |a' - hi| of both rows (a' =
// fl(x - c), hi = bf16(a'), both per row, rounded up), which are typically
// ~0.4 u |a| rather than the worst case u |a|. With e = a - a' (|e| <=
// 2^-24 |a|), t = r - lo (|t| <= u |r|) and |r| <= u (1 + 2^-23) |a|:
//   NS = 1: a.b - hi_a.hi_b = (e_a + r_a).b + hi_a.(e_b + r_b), so
//           |.| <= (1 + 2^-7)(|r_a||b| + |a||r_b|) + 3 2^-24 |a||b|;
//   NS = 3: a.b - P = lo_a.lo_b + (hi_a + lo_a).(t_b + e_b) + (t_a + e_a).b, so
//           |.| <= (1 + 2^-6)|r_a||r_b| + u (1 + 2^-6)(|a||r_b| + |r_a||b|) + 2^-22 |a||b|.
// E = K2 |r_a||r_b| + K1 (|r_a||b| + |a||r_b|) + K0 |a||b| + A2 (|a|^2 + |b|^2) + A3,
// with the accumulation, screen and norm terms and the 1.25 margin of tc_bound.
void tc_bound_resid(int ns, int dp, double eps2, double* K0, double* K1, double* K2, double* A2, double* A3)
{
    const double u = std::ldexp(1.0, -8), v = std::ldexp(1.0, -24);
    const double accu = accu_model(ns, dp);
    double o2, o1, o0;
    if (ns == 1) {
        o2 = 0.0;
        o1 = 1.0 + std::ldexp(1.0, -7);
        o0 = 3.0 * v;
    } else {
        o2 = 1.0 + std::ldexp(1.0, -6);
        o1 = u * (1.0 + std::ldexp(1.0, -6));
        o0 = std::ldexp(1.0, -22);
    }
    *K2 = 1.25 * 2.0 * o2;
    *K1 = 1.25 * 2.0 * o1;
    *K0 = 1.25 * (2.0 * (o0 + accu) + 4.0 * v);
    *A2 = 2.0 * (dp / 32 + 16) * v + 4.0 * v;
    *A3 = std::ldexp(1.0, -40) * eps2 + 1e-30;
}

// FP8 E4M3 screen (three products of per-tile scaled rows: a / s_a = hi + lo
// + t, hi = e4m3(a / s_a), r = a / s_a - hi, lo = e4m3(r)). E4M3 rounds to
// 2^-4 relative above 2^-6 and to 2^-10 absolute below, so per row |t| <=
// 2^-4 |r| + f with f = 2^-10 sqrt(dp). With R = |r| and N = |a / s| (scaled
// norms) the algebra of tc_bound_resid gives
//   |a.b / (s_a s_b) - P| <= 1.14 R_a R_b + 2^-4 1.001 (N_a R_b + R_a N_b)
//                            + 1.2 f (N_a + N_b) + 6 f^2 + 2^-22 N_a N_b,
// which times s_a s_b is, in the rows' own units (frl = s R, rn = s N),
//   K2 frl_a frl_b + K1 (rn_a frl_b + frl_a rn_b) + K4 (s_b rn_a + s_a rn_b) + K5 s_a s_b + K0 rn_a rn_b
// with the 2 x 1.25 factor, the accumulation (dp / 128 * 4 instructions of
// K = 32 per product) and the screen and norm terms as for BF16.

void tc_bound_f8(int dp, double eps2, double* K0, double* K1, double* K2, double* K4, double* K5, double* A2,
                 double* A3)
{
    const double v = std::ldexp(1.0, -24);
    const double f = std::ldexp(1.0, -10) * std::sqrt((double)dp);
    *K2 = 2.5 * 1.14;
    *K1 = 2.5 * std::ldexp(1.0, -4) * 1.001;
    *K4 = 2.5 * 1.2 * f;
    *K5 = 2.5 * 6.0 * f * f;
    *K0 = 1.25 * (2.0 * (std::ldexp(1.0, -22) + accu_model_f8(3, dp)) + 4.0 * v);
    *A2 = 2.0 * (dp / 32 + 16) * v + 4.0 * v;
    *A3 = std::ldexp(1.0, -40) * eps2 + 1e-30;
}

int tc_pass(int mode, const PassArgs& a, const TcArgs& t, int64_t n_pairs, cudaStream_t s)
{
    if (n_pairs == 0) return MAPPER_OK;
    if (t.R >= (int64_t(1) << 30)) {
        set_error("tensor-core screen: more than 2^30 rows");
        return MAPPER_ENOMEM;
    }
    if (t.f8 && (mode != 1 || t.ns != 3 || !t.rl || !t.tmax)) {
        set_error("tensor-core pass: the FP8 screen is a three-product count pass");
        return MAPPER_EINTERNAL;
    }
    if (mode == 5) {
        bool ok = t.n_radii >= 1 && t.n_radii <= kMaxRadii && !t.f8;
        for (int e = 0; ok && e < t.n_radii; ++e) {
            const RadiusOut& o = t.radii[e];
            ok = o.count && o.queue && o.queue_n && o.stats && (a.cap == 0 || o.nbr) && o.eps2 > 0.0 &&
                 std::isfinite(o.eps2) && (e == 0 || o.eps2 >= t.radii[e - 1].eps2);
        }
        if (!ok) {
            set_error("tensor-core pass: bad radii for the count pass over several radii");
            return MAPPER_EINTERNAL;
        }
    }
    // the error bound grows with eps^2 (its A3 term): the largest radius's
    // bound holds for every radius of a mode-5 pass
    const double eps2_b = mode == 5 ? t.radii[t.n_radii - 1].eps2 : a.eps2;
    // FP8 rows of dp bytes are moved as rows of dp / 2 BF16 columns (the same
    // bytes, the same 128-byte swizzled K blocks, each holding 128 FP8 columns)
    const int dcols = t.f8 ? a.dp / 2 : a.dp;
    CUtensorMap mh, ml;
    if (!make_map(&mh, t.Ah, t.R, dcols) || !make_map(&ml, t.ns == 3 ? t.Al : t.Ah, t.R, dcols)) {
        set_error("cuTensorMapEncodeTiled failed (or is unavailable)");
        return MAPPER_ECUDA;
    }
    TcParams p{};
    p.A = a;
    p.rn2 = t.rn2;
    p.rn = t.rn;
    p.n_pairs = n_pairs;
    p.nkb = (dcols + kKB - 1) / kKB;
    tc_bound(t.ns, a.dp, eps2_b, &p.A1, &p.A2, &p.A3);
    p.A1f = std::nextafter((float)p.A1, INFINITY);
    p.A2f = std::nextafter((float)p.A2, INFINITY);
    p.A3f = std::nextafter((float)p.A3, INFINITY);
    p.rl = t.rl;
    if (t.f8) {
        double K0, K1, K2, K4, K5, A2, A3;
        tc_bound_f8(a.dp, a.eps2, &K0, &K1, &K2, &K4, &K5, &A2, &A3);
        p.K0f = std::nextafter((float)K0, INFINITY);
        p.K1f = std::nextafter((float)K1, INFINITY);
        p.K2f = std::nextafter((float)K2, INFINITY);
        p.K4f = std::nextafter((float)K4, INFINITY);
        p.K5f = std::nextafter((float)K5, INFINITY);
    } else if (t.rl) {
        double K0, K1, K2, A2, A3;
        tc_bound_resid(t.ns, a.dp, eps2_b, &K0, &K1, &K2, &A2, &A3);
        p.K0f = std::nextafter((float)K0, INFINITY);
        p.K1f = std::nextafter((float)K1, INFINITY);
        p.K2f = std::nextafter((float)K2, INFINITY);
    }
    auto f32_lo = [](double x) {
        float f = (float)x;
        return (double)f > x ? std::nextafter(f, -INFINITY) : f;
    };
    auto f32_hi = [](double x) {
        float f = (float)x;
        return (double)f < x ? std::nextafter(f, INFINITY) : f;
    };
    p.eps2_lo = f32_lo(a.eps2);
    p.eps2_hi = f32_hi(a.eps2);
    if (mode == 5) {
        p.n_rad = t.n_radii;
        for (int e = 0; e < t.n_radii; ++e) {
            const RadiusOut& o = t.radii[e];
            p.rad[e] = {o.count, o.nbr, o.pair_hit, o.queue, o.queue_n, o.stats, o.eps2, 1e-12 * o.eps2,
                        f32_lo(o.eps2), f32_hi(o.eps2)};
        }
    }
    p.queue = t.queue;
    p.queue_n = t.queue_n;
    p.queue_cap = t.queue_cap;
    p.err = t.err;
    const bool count_pass = mode == 1 || mode == 5;
    const bool defer = count_pass && t.defer && (t.ns == 1 || t.f8);
    p.defer = defer ? (t.defer_mixed ? 2 : 1) : 0;
    p.redo_mask = t.redo_mask;
    p.sub_mask = t.sub_mask;
    p.sub_q = t.sub_q;
    p.tmax = t.tmax;
    p.tn2min = t.tn2min;
    if ((t.defer && !defer) || (count_pass && (!t.tmax || !t.tn2min)) || (t.sub_mask && !t.sub_q) || (defer && !t.redo_mask)) {
        set_error("tensor-core pass: inconsistent arguments");
        return MAPPER_EINTERNAL;
    }
    cudaError_t e = cudaSuccess;
    if (mode == 5) {
        for (int r = 0; r < t.n_radii && e == cudaSuccess; ++r)
            e = cudaMemsetAsync(t.radii[r].queue_n, 0, sizeof(unsigned long long), s);
    } else {
        e = cudaMemsetAsync(t.queue_n, 0, sizeof(unsigned long long), s);
    }
    if (e != cudaSuccess) { set_error(cudaGetErrorString(e)); return MAPPER_ECUDA; }
    const bool grouped = (mode == 1 || mode == 5) && t.groups != nullptr;
    p.groups = grouped ? t.groups : nullptr;
    p.n_groups = grouped ? t.n_groups : 0;
    p.n_dev = grouped ? t.groups_dev : t.n_dev;
    const int grid = (int)std::min<int64_t>(grouped ? t.n_groups : n_pairs, t.num_sms);
    if (grid < 1) return MAPPER_OK;
    if (t.ev_begin) cudaEventRecord(t.ev_begin, s);
    if (t.f8)
        e = grouped ? launch<3, 1, 2, 1>(mh, ml, p, grid, s) : launch<3, 1, 1, 1>(mh, ml, p, grid, s);
    else if (mode == 5)
        e = grouped ? (t.ns == 3 ? launch<3, 5, 2>(mh, ml, p, grid, s) : launch<1, 5, 2>(mh, ml, p, grid, s))
                    : (t.ns == 3 ? launch<3, 5, 1>(mh, ml, p, grid, s) : launch<1, 5, 1>(mh, ml, p, grid, s));
    else if (grouped)
        e = t.ns == 3 ? launch<3, 1, 2>(mh, ml, p, grid, s) : launch<1, 1, 2>(mh, ml, p, grid, s);
    else if (t.ns == 3)
        e = mode == 1 ? launch<3, 1, 1>(mh, ml, p, grid, s) : launch<3, 2, 1>(mh, ml, p, grid, s);
    else
        e = mode == 1 ? launch<1, 1, 1>(mh, ml, p, grid, s) : launch<1, 2, 1>(mh, ml, p, grid, s);
    if (t.ev_end) cudaEventRecord(t.ev_end, s);
    note_launch();
    if (e != cudaSuccess) {
        set_error(std::string("tensor-core pass: ") + cudaGetErrorString(e));
        return MAPPER_ECUDA;
    }
    if (defer) return MAPPER_OK;              // no pair reaches the band queue
    // FP32 limits of the recheck's lane-split sum (relative error (dp/8 + 5) 2^-24)
    const double eta = 1.5 * (a.dp / 8 + 5) * std::ldexp(1.0, -24);
    const double tiny = 3.0 * (a.d + 2) * std::ldexp(1.0, -149);
    const int rgrid = t.num_sms * 16;
    auto recheck = [&](const PassArgs& ar, const uint2* queue, const unsigned long long* queue_n) {
        float lo32 = (float)(ar.eps2 * (1.0 - eta) - tiny), hi32 = (float)(ar.eps2 * (1.0 + eta) + tiny);
        if ((double)lo32 > ar.eps2 * (1.0 - eta) - tiny) lo32 = std::nextafter(lo32, -INFINITY);
        if ((double)hi32 < ar.eps2 * (1.0 + eta) + tiny) hi32 = std::nextafter(hi32, INFINITY);
        if (mode == 2) recheck_kernel<2><<<rgrid, 256, 0, s>>>(ar, queue, queue_n, t.queue_cap, lo32, hi32);
        else recheck_kernel<1><<<rgrid, 256, 0, s>>>(ar, queue, queue_n, t.queue_cap, lo32, hi32);
        note_launch();
    };
    if (mode == 5) {
        for (int r = 0; r < t.n_radii; ++r) {
            const RadiusOut& o = t.radii[r];
            PassArgs ar = a;
            ar.count = o.count;
            ar.nbr = o.nbr;
            ar.pair_hit = o.pair_hit;
            ar.stats = o.stats;
            ar.eps2 = o.eps2;
            ar.tie_thr = 1e-12 * o.eps2;
            recheck(ar, o.queue, o.queue_n);
        }
    } else {
        recheck(a, t.queue, t.queue_n);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error(std::string("band recheck: ") + cudaGetErrorString(e));
        return MAPPER_ECUDA;
    }
    return MAPPER_OK;
}

namespace {

// The bounded wait of the tensor-core passes, run out on purpose: one thread
// arms an mbarrier for one arrival that nothing makes and waits on it with
// the same helper; status = 1 when the wait gave up and raised the abort
// flag (as a pass that lost its producer would), 0 if it completed.
__global__ void wait_selftest_kernel(int* status)
{
    __shared__ uint64_t bar;
    __shared__ int abort_flag;
    if (threadIdx.x == 0) {
        abort_flag = 0;
        mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        const bool done = mbar_wait(&bar, 0, &abort_flag);
        *status = done ? 0 : (abort_flag ? 1 : 2);
    }
}

}  // namespace

int tc_wait_selftest(cudaStream_t s)
{
    Buf st;
    cudaError_t e = st.alloc(sizeof(int), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(st.p, 0xff, sizeof(int), s);
    if (e != cudaSuccess) { set_error(cudaGetErrorString(e)); return MAPPER_ECUDA; }
    wait_selftest_kernel<<<1, 32, 0, s>>>(st.as<int>());
    note_launch();
    int h = -1;
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, st.p, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) { set_error(cudaGetErrorString(e)); return MAPPER_ECUDA; }
    if (h == 1) {
        set_error("bounded wait gave up as designed (self-test)");
        return MAPPER_ETIMEOUT;
    }
    set_error("bounded-wait self-test: the wait did not run out");
    return MAPPER_EINTERNAL;
}

int tc_knn_screen(const KnnScreen& k, cudaStream_t s)
{
    if (k.q == 0 || k.n_tiles == 0) return MAPPER_OK;
    const int64_t Tq = (k.q + kT - 1) / kT;
    if (k.rows >= (int64_t(1) << 30) || k.chunk_tiles < 2 || (k.chunk_tiles & 1) || k.chunks < 1 ||
        Tq * k.chunks > INT32_MAX || k.tile_stride < 1 || (k.n_tiles - 1) * k.tile_stride >= k.q_tile0 ||
        (k.q_tile0 + Tq) * kT > k.rows || (k.tau && ((k.cap < 1 && !k.off) || !k.count))) {
        set_error("k-distance tensor-core screen: sizes out of range");
        return MAPPER_EINVAL;
    }
    CUtensorMap mh, ml;
    if (!make_map(&mh, k.Ah, k.rows, k.dp) || !make_map(&ml, k.Al, k.rows, k.dp)) {
        set_error("cuTensorMapEncodeTiled failed (or is unavailable)");
        return MAPPER_ECUDA;
    }
    TcParams p{};
    p.A.tile_n = k.tile_n;
    p.A.dp = k.dp;
    p.rn2 = k.rn2;
    p.nkb = (k.dp + kKB - 1) / kKB;
    p.err = k.err;
    p.A3f = k.A3f;
    p.kq_tp = k.n_tiles;
    p.kq_stride = k.tile_stride;
    p.kq_qt0 = k.q_tile0;
    p.kq_q = k.q;
    p.kq_ct = k.chunk_tiles;
    p.kq_chunks = k.chunks;
    p.kq_m = k.m;
    p.kq_c2 = k.c2;
    p.kq_tau = k.tau;
    p.kq_cap = k.cap;
    p.kq_off = k.off;
    p.kq_cnt = k.count;
    p.kq_v = k.cand_v;
    p.kq_i = k.cand_i;
    const cudaError_t e = launch<3, 3, 2>(mh, ml, p, (int)(Tq * k.chunks), s);
    note_launch();
    if (e != cudaSuccess) {
        set_error(std::string("k-distance tensor-core screen: ") + cudaGetErrorString(e));
        return MAPPER_ECUDA;
    }
    return MAPPER_OK;
}

namespace {

uint64_t splitmix(uint64_t x)
{
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}

uint16_t bf16_bits_rn(float f)                // round to nearest even (finite f)
{
    uint32_t u;
    std::memcpy(&u, &f, 4);
    u += 0x7FFFu + ((u >> 16) & 1u);
    return (uint16_t)(u >> 16);
}

float bf16_value(uint16_t b)
{
    const uint32_t u = (uint32_t)b << 16;
    float f;
    std::memcpy(&f, &u, 4);
    return f;
}

}  // namespace

// value of an E4M3 byte (sign, 4 exponent bits of bias 7, 3 mantissa bits;
// exponent 0 subnormal; S.1111.111 is NaN and never generated here)
double e4m3_value(uint8_t b)
{
    const int e = (b >> 3) & 15, m = b & 7;
    const double v = e ? std::ldexp(1.0 + m / 8.0, e - 7) : std::ldexp(m / 8.0, -6);
    return (b & 0x80) ? -v : v;
}

uint8_t e4m3_random(uint64_t h, int e_lo, int e_hi)        // a normal value 2^e (1 + m/8), e in [e_lo, e_hi]
{
    const int e = e_lo + (int)((h >> 8) % (uint64_t)(e_hi - e_lo + 1));
    const int m = (int)(h & 7);
    return (uint8_t)(((h >> 63) ? 0x80 : 0) | ((e + 7) << 3) | m);
}

int tc_mma_probe(int ns, int fmt, int dp, uint64_t seed, int num_sms, double* observed, double* modelled,
                 cudaStream_t s)
{
    if ((ns != 1 && ns != 3) || (fmt != 0 && fmt != 1) || dp < 32 || dp % 32 || dp > 4096) {
        set_error("accumulation probe: products must be 1 or 3, the format 0 (BF16) or 1 (FP8) and the pitch a "
                  "multiple of 32 in [32, 4096]");
        return MAPPER_EINVAL;
    }
    constexpr int kPairs = 4, kTiles = 2 * kPairs, R = kTiles * kT;
    // random rows: BF16 values sign * 2^e * m with e in [-4, 4] split into hi + lo;
    // FP8 E4M3 hi parts with exponents in [-4, 5] and lo parts in [-8, 1]
    const int esz = fmt ? 1 : 2;
    std::vector<uint16_t> hi((size_t)R * dp), lo((size_t)R * dp);
    std::vector<uint8_t> hi8(fmt ? (size_t)R * dp : 0), lo8(fmt ? (size_t)R * dp : 0);
    for (size_t i = 0; i < hi.size(); ++i) {
        const uint64_t h = splitmix(seed * 0x100000001B3ull + i);
        if (fmt) {
            hi8[i] = e4m3_random(h, -4, 5);
            lo8[i] = e4m3_random(splitmix(h), -8, 1);
            continue;
        }
        const float m = 1.0f + (float)((h >> 11) & 0xFFFFFF) / 16777216.0f;
        const int e = (int)((h >> 40) % 9) - 4;
        const float v = std::ldexp(m, e) * ((h >> 63) ? -1.0f : 1.0f);
        hi[i] = bf16_bits_rn(v);
        lo[i] = bf16_bits_rn(v - bf16_value(hi[i]));
    }
    auto hv = [&](size_t i) { return fmt ? e4m3_value(hi8[i]) : (double)bf16_value(hi[i]); };
    auto lv = [&](size_t i) { return fmt ? e4m3_value(lo8[i]) : (double)bf16_value(lo[i]); };
    std::vector<int2> pairs(kPairs);
    for (int k = 0; k < kPairs; ++k) pairs[k] = make_int2(2 * k, 2 * k + 1);
    std::vector<int32_t> tile_n(kTiles, kT);
    Buf dAh, dAl, dpairs, dtn, ddump, derr;
#define PK(expr)                                                                  \
    do {                                                                          \
        cudaError_t e_ = (expr);                                                  \
        if (e_ != cudaSuccess) {                                                  \
            set_error(std::string("accumulation probe: ") + cudaGetErrorString(e_)); \
            return e_ == cudaErrorMemoryAllocation ? MAPPER_ENOMEM : MAPPER_ECUDA; \
        }                                                                         \
    } while (0)
    PK(dAh.alloc(hi.size() * esz, s));
    PK(dAl.alloc(lo.size() * esz, s));
    PK(dpairs.alloc(sizeof(int2) * kPairs, s));
    PK(dtn.alloc(sizeof(int32_t) * kTiles, s));
    PK(ddump.alloc(sizeof(float) * (size_t)kPairs * kT * kT, s));
    PK(derr.alloc(sizeof(int), s));
    PK(cudaMemcpyAsync(dAh.p, fmt ? (const void*)hi8.data() : (const void*)hi.data(), hi.size() * esz,
                       cudaMemcpyHostToDevice, s));
    PK(cudaMemcpyAsync(dAl.p, fmt ? (const void*)lo8.data() : (const void*)lo.data(), lo.size() * esz,
                       cudaMemcpyHostToDevice, s));
    PK(cudaMemcpyAsync(dpairs.p, pairs.data(), sizeof(int2) * kPairs, cudaMemcpyHostToDevice, s));
    PK(cudaMemcpyAsync(dtn.p, tile_n.data(), sizeof(int32_t) * kTiles, cudaMemcpyHostToDevice, s));
    PK(cudaMemsetAsync(derr.p, 0, sizeof(int), s));
    const int dcols = fmt ? dp / 2 : dp;                 // FP8 rows moved as BF16 columns of two bytes
    CUtensorMap mh, ml;
    if (!make_map(&mh, dAh.p, R, dcols) || !make_map(&ml, ns == 3 ? dAl.p : dAh.p, R, dcols)) {
        set_error("cuTensorMapEncodeTiled failed (or is unavailable)");
        return MAPPER_ECUDA;
    }
    TcParams p{};
    p.A.pairs = dpairs.as<int2>();
    p.A.tile_n = dtn.as<int32_t>();
    p.A.dp = dp;
    p.n_pairs = kPairs;
    p.nkb = (dcols + kKB - 1) / kKB;
    p.err = derr.as<int>();
    p.dump = ddump.as<float>();
    const int grid = std::min(kPairs, num_sms);
    if (fmt) PK((ns == 3 ? launch<3, 4, 1, 1>(mh, ml, p, grid, s) : launch<1, 4, 1, 1>(mh, ml, p, grid, s)));
    else PK((ns == 3 ? launch<3, 4, 1>(mh, ml, p, grid, s) : launch<1, 4, 1>(mh, ml, p, grid, s)));
    note_launch();
    std::vector<float> acc((size_t)kPairs * kT * kT);
    int h_err = 0;
    PK(cudaMemcpyAsync(acc.data(), ddump.p, acc.size() * sizeof(float), cudaMemcpyDeviceToHost, s));
    PK(cudaMemcpyAsync(&h_err, derr.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    PK(cudaStreamSynchronize(s));
#undef PK
    if (h_err) {
        set_error("accumulation probe gave up waiting on a barrier");
        return MAPPER_ETIMEOUT;
    }
    // exact sums in FP64 (products of BF16 values are exact; the FP64 sum of
    // 3 dp terms errs by < 3 dp 2^-53 of their magnitude sum)
    double worst = 0.0;
    for (int k = 0; k < kPairs; ++k)
        for (int i = 0; i < kT; ++i)
            for (int j = 0; j < kT; ++j) {
                const size_t ra = ((size_t)(2 * k) * kT + i) * dp, rb = ((size_t)(2 * k + 1) * kT + j) * dp;
                double ex = 0.0, mag = 0.0;
                for (int c = 0; c < dp; ++c) {
                    const double ah = hv(ra + c), bh = hv(rb + c);
                    double t = ah * bh;
                    ex += t;
                    mag += std::fabs(t);
                    if (ns == 3) {
                        const double al = lv(ra + c), bl = lv(rb + c);
                        t = ah * bl;
                        ex += t;
                        mag += std::fabs(t);
                        t = al * bh;
                        ex += t;
                        mag += std::fabs(t);
                    }
                }
                const double err = std::fabs((double)acc[((size_t)k * kT + i) * kT + j] - ex);
                if (mag > 0.0) worst = std::max(worst, err / mag);
            }
    *observed = worst;
    *modelled = fmt ? accu_model_f8(ns, dp) : accu_model(ns, dp);
    return MAPPER_OK;
}

int tc_groups(const int2* pairs, int64_t n, Buf* groups, Buf* pos, cudaStream_t s)
{
    if (n == 0) return MAPPER_OK;
    Buf lead;
#define GK(expr)                                                                  \
    do {                                                                          \
        cudaError_t e_ = (expr);                                                  \
        if (e_ != cudaSuccess) {                                                  \
            set_error(std::string("tc_groups: ") + cudaGetErrorString(e_));       \
            return e_ == cudaErrorMemoryAllocation ? MAPPER_ENOMEM : MAPPER_ECUDA; \
        }                                                                         \
    } while (0)
    GK(lead.alloc(sizeof(int32_t) * n, s));
    GK(pos->alloc(sizeof(int64_t) * (n + 1), s));
    const unsigned blocks = (unsigned)div_up(n, 256);
    group_lead_kernel<<<blocks, 256, 0, s>>>(pairs, n, lead.as<int32_t>());
    note_launch();
    GK(cudaGetLastError());
    GK(exclusive_scan_i32_to_i64(lead.as<int32_t>(), pos->as<int64_t>(), n, s));
    GK(groups->alloc(sizeof(int2) * (size_t)n, s));
    group_emit_kernel<<<blocks, 256, 0, s>>>(pairs, n, lead.as<int32_t>(), pos->as<int64_t>(), groups->as<int2>());
    note_launch();
    GK(cudaGetLastError());
#undef GK
    return MAPPER_OK;
}

}  // namespace mgb
