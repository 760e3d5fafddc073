// k_nerve.cu -- nodes and the 1D nerve ("Mapper Interactive" §3: the clusters
// of every cover element are the nodes; an edge joins two nodes whose point
// sets intersect).
//
// Nodes are numbered by the cover slot of their root (slots are ordered by
// element, then point), i.e. by (element, canonical id). Memberships become
// (node << 32 | point) keys, sorted into per-node member lists; the same
// memberships re-keyed as (point << 32 | node) and sorted group the nodes of
// each point, every pair of them is emitted as (u << 32 | v), u < v, and a
// sort-unique of those keys gives the edge list in lexicographic order.
#include "dbscan.cuh"

namespace mgb {

namespace {

__global__ void member_keys_kernel(const int32_t* __restrict__ lab, const int64_t* __restrict__ nid,
                                   const int64_t* __restrict__ mpos,
                                   const int32_t* __restrict__ slot_point,
                                   const int32_t* __restrict__ slot_elem, int64_t M,
                                   uint64_t* __restrict__ keys, int32_t* __restrict__ node_elem)
{
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= M) return;
    const int l = lab[s];
    if (l < 0) return;
    const int64_t node = nid[l];
    keys[mpos[s]] = ((uint64_t)node << 32) | (uint64_t)(uint32_t)slot_point[s];
    if (l == (int)s) node_elem[node] = slot_elem[s];
}

__global__ void node_offsets_kernel(const uint64_t* __restrict__ keys, int64_t G,
                                    int64_t* __restrict__ node_off, int32_t* __restrict__ members,
                                    uint64_t* __restrict__ keys2)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= G) return;
    const uint64_t k = keys[i];
    const int64_t node = (int64_t)(k >> 32);
    members[i] = (int32_t)(uint32_t)k;
    keys2[i] = ((k & 0xffffffffull) << 32) | (uint64_t)node;
    if (i == 0 || (int64_t)(keys[i - 1] >> 32) != node) node_off[node] = i;
}

// Nerve keys (point << 32 | node) of given nodes: member i belongs to the
// node u with node_off[u] <= i < node_off[u + 1].
__global__ void node_member_keys_kernel(const int64_t* __restrict__ node_off, int64_t N, int64_t G,
                                        const int32_t* __restrict__ members, uint64_t* __restrict__ keys2)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= G) return;
    int64_t lo = 0, hi = N;                    // last u with node_off[u] <= i
    while (hi - lo > 1) {
        const int64_t mid = (lo + hi) >> 1;
        if (node_off[mid] <= i) lo = mid; else hi = mid;
    }
    keys2[i] = ((uint64_t)(uint32_t)members[i] << 32) | (uint64_t)lo;
}

// Slot -> element index of a cover whose element offsets are elem_off[0..k].
__global__ void fill_slot_elem_kernel(const int64_t* __restrict__ elem_off, int32_t k, int64_t M,
                                      int32_t* __restrict__ slot_elem)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= M) return;
    int32_t lo = 0, hi = k;                    // last e with elem_off[e] <= i
    while (hi - lo > 1) {
        const int32_t mid = (lo + hi) >> 1;
        if (elem_off[mid] <= i) lo = mid; else hi = mid;
    }
    slot_elem[i] = lo;
}

__global__ void run_pairs_kernel(const uint64_t* __restrict__ keys2, int64_t G,
                                 int64_t* __restrict__ cnt)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= G) return;
    const uint64_t pt = keys2[i] >> 32;
    int64_t c = 0;
    if (i == 0 || (keys2[i - 1] >> 32) != pt) {
        int64_t len = 1;
        while (i + len < G && (keys2[i + len] >> 32) == pt) ++len;
        c = len * (len - 1) / 2;
    }
    cnt[i] = c;
}

__global__ void emit_pairs_kernel(const uint64_t* __restrict__ keys2, int64_t G,
                                  const int64_t* __restrict__ pos, uint64_t* __restrict__ out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= G) return;
    const uint64_t pt = keys2[i] >> 32;
    if (!(i == 0 || (keys2[i - 1] >> 32) != pt)) return;
    int64_t len = 1;
    while (i + len < G && (keys2[i + len] >> 32) == pt) ++len;
    int64_t o = pos[i];
    for (int64_t a = 0; a < len; ++a)
        for (int64_t b = a + 1; b < len; ++b)
            out[o++] = ((keys2[i + a] & 0xffffffffull) << 32) | (keys2[i + b] & 0xffffffffull);
}

__global__ void unique_flags_kernel(const uint64_t* __restrict__ k, int64_t P,
                                    int32_t* __restrict__ flag)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P) return;
    flag[i] = (i == 0 || k[i] != k[i - 1]);
}

__global__ void unique_emit_kernel(const uint64_t* __restrict__ k, const int32_t* __restrict__ flag,
                                   const int64_t* __restrict__ pos, int64_t P,
                                   int32_t* __restrict__ edges)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P || !flag[i]) return;
    const int64_t o = pos[i];
    edges[2 * o] = (int32_t)(k[i] >> 32);
    edges[2 * o + 1] = (int32_t)(uint32_t)k[i];
}

inline unsigned grid_for(int64_t n, int t = 256) { return (unsigned)std::max<int64_t>(1, div_up(n, t)); }

}  // namespace

cudaError_t member_keys(const int32_t* lab, const int64_t* nid, const int64_t* mpos,
                        const int32_t* slot_point, const int32_t* slot_elem, int64_t M,
                        uint64_t* keys, int32_t* node_elem, cudaStream_t s)
{
    if (M == 0) return cudaSuccess;
    { member_keys_kernel<<<grid_for(M), 256, 0, s>>>(lab, nid, mpos, slot_point, slot_elem, M, keys,
                                                   node_elem); note_launch(); }
    return cudaGetLastError();
}

cudaError_t node_offsets(const uint64_t* keys, int64_t G, int64_t* node_off, int32_t* members,
                         uint64_t* keys2, cudaStream_t s)
{
    if (G == 0) return cudaSuccess;
    { node_offsets_kernel<<<grid_for(G), 256, 0, s>>>(keys, G, node_off, members, keys2); note_launch(); }
    return cudaGetLastError();
}

cudaError_t node_member_keys(const int64_t* node_off, int64_t N, int64_t G, const int32_t* members,
                             uint64_t* keys2, cudaStream_t s)
{
    if (G == 0 || N == 0) return cudaSuccess;
    { node_member_keys_kernel<<<grid_for(G), 256, 0, s>>>(node_off, N, G, members, keys2); note_launch(); }
    return cudaGetLastError();
}

cudaError_t fill_slot_elem(const int64_t* elem_off, int32_t k, int64_t M, int32_t* slot_elem, cudaStream_t s)
{
    if (M == 0 || k == 0) return cudaSuccess;
    { fill_slot_elem_kernel<<<grid_for(M), 256, 0, s>>>(elem_off, k, M, slot_elem); note_launch(); }
    return cudaGetLastError();
}

cudaError_t run_pairs(const uint64_t* keys2, int64_t G, int64_t* cnt, cudaStream_t s)
{
    if (G == 0) return cudaSuccess;
    { run_pairs_kernel<<<grid_for(G), 256, 0, s>>>(keys2, G, cnt); note_launch(); }
    return cudaGetLastError();
}

cudaError_t emit_pairs(const uint64_t* keys2, int64_t G, const int64_t* pos, uint64_t* out,
                       cudaStream_t s)
{
    if (G == 0) return cudaSuccess;
    { emit_pairs_kernel<<<grid_for(G), 256, 0, s>>>(keys2, G, pos, out); note_launch(); }
    return cudaGetLastError();
}

cudaError_t unique_flags(const uint64_t* k, int64_t P, int32_t* flag, cudaStream_t s)
{
    if (P == 0) return cudaSuccess;
    { unique_flags_kernel<<<grid_for(P), 256, 0, s>>>(k, P, flag); note_launch(); }
    return cudaGetLastError();
}

cudaError_t unique_emit(const uint64_t* k, const int32_t* flag, const int64_t* pos, int64_t P,
                        int32_t* edges, cudaStream_t s)
{
    if (P == 0) return cudaSuccess;
    { unique_emit_kernel<<<grid_for(P), 256, 0, s>>>(k, flag, pos, P, edges); note_launch(); }
    return cudaGetLastError();
}

}  // namespace mgb
