"""One mapper graph computed by several ranks, each clustering a share of the
cover elements.

The clustering of each cover element is independent ("Mapper Interactive"
§4.3), and §6 names distributing it across several GPUs, with the merge of
the results, as the next step. Here every rank computes the lens and the
cover (cheap, and identical on every rank), clusters the elements it owns
(a longest-processing-time split by the cost n_i^2 d of each element), and
the ranks exchange their nodes (all-gathers of plain tensors): the one
exchange of the path. Every rank then
merges the nodes in element order and computes the nerve of the merged list
on its GPU.

The library calls do the work (lens, cover, cover subset, clustering and
nerve kernels); this module partitions, exchanges and concatenates arrays.
"""
from __future__ import annotations

import numpy as np

import paper_2011_03209_gb300 as mg


def lpt_partition(costs, world: int) -> list:
    """Split elements over `world` ranks, longest processing time first:
    elements by decreasing cost (ties: lower index first), each to the rank
    with the least cost so far (ties: lower rank). Returns, per rank, its
    element indices ascending."""
    costs = np.asarray(costs, dtype=np.float64)
    order = np.lexsort((np.arange(costs.size), -costs))
    load = np.zeros(world, dtype=np.float64)
    owner = np.empty(costs.size, dtype=np.int64)
    for e in order:
        r = int(np.argmin(load))
        owner[e] = r
        load[r] += costs[e]
    return [np.nonzero(owner == r)[0].astype(np.int32) for r in range(world)]


def local_nodes(ctx, X, cover, elements, eps: float, min_pts: int, precision: int) -> dict:
    """Nodes of the given elements (global indices, ascending): members,
    offsets and global element of each node, ordered by (element, canonical
    id) as in a whole graph."""
    elements = np.asarray(elements, dtype=np.int32)
    if elements.size == 0:
        return dict(elements=elements, node_offsets=np.zeros(1, dtype=np.int64),
                    node_members=np.zeros(0, dtype=np.int32), node_elem=np.zeros(0, dtype=np.int32))
    sub = mg.mapper_cover_subset(ctx, cover, elements)
    cl = mg.mapper_cluster(ctx, X, sub, eps, min_pts, precision)
    g = mg.mapper_nerve(ctx, cl).numpy()
    return dict(elements=elements, node_offsets=g["node_offsets"], node_members=g["node_members"],
                node_elem=elements[g["node_elem"]])


def merge_nodes(pieces) -> tuple:
    """Nodes of all pieces (element sets disjoint) in global element order;
    within an element, a piece's order (canonical id). Returns node_offsets,
    node_members, node_elem."""
    elems, sizes, members = [], [], []
    for p in pieces:
        off = np.asarray(p["node_offsets"], dtype=np.int64)
        elems.append(np.asarray(p["node_elem"], dtype=np.int32))
        sizes.append(np.diff(off))
        members.append([np.asarray(p["node_members"][off[u]:off[u + 1]], dtype=np.int32)
                        for u in range(off.size - 1)])
    if not elems:
        return np.zeros(1, dtype=np.int64), np.zeros(0, dtype=np.int32), np.zeros(0, dtype=np.int32)
    node_elem = np.concatenate(elems)
    all_members = [m for ms in members for m in ms]
    order = np.argsort(node_elem, kind="stable")
    sz = np.concatenate(sizes)[order]
    offs = np.zeros(order.size + 1, dtype=np.int64)
    np.cumsum(sz, out=offs[1:])
    mem = (np.concatenate([all_members[i] for i in order]).astype(np.int32) if order.size
           else np.zeros(0, dtype=np.int32))
    return offs, mem, node_elem[order].astype(np.int32)


_FIELDS = (("elements", np.int32), ("node_offsets", np.int64), ("node_members", np.int32), ("node_elem", np.int32))


def exchange(piece: dict, group=None) -> list:
    """Every rank's piece, on every rank (a single piece without a process
    group). Two collectives of plain tensors: an all-gather of the four array
    lengths, then one all-gather of each array padded to the longest rank's
    length; on NCCL the tensors live on the current CUDA device, on gloo on
    the host."""
    import torch
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized():
        return [piece]
    world = dist.get_world_size(group)
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend(group) == "nccl" else torch.device("cpu")
    lens = torch.tensor([len(piece[k]) for k, _ in _FIELDS], dtype=torch.int64, device=dev)
    all_lens = [torch.empty_like(lens) for _ in range(world)]
    dist.all_gather(all_lens, lens, group=group)
    all_lens = torch.stack(all_lens).cpu().numpy()
    out = [dict() for _ in range(world)]
    for f, (key, dtype) in enumerate(_FIELDS):
        width = max(int(all_lens[:, f].max()), 1)
        mine = torch.zeros(width, dtype=torch.int64, device=dev)
        if len(piece[key]):
            mine[:len(piece[key])] = torch.from_numpy(np.asarray(piece[key], dtype=np.int64)).to(dev)
        parts = [torch.empty_like(mine) for _ in range(world)]
        dist.all_gather(parts, mine, group=group)
        for r in range(world):
            out[r][key] = parts[r][:int(all_lens[r, f])].cpu().numpy().astype(dtype)
    return out


def sharded_graph(ctx, X, prm, group=None):
    """The mapper graph of X with parameters `prm`, its elements clustered by
    the ranks of `group` (or by this process alone): equal, node for node and
    edge for edge, to mapper_graph(ctx, X, prm). Returns (graph handle of the
    merged nodes and their nerve, this rank's element indices)."""
    import torch.distributed as dist
    world, rank = 1, 0
    if dist.is_available() and dist.is_initialized():
        world, rank = dist.get_world_size(group), dist.get_rank(group)
    m = int(prm.m)
    kinds = [int(prm.lens_kind[i]) for i in range(m)]
    args = [int(prm.lens_arg[i]) for i in range(m)]
    lens, _ = mg.mapper_lens(ctx, X, kinds, args)
    cover = mg.mapper_cover(ctx, lens, [int(prm.n_intervals[i]) for i in range(m)],
                            [float(prm.overlap[i]) for i in range(m)],
                            balanced=int(prm.cover_kind) == mg.COVER_BALANCED)
    offs, _ = cover.numpy()
    d = int(X.shape[1])
    sizes = np.diff(offs).astype(np.float64)
    mine = lpt_partition(sizes * sizes * d, world)[rank]
    piece = local_nodes(ctx, X, cover, mine, float(prm.eps), int(prm.min_pts), int(prm.precision))
    no, nm, ne = merge_nodes(exchange(piece, group))
    return mg.mapper_nerve_from_nodes(ctx, int(X.shape[0]), no, nm, ne), mine
