"""Element sharding across ranks, on CPU: two (and three) gloo ranks each
cluster their share of the cover elements with the oracle, exchange their
nodes through torch.distributed and merge them; the merged nodes and their
nerve equal the oracle's whole graph. The partition, the exchange and the
merge are the host logic of the multi-GPU path (paper_2011_03209_gb300.sharded);
on GPUs the per-rank clustering runs in the library instead of the oracle."""
import os
import socket

import numpy as np
import pytest

import oracle
from paper_2011_03209_gb300 import sharded, synth

torch = pytest.importorskip("torch")
dist = pytest.importorskip("torch.distributed")


def _free_port() -> int:
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _case():
    X = synth.gaussian_mixture(1200, 6, 5, seed=31, centre_box=6.0, std_lo=0.4, std_hi=1.0,
                               anisotropic=True, noise_frac=0.05)
    eps = synth.eps_at_percentile(X, 6, 31, n_pairs=4000)
    return X, oracle.lens_l2(X).reshape(-1, 1), (9,), (0.3,), eps, 5


def _piece(X, lens, nint, ov, eps, min_pts, elements):
    """This rank's nodes: the oracle's clustering of its elements only."""
    offs, pts = oracle.cover(lens, nint, ov)
    sub_offs = [0]
    sub_pts = []
    for e in elements:
        sub_pts.append(pts[offs[e]:offs[e + 1]])
        sub_offs.append(sub_offs[-1] + int(offs[e + 1] - offs[e]))
    sub_pts = np.concatenate(sub_pts).astype(np.int32) if sub_pts else np.zeros(0, dtype=np.int32)
    labels = np.full(sub_pts.size, -1, dtype=np.int64)
    for j in range(len(elements)):
        s, t = sub_offs[j], sub_offs[j + 1]
        if t > s:
            labels[s:t] = oracle.dbscan(X, sub_pts[s:t], eps, min_pts)[2]
    no, nm, ne = oracle.nodes_from_labels(np.asarray(sub_offs, dtype=np.int64), sub_pts, labels)
    return dict(elements=np.asarray(elements, dtype=np.int32), node_offsets=no, node_members=nm,
                node_elem=np.asarray(elements, dtype=np.int32)[ne] if ne.size else ne)


def _rank(rank, world, port, result_dir):
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        X, lens, nint, ov, eps, min_pts = _case()
        offs, _ = oracle.cover(lens, nint, ov)
        sizes = np.diff(offs).astype(np.float64)
        parts = sharded.lpt_partition(sizes * sizes * X.shape[1], world)
        piece = _piece(X, lens, nint, ov, eps, min_pts, parts[rank])
        pieces = sharded.exchange(piece)
        assert len(pieces) == world
        assert sorted(np.concatenate([p["elements"] for p in pieces]).tolist()) == list(range(len(sizes)))
        no, nm, ne = sharded.merge_nodes(pieces)
        edges = oracle.nerve(no, nm, X.shape[0])
        np.savez(os.path.join(result_dir, f"rank{rank}.npz"), no=no, nm=nm, ne=ne, edges=edges)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_nodes_and_nerve_equal_whole_graph(tmp_path, world):
    mp = pytest.importorskip("torch.multiprocessing")
    port = _free_port()
    mp.spawn(_rank, args=(world, port, str(tmp_path)), nprocs=world, join=True)
    X, lens, nint, ov, eps, min_pts = _case()
    ref = oracle.mapper_graph(X, lens, nint, ov, eps, min_pts)
    assert len(ref["node_elem"]) > 3 and len(ref["edges"]) > 0
    for r in range(world):
        got = np.load(tmp_path / f"rank{r}.npz")
        assert np.array_equal(got["no"], ref["node_offsets"])
        assert np.array_equal(got["nm"], ref["node_members"])
        assert np.array_equal(got["ne"], ref["node_elem"])
        assert np.array_equal(got["edges"], ref["edges"])


def test_lpt_partition():
    costs = np.array([5.0, 1.0, 9.0, 3.0, 3.0, 0.0, 7.0])
    parts = sharded.lpt_partition(costs, 3)
    assert sorted(np.concatenate(parts).tolist()) == list(range(costs.size))
    for p in parts:
        assert np.all(np.diff(p) > 0)
    loads = sorted(float(costs[p].sum()) for p in parts)
    assert loads == [9.0, 9.0, 10.0]                 # {2, 5}, {6, 4}, {0, 3, 1}
    assert [p.tolist() for p in sharded.lpt_partition(costs, 1)] == [list(range(costs.size))]
    assert sum(p.size for p in sharded.lpt_partition(np.zeros(4), 3)) == 4


def test_merge_nodes_orders_by_element():
    a = dict(elements=np.array([2], np.int32), node_offsets=np.array([0, 2, 3]), node_members=np.array([4, 7, 1]),
             node_elem=np.array([2, 2], np.int32))
    b = dict(elements=np.array([0, 5], np.int32), node_offsets=np.array([0, 1, 3]), node_members=np.array([9, 2, 3]),
             node_elem=np.array([0, 5], np.int32))
    no, nm, ne = sharded.merge_nodes([a, b])
    assert no.tolist() == [0, 1, 3, 4, 6]
    assert nm.tolist() == [9, 4, 7, 1, 2, 3]
    assert ne.tolist() == [0, 2, 2, 5]
