"""Pins of the oracle's DBSCAN, node numbering and nerve: hand-derived
fixtures, textbook special cases, an independent library (scikit-learn's
DBSCAN, SciPy's connected components) and geometric invariants with a known
answer (a circle under a height lens is a cycle)."""
import json
import os

import numpy as np
import pytest

import oracle
from paper_2011_03209_gb300 import synth


def _line(x, d=1):
    X = np.zeros((len(x), d), dtype=np.float32)
    X[:, 0] = x
    return X


@pytest.mark.parametrize("d", [1, 3])
def test_dbscan_golden(golden_dir, d):
    g = json.load(open(os.path.join(golden_dir, "dbscan_line.json")))
    for c in g["cases"]:
        X = _line(c["x"], d)
        count, core, label, ties = oracle.dbscan(X, np.arange(len(X)), c["eps"], c["min_pts"])
        assert count.tolist() == c["count"], c["name"]
        assert core.astype(int).tolist() == c["core"], c["name"]
        assert label.tolist() == c["label"], c["name"]
        assert ties == c["near_ties"], c["name"]


def test_dbscan_subset_uses_global_ids():
    # the same cluster seen through a subset: canonical ids are global indices
    X = _line([9.0, 0.0, 9.0, 0.1, 0.2, 9.0])
    _, core, label, _ = oracle.dbscan(X, np.array([1, 3, 4]), 0.5, 2)
    assert core.all() and label.tolist() == [1, 1, 1]


def _core_partition(labels, core_mask):
    parts = {}
    for i in np.nonzero(core_mask)[0]:
        parts.setdefault(int(labels[i]), []).append(int(i))
    return sorted(tuple(v) for v in parts.values())


@pytest.mark.parametrize("seed,eps,min_pts", [(0, 0.25, 4), (1, 0.15, 3), (2, 0.4, 10), (3, 0.3, 1)])
def test_dbscan_core_set_and_partition_match_sklearn(seed, eps, min_pts):
    sk = pytest.importorskip("sklearn.cluster")
    X = synth.tiny_random(600, 3, seed=seed, dup_frac=0.05)
    count, core, label, _ = oracle.dbscan(X, np.arange(len(X)), eps, min_pts)
    ref = sk.DBSCAN(eps=eps, min_samples=min_pts, algorithm="brute").fit(X.astype(np.float64))
    ref_core = np.zeros(len(X), dtype=bool)
    ref_core[ref.core_sample_indices_] = True
    assert np.array_equal(core, ref_core)
    assert _core_partition(label, core) == _core_partition(ref.labels_, ref_core)
    # every non-noise label is the smallest index among that cluster's cores
    for c in set(label[label >= 0].tolist()):
        assert c == np.nonzero(core & (label == c))[0].min()


def test_dbscan_min_pts_one_is_connected_components():
    csgraph = pytest.importorskip("scipy.sparse.csgraph")
    from scipy.spatial.distance import cdist
    X = synth.tiny_random(300, 2, seed=11)
    eps = 0.06
    _, core, label, _ = oracle.dbscan(X, np.arange(len(X)), eps, 1)
    D = cdist(X.astype(np.float64), X.astype(np.float64), "sqeuclidean")
    ncomp, comp = csgraph.connected_components(D <= eps * eps, directed=False)
    assert core.all()
    assert len(set(label.tolist())) == ncomp
    for c in range(ncomp):
        members = np.nonzero(comp == c)[0]
        assert np.all(label[members] == members.min())


def test_dbscan_extreme_radii():
    X = synth.tiny_random(200, 4, seed=12)
    _, core, label, _ = oracle.dbscan(X, np.arange(200), 100.0, 5)
    assert core.all() and np.all(label == 0)          # one cluster
    _, core, label, _ = oracle.dbscan(X, np.arange(200), 1e-6, 2)
    assert not core.any() and np.all(label == -1)     # all noise
    _, core, label, _ = oracle.dbscan(X, np.arange(200), 1e-6, 1)
    assert np.array_equal(label, np.arange(200))      # singletons


def test_graph_golden_line(golden_dir):
    g = json.load(open(os.path.join(golden_dir, "graph_line.json")))
    X = _line(g["x"], 2)
    f = oracle.lens_coord(X, 0)
    out = oracle.mapper_graph(X, f[:, None], [g["n_intervals"]], [g["overlap"]], g["eps"], g["min_pts"])
    offs, pts = out["elem_offsets"], out["elem_points"]
    assert [pts[offs[e]:offs[e + 1]].tolist() for e in range(3)] == g["elements"]
    assert out["node_offsets"].tolist() == g["node_offsets"]
    assert out["node_members"].tolist() == g["node_members"]
    assert out["node_elem"].tolist() == g["node_elem"]
    assert out["edges"].tolist() == g["edges"]


def _components(n_nodes, edges):
    parent = list(range(n_nodes))

    def find(a):
        while parent[a] != a:
            a = parent[a]
        return a
    for u, v in edges:
        parent[find(u)] = find(v)
    return len({find(i) for i in range(n_nodes)})


@pytest.mark.parametrize("n_int", [4, 6, 9])
def test_circle_height_lens_is_a_cycle(n_int):
    # unit circle, lens = height: the two caps give one node each and every
    # inner interval two arcs, so 2n-2 nodes joined in a single cycle
    X = synth.circle(720)
    f = oracle.lens_coord(X, 1)
    out = oracle.mapper_graph(X, f[:, None], [n_int], [0.3], 0.05, 2)
    N = len(out["node_offsets"]) - 1
    E = out["edges"]
    assert N == 2 * n_int - 2 and len(E) == 2 * n_int - 2
    deg = np.bincount(E.ravel(), minlength=N)
    assert np.all(deg == 2)
    assert _components(N, E.tolist()) == 1


def test_separated_blobs_give_one_component_each():
    k = 5
    X = synth.separated_blobs(k, 150, 6, gap=40.0, std=0.3, seed=3)
    f = oracle.lens_l2(X)
    out = oracle.mapper_graph(X, f[:, None], [12], [0.3], 1.5, 3)
    N = len(out["node_offsets"]) - 1
    assert _components(N, out["edges"].tolist()) == k


def _check_nerve_by_definition(out):
    no, nm = out["node_offsets"], out["node_members"]
    sets = [set(nm[no[u]:no[u + 1]].tolist()) for u in range(len(no) - 1)]
    ref = [[u, v] for u in range(len(sets)) for v in range(u + 1, len(sets)) if sets[u] & sets[v]]
    assert out["edges"].tolist() == ref


def test_zero_overlap_and_graph_invariants():
    w = synth.blobs_circle_5k()
    f = oracle.lens(w.X, w.lens_kind, w.lens_arg)
    for p in (0.0, 0.3, 0.6):
        out = oracle.mapper_graph(w.X, f, [15], [p], w.eps, w.min_pts)
        ne, E = out["node_elem"], out["edges"]
        if p == 0.0:
            assert np.all(np.abs(ne[E[:, 0]] - ne[E[:, 1]]) <= 1)
        _check_nerve_by_definition(out)
        # members of nodes of one element are disjoint, and are exactly the
        # non-noise points of that element
        offs, pts, lab = out["elem_offsets"], out["elem_points"], out["labels"]
        no, nm = out["node_offsets"], out["node_members"]
        for e in range(15):
            mem = [nm[no[u]:no[u + 1]] for u in np.nonzero(ne == e)[0]]
            allm = np.concatenate(mem) if mem else np.zeros(0, dtype=np.int32)
            assert len(allm) == len(set(allm.tolist()))
            s, t = offs[e], offs[e + 1]
            assert sorted(allm.tolist()) == sorted(pts[s:t][lab[s:t] >= 0].tolist())
        # nodes are ordered by (element, canonical id = smallest core index)
        keys = []
        for u in range(len(ne)):
            s, t = offs[ne[u]], offs[ne[u] + 1]
            core_pts = set(pts[s:t][out["core"][s:t]].tolist())
            keys.append((ne[u], min(set(nm[no[u]:no[u + 1]].tolist()) & core_pts)))
        assert keys == sorted(keys)


def test_blobs_circle_5k_core_partition_vs_sklearn():
    sk = pytest.importorskip("sklearn.cluster")
    w = synth.blobs_circle_5k()
    f = oracle.lens(w.X, w.lens_kind, w.lens_arg)
    out = oracle.mapper_graph(w.X, f, w.n_intervals, w.overlap, w.eps, w.min_pts)
    offs, pts = out["elem_offsets"], out["elem_points"]
    assert out["near_ties"] == 0
    for e in range(len(offs) - 1):
        s, t = offs[e], offs[e + 1]
        if t - s == 0:
            continue
        ref = sk.DBSCAN(eps=w.eps, min_samples=w.min_pts, algorithm="brute").fit(
            w.X[pts[s:t]].astype(np.float64))
        ref_core = np.zeros(t - s, dtype=bool)
        ref_core[ref.core_sample_indices_] = True
        assert np.array_equal(out["core"][s:t], ref_core)
        assert _core_partition(out["labels"][s:t], ref_core) == \
            _core_partition(ref.labels_, ref_core)


def test_knn_distance_closed_forms():
    """k-th nearest-neighbour distance (the point itself first): points
    0, 1, ..., 9 on a line; duplicates; k = 1 and k = n."""
    X = np.arange(10, dtype=np.float32).reshape(-1, 1)
    q = np.arange(10)
    # from x = i the sorted distances are 0, 1, 1, 2, 2, ... (while both sides last)
    assert oracle.knn_distance(X, q, 1).tolist() == [0.0] * 10
    assert oracle.knn_distance(X, [0, 5, 9], 2).tolist() == [1.0, 1.0, 1.0]
    assert oracle.knn_distance(X, [0, 5, 9], 4).tolist() == [3.0, 2.0, 3.0]
    assert oracle.knn_distance(X, [0, 4, 9], 10).tolist() == [9.0, 5.0, 9.0]
    # a 3-4-5 triangle
    T = np.array([[0, 0], [3, 0], [0, 4]], dtype=np.float32)
    assert oracle.knn_distance(T, [0, 1, 2], 2).tolist() == [3.0, 3.0, 4.0]
    assert oracle.knn_distance(T, [0, 1, 2], 3).tolist() == [4.0, 5.0, 5.0]
    # duplicates count: three copies of a point reach k = 3 at distance 0
    D = np.array([[1, 1], [1, 1], [1, 1], [4, 5]], dtype=np.float32)
    assert oracle.knn_distance(D, [0, 3], 3).tolist() == [0.0, 5.0]
    with pytest.raises(ValueError):
        oracle.knn_distance(D, [0], 5)


def test_knn_distance_is_the_core_threshold():
    """kdist(p) <= eps iff p has at least k neighbours (itself included) in
    the whole cloud, i.e. iff p is core for DBSCAN(eps, k) on one element."""
    X = synth.tiny_random(300, 5, 9, scale=2.0)
    k = 6
    kd = oracle.knn_distance(X, np.arange(300), k)
    for eps in (0.3, 0.45, 0.6):
        _, core, _, _ = oracle.dbscan(X, np.arange(300, dtype=np.int32), eps, k)
        assert np.array_equal(core, kd <= eps)
