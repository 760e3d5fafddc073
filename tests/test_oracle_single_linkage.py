"""Pins of the oracle's single-linkage forest (the minimum spanning forest of
the eps-graph of a cover element, Section 5's single-linkage clusterer):
hand-worked cases with tied distances (tests/golden/single_linkage.json),
SciPy's minimum spanning tree on clouds with distinct distances, the cut
property (the forest cut at h gives the components of the h-graph, i.e.
DBSCAN(h, minPts = 1)), and the forest's size."""
import json
import os

import numpy as np
import pytest

import oracle
from paper_2011_03209_gb300 import synth

scipy_sparse = pytest.importorskip("scipy.sparse")
csgraph = pytest.importorskip("scipy.sparse.csgraph")
spatial = pytest.importorskip("scipy.spatial")


def test_golden_forests(golden_dir):
    g = json.load(open(os.path.join(golden_dir, "single_linkage.json")))
    for c in g["cases"]:
        X = np.asarray(c["points"], dtype=np.float32)
        u, v, d2 = oracle.msf(X, np.arange(len(X), dtype=np.int32), c["eps"])
        got = [[int(a), int(b), float(w)] for a, b, w in zip(u, v, d2)]
        assert got == c["edges"], c["note"]


def _dense_eps_graph(X, eps):
    D = spatial.distance.cdist(X.astype(np.float64), X.astype(np.float64))
    D[D > eps] = 0.0
    return D


@pytest.mark.parametrize("n,d,seed,q", [(300, 3, 0, 5.0), (500, 16, 1, 2.0), (400, 64, 2, 10.0)])
def test_forest_matches_scipy_minimum_spanning_tree(n, d, seed, q):
    X = synth.tiny_random(n, d, seed, scale=2.0)           # distinct distances (no duplicates)
    eps = synth.eps_at_percentile(X, q, seed=seed, n_pairs=20000)
    u, v, d2 = oracle.msf(X, np.arange(n, dtype=np.int32), eps)
    T = csgraph.minimum_spanning_tree(scipy_sparse.csr_matrix(_dense_eps_graph(X, eps))).tocoo()
    ref = sorted((min(a, b), max(a, b)) for a, b in zip(T.row, T.col))
    assert sorted(zip(u.tolist(), v.tolist())) == ref
    np.testing.assert_allclose(np.sqrt(d2).sum(), T.data.sum(), rtol=1e-12)
    # key order and the eps restriction
    keys = list(zip(d2.tolist(), u.tolist(), v.tolist()))
    assert keys == sorted(keys) and np.all(d2 <= eps * eps) and np.all(u < v)
    # size: n minus the components of the eps-graph
    k, _ = csgraph.connected_components(scipy_sparse.csr_matrix(_dense_eps_graph(X, eps)), directed=False)
    assert len(u) == n - k


@pytest.mark.parametrize("seed", [3, 4])
def test_cut_gives_the_components_of_the_h_graph(seed):
    X = synth.gaussian_mixture(600, 8, 5, seed=seed, centre_box=5.0, std_lo=0.3, std_hi=1.0, anisotropic=True)
    pts = np.arange(600, dtype=np.int32)
    eps = synth.eps_at_percentile(X, 8.0, seed=seed, n_pairs=20000)
    u, v, d2 = oracle.msf(X, pts, eps)
    for frac in (0.3, 0.6, 0.9, 1.0):
        h = eps * frac
        lab = oracle.single_linkage(pts, u, v, d2, h)
        _, core, ref, _ = oracle.dbscan(X, pts, h, 1)      # minPts = 1: every point core
        assert core.all() and np.array_equal(lab, ref)
        k, comp = csgraph.connected_components(scipy_sparse.csr_matrix(_dense_eps_graph(X, h)), directed=False)
        assert len(np.unique(lab)) == k


def test_subset_of_points_and_empty_element():
    X = synth.tiny_random(200, 5, 9)
    pts = np.arange(3, 200, 3, dtype=np.int32)               # a cover element: some of the rows
    eps = synth.eps_at_percentile(X, 10.0, seed=9, n_pairs=10000)
    u, v, d2 = oracle.msf(X, pts, eps)
    assert set(u.tolist()) | set(v.tolist()) <= set(pts.tolist())
    sub = X[pts]
    u2, v2, d22 = oracle.msf(sub, np.arange(len(pts), dtype=np.int32), eps)
    assert np.array_equal(pts[u2], u) and np.array_equal(pts[v2], v) and np.array_equal(d22, d2)
    u3, _, _ = oracle.msf(X, np.zeros(0, dtype=np.int32), eps)
    assert len(u3) == 0
