"""Full-size parity of the 2D-lens workload: 500,000 x 128 points from 24
anisotropic Gaussians with Zipf(1.2) weights, lens (PC1, PC2), a 30 x 30 grid
of rectangles at 25 % overlap (900 cover elements of very uneven size, the
largest holding ~133k points), minPts 10, eps at the 1st percentile of
sampled distances.

Against the FP64 oracle: both principal axes (direction within 1e-6), the
lens bit for bit given the GPU's basis, the whole cover bit for bit, and the
DBSCAN of sampled elements (the smallest non-empty one, the median one and two
random ones of at most 20k points) slot by slot. The largest element is too
large for the brute-force oracle within a test, so its rows are checked by
sampling: core flags of 1500 rows from the oracle's neighbour counts, and
labels by properties every DBSCAN labelling has. Nodes and edges are checked
by their definition on the GPU's output."""
import functools

import numpy as np
import pytest

import oracle
from paper_2011_03209_gb300 import synth

torch = pytest.importorskip("torch")
mg = pytest.importorskip("paper_2011_03209_gb300")

pytestmark = pytest.mark.gpu


@functools.lru_cache(maxsize=1)
def _workload():
    w = synth.zipf_mixture_500k()
    omu, oV, _ = oracle.pca(w.X, 2)
    return w, omu, oV


def _check_nodes(res, n_points):
    """Nodes ordered by element, members ascending and disjoint within an
    element, and every edge {u, v} exactly where two nodes share a point."""
    no, nm, ne, E = res["node_offsets"], res["node_members"], res["node_elem"], res["edges"]
    N = len(ne)
    assert N > 0 and np.all(np.diff(no) > 0) and np.all(np.diff(ne) >= 0)
    node_of = np.repeat(np.arange(N), np.diff(no))
    same = node_of[1:] == node_of[:-1]
    assert np.all(nm[1:][same] > nm[:-1][same])
    key = ne[node_of].astype(np.int64) * n_points + nm
    assert len(np.unique(key)) == len(key)
    order = np.lexsort((node_of, nm))
    pts, nodes = nm[order], node_of[order]
    start = np.r_[0, np.nonzero(np.diff(pts))[0] + 1]
    ends = np.r_[start[1:], len(pts)]
    pairs = set()
    for s, t in zip(start, ends):
        ids = nodes[s:t]
        for a in range(len(ids)):
            for b in range(a + 1, len(ids)):
                pairs.add((int(ids[a]), int(ids[b])))
    assert sorted(pairs) == [tuple(e) for e in E.tolist()]


@pytest.mark.parametrize("prec", [mg.BF16, mg.FP32])
def test_zipf_500k_d128_grid_against_the_oracle(prec):
    w, omu, oV = _workload()
    Xd = torch.from_numpy(w.X).to("cuda:0")
    with mg.Context(0) as ctx:
        g = mg.mapper_graph(ctx, Xd, mg.params(w.lens_kind, w.lens_arg, w.n_intervals, w.overlap, w.eps,
                                               w.min_pts, prec))
        res = g.numpy()
        lens, pca = g.lens(w.n, 2)
        offs_g, pts_g = g.cover().numpy()
        labels, core = g.clusters().numpy(len(pts_g))
        st = g.stats()
    d = w.d
    mu, V = pca[:d], np.stack([pca[d:2 * d], pca[2 * d:3 * d]])
    for j in range(2):
        assert 1.0 - abs(V[j] @ oV[j]) <= 1e-6, j
        assert np.array_equal(lens[:, j], oracle.lens_project(w.X, mu, V[j])), j
    offs, pts = oracle.cover(lens, w.n_intervals, w.overlap)
    assert np.array_equal(offs, offs_g) and np.array_equal(pts, pts_g)
    sizes = np.diff(offs)
    assert len(sizes) == 900
    nonempty = np.nonzero(sizes)[0]
    small = nonempty[sizes[nonempty] <= 20_000]
    rng = np.random.default_rng(3)
    picks = {int(nonempty[np.argmin(sizes[nonempty])]),
             int(nonempty[np.argsort(sizes[nonempty])[len(nonempty) // 2]])}
    picks |= {int(e) for e in rng.choice(small, 2, replace=False)}
    for e in sorted(picks):
        s, t = offs[e], offs[e + 1]
        if sizes[e] > 40_000:
            continue
        _, c, lab, ties = oracle.dbscan(w.X, pts[s:t], w.eps, w.min_pts)
        assert ties == 0, e
        assert np.array_equal(core[s:t], c), e
        assert np.array_equal(labels[s:t], lab), e
    # the largest element by sampled rows
    e = int(np.argmax(sizes))
    s, t = offs[e], offs[e + 1]
    members = pts[s:t]
    rows = np.sort(rng.choice(t - s, 1500, replace=False))
    cnt = oracle.density_at(w.X[members], rows, w.eps)
    assert np.array_equal(core[s:t][rows], cnt >= w.min_pts)
    lab = labels[s:t]
    pos = {int(p): i for i, p in enumerate(members)}
    for i in rows:
        l = int(lab[i])
        if core[s + i]:
            # canonical id: a core point of the element at or below this one, its own label
            assert 0 <= l <= int(members[i]) and core[s + pos[l]] and lab[pos[l]] == l
        elif l >= 0:
            assert core[s + pos[l]] and lab[pos[l]] == l
    assert st["near_ties"] == 0
    _check_nodes(res, w.n)
