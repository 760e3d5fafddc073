"""Single linkage on the GPU (mapper_single_linkage, mapper_forest_cut)
against the FP64 oracle: the minimum spanning forest of every cover
element's eps-graph equals the oracle's Kruskal forest edge for edge (the
same point pairs and the same FP64 d2), ties included, and the forest cut at
a height h gives the oracle's single-linkage clusters, whose mapper graph is
the graph of DBSCAN(h, minPts = 1)."""
import numpy as np
import pytest

import oracle
from paper_2011_03209_gb300 import synth

torch = pytest.importorskip("torch")
mg = pytest.importorskip("paper_2011_03209_gb300")

pytestmark = pytest.mark.gpu


def _oracle_forest(X, offs, pts, eps):
    rows = []
    for e in range(len(offs) - 1):
        u, v, d2 = oracle.msf(X, pts[offs[e]:offs[e + 1]], eps)
        rows += [(e, int(a), int(b), float(w)) for a, b, w in zip(u, v, d2)]
    rows.sort(key=lambda t: (t[0], t[3], t[1], t[2]))
    return rows


def _gpu(ctx, X, kinds, args, nint, ov, eps):
    Xd = torch.from_numpy(np.ascontiguousarray(X)).to("cuda:0")
    lens, _ = mg.mapper_lens(ctx, Xd, kinds, args)
    cover = mg.mapper_cover(ctx, lens, nint, ov)
    forest = mg.mapper_single_linkage(ctx, Xd, cover, eps)
    return Xd, lens.cpu().numpy(), cover, forest


CASES = [
    # n, d, seed, cover (kinds, args, n_intervals, overlap), eps percentile, duplicates
    (700, 5, 0, ((1,), (0,), (6,), (0.3,)), 6.0, 0.0),
    (2500, 32, 1, ((0,), (0,), (9,), (0.25,)), 3.0, 0.0),
    (1800, 3, 2, ((1, 1), (0, 1), (4, 3), (0.2, 0.3)), 10.0, 0.1),
    (300, 2, 3, ((1,), (1,), (1,), (0.0,)), 40.0, 0.0),
]


@pytest.mark.parametrize("n,d,seed,cov,q,dup", CASES)
def test_forest_equals_oracle(n, d, seed, cov, q, dup):
    X = synth.tiny_random(n, d, seed, scale=3.0, dup_frac=dup)
    eps = synth.eps_at_percentile(X, q, seed=seed, n_pairs=20000)
    with mg.Context(0) as ctx:
        _, lens, cover, forest = _gpu(ctx, X, *cov, eps)
        got = forest.numpy()
        offs, pts = cover.numpy()
    ref = _oracle_forest(X, offs, pts, eps)
    assert len(ref) > 0
    gl = list(zip(got["elem"].tolist(), got["u"].tolist(), got["v"].tolist(), got["d2"].tolist()))
    assert gl == ref


def test_ties_on_a_grid_follow_the_index_order():
    # a 12 x 12 grid: every nearest-neighbour distance ties at 1
    g = np.stack(np.meshgrid(np.arange(12.0), np.arange(12.0)), axis=-1).reshape(-1, 2).astype(np.float32)
    rng = np.random.default_rng(7)
    X = g[rng.permutation(len(g))]
    with mg.Context(0) as ctx:
        _, _, cover, forest = _gpu(ctx, X, (1,), (0,), (1,), (0.0,), 1.2)
        got = forest.numpy()
        offs, pts = cover.numpy()
    ref = _oracle_forest(X, offs, pts, 1.2)
    assert len(ref) == len(X) - 1
    assert list(zip(got["elem"].tolist(), got["u"].tolist(), got["v"].tolist(), got["d2"].tolist())) == ref


@pytest.mark.parametrize("frac", [0.4, 0.75, 1.0])
def test_cut_equals_oracle_and_dbscan_min_pts_one(frac):
    X = synth.gaussian_mixture(3000, 16, 6, seed=5, centre_box=6.0, std_lo=0.3, std_hi=1.0, anisotropic=True)
    eps = synth.eps_at_percentile(X, 6.0, seed=5, n_pairs=20000)
    h = eps * frac
    with mg.Context(0) as ctx:
        Xd, lens, cover, forest = _gpu(ctx, X, (1,), (0,), (5,), (0.3,), eps)
        offs, pts = cover.numpy()
        cl = forest.cut(ctx, h)
        lab, core = cl.numpy(len(pts))
        g = mg.mapper_nerve(ctx, cl).numpy()
        dbs = mg.mapper_cluster(ctx, Xd, cover, h, 1, mg.FP32)
        g1 = mg.mapper_nerve(ctx, dbs).numpy()
        with pytest.raises(mg.MapperError):
            forest.cut(ctx, eps * 1.01)
    assert core.all()
    for e in range(len(offs) - 1):
        s, t = offs[e], offs[e + 1]
        u, v, d2 = oracle.msf(X, pts[s:t], eps)
        assert np.array_equal(lab[s:t], oracle.single_linkage(pts[s:t], u, v, d2, h)), e
    for k in ("node_offsets", "node_members", "node_elem", "edges"):
        assert np.array_equal(g[k], g1[k]), k
    ref = oracle.mapper_graph(X, lens, (5,), (0.3,), h, 1)
    for k in ("node_offsets", "node_members", "node_elem", "edges"):
        assert np.array_equal(g[k], ref[k]), k


def test_mixture_100k_sampled_elements():
    w = synth.mixture_100k()
    with mg.Context(0) as ctx:
        _, lens, cover, forest = _gpu(ctx, w.X, w.lens_kind, w.lens_arg, w.n_intervals, w.overlap, w.eps)
        got = forest.numpy()
        offs, pts = cover.numpy()
    sizes = np.diff(offs)
    nonempty = np.nonzero(sizes)[0]
    picks = [int(nonempty[np.argmin(sizes[nonempty])]), int(nonempty[np.argsort(sizes[nonempty])[len(nonempty) // 2]]),
             int(np.argmax(sizes))]
    for e in picks:
        s, t = offs[e], offs[e + 1]
        u, v, d2 = oracle.msf(w.X, pts[s:t], w.eps)
        mine = got["elem"] == e
        assert np.array_equal(got["u"][mine], u) and np.array_equal(got["v"][mine], v), e
        assert np.array_equal(got["d2"][mine], d2), e
