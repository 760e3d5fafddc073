"""Parity of the L-infinity-norm, density and L-infinity-centrality filters
(through the C ABI) with the FP64 oracle. All three are exact (a maximum of
magnitudes; integer counts of the points within distance r; the FP64 distance
of the defining expression to the farthest point), so the lens columns equal
the oracle's bit for bit in every screen precision, and the graphs built on
them equal the oracle's."""
import functools

import numpy as np
import pytest

import oracle
from paper_2011_03209_gb300 import synth

torch = pytest.importorskip("torch")
mg = pytest.importorskip("paper_2011_03209_gb300")

pytestmark = pytest.mark.gpu

PRECISIONS = [mg.FP32, mg.BF16, mg.BF16X1, mg.FP8]


@pytest.fixture(scope="module")
def ctx():
    c = mg.Context(0)
    yield c
    c.close()


def _lens(ctx, X, kinds, args, radii=None, prec=mg.BF16):
    Xd = torch.from_numpy(np.ascontiguousarray(X)).to("cuda:0")
    f, _ = mg.mapper_lens(ctx, Xd, kinds, args, radii, prec)
    return f.cpu().numpy()


def _cloud(n, d, seed):
    if n <= 5:
        return synth.tiny_random(n, d, seed, scale=3.0)
    return synth.gaussian_mixture(n, d, 4, seed=90 + seed, centre_box=5.0, std_lo=0.5, std_hi=1.2,
                                  anisotropic=True, noise_frac=0.03)


def _radius(X, q, seed):
    if X.shape[0] < 3:
        return 0.75
    return synth.eps_at_percentile(X, q, seed, n_pairs=min(4000, X.shape[0] * 8))


@pytest.mark.parametrize("n,d,seed", [(1, 1, 0), (5, 3, 1), (1000, 7, 2), (3000, 256, 3), (513, 300, 4)])
def test_linf_lens_exact(ctx, n, d, seed):
    X = _cloud(n, d, seed)
    X[:, -1] *= -2.0                                      # the largest magnitude often negative
    assert np.array_equal(_lens(ctx, X, (mg.LENS_LINF,), (0,))[:, 0], oracle.lens_linf(X))


def test_linf_lens_strided_rows_and_2d(ctx):
    X = _cloud(2000, 40, 5)
    wide = torch.from_numpy(np.ascontiguousarray(np.pad(X, ((0, 0), (0, 7))))).to("cuda:0")
    f, _ = mg.mapper_lens(ctx, wide[:, :40], (mg.LENS_LINF, mg.LENS_COORD), (0, 3))
    f = f.cpu().numpy()
    assert np.array_equal(f[:, 0], oracle.lens_linf(X))
    assert np.array_equal(f[:, 1], X[:, 3].astype(np.float64))


@pytest.mark.parametrize("bad", [np.nan, np.inf, -np.inf])
def test_linf_lens_rejects_non_finite(ctx, bad):
    X = _cloud(300, 9, 6)
    X[17, 4] = bad
    with pytest.raises(mg.MapperError):
        _lens(ctx, X, (mg.LENS_LINF,), (0,))


@pytest.mark.parametrize("prec", PRECISIONS)
@pytest.mark.parametrize("n,d,seed", [(1, 3, 0), (2, 5, 1), (300, 7, 2), (3000, 64, 3), (2500, 130, 4),
                                      (1200, 300, 5)])
def test_density_lens_exact(ctx, n, d, seed, prec):
    X = _cloud(n, d, seed)
    r = _radius(X, 5, seed)
    got = _lens(ctx, X, (mg.LENS_DENSITY,), (0,), (r,), prec)[:, 0]
    ref = oracle.lens_density(X, r)
    assert np.array_equal(got, ref)
    if n > 100:
        assert ref.max() > 1.0


@pytest.mark.parametrize("prec", [mg.FP32, mg.BF16])
def test_density_lens_extremes_and_duplicates(ctx, prec):
    X = synth.tiny_random(700, 6, 7, scale=2.0, dup_frac=0.2)
    diam = float(np.sqrt(((X.max(axis=0) - X.min(axis=0)).astype(np.float64) ** 2).sum()))
    for r in (1e-6, 0.3, 1.1, 2.0 * diam):
        got = _lens(ctx, X, (mg.LENS_DENSITY,), (0,), (r,), prec)[:, 0]
        assert np.array_equal(got, oracle.lens_density(X, r)), r
    assert np.all(_lens(ctx, X, (mg.LENS_DENSITY,), (0,), (2.0 * diam,), prec)[:, 0] == 700.0)


def test_density_lens_rejects_bad_radius(ctx):
    X = _cloud(200, 4, 8)
    Xd = torch.from_numpy(X).to("cuda:0")
    for radii in (None, (0.0,), (-1.0,), (float("nan"),), (float("inf"),)):
        with pytest.raises(mg.MapperError):
            mg.mapper_lens(ctx, Xd, (mg.LENS_DENSITY,), (0,), radii)


@pytest.mark.parametrize("prec", [mg.FP32, mg.BF16])
def test_density_and_linf_graphs(ctx, prec):
    """2D mapper graph on (density, L-infinity norm) and 1D on density: lens,
    cover, clusters, nodes and edges equal the oracle's."""
    X = _cloud(4000, 16, 9)
    r = _radius(X, 4, 9)
    eps = _radius(X, 3, 19)
    for kinds, nint, ov in (((mg.LENS_DENSITY, mg.LENS_LINF), (6, 5), (0.3, 0.25)),
                            ((mg.LENS_DENSITY,), (12,), (0.35,))):
        prm = mg.params(kinds, (0,) * len(kinds), nint, ov, eps, 4, prec, lens_param=(r,) * len(kinds))
        g = mg.mapper_graph(ctx, torch.from_numpy(X).to("cuda:0"), prm)
        res = g.numpy()
        lens, _ = g.lens(X.shape[0], len(kinds))
        ref_lens = oracle.lens(X, kinds, (0,) * len(kinds), radii=(r,) * len(kinds))
        assert np.array_equal(lens, ref_lens)
        ref = oracle.mapper_graph(X, ref_lens, nint, ov, eps, 4)
        offs, pts = g.cover().numpy()
        assert np.array_equal(offs, ref["elem_offsets"]) and np.array_equal(pts, ref["elem_points"])
        for k in ("node_offsets", "node_members", "node_elem", "edges"):
            assert np.array_equal(np.asarray(res[k]), np.asarray(ref[k])), k
        assert len(ref["node_elem"]) > 2


@functools.lru_cache(maxsize=1)
def _mixture():
    return synth.mixture_100k()


@pytest.mark.parametrize("prec", [mg.FP32, mg.BF16])
def test_density_lens_100k_sampled(ctx, prec):
    """100k x 64 mixture, radius = its DBSCAN eps: sampled rows (and the
    least and most dense) against the oracle's counts at those rows."""
    w = _mixture()
    f = _lens(ctx, w.X, (mg.LENS_DENSITY,), (0,), (w.eps,), prec)[:, 0]
    rng = np.random.default_rng(3)
    rows = np.r_[rng.choice(w.n, 300, replace=False), np.argmin(f), np.argmax(f), 0, w.n - 1]
    assert np.array_equal(f[rows], oracle.density_at(w.X, rows, w.eps))
    assert f.min() >= 1.0 and f.max() > 10.0


@pytest.mark.slow
def test_density_lens_1m_d256_sampled(ctx):
    """The 1M x 256 benchmark cloud, radius = its eps, BF16 screen: sampled
    rows against the oracle."""
    w = synth.clusters_1m_d256()
    f = _lens(ctx, w.X, (mg.LENS_DENSITY,), (0,), (w.eps,), mg.BF16)[:, 0]
    rng = np.random.default_rng(4)
    rows = np.r_[rng.choice(w.n, 40, replace=False), np.argmin(f), np.argmax(f)]
    assert np.array_equal(f[rows], oracle.density_at(w.X, rows, w.eps))


@pytest.mark.parametrize("prec", [mg.BF16, mg.FP32])
@pytest.mark.parametrize("n,d,seed", [(1, 3, 0), (2, 5, 1), (300, 1500, 2), (3000, 64, 3), (5000, 17, 4)])
def test_ecc_inf_lens_exact(ctx, n, d, seed, prec):
    """L-infinity centrality max_y |x - y| equals the oracle's brute force bit
    for bit (rows up to 1500 columns, as §5's gene-expression case), through
    the tensor-core screen (BF16) and the CUDA-core one (FP32)."""
    X = _cloud(n, d, seed)
    got = _lens(ctx, X, (mg.LENS_ECC_INF,), (0,), prec=prec)[:, 0]
    assert np.array_equal(got, oracle.lens_ecc_inf(X))


def test_ecc_inf_lens_far_duplicates_and_2d_graph(ctx):
    """Forty copies of one far point make the 16 largest screened values tie
    for every row (the streaming passes decide them); the 2D graph on
    (L-infinity centrality, a column), as in §5, equals the oracle's."""
    X = _cloud(2500, 12, 7)
    X[100:140] = X[:, :].max(axis=0) * 3.0
    ref = oracle.lens(X, (6, 1), (0, 2))
    for prec in (mg.BF16, mg.FP32):
        got = _lens(ctx, X, (mg.LENS_ECC_INF, mg.LENS_COORD), (0, 2), prec=prec)
        assert np.array_equal(got, ref)
    eps = _radius(X, 4, 7)
    prm = mg.params((mg.LENS_ECC_INF, mg.LENS_COORD), (0, 2), (8, 5), (0.65, 0.5), eps, 2, mg.BF16)
    g = mg.mapper_graph(ctx, torch.from_numpy(X).to("cuda:0"), prm)
    res = g.numpy()
    lens, _ = g.lens(X.shape[0], 2)
    assert np.array_equal(lens, ref)
    rg = oracle.mapper_graph(X, ref, (8, 5), (0.65, 0.5), eps, 2)
    for k in ("node_offsets", "node_members", "node_elem", "edges"):
        assert np.array_equal(np.asarray(res[k]), np.asarray(rg[k])), k
