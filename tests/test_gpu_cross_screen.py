"""Mixed tile pairs across two segments of one element screened on the tensor
cores (rows centred per element, a second BF16 operand set) give the same
exact graph as on CUDA cores and as the oracle: forced on and off on small
and medium clouds, and picked automatically for an element holding scattered
points (wide tile spheres, many such pairs). When such pairs are many, the
classification first bounds the outlier tiles' distance to every segment of
their element, which certifies far noise all-out; outliers in a halo around
the clusters keep pairs mixed."""
import numpy as np
import pytest

import oracle
from paper_2011_03209_gb300 import synth

torch = pytest.importorskip("torch")
mg = pytest.importorskip("paper_2011_03209_gb300")

pytestmark = pytest.mark.gpu


def _graph(ctx, X, kinds, args, nint, ov, eps, min_pts, prec):
    g = mg.mapper_graph(ctx, torch.from_numpy(np.ascontiguousarray(X)).to("cuda:0"),
                        mg.params(kinds, args, nint, ov, eps, min_pts, prec))
    out = g.numpy()
    out["lens"], _ = g.lens(X.shape[0], len(kinds))
    out["elem_offsets"], out["elem_points"] = g.cover().numpy()
    out["labels"], out["core"] = g.clusters().numpy(len(out["elem_points"]))
    out["stats"] = g.stats()
    return out


def _check(X, res, nint, ov, eps, min_pts):
    ref = oracle.mapper_graph(X, res["lens"], nint, ov, eps, min_pts)
    for k in ("elem_points", "core", "labels", "node_offsets", "node_members", "node_elem", "edges"):
        assert np.array_equal(np.asarray(res[k]), np.asarray(ref[k])), k
    assert res["stats"]["near_ties"] == ref["near_ties"]
    return ref


def _scattered(n_clustered, n_noise, d, seed, halo=0):
    """Gaussian clusters plus points uniform in a box twice their extent and,
    optionally, `halo` copies of cluster points pushed a few eps away."""
    X = synth.gaussian_mixture(n_clustered, d, 6, seed=seed, centre_box=6.0, std_lo=0.4, std_hi=0.9,
                               anisotropic=False)
    rng = np.random.default_rng(seed + 1)
    lo, hi = X.min(axis=0) * 2.0, X.max(axis=0) * 2.0
    parts = [X, rng.uniform(lo, hi, size=(n_noise, d)).astype(np.float32)]
    if halo:
        r = 5.0 * synth.eps_at_percentile(X, 3, seed, n_pairs=6000)
        u = rng.standard_normal((halo, d))
        u *= r / np.linalg.norm(u, axis=1, keepdims=True)
        parts.append((X[rng.integers(0, n_clustered, size=halo)] + u).astype(np.float32))
    Y = np.concatenate(parts)
    return np.ascontiguousarray(Y[rng.permutation(Y.shape[0])])


CASES = [
    # n_clustered, n_noise, d, seed, n_int, overlap, min_pts
    (600, 200, 8, 0, 1, 0.0, 4),
    (3000, 1500, 24, 1, 3, 0.3, 5),
    (2500, 900, 130, 2, 2, 0.25, 3),
    (5000, 4000, 64, 3, 1, 0.0, 6),
]


@pytest.mark.parametrize("prec", [mg.BF16, mg.BF16X1])
@pytest.mark.parametrize("case", CASES)
def test_cross_screen_on_off_auto_equal_oracle(case, prec):
    nc, nn, d, seed, nint, ov, min_pts = case
    X = _scattered(nc, nn, d, 40 + seed)
    eps = synth.eps_at_percentile(X, 3, seed, n_pairs=6000)
    outs = {}
    for mode in (0, 1, 2):
        with mg.Context(0) as ctx:
            ctx.set_cross_screen(mode)
            outs[mode] = _graph(ctx, X, (mg.LENS_L2,), (0,), (nint,), (ov,), eps, min_pts, prec)
    assert outs[1]["stats"]["tile_pairs_cross"] == outs[1]["stats"]["tile_pairs_simt"]
    assert outs[2]["stats"]["tile_pairs_cross"] == 0
    for mode in (0, 2):
        for k in ("elem_points", "core", "labels", "node_offsets", "node_members", "edges"):
            assert np.array_equal(outs[mode][k], outs[1][k]), (mode, k)
    ref = _check(X, outs[1], (nint,), (ov,), eps, min_pts)
    assert len(ref["node_elem"]) > 0


def test_cross_screen_auto_rule_for_scattered_element():
    """The automatic choice follows its rule (tensor cores iff the pairs are at
    least 1/32 of the rows) and the graph is the oracle's."""
    X = _scattered(20000, 12000, 48, 77, halo=3000)
    eps = synth.eps_at_percentile(X, 2, 7, n_pairs=20000)
    with mg.Context(0) as ctx:
        res = _graph(ctx, X, (mg.LENS_L2,), (0,), (1,), (0.0,), eps, 5, mg.BF16)
    st = res["stats"]
    assert st["tile_pairs_cross"] == (st["tile_pairs_simt"] if st["tile_pairs_simt"] * 32 >= st["n_rows"] else 0)
    _check(X, res, (1,), (0.0,), eps, 5)


@pytest.mark.parametrize("prec", [mg.BF16, mg.BF16X1])
def test_cross_screen_halo_outliers(prec):
    """Outliers a few eps around the clusters keep cross-segment pairs mixed
    after the outlier bounds: forced onto the tensor cores they give the
    CUDA-core graph and the oracle's."""
    X = _scattered(6000, 1000, 32, 55, halo=2500)
    eps = synth.eps_at_percentile(X, 3, 55, n_pairs=8000)
    outs = {}
    for mode in (1, 2):
        with mg.Context(0) as ctx:
            ctx.set_cross_screen(mode)
            outs[mode] = _graph(ctx, X, (mg.LENS_L2,), (0,), (2,), (0.2,), eps, 4, prec)
    assert outs[1]["stats"]["tile_pairs_cross"] == outs[1]["stats"]["tile_pairs_simt"] > 0
    for k in ("elem_points", "core", "labels", "node_offsets", "node_members", "edges"):
        assert np.array_equal(outs[1][k], outs[2][k]), k
    _check(X, outs[1], (2,), (0.2,), eps, 4)


def test_cross_screen_with_density_lens_2d():
    X = _scattered(4000, 2500, 16, 91)
    r = synth.eps_at_percentile(X, 4, 91, n_pairs=8000)
    eps = synth.eps_at_percentile(X, 3, 92, n_pairs=8000)
    with mg.Context(0) as ctx:
        ctx.set_cross_screen(1)
        prm = mg.params((mg.LENS_DENSITY, mg.LENS_L2), (0, 0), (5, 4), (0.3, 0.2), eps, 4, mg.BF16,
                        lens_param=(r, r))
        g = mg.mapper_graph(ctx, torch.from_numpy(X).to("cuda:0"), prm)
        res = g.numpy()
        lens, _ = g.lens(X.shape[0], 2)
    assert np.array_equal(lens[:, 0], oracle.lens_density(X, r))
    ref = oracle.mapper_graph(X, lens, (5, 4), (0.3, 0.2), eps, 4)
    for k in ("node_offsets", "node_members", "node_elem", "edges"):
        assert np.array_equal(np.asarray(res[k]), np.asarray(ref[k])), k


def test_cross_screen_rejects_bad_mode():
    with mg.Context(0) as ctx:
        for mode in (-1, 3):
            with pytest.raises(mg.MapperError):
                ctx.set_cross_screen(mode)
