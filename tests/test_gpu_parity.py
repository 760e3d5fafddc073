"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

The L2 lens is the exact sum of squares rounded once, then a correctly
rounded square root: it must equal sqrt(fsum(x_k^2)) bit for bit and lie
within 1e-12 relative of the oracle's sequential double sum. Every other
comparison is exact: coordinate and projection lenses, the cover
membership, per-slot core flags and cluster labels, node memberships and
edges are equal element by element. The oracle is fed the GPU's lens (and,
for principal-component lenses, checked against the GPU's basis), so a lens
rounding difference could not hide a clustering difference."""
import functools
import math

import numpy as np
import pytest

import oracle
from paper_2011_03209_gb300 import synth

torch = pytest.importorskip("torch")
mg = pytest.importorskip("paper_2011_03209_gb300")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = mg.Context(0)
    c.set_timing(True)
    yield c
    c.close()


def run_gpu(ctx, X, kinds, args, nint, ov, eps, min_pts, prec=mg.FP32, cover_kind=mg.COVER_UNIFORM):
    Xd = torch.from_numpy(np.ascontiguousarray(X)).to("cuda:0")
    g = mg.mapper_graph(ctx, Xd, mg.params(kinds, args, nint, ov, eps, min_pts, prec, cover_kind))
    out = g.numpy()
    out["lens"], out["pca"] = g.lens(X.shape[0], len(kinds))
    out["elem_offsets"], out["elem_points"] = g.cover().numpy()
    out["labels"], out["core"] = g.clusters().numpy(len(out["elem_points"]))
    out["stats"] = g.stats()
    return out


def assert_l2_lens(X, f):
    """L2 lens: correctly rounded exact sum (math.fsum of the squares, which
    are exact in double), and 1e-12 relative of the oracle's sequential sum."""
    X64 = np.asarray(X, dtype=np.float64)
    exact = np.array([np.sqrt(math.fsum(r * r)) for r in X64])
    assert np.array_equal(f, exact)
    ref = oracle.lens_l2(np.asarray(X, dtype=np.float32))
    assert np.all(np.abs(f - ref) <= 1e-12 * np.abs(ref))


def assert_same_graph(X, res, nint, ov, eps, min_pts, balanced=False):
    ref = oracle.mapper_graph(X, res["lens"], nint, ov, eps, min_pts, balanced=balanced)
    for k in ("elem_offsets", "elem_points", "core", "labels", "node_offsets", "node_members",
              "node_elem", "edges"):
        assert np.array_equal(np.asarray(res[k]), np.asarray(ref[k])), k
    assert res["stats"]["near_ties"] == ref["near_ties"]
    return ref


def _eps(X, q, seed):
    if X.shape[0] < 3:
        return 0.5
    return synth.eps_at_percentile(X, q, seed, n_pairs=min(2000, X.shape[0] * 8))


TINY = [
    # n, d, seed, n_int, overlap, q, min_pts
    (1, 3, 0, 4, 0.3, 10, 1),
    (2, 1, 1, 2, 0.0, 50, 2),
    (3, 2, 2, 3, 0.5, 40, 2),
    (17, 5, 3, 5, 0.25, 20, 3),
    (64, 8, 4, 6, 0.3, 10, 4),
    (129, 33, 5, 3, 0.2, 15, 5),
    (300, 2, 6, 10, 0.4, 5, 3),
    (257, 70, 7, 4, 0.1, 8, 2),
    (400, 16, 8, 1, 0.0, 3, 6),
]


PRECISIONS = [mg.FP32, mg.BF16, mg.BF16X1, mg.FP8]


@pytest.mark.parametrize("prec", PRECISIONS)
@pytest.mark.parametrize("n,d,seed,n_int,ov,q,min_pts", TINY)
def test_tiny_l2(ctx, n, d, seed, n_int, ov, q, min_pts, prec):
    X = synth.tiny_random(n, d, seed, scale=2.0)
    eps = _eps(X, q, seed)
    res = run_gpu(ctx, X, (0,), (0,), (n_int,), (ov,), eps, min_pts, prec)
    assert_l2_lens(X, res["lens"][:, 0])
    assert_same_graph(X, res, (n_int,), (ov,), eps, min_pts)


@pytest.mark.parametrize("prec", PRECISIONS)
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_duplicates_min_pts_one_coord_lens(ctx, seed, prec):
    X = synth.tiny_random(350, 4, seed, dup_frac=0.3)
    eps = _eps(X, 5, seed)
    res = run_gpu(ctx, X, (1,), (2,), (7,), (0.35,), eps, 1, prec)
    assert np.array_equal(res["lens"][:, 0], X[:, 2].astype(np.float64))
    assert_same_graph(X, res, (7,), (0.35,), eps, 1)


def test_constant_lens_and_min_pts_above_size(ctx):
    X = synth.tiny_random(200, 3, 9)
    X[:, 1] = 0.25                                   # every lens value equal
    res = run_gpu(ctx, X, (1,), (1,), (5,), (0.2,), 0.3, 4)
    assert res["elem_offsets"][1] == 200 and res["elem_offsets"][-1] == 200
    assert_same_graph(X, res, (5,), (0.2,), 0.3, 4)
    res = run_gpu(ctx, X, (0,), (0,), (5,), (0.2,), 0.3, 500)   # minPts > n: all noise
    assert len(res["node_elem"]) == 0 and len(res["edges"]) == 0
    assert_same_graph(X, res, (5,), (0.2,), 0.3, 500)


def test_many_empty_elements(ctx):
    # three tight blobs 50 apart along axis 0, coordinate lens on that axis:
    # most of the 97 intervals hold no point
    X = synth.tiny_random(120, 4, 2, scale=0.4)
    X[:, 0] += np.repeat(np.array([0.0, 50.0, 100.0], dtype=np.float32), 40)
    res = run_gpu(ctx, X, (1,), (0,), (97,), (0.15,), 0.5, 3)
    sizes = np.diff(res["elem_offsets"])
    assert (sizes == 0).sum() > 80
    assert_same_graph(X, res, (97,), (0.15,), 0.5, 3)


def test_cover_rounding_gap_closed(ctx, golden_dir):
    """The hand-worked case where rounding leaves b_k one ulp below a_{k+1}
    (tests/golden/cover_intervals.json, "rounding_gap"): the device cover
    closes the gap as the oracle does, so the point at a_{k+1} lies in both
    elements."""
    import json
    import os
    c = json.load(open(os.path.join(golden_dir, "cover_intervals.json")))["rounding_gap"]
    lens = torch.tensor([[float.fromhex(x)] for x in c["lens"]], dtype=torch.float64, device="cuda:0")
    offs, pts = mg.mapper_cover(ctx, lens, (c["n"],), (c["p"],)).numpy()
    assert [pts[offs[e]:offs[e + 1]].tolist() for e in range(c["n"])] == c["elements"]


@pytest.mark.parametrize("prec", PRECISIONS)
@pytest.mark.parametrize("seed", [0, 1])
def test_2d_cover(ctx, seed, prec):
    X = synth.tiny_random(900, 6, seed, scale=3.0)
    eps = _eps(X, 4, seed)
    res = run_gpu(ctx, X, (1, 0), (0, 0), (6, 5), (0.3, 0.2), eps, 4, prec)
    assert_same_graph(X, res, (6, 5), (0.3, 0.2), eps, 4)


def test_circle_cycle_graph(ctx):
    X = synth.circle(720)
    res = run_gpu(ctx, X, (1,), (1,), (6,), (0.3,), 0.05, 2)
    ref = assert_same_graph(X, res, (6,), (0.3,), 0.05, 2)
    assert len(ref["node_elem"]) == 10 and len(ref["edges"]) == 10


@pytest.mark.parametrize("d", [1, 7, 33, 256, 700])
def test_l2_lens_exponent_range(ctx, d):
    """L2 lens over rows mixing magnitudes from subnormal to near overflow,
    zero rows and ragged widths; X holding an Inf or a NaN is rejected."""
    rng = np.random.default_rng(d)
    n = 300
    X = (rng.standard_normal((n, d)) * np.exp2(rng.integers(-140, 120, (n, d)))).astype(np.float32)
    X[5] = 0.0
    X[6, 0] = np.float32(1e-45)                      # a lone subnormal
    X[7] = np.float32(3e38) * (rng.random(d) < 0.5)  # near the float maximum
    f, _ = mg.mapper_lens(ctx, torch.from_numpy(X).to("cuda:0"), (0,), (0,))
    f = f.cpu().numpy()[:, 0]
    assert f[5] == 0.0
    assert_l2_lens(X, f)
    for bad in (np.inf, np.nan):
        Y = X.copy()
        Y[8, d // 2] = bad
        with pytest.raises(mg.MapperError):
            mg.mapper_lens(ctx, torch.from_numpy(Y).to("cuda:0"), (0,), (0,))


@pytest.mark.parametrize("prec", [mg.BF16, mg.FP32])
@pytest.mark.parametrize("n,d,seed", [(1, 3, 0), (2, 5, 1), (300, 7, 2), (3000, 64, 3)])
def test_eccentricity_lens(ctx, n, d, seed, prec):
    """Eccentricity filter (exponent 2) within 1e-12 relative of the oracle's
    direct O(n^2 d) form; the graph on it equals the oracle's."""
    X = synth.gaussian_mixture(n, d, 3, seed=60 + seed, centre_box=4.0, std_lo=0.5, std_hi=1.0,
                               anisotropic=False) if n > 2 else synth.tiny_random(n, d, seed, scale=3.0)
    eps = _eps(X, 8, seed)
    res = run_gpu(ctx, X, (mg.LENS_ECC,), (0,), (7,), (0.3,), eps, 4, prec)
    ref = oracle.lens_ecc2(X)
    assert np.all(np.abs(res["lens"][:, 0] - ref) <= 1e-12 * np.abs(ref))
    assert_same_graph(X, res, (7,), (0.3,), eps, 4)


def test_eccentricity_with_l2_2d_cover(ctx):
    X = synth.gaussian_mixture(2500, 16, 4, seed=64, centre_box=5.0, std_lo=0.5, std_hi=1.0,
                               anisotropic=True)
    eps = _eps(X, 6, 64)
    res = run_gpu(ctx, X, (mg.LENS_ECC, mg.LENS_L2), (0, 0), (5, 6), (0.25, 0.2), eps, 5, mg.BF16)
    np.testing.assert_allclose(res["lens"][:, 0], oracle.lens_ecc2(X), rtol=1e-12, atol=0)
    assert_l2_lens(X, res["lens"][:, 1])
    assert_same_graph(X, res, (5, 6), (0.25, 0.2), eps, 5)


@pytest.mark.parametrize("prec", [mg.BF16, mg.FP32])
@pytest.mark.parametrize("n,d,seed,n_int,ov", [(1, 3, 0, 4, 0.25), (2, 4, 1, 3, 0.2), (5, 2, 2, 7, 0.5),
                                               (3000, 12, 3, 9, 0.3), (2000, 8, 4, 1, 0.0)])
def test_balanced_cover(ctx, n, d, seed, n_int, ov, prec):
    """Balanced cover (uniform cover of the filter's ranks): memberships equal
    the oracle's bit for bit, and so does the graph."""
    X = (synth.gaussian_mixture(n, d, 4, seed=70 + seed, centre_box=5.0, std_lo=0.5, std_hi=1.0,
                                anisotropic=False) if n > 5 else synth.tiny_random(n, d, seed, scale=2.0))
    eps = _eps(X, 6, seed)
    res = run_gpu(ctx, X, (0,), (0,), (n_int,), (ov,), eps, 4, prec, mg.COVER_BALANCED)
    offs, pts = oracle.cover(res["lens"], (n_int,), (ov,), balanced=True)
    assert np.array_equal(res["elem_offsets"], offs) and np.array_equal(res["elem_points"], pts)
    assert_same_graph(X, res, (n_int,), (ov,), eps, 4, balanced=True)


def test_balanced_cover_2d_with_ties(ctx):
    """2D balanced cover on a coordinate filter with many equal values (ties
    sit on both sides of a boundary) and the L2 filter."""
    X = synth.gaussian_mixture(2500, 6, 5, seed=77, centre_box=5.0, std_lo=0.5, std_hi=1.0, anisotropic=True)
    X[:, 1] = np.round(X[:, 1])                      # a handful of distinct values
    eps = _eps(X, 5, 77)
    res = run_gpu(ctx, X, (mg.LENS_COORD, mg.LENS_L2), (1, 0), (6, 5), (0.3, 0.2), eps, 5, mg.BF16,
                  mg.COVER_BALANCED)
    offs, pts = oracle.cover(res["lens"], (6, 5), (0.3, 0.2), balanced=True)
    assert np.array_equal(res["elem_offsets"], offs) and np.array_equal(res["elem_points"], pts)
    assert_same_graph(X, res, (6, 5), (0.3, 0.2), eps, 5, balanced=True)


@pytest.mark.parametrize("kinds,args", [((0,), (0,)), ((1, 0), (3, 0)), ((2,), (0,))])
@pytest.mark.parametrize("pinned", [False, True])
def test_host_input_equals_device_input(ctx, kinds, args, pinned):
    """X given in host memory (pageable or pinned; copied in chunks beside the
    filter when the filter is row-local) gives the device-input graph."""
    X = synth.gaussian_mixture(5003, 20, 4, seed=81, centre_box=5.0, std_lo=0.5, std_hi=1.0,
                               anisotropic=False)
    eps = _eps(X, 5, 81)
    nint = (8,) * len(kinds)
    ov = (0.3,) * len(kinds)
    prm = mg.params(kinds, args, nint, ov, eps, 5, mg.BF16)
    dev = mg.mapper_graph(ctx, torch.from_numpy(X).to("cuda:0"), prm)
    host = torch.from_numpy(X).pin_memory().numpy() if pinned else X
    hst = mg.mapper_graph(ctx, host, prm)
    a, b = dev.numpy(), hst.numpy()
    for k in ("node_offsets", "node_members", "node_elem", "edges"):
        assert np.array_equal(a[k], b[k]), k
    la, _ = dev.lens(X.shape[0], len(kinds))
    lb, _ = hst.lens(X.shape[0], len(kinds))
    assert np.array_equal(la, lb)


def test_host_strided_input_equals_device_input(ctx):
    """Host rows with a pitch above d (a column slice of a wider CPU tensor)
    take the two-dimensional chunked copy; the graph and the lens equal those
    of the device input."""
    X = synth.gaussian_mixture(4099, 13, 4, seed=83, centre_box=5.0, std_lo=0.5, std_hi=1.0,
                               anisotropic=False)
    wide = np.zeros((X.shape[0], 16), dtype=np.float32)
    wide[:, :13] = X
    eps = _eps(X, 5, 83)
    prm = mg.params((0,), (0,), (8,), (0.3,), eps, 5, mg.BF16)
    dev = mg.mapper_graph(ctx, torch.from_numpy(X).to("cuda:0"), prm)
    hst = mg.mapper_graph(ctx, torch.from_numpy(wide)[:, :13], prm)
    a, b = dev.numpy(), hst.numpy()
    for k in ("node_offsets", "node_members", "node_elem", "edges"):
        assert np.array_equal(a[k], b[k]), k
    la, _ = dev.lens(X.shape[0], 1)
    lb, _ = hst.lens(X.shape[0], 1)
    assert np.array_equal(la, lb)


def test_pca_lens_basis_and_bits(ctx):
    X = synth.gaussian_mixture(6000, 12, 5, seed=4, centre_box=5.0, std_lo=0.3, std_hi=1.5,
                               anisotropic=True)
    eps = _eps(X, 2, 4)
    res = run_gpu(ctx, X, (2, 2), (0, 1), (8, 6), (0.25, 0.25), eps, 5)
    d = X.shape[1]
    mu, V = res["pca"][:d], res["pca"][d:].reshape(-1, d)
    omu, oV, _ = oracle.pca(X, 2)
    np.testing.assert_allclose(mu, omu, rtol=1e-12, atol=1e-12)
    for c in range(2):
        assert 1.0 - abs(V[c] @ oV[c]) <= 1e-6
        assert V[c][np.argmax(np.abs(V[c]))] > 0
    for c in range(2):                                 # lens bits given the GPU basis
        assert np.array_equal(res["lens"][:, c], oracle.lens_project(X, mu, V[c]))
    assert_same_graph(X, res, (8, 6), (0.25, 0.25), eps, 5)


@pytest.mark.parametrize("prec", PRECISIONS)
@pytest.mark.parametrize("d", [300, 520])
def test_wide_rows_exact(ctx, d, prec):
    """Rows wider than 256 columns: the tile statistics go through the
    gathered FP32 rows, the tensor-core operands span more K blocks."""
    X = synth.gaussian_mixture(3000, d, 6, seed=40 + d, centre_box=4.0, std_lo=0.4, std_hi=1.0,
                               anisotropic=True, noise_frac=0.05)
    eps = _eps(X, 4, d)
    res = run_gpu(ctx, X, (0,), (0,), (6,), (0.3,), eps, 6, prec)
    assert_l2_lens(X, res["lens"][:, 0])
    ref = assert_same_graph(X, res, (6,), (0.3,), eps, 6)
    assert ref["near_ties"] == 0 and len(ref["node_elem"]) > 0


@pytest.mark.parametrize("prec", PRECISIONS)
@pytest.mark.parametrize("d,pad", [(37, 3), (64, 1), (130, 6)])
def test_strided_rows_exact(ctx, d, pad, prec):
    """X as a column slice of a wider array (row stride ld = d + pad): rows
    re-decided from X use unaligned scalar loads."""
    X = synth.gaussian_mixture(4000, d, 5, seed=50 + d, centre_box=5.0, std_lo=0.5, std_hi=1.2,
                               anisotropic=False, noise_frac=0.05)
    wide = np.zeros((X.shape[0], d + pad), dtype=np.float32)
    wide[:, :d] = X
    wide[:, d:] = 7.0                                  # never read
    Xd = torch.from_numpy(wide).to("cuda:0")[:, :d]
    assert Xd.stride(0) == d + pad
    eps = _eps(X, 5, d)
    g = mg.mapper_graph(ctx, Xd, mg.params((0,), (0,), (8,), (0.25,), eps, 5, prec))
    res = g.numpy()
    res["lens"], _ = g.lens(X.shape[0], 1)
    res["elem_offsets"], res["elem_points"] = g.cover().numpy()
    res["labels"], res["core"] = g.clusters().numpy(len(res["elem_points"]))
    res["stats"] = g.stats()
    assert_l2_lens(X, res["lens"][:, 0])
    assert_same_graph(X, res, (8,), (0.25,), eps, 5)


@pytest.mark.parametrize("prec", PRECISIONS)
def test_blobs_circle_5k_exact(ctx, prec):
    w = synth.blobs_circle_5k()
    res = run_gpu(ctx, w.X, w.lens_kind, w.lens_arg, w.n_intervals, w.overlap, w.eps, w.min_pts, prec)
    ref = assert_same_graph(w.X, res, w.n_intervals, w.overlap, w.eps, w.min_pts)
    assert res["stats"]["near_ties"] == 0 and ref["near_ties"] == 0
    assert len(ref["node_elem"]) > 0


@pytest.mark.parametrize("prec", PRECISIONS)
def test_mixture_100k_d64_exact(ctx, prec):
    w = synth.mixture_100k()
    res = run_gpu(ctx, w.X, w.lens_kind, w.lens_arg, w.n_intervals, w.overlap, w.eps, w.min_pts, prec)
    d = w.d
    omu, oV, _ = oracle.pca(w.X, 1)
    assert 1.0 - abs(res["pca"][d:2 * d] @ oV[0]) <= 1e-6
    ref = assert_same_graph(w.X, res, w.n_intervals, w.overlap, w.eps, w.min_pts)
    assert ref["near_ties"] == 0
    assert len(ref["node_elem"]) > 10 and len(ref["edges"]) > 0


@functools.lru_cache(maxsize=1)
def _clusters_1m():
    return synth.clusters_1m_d256()


def _check_graph_properties(res, n_points):
    """Properties that hold at any size, checked on the GPU's own output."""
    no, nm, ne, E = res["node_offsets"], res["node_members"], res["node_elem"], res["edges"]
    N = len(ne)
    assert np.all(np.diff(no) > 0)
    node_of = np.repeat(np.arange(N), np.diff(no))
    # members ascending within a node; nodes ordered by element
    same = node_of[1:] == node_of[:-1]
    assert np.all(nm[1:][same] > nm[:-1][same])
    assert np.all(np.diff(ne) >= 0)
    # nodes of one element are disjoint
    key = ne[node_of].astype(np.int64) * n_points + nm
    assert len(np.unique(key)) == len(key)
    # edge {u, v} iff some point lies in both: rebuild from memberships
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


@pytest.mark.parametrize("prec", [mg.BF16, mg.BF16X1, mg.FP8])
def test_pass1_shapes_agree(prec):
    """Both pass-1 product shapes (one tile pair per item, N = 128; two pairs
    sharing tile A, N = 256) and the autotuner's pick give the same exact
    graph, equal to the oracle's."""
    w = synth.mixture_100k()
    Xd = torch.from_numpy(w.X).to("cuda:0")
    prm = mg.params(w.lens_kind, w.lens_arg, w.n_intervals, w.overlap, w.eps, w.min_pts, prec)
    outs = []
    for tile_n in (128, 256, 0):
        with mg.Context(0) as c:
            c.set_pass1_tile_n(tile_n)
            g = c_graph = mg.mapper_graph(c, Xd, prm)
            st = g.stats()
            assert st["tile_pairs_tc"] > 0
            assert st["pass1_tile_n"] in ((128, 256) if tile_n == 0 else (tile_n,))
            out = g.numpy()
            out["lens"], out["pca"] = g.lens(w.n, 1)
            out["elem_offsets"], out["elem_points"] = g.cover().numpy()
            out["labels"], out["core"] = g.clusters().numpy(len(out["elem_points"]))
            out["stats"] = st
            outs.append(out)
            del g, c_graph
    for o in outs[1:]:
        for k in ("elem_points", "core", "labels", "node_offsets", "node_members", "node_elem", "edges"):
            assert np.array_equal(o[k], outs[0][k]), k
    assert_same_graph(w.X, outs[0], w.n_intervals, w.overlap, w.eps, w.min_pts)
    with mg.Context(0) as c:
        with pytest.raises(mg.MapperError):
            c.set_pass1_tile_n(64)


@pytest.mark.parametrize("first", [mg.BF16, mg.FP8])
@pytest.mark.parametrize("tile_n", [128, 256])
def test_two_phase_count_pass_equals_three_products(tile_n, first):
    """The two-phase count pass (a first screen of one BF16 product, or of
    three FP8 products, then three BF16 products for the 32 x 32 blocks
    holding a pair inside the first screen's band) gives the graph of one
    phase (three products everywhere; FP8: its band re-decided in FP64) and
    the oracle's."""
    w = synth.mixture_100k()
    Xd = torch.from_numpy(w.X).to("cuda:0")
    prm = mg.params(w.lens_kind, w.lens_arg, w.n_intervals, w.overlap, w.eps, w.min_pts, first)
    outs = []
    for mode in (1, 2, 3):
        with mg.Context(0) as c:
            c.set_pass1_tile_n(tile_n)
            c.set_pass1_screen(mode)
            g = mg.mapper_graph(c, Xd, prm)
            st = g.stats()
            out = g.numpy()
            out["lens"], out["pca"] = g.lens(w.n, 1)
            out["elem_offsets"], out["elem_points"] = g.cover().numpy()
            out["labels"], out["core"] = g.clusters().numpy(len(out["elem_points"]))
            out["stats"] = st
            outs.append(out)
            del g
    one, three, mixed = outs
    assert one["stats"]["tile_pairs_screen1"] == one["stats"]["tile_pairs_tc"] + one["stats"]["tile_pairs_cross"]
    assert 0 < one["stats"]["tile_pairs_redo"] < one["stats"]["tile_pairs_screen1"]
    assert 0 < one["stats"]["redo_blocks"] and one["stats"]["redo_parts"] <= one["stats"]["redo_blocks"]
    assert three["stats"]["tile_pairs_screen1"] == 0 and three["stats"]["tile_pairs_redo"] == 0
    # the first phase of mode 3 defers every block its extremes leave open:
    # a superset of mode 1's blocks
    assert mixed["stats"]["redo_blocks"] >= one["stats"]["redo_blocks"]
    # every tile pair is counted once: the same pairs screened either way
    assert one["stats"]["count_kernel_pairs"] == three["stats"]["count_kernel_pairs"]
    assert mixed["stats"]["count_kernel_pairs"] == three["stats"]["count_kernel_pairs"]
    for k in ("elem_points", "core", "labels", "node_offsets", "node_members", "node_elem", "edges"):
        assert np.array_equal(one[k], three[k]), k
        assert np.array_equal(mixed[k], three[k]), k
    assert_same_graph(w.X, one, w.n_intervals, w.overlap, w.eps, w.min_pts)
    with mg.Context(0) as c:
        with pytest.raises(mg.MapperError):
            c.set_pass1_screen(4)


@pytest.mark.parametrize("first", [mg.BF16, mg.FP8])
def test_default_screen_samples_the_first_phase(first):
    """The default count-pass screen samples the first phase on every 64th
    tile pair and takes one phase or two from the fractions that defer a
    block (per bin of the tile-pair statistic for the BF16 first phase,
    overall for the FP8 one); either way the graph is the one of three
    products everywhere."""
    w = synth.mixture_100k()
    Xd = torch.from_numpy(w.X).to("cuda:0")
    prm = mg.params(w.lens_kind, w.lens_arg, w.n_intervals, w.overlap, w.eps, w.min_pts, first)
    outs = []
    for mode in (0, 2):
        with mg.Context(0) as c:
            c.set_pass1_screen(mode)
            g = mg.mapper_graph(c, Xd, prm)
            out = g.numpy()
            out["stats"] = g.stats()
            outs.append(out)
            del g
    auto, three = outs
    st = auto["stats"]
    assert 0.0 <= st["pass1_sample_deferred"] <= 1.0
    if first != mg.BF16:
        assert st["pass1_phases"] == (1 if st["pass1_sample_deferred"] > 0.35 else 2)
    assert st["pass1_phases"] in (1, 2)
    assert (st["tile_pairs_screen1"] > 0) == (st["pass1_phases"] == 2)
    assert st["pass1_phases"] == 2 or st["tile_pairs_direct"] == 0
    assert three["stats"]["pass1_phases"] == 1 and three["stats"]["pass1_sample_deferred"] == -1.0
    for k in ("node_offsets", "node_members", "node_elem", "edges"):
        assert np.array_equal(auto[k], three[k]), k


@pytest.mark.parametrize("prec", [mg.BF16, mg.BF16X1, mg.FP8])
@pytest.mark.parametrize("cap", [1, 16])
def test_band_queue_overflow_exact(prec, cap):
    """A band queue far smaller than the band: the pairs past its capacity are
    decided in FP64 inside the tensor-core kernels (count and union passes)
    instead of by the recheck kernel, and the graph still equals the
    oracle's."""
    w = synth.mixture_100k(40_000)
    Xd = torch.from_numpy(w.X).to("cuda:0")
    prm = mg.params(w.lens_kind, w.lens_arg, w.n_intervals, w.overlap, w.eps, w.min_pts, prec)
    with mg.Context(0) as c:
        c.set_band_queue_cap(cap)
        g = mg.mapper_graph(c, Xd, prm)
        st = g.stats()
        assert st["tile_pairs_tc"] > 0 and st["band_pairs"] > 4 * cap
        out = g.numpy()
        out["lens"], out["pca"] = g.lens(w.n, 1)
        out["elem_offsets"], out["elem_points"] = g.cover().numpy()
        out["labels"], out["core"] = g.clusters().numpy(len(out["elem_points"]))
        out["stats"] = st
        with pytest.raises(mg.MapperError):
            c.set_band_queue_cap(-1)
    assert_same_graph(w.X, out, w.n_intervals, w.overlap, w.eps, w.min_pts)


@pytest.mark.slow
@pytest.mark.parametrize("prec", [mg.BF16, mg.FP32, mg.FP8])
def test_clusters_1m_d256_sampled(ctx, prec):
    """Full-size 1M x 256 workload as the benchmark runs it: lens rows, the
    whole cover, and the DBSCAN of sampled elements against the oracle; the
    nerve by its definition."""
    w = _clusters_1m()
    res = run_gpu(ctx, w.X, w.lens_kind, w.lens_arg, w.n_intervals, w.overlap, w.eps, w.min_pts, prec)
    rng = np.random.default_rng(0)
    rows = rng.choice(w.n, 4000, replace=False)
    assert_l2_lens(w.X[rows], res["lens"][rows, 0])
    offs, pts = oracle.cover(res["lens"], w.n_intervals, w.overlap)
    assert np.array_equal(offs, res["elem_offsets"]) and np.array_equal(pts, res["elem_points"])
    sizes = np.diff(offs)
    nonempty = np.nonzero(sizes)[0]
    picks = [nonempty[np.argmin(sizes[nonempty])],
             nonempty[np.argsort(sizes[nonempty])[len(nonempty) // 3]]]
    picks.append(int(rng.choice(nonempty[sizes[nonempty] <= 16000])))
    for e in picks:
        s, t = offs[e], offs[e + 1]
        _, core, label, ties = oracle.dbscan(w.X, pts[s:t], w.eps, w.min_pts)
        assert np.array_equal(res["core"][s:t], core), e
        assert np.array_equal(res["labels"][s:t], label), e
        assert ties == 0
    # the largest element by sampled rows: core flags from the oracle's counts,
    # labels by what every DBSCAN labelling satisfies
    e = int(np.argmax(sizes))
    s, t = offs[e], offs[e + 1]
    members = pts[s:t]
    sample = np.sort(rng.choice(t - s, 400, replace=False))
    cnt = oracle.density_at(w.X[members], sample, w.eps)
    assert np.array_equal(res["core"][s:t][sample], cnt >= w.min_pts)
    lab = res["labels"][s:t]
    pos = {int(p): i for i, p in enumerate(members)}
    for i in sample:
        l = int(lab[i])
        if res["core"][s + i]:
            assert 0 <= l <= int(members[i]) and res["core"][s + pos[l]] and lab[pos[l]] == l
        elif l >= 0:
            assert res["core"][s + pos[l]] and lab[pos[l]] == l
    assert res["stats"]["near_ties"] == 0
    _check_graph_properties(res, w.n)


def test_default_screen_sends_deferring_bins_to_three_products():
    """On the 256-column clusters cloud the default screen's sample finds bins
    of the tile-pair statistic whose pairs all defer a block; those pairs skip
    the first phase. The graph equals the one of three products everywhere,
    the first phase screens exactly the other tensor-core pairs, and two
    sampled elements equal the oracle's DBSCAN."""
    w = synth.clusters_1m_d256(200_000)
    Xd = torch.from_numpy(w.X).to("cuda:0")
    prm = mg.params(w.lens_kind, w.lens_arg, w.n_intervals, w.overlap, w.eps, w.min_pts, mg.BF16)
    outs = []
    for mode in (0, 2):
        with mg.Context(0) as c:
            c.set_pass1_screen(mode)
            g = mg.mapper_graph(c, Xd, prm)
            out = g.numpy()
            out["stats"] = g.stats()
            out["elem_offsets"], out["elem_points"] = g.cover().numpy()
            out["labels"], out["core"] = g.clusters().numpy(len(out["elem_points"]))
            outs.append(out)
            del g
    auto, three = outs
    st = auto["stats"]
    assert st["pass1_phases"] == 2 and st["tile_pairs_direct"] > 0
    assert st["tile_pairs_screen1"] == st["tile_pairs_tc"] - st["tile_pairs_direct"] + st["tile_pairs_cross"]
    assert three["stats"]["tile_pairs_direct"] == 0
    for k in ("node_offsets", "node_members", "node_elem", "edges", "labels", "core"):
        assert np.array_equal(auto[k], three[k]), k
    offs, pts = auto["elem_offsets"], auto["elem_points"]
    sizes = np.diff(offs)
    for el in np.nonzero((sizes > 500) & (sizes <= 3000))[0][:2]:
        s0, t0 = offs[el], offs[el + 1]
        _, rc, rl, _ = oracle.dbscan(w.X, pts[s0:t0], w.eps, w.min_pts)
        assert np.array_equal(rc, auto["core"][s0:t0]) and np.array_equal(rl, auto["labels"][s0:t0]), el
