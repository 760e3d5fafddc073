"""Pins of the oracle's lens and cover against things other than itself:
hand-derived fixtures, closed forms and independent library routines."""
import json
import os

import numpy as np
import pytest

import oracle
from paper_2011_03209_gb300 import synth


def test_l2_lens_closed_form_and_numpy():
    X = np.array([[3.0, 4.0, 0.0], [0.0, 0.0, 0.0], [-1.0, -1.0, -1.0]], dtype=np.float32)
    f = oracle.lens_l2(X)
    assert f[0] == 5.0 and f[1] == 0.0
    assert f[2] == np.sqrt(3.0)
    Y = synth.tiny_random(500, 37, seed=3, scale=20.0) - 10.0
    ref = np.linalg.norm(Y.astype(np.float64), axis=1)
    np.testing.assert_allclose(oracle.lens_l2(Y), ref, rtol=1e-14, atol=0)


def test_eccentricity_closed_forms():
    """Eccentricity with exponent 2, pinned by hand-derived values."""
    # two points at distance 5: each has mean squared distance 25 / 2
    f = oracle.lens_ecc2(np.array([[0.0, 0.0], [3.0, 4.0]], dtype=np.float32))
    np.testing.assert_allclose(f, [5.0 / np.sqrt(2.0)] * 2, rtol=1e-15)
    # {-1, 0, 1} on a line: f(0)^2 = (1 + 0 + 1) / 3, f(+-1)^2 = (0 + 1 + 4) / 3
    f = oracle.lens_ecc2(np.array([[-1.0], [0.0], [1.0]], dtype=np.float32))
    np.testing.assert_allclose(f, [np.sqrt(5 / 3), np.sqrt(2 / 3), np.sqrt(5 / 3)], rtol=1e-15)
    # the n unit vectors of R^n: every pair at distance sqrt(2), so f^2 = 2 (n - 1) / n
    n = 7
    f = oracle.lens_ecc2(np.eye(n, dtype=np.float32))
    np.testing.assert_allclose(f, np.sqrt(2.0 * (n - 1) / n), rtol=1e-15)
    # one point: zero
    assert oracle.lens_ecc2(np.array([[2.5, -1.0, 7.0]], dtype=np.float32))[0] == 0.0


def test_eccentricity_invariants():
    """Translation invariance, and the parallel-axis identity
    mean_y |x - y|^2 = |x - mu|^2 + mean_y |y - mu|^2 (mu the mean)."""
    Y = np.round(synth.tiny_random(400, 11, seed=8, scale=3.0) * 64.0).astype(np.float32) / 64.0
    f = oracle.lens_ecc2(Y)
    shifted = Y + np.float32(2.0)                      # exact: multiples of 1/64 below 8
    np.testing.assert_allclose(oracle.lens_ecc2(shifted), f, rtol=1e-12)
    Y64 = Y.astype(np.float64)
    mu = Y64.mean(axis=0)
    ident = np.sqrt(((Y64 - mu) ** 2).sum(axis=1) + ((Y64 - mu) ** 2).sum(axis=1).mean())
    np.testing.assert_allclose(f, ident, rtol=1e-12)


def test_linf_lens_closed_forms_and_numpy():
    """L-infinity norm of each row: hand values, numpy's ord=inf norm, and the
    norm inequalities |x|_inf <= |x|_2 <= sqrt(d) |x|_inf (equal on scaled unit
    vectors)."""
    X = np.array([[0, 0, 0], [1, -3, 2], [-0.5, 0.25, 0.5], [-7, 7, -7]], dtype=np.float32)
    assert oracle.lens_linf(X).tolist() == [0.0, 3.0, 0.5, 7.0]
    Y = synth.tiny_random(500, 9, seed=12, scale=5.0)
    f = oracle.lens_linf(Y)
    assert np.array_equal(f, np.linalg.norm(Y.astype(np.float64), ord=np.inf, axis=1))
    l2 = oracle.lens_l2(Y)
    assert np.all(f <= l2) and np.all(l2 <= np.sqrt(9.0) * f * (1 + 1e-15))
    E = np.diag(np.arange(1, 6, dtype=np.float32)) * np.float32(-1.5)
    assert np.array_equal(oracle.lens_linf(E), oracle.lens_l2(E))


def test_density_lens_closed_forms():
    """Ball counts (self included), pinned by hand: points 0..9 on a line with
    r = 1.5 have 3 points within r, 2 at the ends; r below every distance
    gives 1; r at least the diameter gives n; a hand-worked planar case."""
    line = np.arange(10, dtype=np.float32).reshape(-1, 1)
    assert oracle.lens_density(line, 1.5).tolist() == [2.0] + [3.0] * 8 + [2.0]
    assert oracle.lens_density(line, 2.0).tolist() == [3.0, 4.0] + [5.0] * 6 + [4.0, 3.0]
    assert np.all(oracle.lens_density(line, 0.5) == 1.0)
    assert np.all(oracle.lens_density(line, 9.0) == 10.0)
    # (0,0) (1,0) (3,0) (3,4), r = 2: the distance 2 between (1,0) and (3,0) counts
    P = np.array([[0, 0], [1, 0], [3, 0], [3, 4]], dtype=np.float32)
    assert oracle.lens_density(P, 2.0).tolist() == [2.0, 3.0, 2.0, 1.0]
    # duplicates count once each
    D = np.array([[1, 1], [1, 1], [1, 1], [5, 5]], dtype=np.float32)
    assert oracle.lens_density(D, 0.1).tolist() == [3.0, 3.0, 3.0, 1.0]


def test_density_lens_against_kdtree_and_pair_count():
    """On a cloud of multiples of 1/8 every squared distance is exact in
    double; with r^2 halfway between two multiples of 1/64 no pair is on the
    sphere, so scipy's k-d tree ball counts are exact too, and the counts sum
    to n + 2 x (pairs within r)."""
    spatial = pytest.importorskip("scipy.spatial")
    Y = np.round(synth.tiny_random(600, 5, seed=21, scale=2.0) * 8.0).astype(np.float32) / 8.0
    r2 = 60.0 / 64.0 + 1.0 / 128.0
    f = oracle.lens_density(Y, np.sqrt(r2))
    Y64 = Y.astype(np.float64)
    tree = spatial.cKDTree(Y64)
    ref = tree.query_ball_point(Y64, np.sqrt(r2), return_length=True)
    assert np.array_equal(f, ref.astype(np.float64))
    pairs = int((spatial.distance.pdist(Y64, "sqeuclidean") <= r2).sum())
    assert int(f.sum()) == Y.shape[0] + 2 * pairs
    assert f.min() >= 1.0 and f.max() > 2.0
    rows = np.array([0, 599, 17, 17, 300])
    assert np.array_equal(oracle.density_at(Y, rows, np.sqrt(r2)), ref[rows].astype(np.float64))
    with pytest.raises(ValueError):
        oracle.density_at(Y, [600], 1.0)


def test_ecc_inf_lens_closed_forms_and_scipy():
    """Largest distance to the cloud: on a line max(x - min, max - x); the
    hand-worked planar case; scipy's cdist row maxima; its maximum is the
    diameter and it bounds the exponent-2 eccentricity from above."""
    spatial = pytest.importorskip("scipy.spatial")
    line = np.array([[-2.0], [0.0], [1.0], [5.0]], dtype=np.float32)
    assert oracle.lens_ecc_inf(line).tolist() == [7.0, 5.0, 4.0, 7.0]
    P = np.array([[0, 0], [1, 0], [3, 0], [3, 4]], dtype=np.float32)
    np.testing.assert_allclose(oracle.lens_ecc_inf(P), [5.0, np.sqrt(20.0), 4.0, 5.0], rtol=1e-15)
    assert oracle.lens_ecc_inf(np.array([[1.0, 2.0]], dtype=np.float32)).tolist() == [0.0]
    Y = synth.tiny_random(300, 7, seed=22, scale=3.0)
    f = oracle.lens_ecc_inf(Y)
    Dm = spatial.distance.cdist(Y.astype(np.float64), Y.astype(np.float64))
    np.testing.assert_allclose(f, Dm.max(axis=1), rtol=1e-14)
    np.testing.assert_allclose(f.max(), Dm.max(), rtol=1e-14)
    assert np.all(f >= oracle.lens_ecc2(Y) * (1 - 1e-14))


def test_coord_lens_is_the_column():
    Y = synth.tiny_random(100, 5, seed=4)
    for j in range(5):
        assert np.array_equal(oracle.lens_coord(Y, j), Y[:, j].astype(np.float64))


def test_projection_lens_matches_matmul():
    Y = synth.tiny_random(300, 16, seed=5, scale=4.0)
    rng = np.random.default_rng(0)
    mu = rng.standard_normal(16)
    v = rng.standard_normal(16)
    ref = (Y.astype(np.float64) - mu) @ v
    got = oracle.lens_project(Y, mu, v)
    np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())


def test_pca_axis_aligned_closed_form():
    # four points (+-a, 0), (0, +-b): mean 0, covariance diag(a^2/2, b^2/2)
    a, b = 3.0, 1.0
    X = np.array([[a, 0], [-a, 0], [0, b], [0, -b]], dtype=np.float32)
    mu, V, lam = oracle.pca(X, 2)
    np.testing.assert_allclose(mu, [0, 0], atol=0)
    np.testing.assert_allclose(lam, [a * a / 2, b * b / 2], rtol=1e-15)
    np.testing.assert_allclose(V, [[1, 0], [0, 1]], atol=1e-15)


def test_pca_against_numpy_eigh_and_sign_rule():
    w = synth.gaussian_mixture(3000, 12, 4, seed=9, centre_box=5.0, std_lo=0.3,
                               std_hi=1.5, anisotropic=True)
    mu, V, lam = oracle.pca(w, 2)
    X64 = w.astype(np.float64)
    np.testing.assert_allclose(mu, X64.mean(axis=0), rtol=1e-12, atol=1e-12)
    C = np.cov(X64, rowvar=False, bias=True)
    ev, evec = np.linalg.eigh(C)
    np.testing.assert_allclose(lam, ev[::-1][:2], rtol=1e-10)
    for c in range(2):
        ref = evec[:, -1 - c]
        assert abs(abs(ref @ V[c]) - 1.0) < 1e-10
        assert abs(np.linalg.norm(V[c]) - 1.0) < 1e-12
        k = np.argmax(np.abs(V[c]))
        assert V[c][k] > 0
    assert abs(V[0] @ V[1]) < 1e-10


def test_pca_line_direction():
    # points along a known unit direction u, plus tiny orthogonal jitter
    rng = np.random.default_rng(2)
    u = np.array([1.0, -2.0, 2.0]) / 3.0
    t = rng.uniform(-5, 5, size=400)
    X = (np.outer(t, u) + 1e-3 * rng.standard_normal((400, 3))).astype(np.float32)
    _, V, _ = oracle.pca(X, 1)
    assert abs(abs(V[0] @ u) - 1.0) < 1e-6
    assert V[0][np.argmax(np.abs(V[0]))] > 0


def test_interval_bounds_golden(golden_dir):
    g = json.load(open(os.path.join(golden_dir, "cover_intervals.json")))
    for c in g["cases"]:
        a, b = oracle.interval_bounds(c["lo"], c["hi"], c["n"], c["p"])
        np.testing.assert_allclose(a, c["a"], rtol=4e-16, atol=4e-16, err_msg=c["note"])
        np.testing.assert_allclose(b, c["b"], rtol=4e-16, atol=4e-16, err_msg=c["note"])
    m = g["membership"]
    offs, pts = oracle.cover(np.array(m["lens"]), [m["n"]], [m["p"]])
    got = [pts[offs[e]:offs[e + 1]].tolist() for e in range(m["n"])]
    assert got == m["elements"]


def test_interval_rounding_gap_is_closed(golden_dir):
    """A case where rounding leaves b_k one ulp below a_{k+1}; the bounds are
    compared bit for bit and the point at a_{k+1} must lie in both elements."""
    c = json.load(open(os.path.join(golden_dir, "cover_intervals.json")))["rounding_gap"]
    h = float.fromhex
    a, b = oracle.interval_bounds(h(c["lo"]), h(c["hi"]), c["n"], c["p"])
    assert [x.hex() for x in map(float, a)] == [h(x).hex() for x in c["a"]]
    assert [x.hex() for x in map(float, b)] == [h(x).hex() for x in c["b"]]
    lens = np.array([h(x) for x in c["lens"]])
    offs, pts = oracle.cover(lens, [c["n"]], [c["p"]])
    assert [pts[offs[e]:offs[e + 1]].tolist() for e in range(c["n"])] == c["elements"]


@pytest.mark.parametrize("n_int,p", [(1, 0.0), (7, 0.0), (20, 0.3), (50, 0.25), (13, 0.6), (4, 0.95)])
def test_cover_invariants(n_int, p):
    rng = np.random.default_rng(n_int)
    f = rng.normal(size=2000) * 3.0 + 1.0
    offs, pts = oracle.cover(f, [n_int], [p])
    assert len(offs) == n_int + 1
    times = np.bincount(pts, minlength=len(f))
    assert times.min() >= 1                           # the cover covers f(X)
    lo, hi = f.min(), f.max()
    a, b = oracle.interval_bounds(lo, hi, n_int, p)
    L = (hi - lo) / (n_int - (n_int - 1) * p)
    np.testing.assert_allclose(b[:-1] - a[:-1], L, rtol=1e-12)
    np.testing.assert_allclose(a[1:] - a[:-1], L * (1 - p), rtol=1e-12)
    assert a[0] == lo and b[-1] == hi
    for e in range(n_int):                            # brute-force membership
        ref = np.nonzero((f >= a[e]) & (f <= b[e]))[0]
        assert np.array_equal(pts[offs[e]:offs[e + 1]], ref)
    if p == 0.0:
        on_boundary = np.isin(f, a[1:]) | np.isin(f, b[:-1])
        assert np.all(times[~on_boundary] == 1)
    # a point lies in at most ceil(1/(1-p)) + 1 intervals
    assert times.max() <= int(np.ceil(1.0 / (1.0 - p))) + 1


def test_cover_2d_is_product_in_row_major_order():
    rng = np.random.default_rng(7)
    f = rng.uniform(-1, 1, size=(800, 2))
    offs, pts = oracle.cover(f, [5, 3], [0.2, 0.4])
    o1, p1 = oracle.cover(f[:, 0], [5], [0.2])
    o2, p2 = oracle.cover(f[:, 1], [3], [0.4])
    for i in range(5):
        for j in range(3):
            e = i * 3 + j
            ref = np.intersect1d(p1[o1[i]:o1[i + 1]], p2[o2[j]:o2[j + 1]])
            assert np.array_equal(pts[offs[e]:offs[e + 1]], ref)


def test_balanced_cover_hand_worked():
    """Ten distinct values 0..9, three intervals, overlap 0.2: rank range
    [0, 9], L = 9 / 2.6, s = 0.8 L, rank intervals [0, 3.46], [2.77, 6.23],
    [5.54, 9] -> ranks {0..3}, {3..6}, {6..9}."""
    f = np.array([5.0, 0.0, 9.0, 3.0, 7.0, 1.0, 8.0, 2.0, 6.0, 4.0])   # a permutation of 0..9
    offs, pts = oracle.cover(f, (3,), (0.2,), balanced=True)
    got = [sorted(f[pts[offs[e]:offs[e + 1]]].tolist()) for e in range(3)]
    assert got == [[0, 1, 2, 3], [3, 4, 5, 6], [6, 7, 8, 9]]
    a, b = oracle.balanced_bounds(f, 3, 0.2)
    assert a.tolist() == [0.0, 3.0, 6.0] and b.tolist() == [3.0, 6.0, 9.0]


def test_balanced_cover_invariants():
    rng = np.random.default_rng(11)
    f = rng.standard_normal(1000) * 3.0
    for n_int, p in [(1, 0.0), (7, 0.0), (10, 0.3), (25, 0.5)]:
        offs, pts = oracle.cover(f, (n_int,), (p,), balanced=True)
        # every point covered; equal counts up to one (distinct values)
        assert set(pts.tolist()) == set(range(f.size))
        sizes = np.diff(offs)
        L = (f.size - 1) / (n_int - (n_int - 1) * p)
        assert sizes.min() >= np.floor(L) and sizes.max() <= np.ceil(L) + 1
        # invariant under a strictly increasing transform of the filter
        offs2, pts2 = oracle.cover(np.exp(f / 4.0), (n_int,), (p,), balanced=True)
        assert np.array_equal(offs, offs2) and np.array_equal(pts, pts2)
    # all values equal: each element's value interval is [2, 2], so (closed
    # membership) every element holds every point
    offs, pts = oracle.cover(np.full(5, 2.0), (3,), (0.2,), balanced=True)
    assert np.diff(offs).tolist() == [5, 5, 5]
    # a single point lies in the first element only
    offs, _ = oracle.cover(np.array([1.5]), (4,), (0.25,), balanced=True)
    assert np.diff(offs).tolist() == [1, 0, 0, 0]


def test_balanced_bounds_nondecreasing_and_covering():
    """Bounds nondecreasing in k (the membership search relies on it) and every
    point covered, down to one and two points."""
    rng = np.random.default_rng(12)
    for n in (1, 2, 3, 7, 40):
        f = rng.standard_normal(n)
        for n_int in (1, 2, 3, 6):
            for p in (0.0, 0.3, 0.6):
                a, b = oracle.balanced_bounds(f, n_int, p)
                assert np.all(a[1:] >= a[:-1]) and np.all(b[1:] >= b[:-1])
                offs, pts = oracle.cover(f, (n_int,), (p,), balanced=True)
                assert set(pts.tolist()) == set(range(n))
    # two points, four intervals of overlap 0.25: rank intervals [0, .31], [.23, .54],
    # [.46, .77], [.69, 1] hold ranks {0}, {}, {}, {1}
    offs, _ = oracle.cover(np.array([3.0, -1.0]), (4,), (0.25,), balanced=True)
    assert np.diff(offs).tolist() == [1, 0, 0, 1]
