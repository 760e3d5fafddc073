"""Parameter sweeps: graphs that share the lens, covers and tile layouts
equal the graphs computed one call at a time, and each equals the FP64
oracle's graph."""
import numpy as np
import pytest

import oracle
from paper_2011_03209_gb300 import synth

torch = pytest.importorskip("torch")
mg = pytest.importorskip("paper_2011_03209_gb300")

pytestmark = pytest.mark.gpu


def _same(a, b):
    for k in ("node_offsets", "node_members", "node_elem", "edges"):
        assert np.array_equal(a[k], b[k]), k


@pytest.mark.parametrize("prec", [mg.BF16, mg.FP32])
def test_sweep_2d_pca_grid_equals_single_calls(prec):
    w = synth.zipf_mixture_500k(20000)
    sq = synth.pair_sample(w.X, 3, 20000)
    eps = [synth.eps_from_sample(sq, q) for q in (0.5, 1.0, 2.0, 4.0) for _ in (0.1, 0.3)]
    ov = [p for _ in (0.5, 1.0, 2.0, 4.0) for p in (0.1, 0.3)]
    Xd = torch.from_numpy(w.X).to("cuda:0")
    with mg.Context(0) as ctx:
        base = mg.params(w.lens_kind, w.lens_arg, (8, 8), (0.25, 0.25), eps[0], w.min_pts, prec)
        graphs = mg.mapper_graph_sweep(ctx, Xd, base, eps, ov)
        assert len(graphs) == len(eps)
        for k, (g, e, p) in enumerate(zip(graphs, eps, ov)):
            got = g.numpy()
            one = mg.mapper_graph(ctx, Xd, mg.params(w.lens_kind, w.lens_arg, (8, 8), (p, p), e, w.min_pts, prec))
            _same(got, one.numpy())
            # every sweep graph against the oracle, given the sweep's lens
            lens, _ = g.lens(w.n, 2)
            ref = oracle.mapper_graph(w.X, lens, (8, 8), (p, p), e, w.min_pts)
            _same(got, ref)
            assert ref["near_ties"] == 0 and len(ref["node_elem"]) > 0, k


def test_sweep_rejects_bad_arguments():
    X = torch.zeros((100, 4), dtype=torch.float32, device="cuda:0")
    with mg.Context(0) as ctx:
        base = mg.params((0,), (0,), (4,), (0.2,), 0.5, 3, mg.BF16)
        with pytest.raises(mg.MapperError):
            mg.mapper_graph_sweep(ctx, X, base, [0.5, -1.0], [0.2, 0.2])


def _against_oracle(w, g, grid, p, e, min_pts):
    got = g.numpy()
    lens, _ = g.lens(w.n, len(grid))
    ref = oracle.mapper_graph(w.X, lens, grid, (p,) * len(grid), e, min_pts)
    _same(got, ref)
    return got, ref


# Radii of one overlap share one count pass (up to four per pass, the rest in
# a second): five distinct radii, one of them twice, in every pass-1 screen.
@pytest.mark.parametrize("prec,screen", [(mg.BF16, 0), (mg.BF16, 1), (mg.BF16, 2), (mg.BF16, 3),
                                         (mg.BF16X1, 0)])
def test_sweep_radii_share_a_count_pass(prec, screen):
    w = synth.mixture_100k(30_000)
    eps = [w.eps * f for f in (1.2, 0.8, 1.0, 0.9, 1.1, 1.0)]
    ov = [w.overlap[0]] * len(eps)
    Xd = torch.from_numpy(w.X).to("cuda:0")
    with mg.Context(0) as ctx:
        ctx.set_pass1_screen(screen)
        base = mg.params(w.lens_kind, w.lens_arg, w.n_intervals, w.overlap, eps[0], w.min_pts, prec)
        graphs = mg.mapper_graph_sweep(ctx, Xd, base, eps, ov)
        band = 0
        for g, e in zip(graphs, eps):
            got, ref = _against_oracle(w, g, w.n_intervals, ov[0], e, w.min_pts)
            assert len(ref["node_elem"]) > 0
            band += g.stats()["band_pairs"]
        assert band > 0


# The fused count pass without neighbour lists (minPts 1: no lists; minPts
# 70: no lists, border rows from pass 3) and with the band queue far smaller
# than the band (pairs past it decided in FP64 inside the kernel).
@pytest.mark.parametrize("min_pts,queue_cap", [(1, 0), (70, 0), (10, 64)])
def test_sweep_radii_lists_and_queue(min_pts, queue_cap):
    w = synth.mixture_100k(30_000)
    eps = [w.eps * f for f in (0.85, 1.0, 1.15)]
    ov = [w.overlap[0]] * len(eps)
    Xd = torch.from_numpy(w.X).to("cuda:0")
    with mg.Context(0) as ctx:
        if queue_cap:
            ctx.set_band_queue_cap(queue_cap)
        base = mg.params(w.lens_kind, w.lens_arg, w.n_intervals, w.overlap, eps[0], min_pts, mg.BF16)
        graphs = mg.mapper_graph_sweep(ctx, Xd, base, eps, ov)
        for g, e in zip(graphs, eps):
            _against_oracle(w, g, w.n_intervals, ov[0], e, min_pts)
            if queue_cap:
                assert g.stats()["band_pairs"] > 4 * queue_cap


# Cross-segment pairs (scattered points and a halo of outliers around
# clusters) on the tensor cores with their own operands, radii fused, and on
# CUDA cores; then the FP8 screen on a 2D lens, whose sweep runs one count
# pass per radius.
def _halo_cloud(seed=55):
    X = synth.gaussian_mixture(6000, 32, 6, seed=seed, centre_box=6.0, std_lo=0.4, std_hi=0.9, anisotropic=False)
    rng = np.random.default_rng(seed + 1)
    lo, hi = X.min(axis=0) * 2.0, X.max(axis=0) * 2.0
    r = 5.0 * synth.eps_at_percentile(X, 3, seed, n_pairs=6000)
    u = rng.standard_normal((2500, 32))
    u *= r / np.linalg.norm(u, axis=1, keepdims=True)
    Y = np.concatenate([X, rng.uniform(lo, hi, size=(1000, 32)).astype(np.float32),
                        (X[rng.integers(0, 6000, size=2500)] + u).astype(np.float32)])
    return np.ascontiguousarray(Y[rng.permutation(Y.shape[0])])


@pytest.mark.parametrize("prec,cross", [(mg.BF16, 1), (mg.BF16, 2), (mg.BF16X1, 1)])
def test_sweep_radii_cross_segment_pairs(prec, cross):
    X = _halo_cloud()
    w = synth.Workload("halo", X, (mg.LENS_L2,), (0,), (2,), (0.2,), 1.0, 4)
    eps = [synth.eps_at_percentile(X, q, 55, n_pairs=8000) for q in (2.5, 3.0, 3.5)]
    ov = [0.2] * len(eps)
    with mg.Context(0) as ctx:
        ctx.set_cross_screen(cross)
        base = mg.params(w.lens_kind, w.lens_arg, (2,), (0.2,), eps[0], 4, prec)
        graphs = mg.mapper_graph_sweep(ctx, torch.from_numpy(X).to("cuda:0"), base, eps, ov)
        for g, e in zip(graphs, eps):
            _against_oracle(w, g, (2,), 0.2, e, 4)
            st = g.stats()
            assert st["tile_pairs_cross"] == (st["tile_pairs_simt"] if cross == 1 else 0)
            if cross == 1:
                assert st["tile_pairs_cross"] > 0


def test_sweep_radii_fp8_2d():
    w = synth.zipf_mixture_500k(20_000)
    sq = synth.pair_sample(w.X, 3, 20_000)
    eps = [synth.eps_from_sample(sq, q) for q in (0.7, 1.0, 1.4)]
    ov = [0.3] * len(eps)
    Xd = torch.from_numpy(w.X).to("cuda:0")
    with mg.Context(0) as ctx:
        base = mg.params(w.lens_kind, w.lens_arg, (8, 8), (0.3, 0.3), eps[0], w.min_pts, mg.FP8)
        graphs = mg.mapper_graph_sweep(ctx, Xd, base, eps, ov)
        for g, e in zip(graphs, eps):
            _against_oracle(w, g, (8, 8), 0.3, e, w.min_pts)


# The bench's 16-graph sweep at full size (500k x 128, (PC1, PC2) on a 30 x 30
# grid, four radii fused per overlap): the cover of each overlap bit for bit
# and the DBSCAN of two sampled elements of every graph against the oracle,
# and every graph equal to its own single call on two of the radii.
@pytest.mark.slow
def test_sweep_500k_grid_fused_radii_sampled():
    w, eps, ov = synth.zipf_sweep()
    Xd = torch.from_numpy(w.X).to("cuda:0")
    rng = np.random.default_rng(11)
    with mg.Context(0) as ctx:
        base = mg.params(w.lens_kind, w.lens_arg, w.n_intervals, w.overlap, eps[0], w.min_pts, mg.BF16)
        graphs = mg.mapper_graph_sweep(ctx, Xd, base, eps, ov)
        lens, _ = graphs[0].lens(w.n, 2)
        covers = {}
        for k, (g, e, p) in enumerate(zip(graphs, eps, ov)):
            offs, pts = g.cover().numpy()
            if p not in covers:
                ro, rp = oracle.cover(lens, w.n_intervals, (p, p))
                assert np.array_equal(ro, offs) and np.array_equal(rp, pts), p
                covers[p] = True
            lab, core = g.clusters().numpy(len(pts))
            sizes = np.diff(offs)
            cand = np.nonzero((sizes > 0) & (sizes <= 3000))[0]
            for el in rng.choice(cand, 2, replace=False):
                s0, t0 = offs[el], offs[el + 1]
                _, rc, rl, _ = oracle.dbscan(w.X, pts[s0:t0], e, w.min_pts)
                assert np.array_equal(rc, core[s0:t0]) and np.array_equal(rl, lab[s0:t0]), (k, el)
        for k in (3, 12):
            one = mg.mapper_graph(ctx, Xd, mg.params(w.lens_kind, w.lens_arg, w.n_intervals, (ov[k], ov[k]), eps[k],
                                                     w.min_pts, mg.BF16))
            _same(graphs[k].numpy(), one.numpy())


# Radii from below the nearest-neighbour distance (no pair in) to beyond the
# cloud's diameter in parts (every pair in), on rows of odd width (padded
# operand columns), two overlaps and two screens: the fused pass's early exit
# at the smaller radii and the all-in lists of the larger ones.
@pytest.mark.parametrize("prec", [mg.BF16, mg.BF16X1])
def test_sweep_radii_extremes_odd_width(prec):
    X = synth.gaussian_mixture(3000, 37, 5, seed=21, centre_box=8.0, std_lo=0.3, std_hi=1.2, anisotropic=True)
    w = synth.Workload("odd", X, (mg.LENS_L2,), (0,), (6,), (0.3,), 1.0, 4)
    sq = synth.pair_sample(X, 5, 20_000)
    Y = X.astype(np.float64)
    g2 = (Y * Y).sum(1)
    d2 = g2[:, None] + g2[None, :] - 2.0 * Y @ Y.T
    np.fill_diagonal(d2, np.inf)
    nearest = float(np.sqrt(max(d2.min(), 0.0)))               # every pair is farther than this
    diameter = 2.0 * float(np.sqrt(((Y - Y.mean(0)) ** 2).sum(1).max()))   # no pair is farther
    radii = [0.5 * nearest, synth.eps_from_sample(sq, 1.0), synth.eps_from_sample(sq, 20.0), 1.01 * diameter]
    eps = radii * 2
    ov = [0.3] * 4 + [0.15] * 4
    with mg.Context(0) as ctx:
        base = mg.params(w.lens_kind, w.lens_arg, w.n_intervals, w.overlap, eps[0], w.min_pts, prec)
        graphs = mg.mapper_graph_sweep(ctx, torch.from_numpy(X).to("cuda:0"), base, eps, ov)
        for g, e, p in zip(graphs, eps, ov):
            got, ref = _against_oracle(w, g, w.n_intervals, p, e, w.min_pts)
        assert graphs[0].stats()["n_core"] == 0 and graphs[3].stats()["tile_pairs_out"] == 0
        # the same sweep from host memory (copied inside the call)
        for gh, g in zip(mg.mapper_graph_sweep(ctx, X, base, eps, ov), graphs):
            _same(gh.numpy(), g.numpy())


# Radii fused on a cloud whose sample sends the tile pairs of mostly-deferring
# bins straight to three products and runs the rest in two phases: every graph
# equals its own single call.
def test_sweep_radii_with_pairs_sent_straight():
    w = synth.clusters_1m_d256(200_000)
    eps = [w.eps * f for f in (0.9, 1.0, 1.1)]
    ov = [w.overlap[0]] * 3
    Xd = torch.from_numpy(w.X).to("cuda:0")
    with mg.Context(0) as ctx:
        base = mg.params(w.lens_kind, w.lens_arg, w.n_intervals, w.overlap, eps[0], w.min_pts, mg.BF16)
        graphs = mg.mapper_graph_sweep(ctx, Xd, base, eps, ov)
        st = graphs[0].stats()
        assert st["pass1_phases"] == 2 and st["tile_pairs_direct"] > 0
        for g, e in zip(graphs, eps):
            one = mg.mapper_graph(ctx, Xd, mg.params(w.lens_kind, w.lens_arg, w.n_intervals, w.overlap, e,
                                                     w.min_pts, mg.BF16))
            _same(g.numpy(), one.numpy())
