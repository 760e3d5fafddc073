"""k-th nearest-neighbour distances on the GPU (§5's module for choosing
eps): equal to the oracle's brute-force FP64 values bit for bit, with either
screen."""
import numpy as np
import pytest

import oracle
from paper_2011_03209_gb300 import synth

torch = pytest.importorskip("torch")
mg = pytest.importorskip("paper_2011_03209_gb300")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", params=[1, 3, 2], ids=["tensor-cores", "tensor-lists", "cuda-cores"])
def ctx(request):
    """Every test runs with each screen: BF16 tensor-core products (three per
    tile pair; large clouds with a threshold per query from a sample of the
    points, or with per-part lists only) and the FP32 CUDA-core sums."""
    c = mg.Context(0)
    c.set_knn_screen(request.param)
    c.knn_mode = request.param
    yield c
    c.close()


@pytest.mark.parametrize("n,d,k,seed", [(1, 3, 1, 0), (40, 2, 16, 1), (3001, 17, 5, 2),
                                        (5000, 64, 1, 3), (4000, 130, 16, 4), (2500, 600, 5, 5)])
def test_knn_distance_equals_oracle(ctx, n, d, k, seed):
    X = (synth.gaussian_mixture(n, d, 6, seed=90 + seed, centre_box=4.0, std_lo=0.3, std_hi=1.0,
                                anisotropic=True, noise_frac=0.05)
         if n > 40 else synth.tiny_random(n, d, seed, scale=3.0))
    rng = np.random.default_rng(seed)
    q = np.unique(rng.integers(0, n, size=min(n, 300))).astype(np.int32)
    got = mg.mapper_knn_distance(ctx, torch.from_numpy(X).to("cuda:0"), q, k)
    ref = oracle.knn_distance(X, q, k)
    assert np.array_equal(got, ref)


def test_knn_distance_duplicates_and_all_points(ctx):
    X = synth.tiny_random(64, 5, 7, dup_frac=0.5)
    Xd = torch.from_numpy(X).to("cuda:0")
    q = np.arange(64, dtype=np.int32)
    for k in (1, 2, 3, 8, 16):
        assert np.array_equal(mg.mapper_knn_distance(ctx, Xd, q, k), oracle.knn_distance(X, q, k))
    # queries given in device memory
    qd = torch.from_numpy(q).to("cuda:0")
    out = np.empty(64)
    lib = ctx._lib
    import ctypes
    p = ctypes.c_void_p(Xd.data_ptr())
    assert lib.mapper_knn_distance(ctx.h, p, 64, 5, 5, ctypes.c_void_p(qd.data_ptr()), 64, 4,
                                   ctypes.c_void_p(out.ctypes.data)) == 0
    assert np.array_equal(out, oracle.knn_distance(X, q, 4))


def test_knn_distance_core_threshold_matches_dbscan(ctx):
    """kdist(p) <= eps exactly when p is core for DBSCAN(eps, k) on the whole
    cloud (one cover element)."""
    X = synth.gaussian_mixture(3000, 12, 5, seed=95, centre_box=4.0, std_lo=0.4, std_hi=1.0, anisotropic=False)
    Xd = torch.from_numpy(X).to("cuda:0")
    k = 6
    kd = mg.mapper_knn_distance(ctx, Xd, np.arange(3000), k)
    s = np.unique(kd)
    i = int(0.4 * s.size)
    eps = float((s[i] + s[i + 1]) / 2)                 # halfway between two k-distances
    prm = mg.params((mg.LENS_COORD,), (0,), (1,), (0.0,), eps, k, mg.BF16)
    g = mg.mapper_graph(ctx, Xd, prm)
    offs, pts = g.cover().numpy()
    _, core = g.clusters().numpy(len(pts))
    assert np.array_equal(core[np.argsort(pts)], kd <= eps)


def test_knn_distance_rejects_bad_input(ctx):
    X = synth.tiny_random(20, 4, 1)
    Xd = torch.from_numpy(X).to("cuda:0")
    for q, k in (([0], 0), ([0], 21), ([0], 17), ([20], 3), ([-1], 3)):
        with pytest.raises(mg.MapperError):
            mg.mapper_knn_distance(ctx, Xd, q, k)
    Y = X.copy()
    Y[3, 2] = np.nan
    with pytest.raises(mg.MapperError):
        mg.mapper_knn_distance(ctx, torch.from_numpy(Y).to("cuda:0"), [0], 3)


def test_knn_distance_huge_finite_rows(ctx):
    """Finite rows whose squared norms pass FP32 (values near 1e20): the
    tensor-core path flags them while building its operands and the call
    falls back to the CUDA-core screen; still exact."""
    X = synth.tiny_random(300, 6, 21, scale=2.0)
    X[::37] *= np.float32(3e19)
    q = np.arange(0, 300, 3, dtype=np.int32)
    for k in (1, 4):
        got = mg.mapper_knn_distance(ctx, torch.from_numpy(X).to("cuda:0"), q, k)
        assert np.array_equal(got, oracle.knn_distance(X, q, k))


@pytest.mark.parametrize("k", [1, 5, 16])
def test_knn_distance_many_chunks(ctx, k):
    """150k points: the screen splits the points into many chunks per query
    tile, each with its own candidate lists; the merged result is exact."""
    X = synth.gaussian_mixture(150_000, 24, 12, seed=97, centre_box=5.0, std_lo=0.4, std_hi=1.1,
                               anisotropic=True, noise_frac=0.05)
    rng = np.random.default_rng(k)
    q = rng.integers(0, X.shape[0], size=200).astype(np.int32)
    got = mg.mapper_knn_distance(ctx, torch.from_numpy(X).to("cuda:0"), q, k)
    assert np.array_equal(got, oracle.knn_distance(X, q, k))
    info = ctx.knn_info()
    if ctx.knn_mode == 1 and k <= 8:
        # 1172 point tiles: the sampled threshold, no query over capacity
        assert info["path"] == 2 and info["sample_stride"] == 4 and info["over_capacity"] == 0, info
    else:
        assert info["path"] == (0 if ctx.knn_mode == 2 or k > 8 else 1), info


def _near_duplicate_clusters(n_centres, copies, d, jitter, seed):
    rng = np.random.default_rng(seed)
    C = rng.uniform(-5.0, 5.0, size=(n_centres, d))
    X = np.repeat(C, copies, axis=0) + rng.normal(0.0, jitter, size=(n_centres * copies, d))
    return X[rng.permutation(len(X))].astype(np.float32)


@pytest.mark.parametrize("k", [1, 5, 8])
def test_knn_distance_sampled_threshold_over_capacity(ctx, k):
    """80,000 points in 40 tight clusters of 2000 (spread 0.01 against centres
    10 apart): every point of a query's cluster is within the screen's error
    band of its k-th neighbour, far more keys below the sampled threshold than
    the capacity, so those queries go through the list screen; exact all
    the same."""
    X = _near_duplicate_clusters(40, 2000, 32, 0.01, seed=101 + k)
    q = np.random.default_rng(k).integers(0, X.shape[0], size=300).astype(np.int32)
    got = mg.mapper_knn_distance(ctx, torch.from_numpy(X).to("cuda:0"), q, k)
    assert np.array_equal(got, oracle.knn_distance(X, q, k))
    if ctx.knn_mode == 1:
        info = ctx.knn_info()
        assert info["path"] == 2 and info["over_capacity"] > 0, info


def test_ecc_inf_lens_sampled_threshold():
    """The L-infinity centrality (the largest distance, the k = 1 farthest
    screen) of 70,000 points: 68,000 from a Gaussian mixture and 2000 tight
    copies of a far point, so for most rows the farthest keys crowd the
    threshold beyond the capacity; sampled rows equal the oracle's."""
    rng = np.random.default_rng(103)
    G = synth.gaussian_mixture(68_000, 8, 5, seed=104, centre_box=3.0, std_lo=0.3, std_hi=1.0, anisotropic=True)
    far = np.full(8, 40.0) + rng.normal(0.0, 1e-3, size=(2000, 8))
    X = np.concatenate([G, far.astype(np.float32)])[rng.permutation(70_000)].astype(np.float32)
    rows = np.sort(rng.choice(70_000, size=48, replace=False)).astype(np.int32)
    with mg.Context(0) as c:
        f, _ = mg.mapper_lens(c, torch.from_numpy(X).to("cuda:0"), (mg.LENS_ECC_INF,), (0,))
        got = f.cpu().numpy()[:, 0]
    assert np.array_equal(got[rows], oracle.knn_distance(X, rows, X.shape[0]))


def test_knn_distance_strided_rows_and_ties(ctx):
    """Rows with a pitch that is not a multiple of 4 floats (scalar loads) and
    a cloud of many exact duplicates (ties at the k-th value send queries to
    the two streaming passes)."""
    base = synth.tiny_random(3000, 13, 11, scale=2.0, dup_frac=0.6)
    base[100:140] = base[100]                            # 40 copies: the 16 smallest values all 0
    X = np.concatenate([base, base[:1500]])              # every point at least twice, many more
    wide = np.zeros((X.shape[0], 16), dtype=np.float32)
    wide[:, :13] = X
    Xd = torch.from_numpy(wide).to("cuda:0")[:, :13]
    q = np.r_[np.arange(0, X.shape[0], 7), np.arange(100, 140)].astype(np.int32)
    for k in (2, 3, 16):
        assert np.array_equal(mg.mapper_knn_distance(ctx, Xd, q, k), oracle.knn_distance(X, q, k)), k


def test_knn_distance_wide_rows(ctx):
    """1500 columns (the row length of §5's gene-expression case): the
    streaming passes stage columns in chunks."""
    X = synth.gaussian_mixture(300, 1500, 3, seed=98, centre_box=3.0, std_lo=0.5, std_hi=1.0, anisotropic=False)
    Xd = torch.from_numpy(X).to("cuda:0")
    q = np.arange(300, dtype=np.int32)
    for k in (1, 2, 5):
        assert np.array_equal(mg.mapper_knn_distance(ctx, Xd, q, k), oracle.knn_distance(X, q, k))


def test_knn_screen_rejects_bad_mode():
    with mg.Context(0) as c:
        for mode in (-1, 4):
            with pytest.raises(mg.MapperError):
                c.set_knn_screen(mode)


@pytest.mark.parametrize("k", [7, 8, 9])
def test_knn_distance_list_length_boundary(ctx, k):
    """k up to 8 runs on the tensor-core screen's 8-entry lists, k = 9 on the
    CUDA-core screen: both exact on either side of the switch."""
    X = synth.gaussian_mixture(20_000, 40, 8, seed=99, centre_box=4.0, std_lo=0.3, std_hi=0.9,
                               anisotropic=True, noise_frac=0.05)
    q = np.random.default_rng(k).integers(0, X.shape[0], size=257).astype(np.int32)
    got = mg.mapper_knn_distance(ctx, torch.from_numpy(X).to("cuda:0"), q, k)
    assert np.array_equal(got, oracle.knn_distance(X, q, k))


def test_knn_distance_k_equals_n(ctx):
    """k = n: the largest distance from each point (the L-infinity centrality)."""
    X = synth.tiny_random(16, 6, 12, scale=2.0)
    q = np.arange(16, dtype=np.int32)
    got = mg.mapper_knn_distance(ctx, torch.from_numpy(X).to("cuda:0"), q, 16)
    assert np.array_equal(got, oracle.knn_distance(X, q, 16))
    assert np.array_equal(got, oracle.lens_ecc_inf(X))
