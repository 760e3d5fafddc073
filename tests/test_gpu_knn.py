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


@pytest.fixture(scope="module", params=[1, 2], ids=["tensor-cores", "cuda-cores"])
def ctx(request):
    """Every test runs with both screens: BF16 tensor-core products (three per
    tile pair) and the FP32 CUDA-core sums."""
    c = mg.Context(0)
    c.set_knn_screen(request.param)
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
        for mode in (-1, 3):
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
