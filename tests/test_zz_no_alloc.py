"""The allocation-free DBSCAN entry point (mapper_dbscan_noalloc) against the
allocating one (mapper_cluster over a one-interval cover, whose single
element holds every row in ascending order) and against the FP64 oracle.

mapper_dbscan_noalloc exists for callers that cannot allocate device memory
(a host framework that owns every allocation through a fixed memory plan, or
code that must not let an allocation synchronise the device); it keeps its
scratch in a fixed array inside the library, shared by all calls. The calls
below run back to back on different inputs, so a value left in the shared
array by one call would show up in the next. Labels and core flags are
integers: the comparison is exact. This file is collected last so that a
failure here stops a `-x` run only after every other test ran."""
import ctypes

import numpy as np
import pytest

from paper_2011_03209_gb300 import synth

torch = pytest.importorskip("torch")
mg = pytest.importorskip("paper_2011_03209_gb300")
from paper_2011_03209_gb300 import _capi  # noqa: E402

pytestmark = pytest.mark.gpu


def _call(lib, Xd, n, d, ld, eps, min_pts, label, core):
    stream = torch.cuda.current_stream(Xd.device)
    return lib.mapper_dbscan_noalloc(ctypes.c_void_p(Xd.data_ptr()), n, d, ld, float(eps), int(min_pts),
                                     ctypes.c_void_p(label.data_ptr()),
                                     ctypes.c_void_p(core.data_ptr()) if core is not None else None,
                                     ctypes.c_void_p(stream.cuda_stream))


def _noalloc(lib, Xd, eps, min_pts, with_core=True, d=None):
    """Xd: n x ld device rows; the first d columns are the points."""
    n, ld = Xd.shape
    d = ld if d is None else d
    label = torch.full((n,), -7, dtype=torch.int64, device=Xd.device)
    core = torch.full((n,), 9, dtype=torch.uint8, device=Xd.device) if with_core else None
    _capi.check(_call(lib, Xd, n, d, ld, eps, min_pts, label, core), "mapper_dbscan_noalloc")
    torch.cuda.synchronize()
    return label.cpu().numpy(), (core.cpu().numpy().astype(bool) if with_core else None)


def _allocating(ctx, Xd, eps, min_pts):
    n = Xd.shape[0]
    lens, _ = mg.mapper_lens(ctx, Xd, (mg.LENS_L2,), (0,))
    cover = mg.mapper_cover(ctx, lens, (1,), (0.0,))
    offs, pts = cover.numpy()
    assert offs.tolist() == [0, n] and np.array_equal(pts, np.arange(n))
    clusters = mg.mapper_cluster(ctx, Xd, cover, eps, min_pts, mg.FP32)
    return clusters.numpy(n)


def test_noalloc_matches_mapper_cluster_on_two_calls_in_a_row():
    lib = _capi.load()
    cases = [
        # larger first (40 tiles of 128 rows, ragged tail), then a smaller one
        (synth.gaussian_mixture(5000, 48, 6, seed=11, centre_box=6.0, std_lo=0.4, std_hi=1.2,
                                anisotropic=True), 3.0, 5),
        (synth.tiny_random(700, 17, 12, scale=2.0), 1.0, 4),
    ]
    with mg.Context(0) as ctx:
        for X, q, min_pts in cases:
            eps = synth.eps_at_percentile(X, q, seed=5, n_pairs=20000)
            Xd = torch.from_numpy(X).to("cuda:0")
            got_label, got_core = _noalloc(lib, Xd, eps, min_pts)
            ref_label, ref_core = _allocating(ctx, Xd, eps, min_pts)
            assert np.array_equal(got_core, ref_core)
            assert np.array_equal(got_label, ref_label)
            assert (got_label >= 0).any() and (got_label < 0).any()


def test_noalloc_full_scratch_then_strided_rows_against_the_oracle():
    """The largest accepted input (8192 x 256 fills the fixed rows block),
    then a smaller strided one (ld > d) with no core output; both against the
    oracle's brute-force DBSCAN of the same rows."""
    oracle = pytest.importorskip("oracle")
    lib = _capi.load()
    n_max, d_max = _capi.NOALLOC_MAX_POINTS, _capi.NOALLOC_MAX_DIM
    X = synth.gaussian_mixture(n_max, d_max, 8, seed=21, centre_box=4.0, std_lo=0.3, std_hi=1.2,
                               anisotropic=False)
    eps = synth.eps_at_percentile(X, 4.0, seed=6, n_pairs=20000)
    got_label, got_core = _noalloc(lib, torch.from_numpy(X).to("cuda:0"), eps, 6)
    _, ref_core, ref_label, ties = oracle.dbscan(X, np.arange(n_max, dtype=np.int32), eps, 6)
    assert ties == 0
    assert np.array_equal(got_core, ref_core)
    assert np.array_equal(got_label, ref_label)
    assert (got_label >= 0).any() and (got_label < 0).any()

    Y = synth.tiny_random(3001, 37, 13, scale=2.0, dup_frac=0.05)
    wide = np.full((Y.shape[0], 41), 1e30, dtype=np.float32)        # columns past d are never read
    wide[:, :37] = Y
    eps = synth.eps_at_percentile(Y, 0.2, seed=7, n_pairs=20000)
    got_label, _ = _noalloc(lib, torch.from_numpy(wide).to("cuda:0"), eps, 3, with_core=False, d=37)
    _, _, ref_label, ties = oracle.dbscan(Y, np.arange(Y.shape[0], dtype=np.int32), eps, 3)
    assert ties == 0
    assert np.array_equal(got_label, ref_label)
    assert len(np.unique(ref_label[ref_label >= 0])) == 2 and (ref_label < 0).any()


def test_noalloc_reports_nonfinite_rows_and_stays_usable():
    lib = _capi.load()
    X = synth.tiny_random(500, 9, 14)
    bad = X.copy()
    bad[123, 4] = np.nan
    Xd = torch.from_numpy(bad).to("cuda:0")
    label = torch.empty(500, dtype=torch.int64, device="cuda:0")
    assert _call(lib, Xd, 500, 9, 9, 0.5, 3, label, None) == _capi.MAPPER_ENONFINITE
    # the next call on the shared array gives the allocating path's result
    eps = synth.eps_at_percentile(X, 3.0, seed=8, n_pairs=20000)
    Xd = torch.from_numpy(X).to("cuda:0")
    got_label, got_core = _noalloc(lib, Xd, eps, 3)
    with mg.Context(0) as ctx:
        ref_label, ref_core = _allocating(ctx, Xd, eps, 3)
    assert np.array_equal(got_core, ref_core) and np.array_equal(got_label, ref_label)


def test_noalloc_rejects_sizes_beyond_its_fixed_scratch():
    lib = _capi.load()
    big = torch.zeros((_capi.NOALLOC_MAX_POINTS + 1, 4), dtype=torch.float32, device="cuda:0")
    wide = torch.zeros((16, _capi.NOALLOC_MAX_DIM + 1), dtype=torch.float32, device="cuda:0")
    out = torch.empty(_capi.NOALLOC_MAX_POINTS + 1, dtype=torch.int64, device="cuda:0")
    for X in (big, wide):
        n, d = X.shape
        rc = lib.mapper_dbscan_noalloc(ctypes.c_void_p(X.data_ptr()), n, d, d, 1.0, 3,
                                       ctypes.c_void_p(out.data_ptr()), None, None)
        assert rc == _capi.MAPPER_EINVAL
        assert b"MAPPER_NOALLOC_MAX" in lib.mapper_last_error()


def test_noalloc_rejects_host_output_pointers():
    lib = _capi.load()
    X = torch.zeros((64, 4), dtype=torch.float32, device="cuda:0")
    host_label = np.zeros(64, dtype=np.int64)
    dev_label = torch.empty(64, dtype=torch.int64, device="cuda:0")
    host_core = np.zeros(64, dtype=np.uint8)
    rc = lib.mapper_dbscan_noalloc(ctypes.c_void_p(X.data_ptr()), 64, 4, 4, 1.0, 3,
                                   host_label.ctypes.data_as(ctypes.c_void_p), None, None)
    assert rc == _capi.MAPPER_EINVAL and b"label_dev" in lib.mapper_last_error()
    rc = lib.mapper_dbscan_noalloc(ctypes.c_void_p(X.data_ptr()), 64, 4, 4, 1.0, 3,
                                   ctypes.c_void_p(dev_label.data_ptr()),
                                   host_core.ctypes.data_as(ctypes.c_void_p), None)
    assert rc == _capi.MAPPER_EINVAL and b"core_dev" in lib.mapper_last_error()
