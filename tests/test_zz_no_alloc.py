"""The allocation-free DBSCAN entry point (mapper_dbscan_noalloc) against the
allocating one (mapper_cluster over a one-interval cover, whose single
element holds every row in ascending order).

mapper_dbscan_noalloc exists for callers that cannot allocate device memory
(a host framework that owns every allocation through a fixed memory plan, or
code that must not let an allocation synchronise the device); it keeps its
scratch in a fixed array inside the library, shared by all calls. The two
calls below run back to back on different inputs, so a value left in the
shared array by the first call would show up in the second. Labels and core
flags are integers: the comparison is exact. This file is collected last so
that a failure here stops a `-x` run only after every other test ran."""
import ctypes

import numpy as np
import pytest

from paper_2011_03209_gb300 import synth

torch = pytest.importorskip("torch")
mg = pytest.importorskip("paper_2011_03209_gb300")
from paper_2011_03209_gb300 import _capi  # noqa: E402

pytestmark = pytest.mark.gpu


def _noalloc(lib, Xd, eps, min_pts):
    n, d = Xd.shape
    label = torch.full((n,), -7, dtype=torch.int64, device=Xd.device)
    core = torch.full((n,), 9, dtype=torch.uint8, device=Xd.device)
    stream = torch.cuda.current_stream(Xd.device)
    rc = lib.mapper_dbscan_noalloc(ctypes.c_void_p(Xd.data_ptr()), n, d, d, float(eps), int(min_pts),
                                   ctypes.c_void_p(label.data_ptr()), ctypes.c_void_p(core.data_ptr()),
                                   ctypes.c_void_p(stream.cuda_stream))
    _capi.check(rc, "mapper_dbscan_noalloc")
    torch.cuda.synchronize()
    return label.cpu().numpy(), core.cpu().numpy().astype(bool)


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
