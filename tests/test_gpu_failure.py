"""Failure detection on the GPU without a fault: every spin-wait of the
tensor-core passes is bounded; a wait that runs out raises an abort flag, the
kernel's roles stop, and the call returns MAPPER_ETIMEOUT. Here the library's
self-test runs that wait on an mbarrier that nothing completes (the limit is
4 s), and the same context then computes an exact graph."""
import time

import numpy as np
import pytest

import oracle
from paper_2011_03209_gb300 import synth

torch = pytest.importorskip("torch")
mg = pytest.importorskip("paper_2011_03209_gb300")
from paper_2011_03209_gb300 import _capi  # noqa: E402

pytestmark = pytest.mark.gpu


def test_bounded_wait_runs_out_and_context_survives():
    w = synth.blobs_circle_5k()
    Xd = torch.from_numpy(w.X).to("cuda:0")
    with mg.Context(0) as ctx:
        t0 = time.perf_counter()
        rc = ctx._lib.mapper_selftest_wait(ctx.h)
        dt = time.perf_counter() - t0
        assert rc == _capi.MAPPER_ETIMEOUT
        assert 3.5 < dt < 30.0
        assert b"self-test" in ctx._lib.mapper_last_error()
        prm = mg.params(w.lens_kind, w.lens_arg, w.n_intervals, w.overlap, w.eps, w.min_pts, mg.BF16)
        g = mg.mapper_graph(ctx, Xd, prm)
        got = g.numpy()
        lens, _ = g.lens(w.n, 1)
    ref = oracle.mapper_graph(w.X, lens, w.n_intervals, w.overlap, w.eps, w.min_pts)
    for k in ("node_offsets", "node_members", "node_elem", "edges"):
        assert np.array_equal(got[k], ref[k]), k
