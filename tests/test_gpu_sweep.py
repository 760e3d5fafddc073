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
