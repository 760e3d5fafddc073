"""Element sharding on the GPU: the elements of one cover split over 2 or 3
shares (as ranks would hold them), each share clustered through a cover
subset, the shares' nodes merged in element order and the nerve of the merged
nodes computed by the library equal the single-call graph, node for node and
edge for edge. The exchange between ranks is covered on CPU ranks
(test_sharded_gloo.py); here the shares run one after the other on one GPU."""
import numpy as np
import pytest

from paper_2011_03209_gb300 import synth

torch = pytest.importorskip("torch")
mg = pytest.importorskip("paper_2011_03209_gb300")
sharded = pytest.importorskip("paper_2011_03209_gb300.sharded")

pytestmark = pytest.mark.gpu


def _same(a, b):
    for k in ("node_offsets", "node_members", "node_elem", "edges"):
        assert np.array_equal(np.asarray(a[k]), np.asarray(b[k])), k


@pytest.mark.parametrize("prec", [mg.BF16, mg.FP32])
@pytest.mark.parametrize("world", [2, 3])
def test_shares_merge_to_the_whole_graph(prec, world):
    w = synth.mixture_100k()
    Xd = torch.from_numpy(w.X).to("cuda:0")
    prm = mg.params(w.lens_kind, w.lens_arg, w.n_intervals, w.overlap, w.eps, w.min_pts, prec)
    with mg.Context(0) as ctx:
        whole = mg.mapper_graph(ctx, Xd, prm).numpy()
        lens, _ = mg.mapper_lens(ctx, Xd, w.lens_kind, w.lens_arg)
        cover = mg.mapper_cover(ctx, lens, w.n_intervals, w.overlap)
        offs, _ = cover.numpy()
        sizes = np.diff(offs).astype(np.float64)
        parts = sharded.lpt_partition(sizes * sizes * w.d, world)
        assert all(p.size > 0 for p in parts)
        pieces = [sharded.local_nodes(ctx, Xd, cover, p, w.eps, w.min_pts, prec) for p in parts]
        no, nm, ne = sharded.merge_nodes(pieces)
        g = mg.mapper_nerve_from_nodes(ctx, w.n, no, nm, ne).numpy()
    assert len(whole["edges"]) > 0
    _same(g, whole)


@pytest.mark.parametrize("cover_kind", [mg.COVER_UNIFORM, mg.COVER_BALANCED])
def test_sharded_graph_single_process(cover_kind):
    w = synth.blobs_circle_5k()
    Xd = torch.from_numpy(w.X).to("cuda:0")
    prm = mg.params(w.lens_kind, w.lens_arg, w.n_intervals, w.overlap, w.eps, w.min_pts, mg.BF16,
                    cover_kind=cover_kind)
    with mg.Context(0) as ctx:
        whole = mg.mapper_graph(ctx, Xd, prm).numpy()
        g, mine = sharded.sharded_graph(ctx, Xd, prm)
        assert mine.size == len(np.unique(mine)) > 0
        _same(g.numpy(), whole)


def test_cover_subset_and_nodes_reject_bad_input():
    w = synth.blobs_circle_5k()
    Xd = torch.from_numpy(w.X).to("cuda:0")
    with mg.Context(0) as ctx:
        lens, _ = mg.mapper_lens(ctx, Xd, w.lens_kind, w.lens_arg)
        cover = mg.mapper_cover(ctx, lens, w.n_intervals, w.overlap)
        E, _ = cover.sizes()
        with pytest.raises(mg.MapperError):
            mg.mapper_cover_subset(ctx, cover, [0, 0])
        with pytest.raises(mg.MapperError):
            mg.mapper_cover_subset(ctx, cover, [E])
        sub = mg.mapper_cover_subset(ctx, cover, [E - 1, 0])
        so, sp = sub.numpy()
        fo, fp = cover.numpy()
        assert np.array_equal(sp, np.concatenate([fp[fo[E - 1]:fo[E]], fp[fo[0]:fo[1]]]))
        assert so.tolist() == [0, int(fo[E] - fo[E - 1]), int(fo[E] - fo[E - 1] + fo[1] - fo[0])]
        empty = mg.mapper_nerve_from_nodes(ctx, w.n, [0], [], []).numpy()
        assert empty["edges"].shape == (0, 2) and empty["node_offsets"].tolist() == [0]
