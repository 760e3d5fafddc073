"""Element sharding on the GPU: the elements of one cover split over 2 or 3
shares (as ranks would hold them), each share clustered through a cover
subset, the shares' nodes merged in element order and the nerve of the merged
nodes computed by the library equal the single-call graph and the FP64
oracle's graph, node for node and edge for edge. The exchange between ranks is covered on CPU ranks
(test_sharded_gloo.py); here the shares run one after the other on one GPU."""
import functools

import numpy as np
import pytest

import oracle
from paper_2011_03209_gb300 import synth

torch = pytest.importorskip("torch")
mg = pytest.importorskip("paper_2011_03209_gb300")
sharded = pytest.importorskip("paper_2011_03209_gb300.sharded")

pytestmark = pytest.mark.gpu


@functools.lru_cache(maxsize=2)
def _oracle_graph(lens_bytes, shape):
    w = synth.mixture_100k()
    lens = np.frombuffer(lens_bytes, dtype=np.float64).reshape(shape)
    return oracle.mapper_graph(w.X, lens, w.n_intervals, w.overlap, w.eps, w.min_pts)


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
        lens_h = lens.cpu().numpy()
    assert len(whole["edges"]) > 0
    _same(g, whole)
    # and the merged graph against the oracle's, given the same lens
    _same(g, _oracle_graph(lens_h.tobytes(), lens_h.shape))


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
        got = g.numpy()
        _same(got, whole)
        lens, _ = mg.mapper_lens(ctx, Xd, w.lens_kind, w.lens_arg)
        lens_h = lens.cpu().numpy()
    _same(got, oracle.mapper_graph(w.X, lens_h, w.n_intervals, w.overlap, w.eps, w.min_pts,
                                   balanced=cover_kind == mg.COVER_BALANCED))


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
