"""The request server: graphs computed while other requests run beside them
on the device equal the graphs computed alone (exact integer outputs), and
equal the FP64 oracle's."""
import numpy as np
import pytest

import oracle
from paper_2011_03209_gb300 import synth

torch = pytest.importorskip("torch")
mg = pytest.importorskip("paper_2011_03209_gb300")

pytestmark = pytest.mark.gpu


def _datasets():
    return [
        synth.gaussian_mixture(6000, 32, 8, seed=21, centre_box=8.0, std_lo=0.3, std_hi=1.2, anisotropic=True),
        synth.gaussian_mixture(15000, 64, 12, seed=22, centre_box=10.0, std_lo=0.3, std_hi=1.5,
                               anisotropic=True),
        synth.blobs_circle_5k().X,
    ]


def _requests(samples, n):
    reqs = synth.serving_requests(samples, n, rate=1000.0, seed=7)
    for k, r in enumerate(reqs):
        r["n_intervals"] = (10 + (r["n_intervals"][0] % 30),)    # keep elements several tiles wide
        r["precision"] = mg.FP32 if k % 5 == 4 else mg.BF16
    return reqs


def _params(r):
    return mg.params(r["lens_kind"], r["lens_arg"], r["n_intervals"], r["overlap"], r["eps"], r["min_pts"],
                     r["precision"])


def _same(a, b):
    for k in ("node_offsets", "node_members", "node_elem", "edges"):
        assert np.array_equal(a[k], b[k]), k


@pytest.fixture(scope="module")
def data():
    Xs = _datasets()
    samples = [synth.pair_sample(X, 3 + i, 20000) for i, X in enumerate(Xs)]
    Xd = [torch.from_numpy(X).to("cuda:0") for X in Xs]
    return Xs, Xd, _requests(samples, 16)


def test_server_results_equal_alone_and_oracle(data):
    Xs, Xd, reqs = data
    with mg.Server(0, n_slots=4) as srv:
        ids = [srv.add_dataset(X) for X in Xd]
        tickets = [srv.submit(ids[r["dataset"]], _params(r)) for r in reqs]
        mixed = []
        for t in tickets:
            g, info = srv.wait(t, timeout=120.0)
            assert info["status"] == 0 and info["latency_s"] >= info["run_s"] >= 0.0
            mixed.append(g.numpy())
    with mg.Context(0) as ctx:
        for k, (r, got) in enumerate(zip(reqs, mixed)):
            alone = mg.mapper_graph(ctx, Xd[r["dataset"]], _params(r))
            _same(got, alone.numpy())
            if k < 4:                                    # and the oracle, on the GPU's lens
                lens, _ = alone.lens(Xs[r["dataset"]].shape[0], 1)
                ref = oracle.mapper_graph(Xs[r["dataset"]], lens, r["n_intervals"], r["overlap"], r["eps"],
                                          r["min_pts"])
                _same(got, ref)


def test_tiny_budget_runs_one_at_a_time_and_stays_exact(data):
    Xs, Xd, reqs = data
    with mg.Server(0, n_slots=3, hbm_budget=1) as srv:
        ids = [srv.add_dataset(X) for X in Xd]
        tickets = [srv.submit(ids[r["dataset"]], _params(r)) for r in reqs[:6]]
        got = [srv.wait(t, timeout=120.0)[0].numpy() for t in tickets]
    with mg.Context(0) as ctx:
        for r, g in zip(reqs[:6], got):
            _same(g, mg.mapper_graph(ctx, Xd[r["dataset"]], _params(r)).numpy())


def test_server_rejects_unknown_dataset_and_request(data):
    _, Xd, reqs = data
    with mg.Server(0, n_slots=1) as srv:
        srv.add_dataset(Xd[0])
        with pytest.raises(mg.MapperError):
            srv.submit(5, _params(reqs[0]))
        with pytest.raises(mg.MapperError):
            srv.wait(12345, timeout=0.1)


def test_small_request_overtakes_a_blocked_large_one(data):
    """Budget for one large and one small request: while the first large
    request runs, a second large one cannot start, and a small request
    submitted after it starts first (it fits beside the running one)."""
    _, Xd, reqs = data
    big = mg.params((mg.LENS_L2,), (0,), (12,), (0.3,), reqs[0]["eps"], 5, mg.FP32)
    small = mg.params((mg.LENS_L2,), (0,), (4,), (0.2,), 0.5, 5, mg.BF16)
    fb = mg.graph_footprint(Xd[1].shape[0], Xd[1].shape[1], big)
    fs = mg.graph_footprint(Xd[2].shape[0], Xd[2].shape[1], small)
    assert fs < fb
    with mg.Server(0, n_slots=2, hbm_budget=fb + fs) as srv:
        ids = [srv.add_dataset(X) for X in Xd]
        t1 = srv.submit(ids[1], big)
        t2 = srv.submit(ids[1], big)
        t3 = srv.submit(ids[2], small)
        i1, i2, i3 = (srv.wait(t, timeout=120.0)[1] for t in (t1, t2, t3))
    assert i1["status"] == i2["status"] == i3["status"] == 0
    # the second large request waited for the first; the small one did not
    assert i2["queue_s"] >= 0.9 * i1["run_s"]
    assert i3["queue_s"] < i2["queue_s"]


def test_destroy_completes_a_pending_waiter(data):
    """A thread waiting without a time limit on a request that is still
    queued when the server is destroyed returns MAPPER_ECANCELED (or the
    graph, had the request started); destroy does not leave it waiting."""
    import threading
    _, Xd, reqs = data
    srv = mg.Server(0, n_slots=1)
    ids = [srv.add_dataset(X) for X in Xd]
    tickets = [srv.submit(ids[r["dataset"]], _params(r)) for r in reqs[:8]]
    result = {}

    def waiter():
        try:
            g, info = srv.wait(tickets[-1])
            result["status"] = info["status"]
        except mg.MapperError as e:
            result["status"] = e.status

    th = threading.Thread(target=waiter)
    th.start()
    srv.close()
    th.join(timeout=120.0)
    assert not th.is_alive()
    assert result["status"] in (0, mg._capi.MAPPER_ECANCELED)


@pytest.mark.slow
def test_full_size_serving_mix_against_single_calls_and_oracle():
    """The serving mix at full size (the 1M x 256 cloud and eight mixtures up
    to 5e5 points): twelve requests through four slots equal the same requests
    alone; on three of them the DBSCAN of the smallest and of a median element
    equals the oracle's."""
    Xs = synth.serving_datasets(seed=4)
    samples = [synth.pair_sample(X, 4 + i, 20000) for i, X in enumerate(Xs)]
    reqs = synth.serving_requests(samples, 12, rate=1000.0, seed=11)
    Xd = [torch.from_numpy(X).to("cuda:0") for X in Xs]

    def prm(r):
        return mg.params(r["lens_kind"], r["lens_arg"], r["n_intervals"], r["overlap"], r["eps"], r["min_pts"],
                         mg.BF16)

    with mg.Server(0, n_slots=4) as srv:
        ids = [srv.add_dataset(X) for X in Xd]
        tickets = [srv.submit(ids[r["dataset"]], prm(r)) for r in reqs]
        got = []
        for t in tickets:
            g, info = srv.wait(t, timeout=300.0)
            assert info["status"] == 0
            got.append((g.numpy(), g))
    with mg.Context(0) as ctx:
        for k, (r, (out, g)) in enumerate(zip(reqs, got)):
            alone = mg.mapper_graph(ctx, Xd[r["dataset"]], prm(r))
            _same(out, alone.numpy())
            if k < 3:
                X = Xs[r["dataset"]]
                offs, pts = g.cover().numpy()
                lab, core = g.clusters().numpy(len(pts))
                sizes = np.diff(offs)
                ne = np.nonzero(sizes)[0]
                for e in (int(ne[np.argmin(sizes[ne])]), int(ne[np.argsort(sizes[ne])[len(ne) // 2]])):
                    s, t = offs[e], offs[e + 1]
                    if t - s > 20000:
                        continue
                    _, rc, rl, ties = oracle.dbscan(X, pts[s:t], r["eps"], r["min_pts"])
                    assert ties == 0 and np.array_equal(core[s:t], rc) and np.array_equal(lab[s:t], rl), (k, e)
