"""The autotuner's pass-1 shape survives the context through the file named
by MAPPER_TUNE_CACHE: a first context tunes and writes it on destruction, a
second one reads it (and, given a forced shape in the file, uses that shape
without timing anything)."""
import os

import numpy as np
import pytest

from paper_2011_03209_gb300 import synth

torch = pytest.importorskip("torch")
mg = pytest.importorskip("paper_2011_03209_gb300")

pytestmark = pytest.mark.gpu


def test_tune_cache_round_trip(tmp_path, monkeypatch):
    path = tmp_path / "tune.txt"
    monkeypatch.setenv("MAPPER_TUNE_CACHE", str(path))
    w = synth.mixture_100k()
    Xd = torch.from_numpy(w.X).to("cuda:0")
    prm = mg.params(w.lens_kind, w.lens_arg, w.n_intervals, w.overlap, w.eps, w.min_pts, mg.BF16)
    with mg.Context(0) as c:
        first = mg.mapper_graph(c, Xd, prm)
        tile_n = first.stats()["pass1_tile_n"]
        ref = first.numpy()
        del first
    lines = path.read_text().splitlines()
    assert lines[0].startswith("mapper-tune-v1 ") and len(lines) >= 2
    keys = {int(a): int(b) for a, b in (ln.split() for ln in lines[1:])}
    assert tile_n in keys.values()
    # a file that prescribes the other shape for every key: the next context uses it
    other = 384 - tile_n
    path.write_text("\n".join([lines[0]] + [f"{k} {other}" for k in keys]) + "\n")
    with mg.Context(0) as c:
        g = mg.mapper_graph(c, Xd, prm)
        assert g.stats()["pass1_tile_n"] == other
        got = g.numpy()
    for k in ("node_offsets", "node_members", "node_elem", "edges"):
        assert np.array_equal(got[k], ref[k]), k
    # a header for another device is ignored (the context tunes again)
    path.write_text("mapper-tune-v1 some other device sms=1\n" + "\n".join(f"{k} {other}" for k in keys) + "\n")
    with mg.Context(0) as c:
        assert mg.mapper_graph(c, Xd, prm).stats()["pass1_tile_n"] in (128, 256)
    assert os.path.exists(path)
