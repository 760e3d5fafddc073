"""The bench line's roofline arithmetic, on CPU: the count pass's DRAM
traffic scaled from the recorded per-launch captures by each launch's tile
pairs, and its algorithmic and executed flop rates for a count pass whose
tile pairs are split between a straight three-product launch and two phases."""
import hashlib
import json
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

bench = pytest.importorskip("bench")


def _record():
    with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
        rec = json.load(f)["tc_kernel_count"]
    with open(os.path.join(ROOT, "paper_2011_03209_gb300", "csrc", "k_tc.cu"), "rb") as f:
        current = hashlib.sha1(f.read()).hexdigest() == rec["source_sha1"]
    return rec, current


def test_traffic_scales_each_launch_by_its_tile_pairs():
    rec, current = _record()
    st = {"tile_pairs_screen1": 1000, "tile_pairs_redo": 30, "tile_pairs_direct": 400}
    got = bench._traffic(st)
    if not current:                       # the kernel changed since the captures
        assert got is None
        return
    want = (rec["bytes_per_tile_pair_first"] * 1000 + rec["bytes_per_tile_pair_second"] * 30 +
            rec["bytes_per_tile_pair_direct"] * 400)
    assert got == pytest.approx(want, rel=1e-12)
    # a one-phase pass has no first-phase launch to scale
    assert bench._traffic({"tile_pairs_screen1": 0, "tile_pairs_redo": 0, "tile_pairs_direct": 0}) is None


def test_traffic_record_names_every_launch():
    rec, _ = _record()
    for k in ("bytes_per_tile_pair_first", "bytes_per_tile_pair_second", "bytes_per_tile_pair_direct"):
        assert rec[k] > 0.0, k
    assert "ncu" in rec["command"] and "--clock-control none" in rec["command"]


def test_roofline_counts_three_products_for_pairs_sent_straight():
    mg = pytest.importorskip("paper_2011_03209_gb300")

    class W:
        d = 256

    st = {"count_kernel_pairs": 5_000_000, "tile_pairs_tc": 1500, "tile_pairs_screen1": 1000,
          "tile_pairs_redo": 30, "tile_pairs_direct": 500}
    kms, roof = bench._roofline(mg.BF16, W(), st, [{"ms_count_kernel": 2.0}], 152)
    assert kms == 2.0
    secs = 2.0e-3
    assert roof["achieved"] == pytest.approx(2.0 * 256 * 5_000_000 / secs / 1e12)
    per_product = 256 * 128.0 * 128.0 * 2.0            # one product of a 128 x 128 tile pair at d = 256
    want = (1000 * 1 + (30 + 500) * 3) * per_product / secs / 1e12
    assert roof["executed_tflops"] == pytest.approx(want)
    assert roof["frac"] == pytest.approx(roof["achieved"] / roof["peak"])
    # one phase: three products over every tensor-core pair
    st1 = dict(st, tile_pairs_screen1=0, tile_pairs_redo=0, tile_pairs_direct=0)
    _, roof1 = bench._roofline(mg.BF16, W(), st1, [{"ms_count_kernel": 2.0}], 152)
    assert roof1["executed_tflops"] == pytest.approx(1500 * 3 * per_product / secs / 1e12)
