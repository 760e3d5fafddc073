"""The empirical leg of the screen's error bound. The bound assumes that the
tcgen05 accumulator adds at most 2^-22 of the products' magnitude sum per
MMA instruction (16 BF16 or 32 FP8 products of K), with a floor of 8 such
units; this measures the accumulation error of the hardware on random BF16
and FP8 E4M3 rows, through the same TMA and MMA path the screen uses, and
requires it to stay below a quarter of the modelled term at every row pitch
and for one and three products."""
import pytest

torch = pytest.importorskip("torch")
mg = pytest.importorskip("paper_2011_03209_gb300")

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("fmt", [0, 1], ids=["bf16", "fp8"])
@pytest.mark.parametrize("products", [1, 3])
@pytest.mark.parametrize("dp", [32, 64, 256, 1024])
def test_accumulation_error_below_a_quarter_of_the_model(dp, products, fmt):
    with mg.Context(0) as ctx:
        worst = 0.0
        for seed in (1, 2, 3):
            observed, modelled = ctx.selftest_mma_error(dp, products, seed, fmt)
            assert modelled > 0.0
            worst = max(worst, observed)
    assert worst <= modelled / 4, (worst, modelled)


def test_accumulation_probe_rejects_bad_shapes():
    with mg.Context(0) as ctx:
        for dp, products, fmt in ((48, 1, 0), (64, 2, 0), (0, 3, 0), (8192, 1, 0), (64, 1, 2)):
            with pytest.raises(mg.MapperError):
                ctx.selftest_mma_error(dp, products, 1, fmt)
