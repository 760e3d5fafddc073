"""The empirical leg of the screen's error bound. The bound assumes that the
tcgen05 accumulator adds at most 2^-22 of the products' magnitude sum per
MMA step (16 products of K per step); this measures the accumulation error
of the hardware on random BF16 rows, through the same TMA and MMA path the
screen uses, and requires it to stay below a quarter of the modelled term
at every row pitch and for one and three products."""
import pytest

torch = pytest.importorskip("torch")
mg = pytest.importorskip("paper_2011_03209_gb300")

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("products", [1, 3])
@pytest.mark.parametrize("dp", [32, 64, 256, 1024])
def test_accumulation_error_below_a_quarter_of_the_model(dp, products):
    with mg.Context(0) as ctx:
        worst = 0.0
        for seed in (1, 2, 3):
            observed, modelled = ctx.selftest_mma_error(dp, products, seed)
            assert modelled > 0.0
            worst = max(worst, observed)
    assert worst <= modelled / 4, (worst, modelled)


def test_accumulation_probe_rejects_bad_shapes():
    with mg.Context(0) as ctx:
        for dp, products in ((48, 1), (64, 2), (0, 3), (8192, 1)):
            with pytest.raises(mg.MapperError):
                ctx.selftest_mma_error(dp, products)
