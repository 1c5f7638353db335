"""hmc_measure_fma_peak: the measured CUDA-core multiply-add ceilings the
benchmark divides the arithmetic-bound kernels by.  Sanity only: positive,
FP32 above FP64 (the FP64 units of this GPU are a small fraction of its FP32
units), paired FP32 at least as fast as scalar FP32, and a bad kind
refused."""
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1805_03560_gb300 import hmc
    return hmc.Context(0)


def test_fma_peaks_ordered(ctx):
    f64, f32, f32x2 = (ctx.fma_peak(k) for k in range(3))
    assert 0 < f64 < f32
    assert f32x2 >= 0.9 * f32


def test_fma_peak_bad_kind(ctx):
    from paper_1805_03560_gb300 import hmc
    with pytest.raises(hmc.HmcError) as e:
        ctx.fma_peak(3)
    assert e.value.status == hmc.EINVAL
