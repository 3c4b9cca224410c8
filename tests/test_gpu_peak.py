"""fil_fma_peak, the measured counterpart of the derived FMA peaks: the rates it
measures agree with the unit counts of the GPU (per SM 128 FP32 lanes, 2 FP64
lanes, an FMA = 2 flops) at the SM clock it measures during the run."""
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fil():
    assert torch.cuda.is_available()
    from paper_1903_12609_gb300 import fil as _fil
    return _fil


@pytest.mark.parametrize("fp64,lanes", [(False, 128), (True, 2)])
def test_fma_peak_matches_unit_counts(fil, fp64, lanes):
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    flops, mhz = fil.fil_fma_peak(fp64)
    assert 500.0 < mhz < 3000.0
    derived = sms * lanes * 2 * mhz * 1e6
    assert 0.7 * derived < flops < 1.05 * derived
