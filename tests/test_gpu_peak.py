"""fv_maxplus_peak: the register-only ceiling of the max-plus cell (one
add.f32x2 + one 3-input max per two cells) on every SM.  Checks that it
reports the device's SM count and a per-SM rate between a quarter of and the
unit-count limit of 128 cells per clock (two FP32 lanes' worth per cell pair
on each of the four SM sub-partitions)."""
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_maxplus_peak_is_plausible():
    import paper_2510_19301_gb300 as fv
    cps, per_clk, sms = fv.maxplus_peak(50000)
    assert sms == torch.cuda.get_device_properties(0).multi_processor_count
    assert 32.0 <= per_clk <= 128.5, per_clk
    # cells/s agrees with cells/clk/SM x SMs x a clock between 0.5 and 2.2 GHz
    mhz = cps / (per_clk * sms) / 1e6
    assert 500.0 <= mhz <= 2200.0, mhz
