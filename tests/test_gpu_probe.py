"""The arithmetic-rate probe used as the denominator of the FP64 / FP32
ALU-bound rooflines: it must report a rate in the range the device can
deliver (GB300: FP64 about 1.2 TFLOP/s, FP32 in the tens of TFLOP/s), and
FP32 must be well above FP64 on this part."""
import pytest

from paper_1511_07174_gb300 import api

pytestmark = pytest.mark.gpu


def test_fma_peak_plausible():
    f64 = api.fma_peak("fp64", iters=1 << 14)
    f32 = api.fma_peak("fp32", iters=1 << 14)
    assert 0.05 < f64 < 20.0, f64
    assert 5.0 < f32 < 500.0, f32
    assert f32 > 4 * f64
