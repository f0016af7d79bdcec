"""The measured roofline denominators (FP64 FMA rate, L2-resident copy
bandwidth) come out positive and within what the B300 can do."""
import pytest

pytestmark = pytest.mark.gpu


def test_measured_fp64_rate(hw):
    r = hw.hw_measure_fp64()
    # nominal 1.25 TFLOP/s = 0.625e12 FMA/s; a measurement far off means the probe is wrong
    assert 0.2e12 < r < 0.8e12, r


def test_measured_l2_copy_bandwidth(hw):
    g = hw.hw_measure_l2()
    # above the HBM copy rate (~6.5 TB/s) is expected for an L2-resident set
    assert 3000 < g < 60000, g
