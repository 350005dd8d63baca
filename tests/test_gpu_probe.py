"""hodlrdd_probe_peaks: the measured pipe rates bench.py divides by. Checked
against what GB300's unit counts allow at its clock range (152 SMs; per SM and
clock 128 FP32 FMA lanes, 16 MUFU operations; FP64 at most 1/2 of FP32): the
probe must land inside, not above, those limits."""
import pytest

from gpu_util import require_cuda

pytestmark = pytest.mark.gpu


def test_probe_rates_are_physical():
    require_cuda()
    import paper_2209_05819_gb300 as hd

    p = hd.probe_peaks()
    sms = 152
    f_max = 2.2e9  # above the 2070 MHz boost clock
    fp32_max = sms * 128 * 2 * f_max / 1e12
    assert 0.2 * fp32_max < p["fp32_tflops"] <= fp32_max
    assert 0.0 < p["fp64_tflops"] <= 0.5 * p["fp32_tflops"]
    mufu_max = sms * 32 * f_max / 1e9  # generous: twice the 16 per SM and clock
    assert 0.0 < p["mufu_rsqrt_gops"] <= mufu_max
    assert 0.0 < p["mufu_ex2_gops"] <= mufu_max
