"""The library's measurement kernels: the copy bandwidth and FP64 FMA rate
come out finite, positive and of the right order for the GPU they ran on
(the copy time is the time of real traffic: a buffer above the L2)."""
import math

import pytest

pytestmark = pytest.mark.gpu


def test_copy_bandwidth_is_plausible():
    from paper_2103_02119_gb300 import lbm
    gbs = lbm.lbm_peak_copy_gbs(512 << 20, 5)
    assert math.isfinite(gbs) and 100.0 < gbs < 20000.0, gbs


def test_fp64_fma_rate_is_plausible():
    from paper_2103_02119_gb300 import lbm
    gf = lbm.lbm_peak_fp64_gflops(2000)
    assert math.isfinite(gf) and 10.0 < gf < 200000.0, gf
