"""The FP64 FMA calibration (lbm_measure_fp64_fma), the peak of the FP64 storage
form's arithmetic roofline: on a GB300 it must land near the nominal FP64 rate,
1.25 TFLOP/s (152 SMs x 2 FP64 FMA a clock x 2 x 2.07 GHz), and repeat."""
import pytest

pytestmark = pytest.mark.gpu
NOMINAL = 152 * 2 * 2 * 2.07e9 / 1e12


@pytest.fixture(scope="module")
def L():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1902_08933_gb300 import build, lbm
    build.build()
    return lbm


def test_fp64_fma_rate_is_near_nominal(L, report):
    a = L.lbm_measure_fp64_fma()
    b = L.lbm_measure_fp64_fma()
    report(fp64_tflops_first=a, fp64_tflops_second=b, nominal=NOMINAL)
    assert 0.5 * NOMINAL < a < 1.2 * NOMINAL, a
    assert abs(a - b) < 0.1 * a
