"""The arithmetic-roofline denominator: fmx_fma_peak measures the device's
FMA rate.  FP32 must land near the unit-count figure (SMs x 128 lanes x 2
flops x SM clock) and FP64 below it."""
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fmx():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1907_13088_gb300 import build
    build.build()
    from paper_1907_13088_gb300 import fmx as m
    return m


def test_fma_peak_fp32_near_unit_count_and_fp64_below(fmx):
    import torch
    props = torch.cuda.get_device_properties(0)
    f32 = fmx.fma_peak(fmx.FMX_F32)
    f64 = fmx.fma_peak(fmx.FMX_F64)
    # 128 FP32 lanes per SM at up to ~2.1 GHz
    nominal = props.multi_processor_count * 128 * 2 * 2.1e9
    assert 0.4 * nominal < f32 < 1.1 * nominal, (f32, nominal)
    assert 0.0 < f64 < f32, (f64, f32)
