"""Host-side arithmetic of bench.py's roofline objects (no GPU needed)."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    sys.path.insert(0, ROOT)
    import bench
    return bench


def test_alu_roofline_of_the_3d_step():
    b = _bench()
    # the stencils as written, one FMA per tap: filter 54, source 78, four sweeps
    # of 201, update 3, Faraday 24
    assert b.FLOPS_PER_CELL_STEP_3D == 963
    assert abs(b.FP32_PEAK_TFLOPS - 80.548) < 1e-3
    r = b.alu_roofline(512 ** 3, 7.5e-3)
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    assert abs(r["achieved"] - 963 * 512 ** 3 / 7.5e-3 / 1e12) < 0.01
    assert abs(r["frac"] - r["achieved"] / b.FP32_PEAK_TFLOPS) < 1e-3
    # above the ridge: flops per algorithmic byte exceed peak flops per HBM byte
    assert b.FLOPS_PER_CELL_STEP_3D / b.BYTES_PER_CELL > b.FP32_PEAK_TFLOPS * 1e12 / (6779.4e9)
