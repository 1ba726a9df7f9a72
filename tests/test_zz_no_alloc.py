"""fmx_step_static: the step for callers that may not allocate device memory
(their device memory comes from their own pool or a budget fixed up front).
It must give what fmx_step gives on the same inputs, call after call, while
its intermediates live in the library's fixed device scratch array."""
import ctypes

import numpy as np
import pytest

from oracle import core
from paper_1907_13088_gb300 import synth
from tests.helpers import rel_l2

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


def _device_fields(shape, arr, dtype, pitch):
    import torch
    nx, ny = shape
    t = torch.zeros((3, ny, pitch), dtype=dtype, device="cuda")
    t[:, :, :nx] = torch.from_numpy(np.ascontiguousarray(arr[:, 0])).to("cuda")
    return t


def _ptrs(t):
    return (ctypes.c_void_p * 3)(*[t[c].data_ptr() for c in range(3)])


CASES = [
    # the 64 x 64 FP64 residual-mode case (tol 1e-13), vacuum
    dict(shape=(64, 64), prec=1, tol_rel=1e-12, kw=dict(iter_mode=1, tol=1e-13, m_max=10000, courant=0.5),
         current=False),
    # an FP32 grid with a filtered current and 4 fixed sweeps
    dict(shape=(96, 80), prec=0, tol_rel=1e-5, kw=dict(m=4, filter_passes=3, courant=0.5), current=True),
]


@pytest.mark.parametrize("case", CASES, ids=["fp64_residual_64", "fp32_fixed_96x80"])
def test_step_static_matches_fmx_step_two_calls(fmx, case):
    import torch
    shape, prec = case["shape"], case["prec"]
    dtype = torch.float64 if prec == 1 else torch.float32
    ndt = np.float64 if prec == 1 else np.float32
    if case["current"]:
        E, B = synth.power_law_fields(shape, 8, 1907021, dtype=ndt)
        J = synth.solenoidal_current(shape, 1907022, width=4.0, rms=1e-2, dtype=ndt)
    else:
        po = core.Params(shape=shape, courant=0.5)
        E, B, _ = synth.tm_plane_waves(shape, po.time_step(), seed=1907001)
        E, B, J = E.astype(ndt), B.astype(ndt), None
    q = 2 if prec == 1 else 4
    pitch = (shape[0] + q - 1) // q * q
    p = fmx.make_params(shape, precision=prec, engine=fmx.FMX_ENGINE_STAGED,
                        stream=ctypes.c_void_p(torch.cuda.current_stream().cuda_stream), **case["kw"])
    Ed = _device_fields(shape, E, dtype, pitch)
    Bd = _device_fields(shape, B, dtype, pitch)
    Jd = _device_fields(shape, J, dtype, pitch) if J is not None else None
    ref = fmx.Grid(shape, with_current=J is not None, precision=prec, engine=fmx.FMX_ENGINE_STAGED, **case["kw"])
    ref.set_fields(E, B)
    if J is not None:
        ref.set_current(J)
    for call in range(2):
        st = fmx.fmx_step_static(ctypes.byref(p), _ptrs(Ed), _ptrs(Bd), _ptrs(Jd) if Jd is not None else None, 10)
        assert st == fmx.FMX_OK, fmx.fmx_last_error()
        torch.cuda.synchronize()
        ref.step(10)
        Er, Br, _ = ref.get_fields()
        Eg = Ed[:, :, :shape[0]].cpu().numpy()
        Bg = Bd[:, :, :shape[0]].cpu().numpy()
        for c in range(3):
            assert rel_l2(Eg[c], Er[c][0]) <= case["tol_rel"], (call, "E", c)
            assert rel_l2(Bg[c], Br[c][0]) <= case["tol_rel"], (call, "B", c)


def test_step_static_rejects_grids_beyond_its_scratch(fmx):
    import torch
    shape = (512, 512)  # FP64 staged workspace ~27 MB > 4 MiB
    p = fmx.make_params(shape, precision=1, m=4)
    t = torch.zeros((3, 512, 512), dtype=torch.float64, device="cuda")
    st = fmx.fmx_step_static(ctypes.byref(p), _ptrs(t), _ptrs(t), None, 1)
    assert st == fmx.FMX_EINVAL
    msg = fmx.fmx_last_error().decode()
    assert "scratch" in msg and str(fmx.FMX_STATIC_SCRATCH_BYTES) in msg
