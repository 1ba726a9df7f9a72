"""fmx_step_static: the step for callers that may not allocate device memory
(their device memory comes from their own pool or a budget fixed up front).
It must give what fmx_step gives on the same inputs, call after call, while
its intermediates live in the library's fixed device scratch array -- also
when calls on different grids and iteration modes alternate on that array."""
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


def _device_fields(arr, dtype, pitch):
    import torch
    _, nz, ny, nx = arr.shape
    t = torch.zeros((3, nz, ny, pitch), dtype=dtype, device="cuda")
    t[..., :nx] = torch.from_numpy(np.ascontiguousarray(arr)).to("cuda")
    return t


def _ptrs(t):
    return (ctypes.c_void_p * 3)(*[t[c].data_ptr() for c in range(3)])


CASES = {
    # the 64 x 64 FP64 residual-mode case (tol 1e-13), vacuum
    "fp64_residual_64": dict(shape=(64, 64), prec=1, tol_rel=1e-12, current=False,
                             kw=dict(iter_mode=1, tol=1e-13, m_max=10000, courant=0.5)),
    # an FP32 grid with a filtered current and 4 fixed sweeps
    "fp32_fixed_96x80": dict(shape=(96, 80), prec=0, tol_rel=1e-5, current=True,
                             kw=dict(m=4, filter_passes=3, courant=0.5)),
    # Chebyshev semi-iteration, fixed sweep count and residual stop (FP64)
    "fp64_cheb_fixed_48x40": dict(shape=(48, 40), prec=1, tol_rel=1e-12, current=True,
                                  kw=dict(iter_mode=2, m=8, filter_passes=1, courant=0.7)),
    "fp64_cheb_residual_48x40": dict(shape=(48, 40), prec=1, tol_rel=1e-12, current=True,
                                     kw=dict(iter_mode=3, tol=1e-13, m_max=10000, courant=0.7)),
    # 3D FP32 through the z-marching kernels (fixed m, one filter pass)
    "fp32_3d_24": dict(shape=(24, 24, 24), prec=0, tol_rel=1e-5, current=True,
                       kw=dict(m=4, filter_passes=1, courant=0.5)),
}


class _Case:
    """One grid advanced both by fmx_step_static (on caller-owned tensors)
    and by fmx_step (a bound Grid with its own workspace)."""

    def __init__(self, fmx, case):
        import torch
        shape, prec = case["shape"], case["prec"]
        self.fmx, self.case, self.shape = fmx, case, shape
        dtype = torch.float64 if prec == 1 else torch.float32
        ndt = np.float64 if prec == 1 else np.float32
        if case["current"]:
            E, B = synth.power_law_fields(shape, max(2, min(shape) // 8), 1907021, dtype=ndt)
            J = synth.solenoidal_current(shape, 1907022, width=4.0, rms=1e-2, dtype=ndt)
        else:
            po = core.Params(shape=shape, courant=0.5)
            E, B, _ = synth.tm_plane_waves(shape, po.time_step(), seed=1907001)
            E, B, J = E.astype(ndt), B.astype(ndt), None
        q = 2 if prec == 1 else 4
        pitch = (shape[0] + q - 1) // q * q
        self.p = fmx.make_params(shape, precision=prec, engine=fmx.FMX_ENGINE_STAGED,
                                 stream=ctypes.c_void_p(torch.cuda.current_stream().cuda_stream), **case["kw"])
        self.Ed = _device_fields(E, dtype, pitch)
        self.Bd = _device_fields(B, dtype, pitch)
        self.Jd = _device_fields(J, dtype, pitch) if J is not None else None
        self.ref = fmx.Grid(shape, with_current=J is not None, precision=prec, engine=fmx.FMX_ENGINE_STAGED,
                            **case["kw"])
        self.ref.set_fields(E, B)
        if J is not None:
            self.ref.set_current(J)

    def call_and_check(self, nsteps, tag):
        import torch
        fmx = self.fmx
        st = fmx.fmx_step_static(ctypes.byref(self.p), _ptrs(self.Ed), _ptrs(self.Bd),
                                 _ptrs(self.Jd) if self.Jd is not None else None, nsteps)
        assert st == fmx.FMX_OK, fmx.fmx_last_error()
        torch.cuda.synchronize()
        self.ref.step(nsteps)
        Er, Br, _ = self.ref.get_fields()
        nx = self.shape[0]
        Eg = self.Ed[..., :nx].cpu().numpy()
        Bg = self.Bd[..., :nx].cpu().numpy()
        tol = self.case["tol_rel"]
        for c in range(3):
            if np.any(Er[c]):
                assert rel_l2(Eg[c], Er[c]) <= tol, (tag, "E", c, rel_l2(Eg[c], Er[c]))
            if np.any(Br[c]):
                assert rel_l2(Bg[c], Br[c]) <= tol, (tag, "B", c, rel_l2(Bg[c], Br[c]))


@pytest.mark.parametrize("name", list(CASES))
def test_step_static_matches_fmx_step_two_calls(fmx, name):
    c = _Case(fmx, CASES[name])
    for call in range(2):
        c.call_and_check(10, (name, call))


def test_step_static_alternating_grids_and_modes(fmx):
    """Calls on different grid sizes, precisions and iteration modes take
    turns on the one scratch array; none may see another's leftovers."""
    cases = [_Case(fmx, CASES[n]) for n in CASES]
    for rnd in range(2):
        for name, c in zip(CASES, cases):
            c.call_and_check(3, (name, rnd))


def _staged_need(fmx, shape, prec):
    q = fmx.make_params(shape, precision=prec, m=4, engine=fmx.FMX_ENGINE_STAGED)
    return fmx.fmx_workspace_bytes(ctypes.byref(q))


def test_step_static_capacity_is_the_staged_workspace(fmx):
    """The largest square FP64 grid whose staged workspace fits the scratch
    runs; one cell wider per side is rejected."""
    import torch
    limit = fmx.FMX_STATIC_SCRATCH_BYTES
    n = 16
    while _staged_need(fmx, (n + 1, n + 1), 1) <= limit:
        n += 1
    assert _staged_need(fmx, (n, n), 1) <= limit < _staged_need(fmx, (n + 1, n + 1), 1)
    case = dict(shape=(n, n), prec=1, tol_rel=1e-12, current=True, kw=dict(m=4, filter_passes=1, courant=0.5))
    _Case(fmx, case).call_and_check(2, ("fits", n))
    big = n + 1
    p = fmx.make_params((big, big), precision=1, m=4)
    t = torch.zeros((3, big, (big + 1) // 2 * 2), dtype=torch.float64, device="cuda")
    st = fmx.fmx_step_static(ctypes.byref(p), _ptrs(t), _ptrs(t), None, 1)
    assert st == fmx.FMX_EINVAL
    msg = fmx.fmx_last_error().decode()
    assert "scratch" in msg and str(fmx.FMX_STATIC_SCRATCH_BYTES) in msg


def test_step_static_rejects_grids_beyond_its_scratch(fmx):
    import torch
    shape = (512, 512)  # FP64 staged workspace ~27 MB > 4 MiB
    p = fmx.make_params(shape, precision=1, m=4)
    t = torch.zeros((3, 512, 512), dtype=torch.float64, device="cuda")
    st = fmx.fmx_step_static(ctypes.byref(p), _ptrs(t), _ptrs(t), None, 1)
    assert st == fmx.FMX_EINVAL
    msg = fmx.fmx_last_error().decode()
    assert "scratch" in msg and str(fmx.FMX_STATIC_SCRATCH_BYTES) in msg


def test_step_static_rejects_host_fields(fmx):
    """The scratch is device memory of the current GPU: fields elsewhere are
    refused before anything is launched."""
    import torch
    shape = (32, 32)
    p = fmx.make_params(shape, precision=1, m=4)
    t = torch.zeros((3, 32, 32), dtype=torch.float64).pin_memory()
    st = fmx.fmx_step_static(ctypes.byref(p), _ptrs(t), _ptrs(t), None, 1)
    assert st == fmx.FMX_EINVAL
    assert b"device" in fmx.fmx_last_error()
