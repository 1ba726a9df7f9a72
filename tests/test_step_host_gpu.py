"""fmx_step_host (steps streamed from and to host memory) against the same
steps made with fmx_set_fields / fmx_set_current / fmx_step / fmx_get_fields:
identical results on the fused engine (pipelined copies, state sets 0 -> 1)
and on the staged engine (copies in order), with a new current every step,
with the bound current kept, and with read-back skipped for some steps."""
import numpy as np
import pytest

from paper_1907_13088_gb300 import synth

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


def _pinned(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()


@pytest.mark.parametrize("engine,prec,shape", [(2, 0, (256, 200)), (2, 1, (96, 80)), (1, 0, (60, 44)),
                                               (2, 0, (131, 70))])
def test_step_host_equals_separate_calls(fmx, engine, prec, shape):
    dt = np.float64 if prec else np.float32
    kw = dict(precision=prec, m=4, filter_passes=2, courant=0.5, engine=engine)
    steps_in = []
    for i in range(4):
        E, B, J = synth.random_fields(shape, 300 + i)
        J = J * 0.01 if i != 2 else None  # step 2 keeps the bound current
        arr = np.concatenate([E, B] + ([J] if J is not None else [])).astype(dt)
        steps_in.append(_pinned(arr))
    outs = [_pinned(np.zeros((6, 1, shape[1], shape[0]), dt)) for _ in range(4)]
    outs[1] = None  # no read-back of step 1
    g = fmx.Grid(shape, with_current=True, **kw)
    g.step_host(list(zip(steps_in, outs)))
    ref = fmx.Grid(shape, with_current=True, **kw)
    for i, a in enumerate(steps_in):
        ref.set_fields(a[0:3], a[3:6])
        if len(a) == 9:
            ref.set_current(a[6:9])
        ref.step(1)
        if outs[i] is None:
            continue
        Er, Br, _ = ref.get_fields()
        np.testing.assert_array_equal(outs[i][0:3], Er, err_msg=f"E step {i}")
        np.testing.assert_array_equal(outs[i][3:6], Br, err_msg=f"B step {i}")
    # the grid is left holding the last step's state
    E2, B2, _ = g.get_fields()
    np.testing.assert_array_equal(E2, outs[3][0:3])
    g.step(2)
    ref.step(2)
    np.testing.assert_array_equal(g.get_fields()[0], ref.get_fields()[0])
    assert g.diagnostics()["steps"] == 6


def test_step_host_argument_checks(fmx):
    import ctypes
    g = fmx.Grid((32, 32), with_current=False, precision=0, m=4)
    rec = (fmx.fmx_host_step * 1)()
    assert fmx.fmx_step_host(g.handle, rec, 1) == fmx.FMX_EINVAL  # NULL inputs
    a = np.zeros((9, 1, 32, 32), np.float32)
    for c in range(9):
        rec[0].inp[c] = a[c].ctypes.data
    assert fmx.fmx_step_host(g.handle, rec, 1) == fmx.FMX_ESTATE  # a current but no J bound
    rec[0].inp[7] = None
    assert fmx.fmx_step_host(g.handle, rec, 1) == fmx.FMX_EINVAL  # partial current
    assert fmx.fmx_step_host(g.handle, rec, -1) == fmx.FMX_EINVAL
    assert fmx.fmx_step_host(g.handle, ctypes.cast(None, ctypes.POINTER(fmx.fmx_host_step)), 0) == fmx.FMX_OK
