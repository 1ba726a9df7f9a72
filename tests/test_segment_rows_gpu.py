"""The segment height of the FP32 2D fused engine (FMX_OPT_SEGMENT_ROWS):
every CTA marches a segment of rows and recomputes the warm-up rows of its
pipeline, and each row's arithmetic does not depend on where a segment
starts, so any height gives the same fields to the bit, forward and
adjoint, and the automatic height matches the oracle."""
import ctypes

import numpy as np
import pytest

from oracle import core
from paper_1907_13088_gb300 import synth
from tests.helpers import assert_parity

pytestmark = pytest.mark.gpu

# a ragged grid: two strips (the second partial), 230 rows
SHAPE = (300, 230)
HEIGHTS = (0, 1, 7, 26, 100, 229, 230, 1000)


@pytest.fixture(scope="module")
def fmx():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1907_13088_gb300 import build
    build.build()
    from paper_1907_13088_gb300 import fmx as m
    return m


def _forward(fmx, rows, E, B, J, nsteps):
    g = fmx.Grid(SHAPE, precision=0, m=4, filter_passes=3, engine=fmx.FMX_ENGINE_FUSED, courant=0.5)
    g.set_option(fmx.FMX_OPT_SEGMENT_ROWS, rows)
    assert g.get_option(fmx.FMX_OPT_SEGMENT_ROWS) == rows
    g.set_fields(E, B)
    g.set_current(J)
    g.step(nsteps)
    Eg, Bg, _ = g.get_fields()
    g.close()
    return np.array(Eg), np.array(Bg)


def test_forward_any_segment_height_same_bits(fmx):
    E, B = synth.power_law_fields(SHAPE, 32, 1907031)
    J = synth.solenoidal_current(SHAPE, 1907032, width=8.0, rms=1e-2)
    ref = _forward(fmx, 0, E, B, J, 6)
    for rows in HEIGHTS[1:]:
        Eg, Bg = _forward(fmx, rows, E, B, J, 6)
        assert np.array_equal(Eg, ref[0]) and np.array_equal(Bg, ref[1]), rows
    p = core.Params(shape=SHAPE, courant=0.5, m=4, filter_passes=3, coef_f32=True)
    Eo, Bo, _, _ = core.step(p, E.astype(np.float64), B.astype(np.float64), J.astype(np.float64), 6)
    assert_parity(ref[0].astype(np.float64), ref[1].astype(np.float64), Eo, Bo, 1e-5, "segment rows automatic")


def _adjoint(fmx, rows, Ebar, Bbar):
    import torch
    g = fmx.Grid(SHAPE, precision=0, m=4, filter_passes=3, engine=fmx.FMX_ENGINE_FUSED, courant=0.5)
    g.set_option(fmx.FMX_OPT_SEGMENT_ROWS, rows)
    nx = SHAPE[0]
    pitch = (nx + 3) // 4 * 4
    dev = lambda a: torch.nn.functional.pad(torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)),
                                            (0, pitch - nx)).to("cuda").contiguous()
    Eb, Bb = dev(Ebar), dev(Bbar)
    jb = torch.zeros_like(Eb)
    wb = fmx.fmx_adjoint_workspace_bytes(ctypes.byref(g.params))
    work = torch.zeros(wb + 256, dtype=torch.uint8, device="cuda")
    wp = (work.data_ptr() + 255) // 256 * 256
    vp = lambda t: (ctypes.c_void_p * 3)(*[t[c].data_ptr() for c in range(3)])
    fmx.check(fmx.fmx_adjoint_step(g.handle, vp(Eb), vp(Bb), vp(jb), wp, wb))
    torch.cuda.synchronize()
    out = [t[..., :nx].cpu().numpy() for t in (Eb, Bb, jb)]
    g.close()
    return out


def test_adjoint_any_segment_height_same_bits(fmx):
    Ebar, Bbar, _ = (x.astype(np.float32) for x in synth.random_fields(SHAPE, seed=1907033))
    ref = _adjoint(fmx, 0, Ebar, Bbar)
    for rows in HEIGHTS[1:]:
        got = _adjoint(fmx, rows, Ebar, Bbar)
        for a, b, name in zip(got, ref, ("Ebar", "Bbar", "jbar")):
            assert np.array_equal(a, b), (rows, name)
    Eo, Bo, jo = core.adjoint_step(core.Params(shape=SHAPE, courant=0.5, m=4, filter_passes=3, coef_f32=True),
                                   Ebar.astype(np.float64), Bbar.astype(np.float64))
    for a, b in ((ref[0], Eo), (ref[1], Bo), (ref[2], jo)):
        a = a.astype(np.float64).reshape(b.shape)
        assert np.linalg.norm(a - b) <= 1e-5 * np.linalg.norm(b)
