"""Two sweeps of Algorithm 1 per z-march pass (FMX_OPT_SWEEPS_PER_PASS = 2,
3D FP32): the temporally blocked kernels against the FP64 oracle (FP32
rounded inputs and coefficients) and against the one-sweep-per-pass kernels,
per component at the FP32 tolerance, 1e-5 relative L2: even and odd m,
partial tiles with periodic wrap in x, y and z, a current with the one-pass
filter, the 200-step 64^3 recipe, and windows of the 512^3 workload."""
import numpy as np
import pytest

from oracle import core
from paper_1907_13088_gb300 import synth
from tests.helpers import assert_parity, rel_l2

pytestmark = pytest.mark.gpu
TOL32 = 1e-5


@pytest.fixture(scope="module")
def fmx():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1907_13088_gb300 import build
    build.build()
    from paper_1907_13088_gb300 import fmx as m
    return m


def _run(fmx, shape, E, B, J, nsteps, spp, **kw):
    g = fmx.Grid(shape, with_current=J is not None, precision=0, **kw)
    g.set_option(fmx.FMX_OPT_SWEEPS_PER_PASS, spp)
    g.set_fields(E, B)
    if J is not None:
        g.set_current(J)
    l0 = g.launches
    g.step(nsteps)
    Eg, Bg, _ = g.get_fields()
    return np.asarray(Eg, np.float64), np.asarray(Bg, np.float64), g.launches - l0


@pytest.mark.parametrize("shape,m,passes", [((64, 24, 20), 4, 1), ((100, 36, 17), 4, 1), ((70, 13, 9), 3, 0),
                                            ((130, 8, 33), 2, 1), ((64, 16, 40), 5, 1)])
def test_two_sweeps_per_pass_match_oracle(fmx, shape, m, passes):
    E, B, J = synth.random_fields(shape, 401)
    E, B, J = (a.astype(np.float32) for a in (E, B, J))
    nsteps = 3
    kw = dict(m=m, filter_passes=passes, courant=0.6)
    Eg, Bg, launches = _run(fmx, shape, E, B, J, nsteps, 2, **kw)
    Eo, Bo, rc, _ = core.step(core.Params(shape=shape, coef_f32=True, **kw), E.astype(np.float64),
                              B.astype(np.float64), J.astype(np.float64), nsteps)
    assert rc == core.OK
    assert_parity(Eg, Bg, Eo, Bo, TOL32, f"2 sweeps/pass {shape} m={m}")
    # source, ceil(m/2) sweep passes (the last with the update), Faraday
    assert launches == nsteps * (2 + (m + 1) // 2), launches
    E1, B1, _ = _run(fmx, shape, E, B, J, nsteps, 1, **kw)
    for c in range(3):
        assert rel_l2(Eg[c], E1[c]) < 2e-6 and rel_l2(Bg[c], B1[c]) < 2e-6, c


def test_two_sweeps_per_pass_64_cubed_200_steps(fmx):
    n, nsteps = 64, 200
    shape = (n, n, n)
    E, B = synth.power_law_fields(shape, n // 8, 1907003, dtype=np.float32)
    J = synth.solenoidal_current(shape, 1907013, width=16.0, rms=1e-3, dtype=np.float32)
    kw = dict(m=4, filter_passes=1, courant=0.5)
    Eg, Bg, _ = _run(fmx, shape, E, B, J, nsteps, 2, **kw)
    Eo, Bo, _, _ = core.step(core.Params(shape=shape, coef_f32=True, **kw), E.astype(np.float64),
                             B.astype(np.float64), J.astype(np.float64), nsteps)
    assert_parity(Eg, Bg, Eo, Bo, TOL32, "3d 64^3 x200, 2 sweeps per pass")


def _window3(a, center, size):
    nz, ny, nx = a.shape[-3:]
    idx = [np.arange(c - size // 2, c - size // 2 + size) % n for c, n in zip(center, (nz, ny, nx))]
    return a[:, idx[0][:, None, None], idx[1][None, :, None], idx[2][None, None, :]]


def test_two_sweeps_per_pass_512_cubed_windows(fmx):
    n, nsteps = 512, 2
    E, B = synth.power_law_fields((n, n, n), n // 8, 1907003, dtype=np.float32)
    J = synth.solenoidal_current((n, n, n), 1907013, width=16.0, rms=1e-3, dtype=np.float32)
    g = fmx.Grid((n, n, n), precision=0, m=4, filter_passes=1, courant=0.5)
    g.set_option(fmx.FMX_OPT_SWEEPS_PER_PASS, 2)
    g.set_fields(E, B)
    g.set_current(J)
    g.step(nsteps)
    Eg, Bg, _ = g.get_fields()
    g.close()
    radius = 7 * nsteps
    size = 2 * radius + 8
    p = core.Params(shape=(size, size, size), courant=0.5, m=4, filter_passes=1, coef_f32=True)
    lo, hi = radius + 1, size - radius - 1
    for ctr in [(0, 0, 0), (511, 511, 511), (300, 63, 64), (17, 448, 200)]:
        w = lambda a: _window3(a, ctr, size).astype(np.float64)
        Eo, Bo, _, _ = core.step(p, w(E), w(B), w(J), nsteps)
        for F_g, F_o in ((Eg, Eo), (Bg, Bo)):
            Fw = _window3(F_g, ctr, size).astype(np.float64)
            for c in range(3):
                e = rel_l2(Fw[c, lo:hi, lo:hi, lo:hi], F_o[c, lo:hi, lo:hi, lo:hi])
                assert e < TOL32, (ctr, c, e)
