"""The resident engine (one thread-block cluster runs every step of an
fmx_step call in one launch, the residual stop decided on the device)
against the FP64 oracle and against the staged engine: fields per component
(FP64 1e-12, FP32 1e-5 relative L2), sweep counts per step equal to the
oracle's, the FMX_ENOCONV path, ragged cell counts that do not divide among
the cluster's threads, 1D/2D/3D, the current filter and the lumped scheme."""
import numpy as np
import pytest

from oracle import core
from paper_1907_13088_gb300 import synth
from tests.helpers import assert_parity

pytestmark = pytest.mark.gpu
TOL64, TOL32 = 1e-12, 1e-5


@pytest.fixture(scope="module")
def fmx():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1907_13088_gb300 import build
    build.build()
    from paper_1907_13088_gb300 import fmx as m
    return m


def _inputs(shape, seed, dtype, with_j=True):
    E, B, J = synth.random_fields(shape, seed)
    return E.astype(dtype), B.astype(dtype), (J.astype(dtype) if with_j else None)


def _run(fmx, shape, E, B, J, nsteps, **kw):
    g = fmx.Grid(shape, with_current=J is not None, **kw)
    g.set_fields(E, B)
    if J is not None:
        g.set_current(J)
    g.step(nsteps)
    Eg, Bg, _ = g.get_fields()
    return np.asarray(Eg, np.float64), np.asarray(Bg, np.float64), g


def test_plane_waves_64_fp64_residual_200_steps(fmx):
    """The 64 x 64 FP64 plane-wave case (tol 1e-13, 200 steps) in one launch:
    the automatic engine choice is the resident one, one launch per call,
    and every step's sweep count equals the oracle's."""
    shape = (64, 64)
    po = core.Params(shape=shape, courant=0.5, residual=True, tol=1e-13, m_max=10000)
    E, B, _ = synth.tm_plane_waves(shape, po.time_step(), seed=1907001)
    kw = dict(precision=1, iter_mode=1, tol=1e-13, m_max=10000, courant=0.5)
    g = fmx.Grid(shape, with_current=False, **kw)
    g.set_fields(E, B)
    g.step(200)
    assert g.launches == 1
    Eg, Bg, _ = g.get_fields()
    d = g.diagnostics()
    Eo, Bo, rc, st = core.step(po, E, B, None, 200)
    assert rc == core.OK
    assert_parity(np.asarray(Eg, np.float64), np.asarray(Bg, np.float64), Eo, Bo, TOL64, "resident 64x64")
    assert d["last_sweeps"] == st["last_sweeps"] and d["total_sweeps"] == st["total_sweeps"]
    assert d["steps"] == 200
    # per-step sweep counts: one call per step against the staged engine
    gr = fmx.Grid(shape, with_current=False, engine=fmx.FMX_ENGINE_RESIDENT, **kw)
    gs = fmx.Grid(shape, with_current=False, engine=fmx.FMX_ENGINE_STAGED, **kw)
    for h in (gr, gs):
        h.set_fields(E, B)
    for n in range(12):
        gr.step(1)
        gs.step(1)
        assert gr.diagnostics()["last_sweeps"] == gs.diagnostics()["last_sweeps"], n


CASES = [
    # shape, precision, iteration, filter passes, lumped
    ((64, 64), 1, "residual", 0, False),
    ((37, 29), 1, "residual", 2, False),   # ragged: 1073 cells over the cluster
    ((37, 29), 0, "residual", 1, False),
    ((50, 44), 1, "fixed", 3, False),
    ((50, 44), 0, "fixed", 3, False),
    ((12, 10, 9), 1, "residual", 1, False),
    ((12, 10, 9), 0, "fixed", 1, False),
    ((257,), 1, "residual", 2, False),
    ((30, 26), 1, "residual", 1, True),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{'x'.join(map(str, c[0]))}-{'f64' if c[1] else 'f32'}-"
                         f"{c[2]}-p{c[3]}{'-lumped' if c[4] else ''}")
def test_resident_matches_oracle(fmx, case):
    shape, prec, it, passes, lumped = case
    dt = np.float64 if prec == 1 else np.float32
    E, B, J = _inputs(shape, 91 + len(shape), dt)
    nsteps = 5
    resid = it == "residual"
    kw = dict(filter_passes=passes, courant=0.7, lumped=lumped)
    gkw = dict(kw, precision=prec, engine=fmx.FMX_ENGINE_RESIDENT)
    if resid:
        gkw.update(iter_mode=1, tol=1e-12 if prec == 1 else 1e-6, m_max=5000)
    else:
        gkw.update(m=4)
    Eg, Bg, g = _run(fmx, shape, E, B, J, nsteps, **gkw)
    assert g.launches == 1
    okw = dict(kw, coef_f32=prec == 0)
    if resid:
        okw.update(residual=True, tol=gkw["tol"], m_max=5000)
    else:
        okw.update(m=4)
    Eo, Bo, rc, st = core.step(core.Params(shape=shape, **okw), E.astype(np.float64), B.astype(np.float64),
                               J.astype(np.float64), nsteps)
    assert rc == core.OK
    assert_parity(Eg, Bg, Eo, Bo, TOL64 if prec == 1 else TOL32, f"resident {case}")
    d = g.diagnostics()
    if prec == 1 or not resid:
        assert d["total_sweeps"] == st["total_sweeps"], (d["total_sweeps"], st["total_sweeps"])


def test_resident_equals_staged_fp64(fmx):
    """Same arithmetic per cell as the staged kernels: the two engines agree
    to round-off over many steps with a current and a filter."""
    shape = (48, 40)
    E, B, J = _inputs(shape, 7, np.float64)
    kw = dict(precision=1, iter_mode=1, tol=1e-12, m_max=5000, filter_passes=2, courant=0.6)
    Er, Br, gr = _run(fmx, shape, E, B, J, 30, engine=fmx.FMX_ENGINE_RESIDENT, **kw)
    Es, Bs, gs = _run(fmx, shape, E, B, J, 30, engine=fmx.FMX_ENGINE_STAGED, **kw)
    assert_parity(Er, Br, Es, Bs, 1e-13, "resident vs staged")
    assert gr.diagnostics()["total_sweeps"] == gs.diagnostics()["total_sweeps"]


def test_resident_noconv(fmx):
    """m_max too small: FMX_ENOCONV, with the failing step applied (as the
    staged engine does) and the launch stopping there."""
    shape = (16, 16)
    E, B, _ = _inputs(shape, 5, np.float64, with_j=False)
    states = []
    for eng in (fmx.FMX_ENGINE_RESIDENT, fmx.FMX_ENGINE_STAGED):
        g = fmx.Grid(shape, with_current=False, precision=1, iter_mode=1, tol=1e-15, m_max=3, engine=eng)
        g.set_fields(E, B)
        with pytest.raises(fmx.FmxError) as ei:
            g.step(4)
        assert ei.value.status == fmx.FMX_ENOCONV
        states.append(g.get_fields()[:2])
    assert_parity(np.asarray(states[0][0], np.float64), np.asarray(states[0][1], np.float64),
                  np.asarray(states[1][0], np.float64), np.asarray(states[1][1], np.float64), 1e-13, "noconv")


def test_resident_time_profile_takes_staged_kernels(fmx):
    """A current time profile (one factor per step) is applied by the staged
    kernels; once it is used up the resident launch takes over again."""
    shape = (32, 24)
    E, B, J = _inputs(shape, 8, np.float64)
    kw = dict(precision=1, iter_mode=1, tol=1e-12, m_max=5000, courant=0.5)
    prof = [0.5, -1.0, 2.0]
    out = []
    for eng in (fmx.FMX_ENGINE_RESIDENT, fmx.FMX_ENGINE_STAGED):
        g = fmx.Grid(shape, with_current=True, engine=eng, **kw)
        g.set_fields(E, B)
        g.set_current(J)
        g.set_current_profile(prof)
        g.step(5)
        g.step(2)
        Eg, Bg, _ = g.get_fields()
        out.append((np.asarray(Eg, np.float64), np.asarray(Bg, np.float64)))
    assert_parity(out[0][0], out[0][1], out[1][0], out[1][1], 1e-13, "profile")


@pytest.mark.parametrize("n", [64, 128])
def test_resident_launch_clusters_and_parity_fp64(fmx, n):
    """FP64 solves above ~4096 cells spread over several clusters in one
    cooperative launch, synchronised by the bounded grid barrier (128^2: four
    clusters); 64^2 stays on one.  The result does not depend on how many."""
    shape = (n, n)
    po = core.Params(shape=shape, courant=0.5, residual=True, tol=1e-13, m_max=10000)
    E, B, _ = synth.tm_plane_waves(shape, po.time_step(), seed=1907001)
    g = fmx.Grid(shape, with_current=False, precision=1, iter_mode=1, tol=1e-13, m_max=10000, courant=0.5,
                 engine=fmx.FMX_ENGINE_RESIDENT)
    g.set_fields(E, B)
    g.step(20)
    ncl = g.get_option(fmx.FMX_OPT_RESIDENT_CLUSTERS)
    print("resident clusters", n, ncl)
    assert ncl == 1 if n == 64 else ncl >= 2
    Eg, Bg, _ = g.get_fields()
    Eo, Bo, rc, st = core.step(po, E, B, None, 20)
    assert_parity(np.asarray(Eg, np.float64), np.asarray(Bg, np.float64), Eo, Bo, TOL64, f"{ncl} clusters")
    assert g.diagnostics()["total_sweeps"] == st["total_sweeps"]


@pytest.mark.parametrize("prec,iter_mode", [(1, 1), (0, 0)])
def test_resident_grid_wait_times_out_and_the_context_survives(fmx, prec, iter_mode):
    """The bounded wait of the grid barrier: with one arrival that never comes
    (the self-test option) the first wait runs out after its limit, the call
    returns FMX_ETIMEOUT, and the same grid then steps normally (the
    context is intact) and matches the staged engine."""
    import time
    shape = (48, 40)
    dt = np.float64 if prec == 1 else np.float32
    E, B, J = _inputs(shape, 9, dt)
    kw = dict(precision=prec, iter_mode=iter_mode, courant=0.6, filter_passes=1)
    if iter_mode == 1:
        kw.update(tol=1e-12, m_max=5000)
    else:
        kw.update(m=4)
    g = fmx.Grid(shape, with_current=True, engine=fmx.FMX_ENGINE_RESIDENT, **kw)
    g.set_fields(E, B)
    g.set_current(J)
    g.set_option(fmx.FMX_OPT_WAIT_LIMIT_US, 20000)
    g.set_option(fmx.FMX_OPT_SELFTEST_LOST_ARRIVAL, 1)
    t0 = time.perf_counter()
    with pytest.raises(fmx.FmxError) as ei:
        g.step(3)
    waited = time.perf_counter() - t0
    assert ei.value.status == fmx.FMX_ETIMEOUT
    assert waited < 5.0, waited  # a 20 ms limit, not a hang
    g.set_option(fmx.FMX_OPT_SELFTEST_LOST_ARRIVAL, 0)
    g.set_fields(E, B)
    g.step(3)
    g.sync()
    Er, Br, _ = g.get_fields()
    Es, Bs, _ = _run(fmx, shape, E, B, J, 3, engine=fmx.FMX_ENGINE_STAGED, **kw)
    assert_parity(np.asarray(Er, np.float64), np.asarray(Br, np.float64), Es, Bs,
                  1e-13 if prec == 1 else 1e-6, "after a time-out")
