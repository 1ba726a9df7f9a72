"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Tolerances, per field component, relative L2 ||gpu - oracle|| / ||oracle||:
FP64 path 1e-12, FP32 path 1e-5.  FP32 runs start from the FP32-rounded
inputs and the oracle uses the FP32-rounded coefficients the kernels
multiply by (the oracle still computes in FP64).
"""
import numpy as np
import pytest

from oracle import core
from paper_1907_13088_gb300 import synth
from tests.helpers import assert_parity, periodic_window, rel_l2

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


def _run_gpu(fmx, shape, E, B, J, nsteps, **kw):
    g = fmx.Grid(shape, with_current=J is not None, **kw)
    g.set_fields(E, B)
    if J is not None:
        g.set_current(J)
    g.step(nsteps)
    E1, B1, _ = g.get_fields()
    info = {"launches": g.launches, "diag": None, "grid": g}
    return np.array(E1, dtype=np.float64), np.array(B1, dtype=np.float64), info


def _oracle(shape, E, B, J, nsteps, **kw):
    p = core.Params(shape=tuple(shape), **kw)
    E1, B1, rc, st = core.step(p, E, B, J, nsteps)
    return E1, B1, rc, st


def _inputs(shape, seed, dtype, with_j=True, smooth=False):
    if smooth:
        kmax = max(2, min(shape) // 8)
        E, B = synth.power_law_fields(shape, kmax, seed, dtype=np.float64)
        J = synth.solenoidal_current(shape, seed + 1, width=2.0, rms=1e-2, dtype=np.float64) if with_j else None
    else:
        E, B, J = synth.random_fields(shape, seed)
        if not with_j:
            J = None
    E = E.astype(dtype)
    B = B.astype(dtype)
    J = J.astype(dtype) if J is not None else None
    return E, B, J


ENGINE = {"staged": 1, "fused": 2}


# ---------------------------------------------------------------------------
# FP64, both engines, 1D/2D/3D, ragged sizes, every filter/sweep count
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("shape", [(37, 29), (5, 3), (1, 8), (7, 1), (300, 41)])
@pytest.mark.parametrize("engine", ["staged", "fused"])
def test_fp64_2d_random(fmx, shape, engine):
    E, B, J = _inputs(shape, 21, np.float64)
    Eg, Bg, _ = _run_gpu(fmx, shape, E, B, J, 6, precision=1, m=4, filter_passes=3, engine=ENGINE[engine])
    Eo, Bo, rc, _ = _oracle(shape, E, B, J, 6, m=4, filter_passes=3)
    assert_parity(Eg, Bg, Eo, Bo, TOL64, f"{engine} {shape}")


@pytest.mark.parametrize("m", [0, 1, 2, 3, 4])
@pytest.mark.parametrize("passes", [0, 1, 2, 3, None])
def test_fused_fp64_every_instantiation(fmx, m, passes):
    shape = (53, 47)
    E, B, J = _inputs(shape, 100 + m, np.float64, with_j=passes is not None)
    p = passes or 0
    Eg, Bg, _ = _run_gpu(fmx, shape, E, B, J, 5, precision=1, m=m, filter_passes=p, engine=2, courant=0.8)
    Eo, Bo, rc, _ = _oracle(shape, E, B, J, 5, m=m, filter_passes=p, courant=0.8)
    assert_parity(Eg, Bg, Eo, Bo, TOL64, f"fused m={m} p={passes}")


@pytest.mark.parametrize("m", [0, 1, 2, 3, 4])
@pytest.mark.parametrize("passes", [0, 1, 2, 3, None])
def test_fused_fp32_every_instantiation(fmx, m, passes):
    """FP32 fused path, the polarisation-split kernels: even n_x (556 has
    three strips, the first and last wrapping the periodic seam) and odd n_x
    (261: seam strips with single-column loads), every (m, passes) pair,
    several strips and segments, against the oracle with FP32-rounded
    coefficients."""
    for shape in ((262, 97), (556, 97), (261, 97)):
        E, B, J = _inputs(shape, 200 + m, np.float32, with_j=passes is not None, smooth=True)
        p = passes or 0
        Eg, Bg, _ = _run_gpu(fmx, shape, E, B, J, 7, precision=0, m=m, filter_passes=p, engine=2, courant=0.8)
        Eo, Bo, rc, _ = _oracle(shape, E.astype(np.float64), B.astype(np.float64),
                                None if J is None else J.astype(np.float64), 7, m=m, filter_passes=p, courant=0.8,
                                coef_f32=True)
        assert_parity(Eg, Bg, Eo, Bo, TOL32, f"fused fp32 {shape} m={m} p={passes}")


@pytest.mark.parametrize("shape", [(2, 2), (4, 3), (2, 9), (600, 2), (1030, 6), (272, 3), (276, 1),
                                   (1, 8), (3, 5), (5, 3), (7, 1), (257, 9), (511, 33), (513, 40)])
def test_fused_fp32_small_and_thin(fmx, shape):
    """Small, thin and odd-n_x FP32 grids on the fused path: with odd n_x the
    strips that cross the periodic seam load single columns (n_x = 1 to 513:
    one strip, two, three with an interior strip)."""
    E, B, J = _inputs(shape, 301, np.float32)
    Eg, Bg, _ = _run_gpu(fmx, shape, E, B, J, 5, precision=0, m=4, filter_passes=3, engine=2)
    Eo, Bo, rc, _ = _oracle(shape, E.astype(np.float64), B.astype(np.float64), J.astype(np.float64), 5, m=4,
                            filter_passes=3, coef_f32=True)
    assert_parity(Eg, Bg, Eo, Bo, TOL32, f"fp32 thin {shape}")


@pytest.mark.parametrize("shape", [(13, 11, 7), (9, 8, 6), (40,), (17, 1, 5)])
def test_staged_fp64_3d_1d(fmx, shape):
    E, B, J = _inputs(shape, 31, np.float64)
    kw = dict(m=3, filter_passes=1, courant=0.7, d=(1.0, 0.8, 1.2))
    Eg, Bg, _ = _run_gpu(fmx, shape, E, B, J, 5, precision=1, engine=1, **kw)
    Eo, Bo, rc, _ = _oracle(shape, E, B, J, 5, **kw)
    assert_parity(Eg, Bg, Eo, Bo, TOL64, f"staged {shape}")


@pytest.mark.parametrize("shape", [(37, 11, 70), (70, 11, 37), (8, 6, 5)])
@pytest.mark.parametrize("kw", [dict(m=4, filter_passes=0), dict(m=2, filter_passes=2), dict(m=1, filter_passes=1),
                                dict(m=0, filter_passes=1)])
def test_3d_march_and_staged_branches(fmx, kw, shape):
    """3D: the z-marching kernels (at most one filter pass on the current;
    several z segments and tiles, ragged in every axis) and the staged
    fallback (two passes), FP64 and FP32, with and without a current.  Odd
    n_x takes the one-column FP32 sweep; even n_x the column-pair sweep
    (with the E update fused into the last sweep), here with a ragged second
    x tile and an odd number of planes in the last z segment (70, 11, 37),
    and with n_x below the tile width (8, 6, 5)."""
    E, B, J = _inputs(shape, 33, np.float64)
    for with_j in (True, False):
        Jw = J if with_j else None
        Eg, Bg, _ = _run_gpu(fmx, shape, E, B, Jw, 3, precision=1, engine=1, courant=0.6, **kw)
        Eo, Bo, rc, _ = _oracle(shape, E, B, Jw, 3, courant=0.6, **kw)
        assert_parity(Eg, Bg, Eo, Bo, TOL64, f"3d fp64 {kw} j={with_j}")
    E32, B32, J32 = (x.astype(np.float32) for x in (E, B, J))
    Eg, Bg, _ = _run_gpu(fmx, shape, E32, B32, J32, 3, precision=0, engine=1, courant=0.6, **kw)
    Eo, Bo, rc, _ = _oracle(shape, E32.astype(np.float64), B32.astype(np.float64), J32.astype(np.float64), 3,
                            courant=0.6, coef_f32=True, **kw)
    assert_parity(Eg, Bg, Eo, Bo, TOL32, f"3d fp32 {kw}")


@pytest.mark.parametrize("shape", [(37, 29), (13, 11, 7), (40,)])
def test_chebyshev_modes(fmx, shape):
    """Chebyshev acceleration (staged engine): m sweeps and residual mode, FP64
    against the oracle's Chebyshev solve; FP32 with the FP32-rounded
    coefficients; residual mode needs fewer sweeps than Algorithm 1."""
    E, B, J = _inputs(shape, 91, np.float64)
    kw = dict(m=5, filter_passes=1, courant=0.8)
    Eg, Bg, _ = _run_gpu(fmx, shape, E, B, J, 3, precision=1, engine=1, iter_mode=fmx.FMX_ITER_CHEB_FIXED, **kw)
    Eo, Bo, rc, _ = _oracle(shape, E, B, J, 3, cheb=True, **kw)
    assert_parity(Eg, Bg, Eo, Bo, TOL64, f"chebyshev fixed fp64 {shape}")
    E32, B32, J32 = (x.astype(np.float32) for x in (E, B, J))
    Eg, Bg, _ = _run_gpu(fmx, shape, E32, B32, J32, 3, precision=0, engine=1, iter_mode=fmx.FMX_ITER_CHEB_FIXED, **kw)
    Eo, Bo, rc, _ = _oracle(shape, E32.astype(np.float64), B32.astype(np.float64), J32.astype(np.float64), 3,
                            cheb=True, coef_f32=True, **kw)
    assert_parity(Eg, Bg, Eo, Bo, TOL32, f"chebyshev fixed fp32 {shape}")
    rk = dict(filter_passes=1, courant=0.8, tol=1e-12, m_max=5000)
    Eg, Bg, info = _run_gpu(fmx, shape, E, B, J, 3, precision=1, engine=1, iter_mode=fmx.FMX_ITER_CHEB_RESIDUAL, **rk)
    Eo, Bo, rc, st = _oracle(shape, E, B, J, 3, cheb=True, residual=True, **rk)
    assert_parity(Eg, Bg, Eo, Bo, TOL64, f"chebyshev residual fp64 {shape}")
    d_cheb = info["grid"].diagnostics()
    _, _, info_j = _run_gpu(fmx, shape, E, B, J, 3, precision=1, engine=1, iter_mode=fmx.FMX_ITER_RESIDUAL, **rk)
    d_jac = info_j["grid"].diagnostics()
    assert d_cheb["last_sweeps"] == st["last_sweeps"]
    assert d_cheb["total_sweeps"] < d_jac["total_sweeps"]


def test_staged_fields_filter_and_lumped(fmx):
    shape = (24, 18)
    E, B, J = _inputs(shape, 41, np.float64)
    kw = dict(m=2, filter_passes=2, filter_target=core.FILTER_FIELDS, courant=0.6)
    Eg, Bg, _ = _run_gpu(fmx, shape, E, B, J, 4, precision=1, engine=1, **kw)
    Eo, Bo, rc, _ = _oracle(shape, E, B, J, 4, **kw)
    assert_parity(Eg, Bg, Eo, Bo, TOL64, "fields filter")
    for eng in (1, 2):
        Eg, Bg, _ = _run_gpu(fmx, shape, E, B, J, 4, precision=1, engine=eng, lumped=True, filter_passes=1)
        Eo, Bo, rc, _ = _oracle(shape, E, B, J, 4, lumped=True, filter_passes=1)
        assert_parity(Eg, Bg, Eo, Bo, TOL64, f"lumped engine {eng}")
    # FP32 lumped with an even n_x: the fused engine's single-kernel path
    E32, B32, J32 = (x.astype(np.float32) for x in (E, B, J))
    Eg, Bg, _ = _run_gpu(fmx, shape, E32, B32, J32, 4, precision=0, engine=2, lumped=True, filter_passes=1)
    Eo, Bo, rc, _ = _oracle(shape, E32.astype(np.float64), B32.astype(np.float64), J32.astype(np.float64), 4,
                            lumped=True, filter_passes=1, coef_f32=True)
    assert_parity(Eg, Bg, Eo, Bo, TOL32, "lumped fp32 fused")


# ---------------------------------------------------------------------------
# residual mode: the 64x64 FP64 plane-wave case (200 steps, tol 1e-13)
# ---------------------------------------------------------------------------

def test_residual_mode_plane_waves_64(fmx):
    shape = (64, 64)
    po = core.Params(shape=shape, courant=0.5, residual=True, tol=1e-13, m_max=10000)
    E, B, _ = synth.tm_plane_waves(shape, po.time_step(), seed=1907001)
    Eg, Bg, info = _run_gpu(fmx, shape, E, B, None, 200, precision=1, iter_mode=1, tol=1e-13, m_max=10000,
                            courant=0.5)
    d = info["grid"].diagnostics()
    Eo, Bo, rc, st = _oracle(shape, E, B, None, 200, courant=0.5, residual=True, tol=1e-13, m_max=10000)
    assert rc == core.OK
    errs = assert_parity(Eg, Bg, Eo, Bo, TOL64, "residual 64x64")
    assert d["last_sweeps"] == st["last_sweeps"] and d["total_sweeps"] == st["total_sweeps"]
    assert d["steps"] == 200
    # TE part stays exactly zero (Sec. 2.2.2 decoupling)
    assert np.all(Eg[:2] == 0) and np.all(Bg[2] == 0)
    del errs


@pytest.mark.parametrize("iter_mode", ["jacobi", "chebyshev"])
@pytest.mark.parametrize("order", ["rough_first", "smooth_first"])
def test_residual_mode_sweep_count_changes(fmx, iter_mode, order):
    """Residual mode when the solve length changes from one step to the next:
    rough fields (high-k content, eigenvalues of A near the Brillouin-zone
    corner) need many more sweeps than smooth ones.  The host launches the
    previous solve's count first, so after rough -> smooth the sweeps past the
    stop must leave the state untouched, and after smooth -> rough further
    chunks must follow.  Every step against the oracle: fields and sweeps."""
    shape = (40, 36)
    cheb = iter_mode == "chebyshev"
    mode = fmx.FMX_ITER_CHEB_RESIDUAL if cheb else fmx.FMX_ITER_RESIDUAL
    kw = dict(filter_passes=1, courant=0.8, tol=1e-12, m_max=5000)
    rough = _inputs(shape, 17, np.float64)
    smooth = _inputs(shape, 18, np.float64, smooth=True)
    seq = [rough, smooth] if order == "rough_first" else [smooth, rough]
    g = fmx.Grid(shape, with_current=True, precision=1, engine=1, iter_mode=mode, **kw)
    counts = []
    for E, B, J in seq + seq[:1]:
        g.set_fields(E, B)
        g.set_current(J)
        g.step(1)
        Eg, Bg, _ = g.get_fields()
        Eo, Bo, rc, st = _oracle(shape, E, B, J, 1, cheb=cheb, residual=True, **kw)
        assert rc == core.OK
        assert_parity(np.asarray(Eg, np.float64), np.asarray(Bg, np.float64), Eo, Bo, TOL64,
                      f"residual {iter_mode} {order} step {len(counts)}")
        d = g.diagnostics()
        assert d["last_sweeps"] == st["last_sweeps"], (d["last_sweeps"], st["last_sweeps"])
        counts.append(d["last_sweeps"])
    # the two inputs need different solve lengths (Algorithm 1: 78 and 33
    # sweeps; Chebyshev: 26 and 24), so one order runs sweeps past the stop
    # and the other a further chunk
    assert counts[0] != counts[1], counts
    assert counts[2] == counts[0]


def test_residual_mode_noconv(fmx):
    shape = (16, 16)
    E, B, J = _inputs(shape, 5, np.float64)
    g = fmx.Grid(shape, with_current=False, precision=1, iter_mode=1, tol=1e-15, m_max=3, engine=1)
    g.set_fields(E, B)
    with pytest.raises(fmx.FmxError) as ei:
        g.step(1)
    assert ei.value.status == fmx.FMX_ENOCONV


# ---------------------------------------------------------------------------
# FP32 against the oracle with FP32-rounded coefficients
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("engine", ["staged", "fused"])
@pytest.mark.parametrize("shape,nsteps", [((96, 80), 100), ((517, 263), 20)])
def test_fp32_smooth_fields(fmx, engine, shape, nsteps):
    E, B, J = _inputs(shape, 51, np.float32, smooth=True)
    Eg, Bg, _ = _run_gpu(fmx, shape, E, B, J, nsteps, precision=0, m=4, filter_passes=3, engine=ENGINE[engine])
    Eo, Bo, rc, _ = _oracle(shape, E.astype(np.float64), B.astype(np.float64), J.astype(np.float64), nsteps,
                            m=4, filter_passes=3, coef_f32=True)
    assert_parity(Eg, Bg, Eo, Bo, TOL32, f"fp32 {engine} {shape}")


def test_engines_agree_fp64(fmx):
    shape = (611, 233)
    E, B, J = _inputs(shape, 61, np.float64, smooth=True)
    E1, B1, _ = _run_gpu(fmx, shape, E, B, J, 8, precision=1, m=4, filter_passes=3, engine=1)
    E2, B2, _ = _run_gpu(fmx, shape, E, B, J, 8, precision=1, m=4, filter_passes=3, engine=2)
    assert_parity(E2, B2, E1, B1, 1e-13, "fused vs staged")


# ---------------------------------------------------------------------------
# the benchmark configuration at full size: 4096^2 FP32, m = 4, 3 passes,
# in the fused launch bench.py times; sampled windows against the oracle
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("nsteps", [1, 3])
def test_full_size_4096_windows(fmx, nsteps):
    shape = (4096, 4096)
    E, B = synth.power_law_fields(shape, 512, 1907002)
    J = synth.solenoidal_current(shape, 1907003, width=16.0, rms=1e-3)
    g = fmx.Grid(shape, precision=0, m=4, filter_passes=3, engine=2, courant=0.5)
    g.set_fields(E, B)
    g.set_current(J)
    g.step(nsteps)
    Eg, Bg, _ = g.get_fields()
    radius = 8 * nsteps  # one step reaches 8 cells (3 filter + 4 sweeps + 1 curl)
    size = 2 * radius + 40
    rng = np.random.default_rng(7)
    centers = [(0, 0), (4095, 4095), (0, 2048), (2048, 4095)] + [tuple(rng.integers(0, 4096, 2)) for _ in range(6)]
    p = core.Params(shape=(size, size), courant=0.5, m=4, filter_passes=3, coef_f32=True)
    worst = 0.0
    for cy, cx in centers:
        w = lambda a: periodic_window(a, (cy, cx), size).astype(np.float64)
        Eo, Bo, rc, _ = core.step(p, w(E), w(B), w(J), nsteps)
        lo, hi = radius + 1, size - radius - 1
        sl = (slice(None), slice(None), slice(lo, hi), slice(lo, hi))
        for F_g, F_o in ((Eg, Eo), (Bg, Bo)):
            Fw = periodic_window(F_g, (cy, cx), size).astype(np.float64)
            for c in range(3):
                e = rel_l2(Fw[c][sl[1:]], F_o[c][sl[1:]])
                worst = max(worst, e)
                assert e < TOL32, (cy, cx, c, e)
    assert g.launches == 2 * nsteps  # one TE and one TM launch per step


# ---------------------------------------------------------------------------
# standalone filter, diagnostics, state handling
# ---------------------------------------------------------------------------

def test_standalone_filter(fmx):
    for shape in ((33, 21), (10, 9, 7)):
        E, B, J = _inputs(shape, 71, np.float64)
        g = fmx.Grid(shape, precision=1, engine=1)
        g.set_fields(E, B)
        g.set_current(J)
        g.filter(fmx.FMX_E | fmx.FMX_JZ, 3)
        Eg, Bg, Jg = g.get_fields(fmx.FMX_E | fmx.FMX_B | fmx.FMX_J)
        p = core.Params(shape=shape)
        assert rel_l2(Eg, core.filter(p, E, 3)) < 1e-14
        assert np.array_equal(np.asarray(Bg), B)
        assert rel_l2(Jg[2], core.filter(p, J[2:3], 3)[0]) < 1e-14
        assert np.array_equal(np.asarray(Jg[:2]), J[:2])


@pytest.mark.parametrize("shape,prec", [((48, 40), 1), ((12, 10, 9), 1), ((64, 56), 0)])
def test_diagnostics_match_oracle(fmx, shape, prec):
    dtype = np.float64 if prec == 1 else np.float32
    E, B, J = _inputs(shape, 81, dtype)
    kw = dict(courant=0.7, m=3)
    g = fmx.Grid(shape, precision=prec, engine=1, **kw)
    g.set_fields(E, B)
    d = g.diagnostics()
    p = core.Params(shape=shape, coef_f32=(prec == 0), **kw)
    E64, B64 = E.astype(np.float64), B.astype(np.float64)
    ws, wp = core.energy(p, E64, B64)
    db = core.div_b(p, B64)
    ge = core.gauss_e(p, E64)
    assert abs(d["w_scheme"] - ws) <= 1e-12 * abs(ws)
    assert abs(d["w_plain"] - wp) <= 1e-12 * abs(wp)
    assert abs(d["divb_max"] - np.max(np.abs(db))) <= 1e-12 * np.max(np.abs(db))
    assert abs(d["divb_l2"] - np.linalg.norm(db)) <= 1e-12 * np.linalg.norm(db)
    assert abs(d["gauss_max"] - np.max(np.abs(ge))) <= 1e-12 * np.max(np.abs(ge))
    assert abs(d["gauss_l2"] - np.linalg.norm(ge)) <= 1e-12 * np.linalg.norm(ge)


def test_zero_steps_and_state_sets(fmx):
    shape = (40, 30)
    E, B, J = _inputs(shape, 91, np.float32)
    g = fmx.Grid(shape, precision=0, m=4, filter_passes=3, engine=2)
    g.set_fields(E, B)
    g.set_current(J)
    g.step(0)
    E0, B0, _ = g.get_fields()
    assert np.array_equal(E0, E) and np.array_equal(B0, B)
    g.step(3)  # odd count: the state now lives in set 1
    E3, B3, _ = g.get_fields()
    g2 = fmx.Grid(shape, precision=0, m=4, filter_passes=3, engine=2)
    g2.set_fields(E, B)
    g2.set_current(J)
    for _ in range(3):
        g2.step(1)
    E3b, B3b, _ = g2.get_fields()
    assert np.array_equal(E3, E3b) and np.array_equal(B3, B3b)
    # set_fields after steps writes the current set
    g.set_fields(E, B)
    g.step(1)
    E1, B1, _ = g.get_fields()
    g3 = fmx.Grid(shape, precision=0, m=4, filter_passes=3, engine=2)
    g3.set_fields(E, B)
    g3.set_current(J)
    g3.step(1)
    E1b, B1b, _ = g3.get_fields()
    assert np.array_equal(E1, E1b) and np.array_equal(B1, B1b)


def test_conservation_on_gpu_fp64(fmx):
    """div B is preserved to round-off by the GPU step for any m (App. A)."""
    shape = (128, 96)
    E, B, J = _inputs(shape, 95, np.float64)
    g = fmx.Grid(shape, precision=1, m=4, filter_passes=3, engine=2)
    g.set_fields(E, B)
    g.set_current(J)
    d0 = g.diagnostics()
    g.step(50)
    d1 = g.diagnostics()
    p = core.Params(shape=shape)
    Eg, Bg, _ = g.get_fields()
    db = core.div_b(p, Bg) - core.div_b(p, B)
    assert np.max(np.abs(db)) < 1e-11
    assert abs(d1["divb_l2"] - d0["divb_l2"]) < 1e-10 * d0["divb_l2"]


@pytest.mark.parametrize("case", [
    dict(shape=(37, 29), precision=1, engine=2, kw=dict(m=4, filter_passes=3)),
    dict(shape=(262, 97), precision=0, engine=2, kw=dict(m=4, filter_passes=3)),
    dict(shape=(70, 11, 37), precision=0, engine=1, kw=dict(m=4, filter_passes=1, courant=0.6)),
    dict(shape=(13, 11, 7), precision=1, engine=1, kw=dict(m=3, filter_passes=2, courant=0.7)),
], ids=["fused-fp64", "pol-fp32", "march3d-fp32", "staged-fp64"])
def test_current_time_profile(fmx, case):
    """fmx_set_current_profile: step k uses table[k] * J for the length of the
    table, J itself afterwards; against the oracle stepped one step at a time
    with the scaled current."""
    shape, prec = case["shape"], case["precision"]
    dt_ = np.float64 if prec == 1 else np.float32
    E, B, J = _inputs(shape, 71, dt_, smooth=prec == 0)
    table = [0.5, -1.25, 2.0, 0.0]
    nsteps = 6
    g = fmx.Grid(shape, precision=prec, engine=case["engine"], **case["kw"])
    g.set_fields(E, B)
    g.set_current(J)
    import ctypes
    bad = (ctypes.c_double * 2)(1.0, float("nan"))
    assert fmx.fmx_set_current_profile(g.handle, bad, 2) == fmx.FMX_EINVAL
    assert fmx.fmx_set_current_profile(g.handle, None, 3) == fmx.FMX_EINVAL
    assert fmx.fmx_set_current_profile(g.handle, bad, -1) == fmx.FMX_EINVAL
    g.set_current_profile(table)
    g.step(nsteps)
    Eg, Bg, _ = g.get_fields()
    g.close()
    p = core.Params(shape=tuple(shape), coef_f32=prec == 0, **case["kw"])
    Eo, Bo = E.astype(np.float64), B.astype(np.float64)
    for k in range(nsteps):
        f = table[k] if k < len(table) else 1.0
        Eo, Bo, _, _ = core.step(p, Eo, Bo, f * J.astype(np.float64), 1)
    assert_parity(np.array(Eg, dtype=np.float64), np.array(Bg, dtype=np.float64), Eo, Bo,
                  TOL64 if prec == 1 else TOL32, f"current profile {case}")
