"""Adjoint of the step on the GPU (fmx_adjoint_step), the Gaussian-envelope
source, and the differentiable run: against the FP64 oracle's adjoint, the
dot-product identity, finite differences, and FP32 against FP64."""
import ctypes
import math

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


def _dev_pitched(a, pitch, dtype):
    import torch
    c, nz, ny, nx = a.shape
    t = torch.zeros((3, nz, ny, pitch), dtype=dtype, device="cuda")
    t[..., :nx] = torch.from_numpy(np.ascontiguousarray(a)).to("cuda")
    return t


def _adjoint_gpu(fmx, shape, Ebar, Bbar, precision=1, with_jbar=True, **kw):
    import torch
    g = fmx.Grid(shape, precision=precision, **kw)
    q = 2 if precision == 1 else 4
    dt_ = torch.float64 if precision == 1 else torch.float32
    nx = shape[0]
    pitch = (nx + q - 1) // q * q
    Eb = _dev_pitched(Ebar, pitch, dt_)
    Bb = _dev_pitched(Bbar, pitch, dt_)
    jb = torch.zeros_like(Eb)
    wb = fmx.fmx_adjoint_workspace_bytes(ctypes.byref(g.params))
    work = torch.zeros(wb + 256, dtype=torch.uint8, device="cuda")
    wp = (work.data_ptr() + 255) // 256 * 256
    vp = lambda t: (ctypes.c_void_p * 3)(*[t[c].data_ptr() for c in range(3)])
    fmx.check(fmx.fmx_adjoint_step(g.handle, vp(Eb), vp(Bb), vp(jb) if with_jbar else None, wp, wb))
    torch.cuda.synchronize()
    f = lambda t: t[..., :nx].double().cpu().numpy()
    return f(Eb), f(Bb), f(jb)


@pytest.mark.parametrize("shape,kw", [((37, 29), dict(m=4, filter_passes=3)), ((12, 10, 7), dict(m=3, filter_passes=1)),
                                      ((40,), dict(m=2, filter_passes=2)), ((16, 16), dict(m=0, filter_passes=0))])
def test_adjoint_step_matches_oracle(fmx, shape, kw):
    Ebar, Bbar, _ = synth.random_fields(shape, seed=41)
    Eg, Bg, jg = _adjoint_gpu(fmx, shape, Ebar, Bbar, courant=0.7, engine=1, **kw)
    Eo, Bo, jo = core.adjoint_step(core.Params(shape=shape, courant=0.7, **kw), Ebar, Bbar)
    assert rel_l2(Eg, Eo) < 1e-12 and rel_l2(Bg, Bo) < 1e-12 and rel_l2(jg, jo) < 1e-12


@pytest.mark.parametrize("m", [0, 1, 2, 3, 4])
@pytest.mark.parametrize("passes", [0, 1, 2, 3])
def test_fused_adjoint_fp32_matches_oracle(fmx, m, passes):
    """FP32 fused TE/TM adjoint kernels (grids on the fused engine), every
    (m, passes) pair, several strips and segments, the periodic seam on both
    sides, with and without jbar, against the oracle's adjoint with the
    FP32-rounded coefficients."""
    for shape in ((262, 97), (556, 61)):
        Ebar, Bbar, _ = synth.random_fields(shape, seed=60 + m)
        Ebar, Bbar = Ebar.astype(np.float32), Bbar.astype(np.float32)
        kw = dict(m=m, filter_passes=passes, courant=0.8)
        Eo, Bo, jo = core.adjoint_step(core.Params(shape=shape, coef_f32=True, **kw), Ebar.astype(np.float64),
                                       Bbar.astype(np.float64))
        Eg, Bg, jg = _adjoint_gpu(fmx, shape, Ebar, Bbar, precision=0, engine=2, **kw)
        assert rel_l2(Eg, Eo) < 1e-5 and rel_l2(Bg, Bo) < 1e-5 and rel_l2(jg, jo) < 1e-5, (shape, m, passes)
        Eg, Bg, _ = _adjoint_gpu(fmx, shape, Ebar, Bbar, precision=0, engine=2, with_jbar=False, **kw)
        assert rel_l2(Eg, Eo) < 1e-5 and rel_l2(Bg, Bo) < 1e-5


def test_dot_product_identity_fp32_fused(fmx):
    """<T d, y> = <d, T^T y> in FP32 with the fused forward (TE/TM) and fused
    adjoint kernels; bound from FP32 rounding of the two sums."""
    shape = (300, 140)
    dE, dB, dJ = (x.astype(np.float32) for x in synth.random_fields(shape, seed=44))
    yE, yB, _ = (x.astype(np.float32) for x in synth.random_fields(shape, seed=45))
    g = fmx.Grid(shape, precision=0, m=4, filter_passes=3, engine=2)
    g.set_fields(dE, dB)
    g.set_current(dJ)
    g.step(1)
    E1, B1, _ = g.get_fields()
    lhs = np.sum(E1.astype(np.float64) * yE) + np.sum(B1.astype(np.float64) * yB)
    Eb, Bb, jb = _adjoint_gpu(fmx, shape, yE, yB, precision=0, m=4, filter_passes=3, engine=2)
    rhs = np.sum(dE * Eb) + np.sum(dB * Bb) + np.sum(dJ * jb)
    assert abs(lhs - rhs) <= 1e-5 * (np.sum(np.abs(E1 * yE)) + np.sum(np.abs(B1 * yB)))


def test_dot_product_identity_gpu(fmx):
    """<T d, y> = <d, T^T y> with T the GPU forward step (fused engine) and
    T^T the GPU adjoint step."""
    shape = (64, 48)
    dE, dB, dJ = synth.random_fields(shape, seed=42)
    yE, yB, _ = synth.random_fields(shape, seed=43)
    g = fmx.Grid(shape, precision=1, m=4, filter_passes=3, engine=2)
    g.set_fields(dE, dB)
    g.set_current(dJ)
    g.step(1)
    E1, B1, _ = g.get_fields()
    lhs = np.sum(E1 * yE) + np.sum(B1 * yB)
    Eb, Bb, jb = _adjoint_gpu(fmx, shape, yE, yB, m=4, filter_passes=3, engine=1)
    rhs = np.sum(dE * Eb) + np.sum(dB * Bb) + np.sum(dJ * jb)
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


@pytest.mark.parametrize("shape,npz,precision,tol", [((96, 80), 8, 1, 1e-13), ((200, 150), 64, 0, 3e-6),
                                                      ((330, 258), 128, 0, 3e-6)])
def test_gauss_source_and_projection(fmx, shape, npz, precision, tol):
    """Separable tiled synthesis and projection against the direct sum of
    periodic Gaussians (ragged tiles in both axes; 128 = the source limit)."""
    import torch
    nx, ny = shape
    cxy, phases, theta = synth.gauss_sources(npz, shape, seed=44)
    w = 6.0
    ii = np.arange(nx)[None, :]
    jj = np.arange(ny)[:, None]
    G = []
    for x, y in cxy:
        dx = (ii - x) - nx * np.floor((ii - x) / nx + 0.5)
        dy = (jj - y) - ny * np.floor((jj - y) / ny + 0.5)
        G.append(np.exp(-(dx * dx + dy * dy) / (2 * w * w)))
    G = np.array(G)
    g = fmx.Grid(shape, precision=precision, engine=1)
    dp = lambda a: np.ascontiguousarray(a).ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    fmx.check(fmx.fmx_gauss_source(g.handle, npz, dp(cxy), dp(theta), w))
    _, _, J = g.get_fields(fmx.FMX_J)
    assert np.max(np.abs(J[:2])) == 0
    assert rel_l2(J[2, 0], np.tensordot(theta, G, 1)) < tol
    f = np.random.default_rng(45).standard_normal((ny, nx))
    esz = 8 if precision == 1 else 4
    pitch = (nx + 16 // esz - 1) // (16 // esz) * (16 // esz)
    ft = torch.zeros((ny, pitch), dtype=torch.float64 if precision == 1 else torch.float32, device="cuda")
    ft[:, :nx] = torch.from_numpy(f)
    out = np.zeros(npz)
    fmx.check(fmx.fmx_gauss_project(g.handle, npz, dp(cxy), w, ctypes.c_void_p(ft.data_ptr()), dp(out)))
    ref = np.einsum("pij,ij->p", G, ft[:, :nx].double().cpu().numpy())
    assert rel_l2(out, ref) < 10 * tol


def test_gauss_run_matches_single_calls_fp64(fmx):
    """fmx_gauss_run (amplitudes formed on the device) against the same steps
    made of fmx_gauss_source with host amplitudes and fmx_step."""
    shape, N, w, om = (96, 80), 7, 6.0, 0.2
    cxy, phases, theta = synth.gauss_sources(8, shape, seed=49)
    E0, B0, _ = synth.random_fields(shape, seed=50)
    dp = lambda a: np.ascontiguousarray(a, dtype=np.float64).ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    res = []
    for mode in ("run", "calls"):
        g = fmx.Grid(shape, precision=1, m=4, filter_passes=3, courant=0.5, engine=2)
        g.set_fields(E0, B0)
        if mode == "run":
            fmx.check(fmx.fmx_gauss_setup(g.handle, 8, dp(cxy), dp(theta), dp(phases), w, om))
            fmx.check(fmx.fmx_gauss_run(g.handle, 3, N))
        else:
            for n in range(3, 3 + N):
                amp = theta * np.sin(om * (n + 0.5) * g.dt + phases)
                fmx.check(fmx.fmx_gauss_source(g.handle, 8, dp(cxy), dp(amp), w))
                g.step(1)
        E, B, _ = g.get_fields(fmx.FMX_E | fmx.FMX_B)
        res.append((E, B))
    assert rel_l2(res[0][0], res[1][0]) < 1e-13 and rel_l2(res[0][1], res[1][1]) < 1e-13


def _oracle_gradient(shape, cxy, phases, theta, E0, B0, N, mask, width, omega0, **kw):
    """dL/dtheta with the oracle alone: forward with the synthesised current,
    then N oracle adjoint steps and the projection on the G_p."""
    p = core.Params(shape=shape, **kw)
    dt = p.time_step()
    nx, ny = shape
    ii = np.arange(nx)[None, :]
    jj = np.arange(ny)[:, None]
    G = []
    for x, y in cxy:
        dx = (ii - x) - nx * np.floor((ii - x) / nx + 0.5)
        dy = (jj - y) - ny * np.floor((jj - y) / ny + 0.5)
        G.append(np.exp(-(dx * dx + dy * dy) / (2 * width * width)))
    G = np.array(G)
    E, B = E0.copy(), B0.copy()
    for n in range(N):
        J = np.zeros(p.array_shape)
        J[2, 0] = np.tensordot(theta * np.sin(omega0 * (n + 0.5) * dt + phases), G, 1)
        E, B, _, _ = core.step(p, E, B, J, 1)
    Eb, Bb = E * mask, B * mask
    loss = 0.5 * (np.sum(Eb * E) + np.sum(Bb * B))
    grad = np.zeros(len(theta))
    for n in range(N - 1, -1, -1):
        Eb, Bb, jb = core.adjoint_step(p, Eb, Bb)
        grad += np.sin(omega0 * (n + 0.5) * dt + phases) * np.einsum("pij,ij->p", G, jb[2, 0])
    return loss, grad


def _gpu_gradient(fmx, shape, cxy, phases, theta, E0, B0, N, mask, precision, K, recompute=False, engine=0):
    import torch
    from paper_1907_13088_gb300.adjoint import GaussSourceRun, make_function
    dt_ = torch.float64 if precision == 1 else torch.float32
    run = GaussSourceRun(shape, cxy, phases, N, width=6.0, omega0=0.2, m=4, passes=3, courant=0.5,
                         precision=precision, checkpoint_every=K, engine=engine)
    FieldRun = make_function()
    th = torch.tensor(theta, dtype=torch.float64, requires_grad=True)
    e0 = torch.from_numpy(np.ascontiguousarray(E0[:, 0])).to("cuda", dt_)
    b0 = torch.from_numpy(np.ascontiguousarray(B0[:, 0])).to("cuda", dt_)
    EN, BN = FieldRun.apply(th, e0, b0, run, recompute)
    mk = torch.from_numpy(mask[:, 0]).to("cuda", dt_)
    loss = 0.5 * ((EN * EN * mk).sum() + (BN * BN * mk).sum())
    loss.backward()
    return float(loss.detach()), th.grad.numpy().copy()


def _setup(shape, N, seed):
    cxy, phases, theta = synth.gauss_sources(8, shape, seed=seed)
    E0, B0, _ = synth.random_fields(shape, seed=seed + 1)
    E0 *= 0.01
    B0 *= 0.01
    mask = np.zeros((3, 1, shape[1], shape[0]))
    mask[:, :, shape[1] // 4:shape[1] // 2, shape[0] // 4:shape[0] // 2] = 1.0
    return cxy, phases, theta, E0, B0, mask


def test_autograd_gradient_matches_oracle_fp64(fmx):
    shape, N = (96, 80), 24
    cxy, phases, theta, E0, B0, mask = _setup(shape, N, 46)
    lo, go = _oracle_gradient(shape, cxy, phases, theta, E0, B0, N, mask, 6.0, 0.2, courant=0.5, m=4,
                              filter_passes=3)
    for engine, recompute in ((2, False), (1, True)):
        lg, gg = _gpu_gradient(fmx, shape, cxy, phases, theta, E0, B0, N, mask, 1, K=5, recompute=recompute,
                               engine=engine)
        assert abs(lg - lo) <= 1e-12 * abs(lo)
        assert rel_l2(gg, go) < 1e-11


def test_autograd_central_differences_fp64(fmx):
    """Central differences (eps = 1e-3) of the GPU FP64 loss along seeded
    directions against the adjoint gradient (the loss is quadratic in theta,
    so the differences are exact up to round-off)."""
    shape, N = (128, 96), 30
    cxy, phases, theta, E0, B0, mask = _setup(shape, N, 47)
    l0, g0 = _gpu_gradient(fmx, shape, cxy, phases, theta, E0, B0, N, mask, 1, K=10, engine=2)
    rng = np.random.default_rng(48)
    eps = 1e-3
    for _ in range(3):
        d = rng.standard_normal(len(theta))
        lp, _ = _gpu_gradient(fmx, shape, cxy, phases, theta + eps * d, E0, B0, N, mask, 1, K=10, engine=2)
        lm, _ = _gpu_gradient(fmx, shape, cxy, phases, theta - eps * d, E0, B0, N, mask, 1, K=10, engine=2)
        fd = (lp - lm) / (2 * eps)
        assert abs(fd - g0 @ d) <= 1e-8 * max(abs(fd), 1e-30)


@pytest.mark.slow
def test_fp32_gradient_1024_against_fp64(fmx):
    """The 1024^2 FP32 run (64 sources, checkpoint every 50 steps) against the
    same run in FP64: relative error of dL/dtheta stated and bounded."""
    from paper_1907_13088_gb300.adjoint import GaussSourceRun
    shape, N = (1024, 1024), 100
    cxy, phases, theta = synth.gauss_sources(64, shape, seed=1907005)
    E0, B0, _ = synth.random_fields(shape, seed=1907006)
    E0 *= 0.01
    B0 *= 0.01
    mask = np.zeros((3, 1, 1024, 1024))
    mask[:, :, 448:576, 448:576] = 1.0
    grads = []
    for prec in (1, 0):
        import torch
        from paper_1907_13088_gb300.adjoint import make_function
        dt_ = torch.float64 if prec == 1 else torch.float32
        run = GaussSourceRun(shape, cxy, phases, N, width=8.0, omega0=0.2, m=4, passes=3, courant=0.5,
                             precision=prec, checkpoint_every=50)
        th = torch.tensor(theta, dtype=torch.float64, requires_grad=True)
        EN, BN = make_function().apply(th, torch.from_numpy(E0[:, 0]).to("cuda", dt_),
                                       torch.from_numpy(B0[:, 0]).to("cuda", dt_), run, False)
        mk = torch.from_numpy(mask[:, 0]).to("cuda", dt_)
        (0.5 * ((EN * EN * mk).sum() + (BN * BN * mk).sum())).backward()
        grads.append(th.grad.numpy().copy())
    assert rel_l2(grads[1], grads[0]) < 1e-3
