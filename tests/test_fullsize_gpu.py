"""The other benchmark configurations at full size, in the launch
configuration bench.py times, against the oracle on sampled outputs or by
properties that hold at any size:

* 512^3 FP32 (m = 4, one filter pass, Courant 0.5, staged engine): periodic
  windows of the GPU result against the oracle run on the same windows;
* the batch of 256 grids (sizes log-uniform 64..1024, Courant 0.3..0.9, FP32,
  vacuum, autotuned tile rows): sampled grids against the oracle;
* the 1024^2 Gaussian-source run (64 sources, 500 steps, checkpoints every 50):
  FP64 adjoint gradient against central differences of the FP64 forward run,
  and the FP32 gradient against the FP64 one.
"""
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


def _window3(a, center, size):
    """(3, nz, ny, nx) -> (3, size, size, size) periodic window whose cell
    (size//2,)*3 is `center` = (k, j, i)."""
    nz, ny, nx = a.shape[-3:]
    idx = [np.arange(c - size // 2, c - size // 2 + size) % n for c, n in zip(center, (nz, ny, nx))]
    return a[:, idx[0][:, None, None], idx[1][None, :, None], idx[2][None, None, :]]


def test_full_size_512_cubed_windows(fmx):
    n, nsteps = 512, 2
    E, B = synth.power_law_fields((n, n, n), n // 8, 1907003, dtype=np.float32)
    J = synth.solenoidal_current((n, n, n), 1907013, width=16.0, rms=1e-3, dtype=np.float32)
    g = fmx.Grid((n, n, n), precision=0, m=4, filter_passes=1, courant=0.5)
    g.set_fields(E, B)
    g.set_current(J)
    g.step(nsteps)
    Eg, Bg, _ = g.get_fields()
    g.close()
    radius = 7 * nsteps  # one step reaches 7 cells per axis (filter 1, source 1, 4 sweeps, curl 1)
    size = 2 * radius + 8
    p = core.Params(shape=(size, size, size), courant=0.5, m=4, filter_passes=1, coef_f32=True)
    rng = np.random.default_rng(11)
    centers = [(0, 0, 0), (511, 511, 511), (256, 0, 511)] + [tuple(rng.integers(0, n, 3)) for _ in range(2)]
    lo, hi = radius + 1, size - radius - 1
    for ctr in centers:
        w = lambda a: _window3(a, ctr, size).astype(np.float64)
        Eo, Bo, _, _ = core.step(p, w(E), w(B), w(J), nsteps)
        for F_g, F_o in ((Eg, Eo), (Bg, Bo)):
            Fw = _window3(F_g, ctr, size).astype(np.float64)
            for c in range(3):
                e = rel_l2(Fw[c, lo:hi, lo:hi, lo:hi], F_o[c, lo:hi, lo:hi, lo:hi])
                assert e < TOL32, (ctr, c, e)


def test_full_batch_256_sampled_grids(fmx):
    sizes = synth.batch_sizes(256, 1907004)
    shapes = [(a, b) for a, b, _ in sizes]
    cfs = [c for _, _, c in sizes]
    bt = fmx.Batch(shapes, cfs, m=4)
    bt.tune(trial_steps=10)
    fields = [synth.power_law_fields(sh, max(2, min(sh) // 8), 1907004 + i) for i, sh in enumerate(shapes)]
    for i, (E, B) in enumerate(fields):
        bt.set_fields(i, E, B)
    nsteps = 3
    bt.step(nsteps)
    area = [a * b for a, b in shapes]
    odd = [i for i, (a, b) in enumerate(shapes) if a % 2 == 1]
    rng = np.random.default_rng(12)
    sample = sorted({int(np.argmin(area)), int(np.argmax(area)), odd[0], odd[-1],
                     int(np.argmin(cfs)), int(np.argmax(cfs))} | set(int(i) for i in rng.integers(0, 256, 4)))
    for i in sample:
        Eg, Bg = bt.get_fields(i)
        E, B = fields[i]
        Eo, Bo, _, _ = core.step(core.Params(shape=shapes[i], courant=cfs[i], m=4, coef_f32=True),
                                 E.astype(np.float64), B.astype(np.float64), None, nsteps)
        assert_parity(Eg, Bg, Eo, Bo, TOL32, f"batch grid {i} {shapes[i]} courant {cfs[i]:.3f}")


def _gauss_loss_and_grad(fmx, theta, precision, N=500, K=50):
    import torch
    from paper_1907_13088_gb300.adjoint import GaussSourceRun, make_function
    shape = (1024, 1024)
    cxy, phases, _ = synth.gauss_sources(64, shape, seed=1907005)
    E0, B0, _ = synth.random_fields(shape, seed=1907006)
    E0 *= 0.01
    B0 *= 0.01
    dt_ = torch.float64 if precision == 1 else torch.float32
    run = GaussSourceRun(shape, cxy, phases, N, width=8.0, omega0=0.2, m=4, passes=3, courant=0.5,
                         precision=precision, checkpoint_every=K)
    th = torch.tensor(theta, dtype=torch.float64, requires_grad=True)
    EN, BN = make_function().apply(th, torch.from_numpy(E0[:, 0]).to("cuda", dt_),
                                   torch.from_numpy(B0[:, 0]).to("cuda", dt_), run, False)
    mk = torch.zeros((3, 1024, 1024), dtype=dt_, device="cuda")
    mk[:, 448:576, 448:576] = 1.0
    loss = 0.5 * ((EN * EN * mk).sum() + (BN * BN * mk).sum())
    loss.backward()
    return float(loss.detach()), th.grad.numpy().copy()


def test_full_size_gauss_run_gradient(fmx):
    """dL/dtheta of the 1024^2, 64-source, 500-step run: FP64 adjoint against
    central differences of the FP64 loss (exact up to round-off: the loss is
    quadratic in theta), and the FP32 gradient against the FP64 one."""
    _, _, theta = synth.gauss_sources(64, (1024, 1024), seed=1907005)
    l0, g0 = _gauss_loss_and_grad(fmx, theta, 1)
    rng = np.random.default_rng(13)
    eps = 1e-3
    for _ in range(2):
        d = rng.standard_normal(64)
        lp, _ = _gauss_loss_and_grad(fmx, theta + eps * d, 1)
        lm, _ = _gauss_loss_and_grad(fmx, theta - eps * d, 1)
        fd = (lp - lm) / (2 * eps)
        assert abs(fd - g0 @ d) <= 1e-7 * abs(fd), (fd, g0 @ d)
    l32, g32 = _gauss_loss_and_grad(fmx, theta, 0)
    assert abs(l32 - l0) <= 1e-3 * abs(l0)
    assert rel_l2(g32, g0) < 1e-2
