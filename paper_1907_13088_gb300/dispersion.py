"""Point-source dispersion experiment of Sec. 4.1 on the GPU step.

A single cell of E_z is set to one on an otherwise empty periodic N x N grid
(Delta x = Delta y, c = 1), so that every wavevector is excited; the fields
advance through the library's step (fmx_step) up to t_max; E_z(t, x, y) is
recorded after every step; the space-time discrete Fourier transform of the
Hann-windowed record, w(t) = sin^2(pi t / t_max), gives per wavevector the
power-weighted frequency over omega >= 0,
    omega_num(k) = sum_omega omega |E~(omega, k)|^2 / sum_omega |E~(omega, k)|^2,
which the paper compares with Eq. dispersion-em-F-2d.  For a fixed number m
of sweeps the exact TM relation is the truncated one,
    sin^2(omega_m dt/2) = (1 - lambda^{m+1}) sin^2(omega_inf dt/2),
lambda the A_zz symbol (App. D, with the factor on the side Eq.
derive_convergence_3 implies).

    python -m paper_1907_13088_gb300.dispersion [--courant 0.5] [--m 4 | --residual]

The stepping runs on the GPU through the C ABI; the Fourier analysis uses
torch.fft on the recorded fields.
"""
from __future__ import annotations

import argparse
import math

import numpy as np

from . import fmx


def _G(theta):
    s2 = np.sin(theta) ** 2
    return s2 / (1.0 - 2.0 / 3.0 * s2)


def theory(courant, n, m=None, d=1.0, c=1.0):
    """omega(kx, ky) of the TM mode on the n x n DFT wavevector grid (fft
    order): Eq. dispersion-em-F-2d for the converged solve (m = None), the
    truncated relation above for m sweeps."""
    dt = courant * d / (c * math.sqrt(2.0))
    k = 2.0 * np.pi * np.fft.fftfreq(n, d)
    kx, ky = np.meshgrid(k, k)  # [iy, ix]
    sig = (c * dt / d) ** 2
    R = c * c * dt * dt * (_G(kx * d / 2) + _G(ky * d / 2)) / (d * d)
    s2inf = R / (1.0 + 2.0 / 3.0 * R)  # sin^2(omega dt / 2), G inverted
    if m is not None:
        sx2, sy2 = np.sin(kx * d / 2) ** 2, np.sin(ky * d / 2) ** 2
        lam = 2.0 / 3.0 * (1 - sig) * sx2 + 2.0 / 3.0 * (1 - sig) * sy2 - 4.0 / 9.0 * (1 - 2 * sig) * sx2 * sy2
        s2inf = (1.0 - lam ** (m + 1)) * s2inf
    return 2.0 / dt * np.arcsin(np.sqrt(np.clip(s2inf, 0.0, 1.0))), kx, ky, dt


def point_source(courant, n=128, t_max=256.0, m=4, residual=False, tol=1e-13, precision=fmx.FMX_F64):
    """Runs the experiment; returns dict(omega=omega_num [iy, ix], kx, ky, dt,
    nsteps, sweeps) with kx, ky in fft order."""
    import torch

    kw = dict(precision=precision, courant=courant, filter_passes=0)
    if residual:
        kw.update(iter_mode=fmx.FMX_ITER_RESIDUAL, tol=tol, m_max=100000, engine=fmx.FMX_ENGINE_STAGED)
    else:
        kw.update(m=m)
    g = fmx.Grid((n, n), with_current=False, **kw)
    dt = g.dt
    nsteps = int(round(t_max / dt))
    dtype = np.float64 if precision == fmx.FMX_F64 else np.float32
    E = np.zeros((3, 1, n, n), dtype=dtype)
    E[2, 0, n // 2, n // 2] = 1.0
    g.set_fields(E, np.zeros_like(E))
    rec = torch.empty((nsteps, n, n), dtype=torch.float64, device=g.device)
    for s in range(nsteps):
        rec[s].copy_(g.field_tensor(2)[0, :, :n])
        g.step(1)
    sweeps = g.diagnostics()["total_sweeps"] if residual else m * nsteps
    t = torch.arange(nsteps, dtype=torch.float64, device=g.device) * dt
    w = torch.sin(math.pi * t / t_max) ** 2
    F = torch.fft.fftn(rec * w[:, None, None], dim=(0, 1, 2))
    P = (F.real ** 2 + F.imag ** 2)
    om = 2.0 * math.pi * torch.fft.fftfreq(nsteps, dt, dtype=torch.float64, device=g.device)
    pos = om >= 0
    Pp = P[pos]
    omega = (om[pos][:, None, None] * Pp).sum(0) / Pp.sum(0)
    k = 2.0 * np.pi * np.fft.fftfreq(n, 1.0)
    kx, ky = np.meshgrid(k, k)
    g.close()
    return dict(omega=omega.cpu().numpy(), kx=kx, ky=ky, dt=dt, nsteps=nsteps, sweeps=sweeps)


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--courant", type=float, default=0.5)
    ap.add_argument("--n", type=int, default=128)
    ap.add_argument("--t-max", type=float, default=256.0)
    ap.add_argument("--m", type=int, default=4)
    ap.add_argument("--residual", action="store_true", help="converged solve (residual mode, FP64 staged engine)")
    a = ap.parse_args(argv)
    r = point_source(a.courant, a.n, a.t_max, a.m, a.residual)
    om_conv, kx, ky, dt = theory(a.courant, a.n, None)
    om_m, _, _, _ = theory(a.courant, a.n, None if a.residual else a.m)
    kk = np.hypot(kx, ky)
    band = (r["omega"] >= 0.3) & (kk > 0)
    rel = np.abs(r["omega"] - om_m)[band] / om_m[band]
    print(f"Courant {a.courant}, {a.n}^2, {r['nsteps']} steps (dt {dt:.5f}), "
          f"{'residual mode' if a.residual else f'm = {a.m}'}, {r['sweeps']} sweeps")
    print(f"measured vs {'Eq. dispersion-em-F-2d' if a.residual else 'truncated relation'}: "
          f"max relative error {rel.max():.2e} over {band.sum()} wavevectors with omega >= 0.3")
    print("  k along x      v_ph measured   v_ph (converged, Eq. dispersion-em-F-2d)")
    for i in range(1, a.n // 2 + 1, max(1, a.n // 16)):
        print(f"  {kx[0, i]:8.4f}       {r['omega'][0, i] / kx[0, i]:10.6f}      {om_conv[0, i] / kx[0, i]:10.6f}")


if __name__ == "__main__":
    main()
