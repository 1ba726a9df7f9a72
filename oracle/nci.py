"""Numerical Cherenkov instability (NCI) of the averaged scheme: resonance
curves (Eqs. reson1, reson2) and the asymptotic growth rate (Sec. 3, App. E).

TEST INFRASTRUCTURE ONLY (see ``oracle/core.py``).  FP64 numpy.

A cold beam drifts along x at v -> c on a 2D grid (dx, dy), time step dt.
The beam mode of alias nu (Eq. aliasing_x), omega = c k_x' with
k_x' = k_x + 2 pi nu / dx (Eq. reson2), resonates with the grid's EM mode
where
    [omega]^2 / (alpha_t c^2) = [k_x]^2 / alpha_x + [k_y]^2 / alpha_y
(Eq. reson1).  The growth rate there follows App. E step by step:
  1. the expansion coefficients xi_0..xi_3 of [omega] and alpha_t about the
     resonance (Eqs. xi0..xi3);
  2. the numerators Q_xx, Q_xy of the beam's dielectric response for the
     momentum-conserving interpolation (S_Jx, S_Bz, S_Ey of Sec. 3);
  3. A_1 to first order in delta omega and C_1 at zeroth order;
  4. dropping B_1, A_1' dw^3 + C_1 = 0, whose root of largest imaginary part
     gives Gamma = (sqrt 3 / 2) |C_1 / A_1'|^(1/3).
The closed form the paper ends with (Eq. NCI-growth-rate) is the same number
after algebra; this module keeps the steps so that each can be checked.

Readings (the paper is terse here):
* Only the temporally unaliased beam, mu = 0, resonates, and only where its
  frequency c k_x' lies in the zone of the EM branch, |c k_x' dt| <= pi.
  Eq. reson1 alone is periodic in omega with period 2 pi / dt, so it would
  also admit the mu != 0 lines; with them the curves reach |k_x| -> 0 and
  |nu| = 2, against Sec. 4.2 (|k_x| > 2.06 / dx, no |nu| >= 2 resonance,
  nu = 0 only above dt_CFL / sqrt 2), which this reading reproduces.
* xi_1 = cos(k~ c dt / 2) (printed without the c; the paper's units set
  c = 1).
* [k]_x, alpha_x are the grid symbols of k_x in the first zone; the shape
  factors s_{l,x} take the aliased k_x' ("dummy variables with aliasing
  wavevector"); nu_y = 0, so k_y' = k_y.
* The beam and the EM mode also meet trivially at k = 0, omega = 0 (the
  uniform static field, where Gamma is 0/0); that point is not a crossing.
* The resonance is solved for k_y >= 0 at each k_x (its mirror -k_y has the
  same Gamma): f(k_y) = [omega]^2/(alpha_t c^2) - [k_x]^2/alpha_x
  - [k_y]^2/alpha_y decreases on [0, pi/dy], so there is at most one root,
  found here by bisection.
"""
from __future__ import annotations

import math

import numpy as np


def dt_cfl(dx, dy, c=1.0):
    """2D time-step limit of the scheme (Sec. 2.1, 2D form of Eq. dt_cfl_3d)."""
    return 1.0 / (c * math.sqrt(1.0 / dx ** 2 + 1.0 / dy ** 2))


def kx_samples(nkx, dx):
    """Cell centres of (-pi/dx, pi/dx): k_x,i = (2 i + 1 - nkx) pi / (nkx dx)."""
    i = np.arange(nkx, dtype=np.float64)
    return (2.0 * i + 1.0 - nkx) * math.pi / (nkx * dx)


def _bracket(k, d):
    """[k] = sin(k d / 2) / (d / 2) (Eq. braket_k)."""
    return np.sin(k * d / 2.0) / (d / 2.0)


def _alpha(k, d):
    """alpha = (2 + cos(k d)) / 3 (Eq. alphax)."""
    return (2.0 + np.cos(k * d)) / 3.0


def beam_frequency(kxp, dt, c=1.0):
    """omega = c k_x' (Eq. reson2 with mu = 0) and whether it lies in the
    zone of the EM branch, |omega dt| <= pi, away from the trivial omega = 0."""
    om = c * kxp
    return om, (np.abs(om * dt) <= math.pi) & (om != 0.0)


def xi(omega, dt):
    """xi_0..xi_3 of Eqs. xi0..xi3 at the grid frequency omega = c k~."""
    x0 = np.sin(omega * dt / 2.0) / (dt / 2.0)
    x1 = np.cos(omega * dt / 2.0)
    x2 = (2.0 + np.cos(omega * dt)) / 3.0
    x3 = -dt * np.sin(omega * dt) / 3.0
    return x0, x1, x2, x3


def resonance_function(kx, ky, nu, dx, dy, dt, c=1.0):
    """Left minus right of Eq. reson1 on the beam line of Eq. reson2."""
    om, _ = beam_frequency(kx + 2.0 * math.pi * nu / dx, dt, c)
    x0, _, x2, _ = xi(om, dt)
    return x0 ** 2 / (x2 * c * c) - _bracket(kx, dx) ** 2 / _alpha(kx, dx) - _bracket(ky, dy) ** 2 / _alpha(ky, dy)


def resonance_ky(kx, nu, dx, dy, dt, c=1.0, iters=200):
    """k_y >= 0 on the resonance curve of alias nu at each k_x (NaN where the
    curve does not cross that k_x), by bisection on [0, pi/dy]."""
    kx = np.asarray(kx, dtype=np.float64)
    _, inzone = beam_frequency(kx + 2.0 * math.pi * nu / dx, dt, c)
    lo = np.zeros_like(kx)
    hi = np.full_like(kx, math.pi / dy)
    f_lo = resonance_function(kx, lo, nu, dx, dy, dt, c)
    f_hi = resonance_function(kx, hi, nu, dx, dy, dt, c)
    ok = inzone & (f_lo >= 0.0) & (f_hi <= 0.0)
    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        if np.all((mid == lo) | (mid == hi)):
            break
        fm = resonance_function(kx, mid, nu, dx, dy, dt, c)
        up = fm > 0.0
        lo = np.where(up, mid, lo)
        hi = np.where(up, hi, mid)
    return np.where(ok, 0.5 * (lo + hi), np.nan)


def shape_factor(k, d, l):
    """s_{l} = (sin(k d / 2) / (k d / 2))^(l + 1), B-spline of order l."""
    h = k * d / 2.0
    return np.where(h == 0.0, 1.0, np.sin(h) / np.where(h == 0.0, 1.0, h)) ** (l + 1)


def growth_terms(kx, ky, nu, dx, dy, dt, omega_p, l, c=1.0):
    """Steps 1-3 of App. E at (k_x, k_y): returns dict with xi_0..xi_3, the S
    factors, Q_xx, Q_xy, A_1' (A_1 = A_1' dw) and C_1."""
    kxp = kx + 2.0 * math.pi * nu / dx
    om, _ = beam_frequency(kxp, dt, c)
    x0, x1, x2, x3 = xi(om, dt)
    bx, by = _bracket(kx, dx), _bracket(ky, dy)
    ax, ay = _alpha(kx, dx), _alpha(ky, dy)
    ss = shape_factor(kxp, dx, l) * shape_factor(ky, dy, l)
    sign = -1.0 if (int(nu) % 2) else 1.0
    s_jx = ss * sign
    s_bz = np.cos(om * dt / 2.0) * ss * sign   # cos(omega' dt / 2) on the beam line
    s_ey = ss
    wp2 = omega_p * omega_p
    q_xx = wp2 * s_jx * s_bz * by * ky * c * c
    q_xy = wp2 * ky * s_jx * (s_ey * x0 - s_bz * bx * c) * c
    a1p = x0 ** 2 * (2.0 * ax * ay * x0 * x1 - x3 * ax * ay * x0 ** 2 / x2)
    c1 = -(ax * x0 ** 2 - x2 * c * c * bx ** 2) * q_xx + x2 * c * c * bx * by * q_xy
    return dict(omega=om, xi=(x0, x1, x2, x3), s_jx=s_jx, s_bz=s_bz, s_ey=s_ey,
                q_xx=q_xx, q_xy=q_xy, a1p=a1p, c1=c1)


def growth_rate(kx, ky, nu, dx, dy, dt, omega_p, l, c=1.0):
    """Step 4: Gamma = (sqrt 3 / 2) |C_1 / A_1'|^(1/3)."""
    t = growth_terms(kx, ky, nu, dx, dy, dt, omega_p, l, c)
    return math.sqrt(3.0) / 2.0 * np.cbrt(np.abs(t["c1"] / t["a1p"]))


def resonance(nkx, courant, dx, dy, omega_p, l, nu_max=1, c=1.0):
    """The resonance curves and the growth rate along them, for every alias
    nu = -nu_max..nu_max on the k_x samples of ``kx_samples``.  Returns dict
    kx [nkx], ky [2 nu_max + 1, nkx] (NaN: no crossing), gamma [same]
    (0 where no crossing), best = (Gamma_max, k_x, k_y, nu)."""
    dt = courant * dt_cfl(dx, dy, c)
    kx = kx_samples(nkx, dx)
    nus = list(range(-nu_max, nu_max + 1))
    ky = np.stack([resonance_ky(kx, nu, dx, dy, dt, c) for nu in nus])
    gam = np.zeros_like(ky)
    for r, nu in enumerate(nus):
        ok = ~np.isnan(ky[r])
        gam[r, ok] = growth_rate(kx[ok], ky[r, ok], nu, dx, dy, dt, omega_p, l, c)
    if np.any(gam > 0):
        r, i = np.unravel_index(np.argmax(gam), gam.shape)
        best = (float(gam[r, i]), float(kx[i]), float(ky[r, i]), float(nus[r]))
    else:
        best = (0.0, float("nan"), float("nan"), float("nan"))
    return dict(kx=kx, ky=ky, gamma=gam, best=best, dt=dt, nus=nus)
