"""Seeded synthetic inputs for the field advance.

This module only draws random numbers and lays out initial fields and
currents.  It holds none of the solver's arithmetic (no averaging operator, no
matrix A, no iteration, no filter) and is the one module that both the CUDA
path's callers and the CPU oracle's callers draw their inputs from.

Arrays are numpy, shape ``(3, nz, ny, nx)`` (x fastest), one plane per
component, at the staggered Yee positions:
  E_x (i+1/2, j, k), E_y (i, j+1/2, k), E_z (i, j, k+1/2),
  B_x (i, j+1/2, k+1/2), B_y (i+1/2, j, k+1/2), B_z (i+1/2, j+1/2, k),
and the current colocated with E.
"""
from __future__ import annotations

import math

import numpy as np

E_POS = ((0.5, 0.0, 0.0), (0.0, 0.5, 0.0), (0.0, 0.0, 0.5))
B_POS = ((0.0, 0.5, 0.5), (0.5, 0.0, 0.5), (0.5, 0.5, 0.0))


def _shape3(shape):
    s = tuple(int(v) for v in shape) + (1,) * (3 - len(shape))
    return s  # (nx, ny, nz)


def tm_plane_waves(shape, dt, nmodes=8, kmax=8, seed=1907001, c=1.0, d=(1.0, 1.0)):
    """Sum of ``nmodes`` vacuum plane waves in the E_z/B_x/B_y polarisation on a
    2D periodic grid: integer mode vectors n with 1 <= |n| <= kmax drawn
    without replacement (a mode and its negative never both), amplitudes
    N(0, 1), phases U[0, 2 pi).  Each wave is the continuum solution
    E_z = a cos(k.r - omega t + phi), B = k_hat x E with omega = c |k|,
    sampled with E at t = 0 and B at t = dt/2.  Returns (E, B, modes)."""
    nx, ny, _ = _shape3(shape)
    rng = np.random.default_rng(seed)
    cand = []
    for mx in range(-kmax, kmax + 1):
        for my in range(-kmax, kmax + 1):
            r2 = mx * mx + my * my
            if 1 <= r2 <= kmax * kmax and (mx > 0 or (mx == 0 and my > 0)):
                cand.append((mx, my))
    pick = rng.choice(len(cand), size=nmodes, replace=False)
    amps = rng.standard_normal(nmodes)
    phis = rng.uniform(0.0, 2.0 * math.pi, nmodes)
    E = np.zeros((3, 1, ny, nx))
    B = np.zeros((3, 1, ny, nx))
    ii = np.arange(nx)[None, :]
    jj = np.arange(ny)[:, None]
    modes = []
    for q, idx in enumerate(pick):
        mx, my = cand[idx]
        kx = 2 * math.pi * mx / (nx * d[0])
        ky = 2 * math.pi * my / (ny * d[1])
        kn = math.hypot(kx, ky)
        w = c * kn
        a, ph = amps[q], phis[q]

        def wave(pos, t):
            x = (ii + pos[0]) * d[0]
            y = (jj + pos[1]) * d[1]
            return a * np.cos(kx * x + ky * y - w * t + ph)

        E[2, 0] += wave(E_POS[2], 0.0)
        B[0, 0] += (ky / kn) * wave(B_POS[0], 0.5 * dt)
        B[1, 0] += (-kx / kn) * wave(B_POS[1], 0.5 * dt)
        modes.append((mx, my, float(a), float(ph)))
    return E, B, modes


def _ifftn(F):
    try:  # multithreaded when scipy is present; the same transform otherwise
        import os
        import scipy.fft
        return scipy.fft.ifftn(F, workers=os.cpu_count() or 1)
    except ImportError:
        return np.fft.ifftn(F)


def _spectrum_plane(rng, shape, weight, dtype):
    """One real field, sum over all DFT modes with |amplitude| = weight(n) and
    uniformly random phases, normalised to unit RMS."""
    nx, ny, nz = shape
    ph = rng.uniform(0.0, 2.0 * math.pi, size=(nz, ny, nx)).astype(np.float32)
    F = (weight * np.exp(1j * ph)).astype(np.complex64)
    f = _ifftn(F).real
    rms = float(np.sqrt(np.mean(f.astype(np.float64) ** 2)))
    return (f / rms).astype(dtype) if rms > 0 else f.astype(dtype)


def _mode_norm(shape):
    nx, ny, nz = shape
    mx = np.fft.fftfreq(nx, 1.0 / nx)[None, None, :]
    my = np.fft.fftfreq(ny, 1.0 / ny)[None, :, None]
    mz = np.fft.fftfreq(nz, 1.0 / nz)[:, None, None]
    return np.sqrt(mx * mx + my * my + mz * mz)


def _back(f, axis):
    """f[i] - f[i-1] along a grid axis (x = 2, y = 1, z = 0 of the array)."""
    if f.shape[axis] == 1:
        return np.zeros_like(f)
    return f - np.roll(f, 1, axis=axis)


def _fwd(f, axis):
    """f[i+1] - f[i] along a grid axis."""
    if f.shape[axis] == 1:
        return np.zeros_like(f)
    return np.roll(f, -1, axis=axis) - f


def _curl_back(p, d):
    """Staggered curl with backward differences: a potential at the B
    positions to a field at the E positions (zero backward divergence)."""
    return np.stack([_back(p[2], 1) / d[1] - _back(p[1], 0) / d[2],
                     _back(p[0], 0) / d[2] - _back(p[2], 2) / d[0],
                     _back(p[1], 2) / d[0] - _back(p[0], 1) / d[1]])


def _curl_fwd(p, d):
    """Staggered curl with forward differences: a potential at the E
    positions to a field at the B positions (zero forward divergence)."""
    return np.stack([_fwd(p[2], 1) / d[1] - _fwd(p[1], 0) / d[2],
                     _fwd(p[0], 0) / d[2] - _fwd(p[2], 2) / d[0],
                     _fwd(p[1], 2) / d[0] - _fwd(p[0], 1) / d[1]])


def power_law_fields(shape, kmax, seed, exponent=-2.0, dtype=np.float32, d=(1.0, 1.0, 1.0)):
    """Divergence-free E and B with random-phase spectra: E = C^T psi_E (the
    backward staggered curl of a potential at the B positions), B = C psi_B
    (the forward curl of a potential at the E positions), so that the
    backward divergence of E and the forward divergence of B vanish
    identically.  Each potential component has amplitude |n|^(exponent/2 - 1)
    on the integer mode vectors 1 <= |n| <= kmax, so the fields' power falls
    as |n|^exponent there (the curl contributes one power of |n|) and is zero
    elsewhere; E and B are each scaled to unit RMS over their three
    components.  Returns (E, B)."""
    s = _shape3(shape)
    nrm = _mode_norm(s)
    w = np.where((nrm >= 1.0) & (nrm <= kmax), np.power(np.maximum(nrm, 1.0), exponent / 2.0 - 1.0), 0.0)
    rng = np.random.default_rng(seed)
    out = []
    for curl in (_curl_back, _curl_fwd):
        psi = [_spectrum_plane(rng, s, w, np.float64) for _ in range(3)]
        F = curl(psi, d)
        r = float(np.sqrt(np.mean(F * F)))
        out.append((F / r if r > 0 else F).astype(dtype))
    return out[0], out[1]


def solenoidal_current(shape, seed, width=16.0, rms=1e-3, dtype=np.float32, d=(1.0, 1.0, 1.0)):
    """A current with zero discrete divergence: the staggered curl of a smooth
    random vector potential psi (psi_a at the B_a position, Gaussian spectrum
    exp(-|k|^2 width^2 / 2) in cells, random phases).  The curl is taken with
    backward differences so that the result sits at the E/j positions and the
    backward divergence of it vanishes identically.  Scaled to the given RMS
    over all three components."""
    s = _shape3(shape)
    nx, ny, nz = s
    kx = 2 * np.pi * np.fft.fftfreq(nx)[None, None, :]
    ky = 2 * np.pi * np.fft.fftfreq(ny)[None, :, None]
    kz = 2 * np.pi * np.fft.fftfreq(nz)[:, None, None]
    w = np.exp(-(kx * kx + ky * ky + kz * kz) * width * width / 2.0)
    w[0, 0, 0] = 0.0
    rng = np.random.default_rng(seed)
    psi = [_spectrum_plane(rng, s, w, np.float64) for _ in range(3)]
    J = _curl_back(psi, d)
    r = float(np.sqrt(np.mean(J ** 2)))
    if r > 0:
        J *= rms / r
    return J.astype(dtype)


def random_fields(shape, seed, dtype=np.float64):
    """Unit-normal white-noise E, B, J (for parity tests of the raw stencils)."""
    nx, ny, nz = _shape3(shape)
    rng = np.random.default_rng(seed)
    a = rng.standard_normal((9, nz, ny, nx))
    return a[:3].astype(dtype), a[3:6].astype(dtype), a[6:].astype(dtype)


def batch_sizes(count, seed, lo=64, hi=1024, courant_lo=0.3, courant_hi=0.9):
    """Sizes drawn log-uniform in [lo, hi] per side and Courant fractions
    uniform in [courant_lo, courant_hi], one per grid."""
    rng = np.random.default_rng(seed)
    nx = np.round(np.exp(rng.uniform(math.log(lo), math.log(hi), count))).astype(int)
    ny = np.round(np.exp(rng.uniform(math.log(lo), math.log(hi), count))).astype(int)
    cf = rng.uniform(courant_lo, courant_hi, count)
    return [(int(a), int(b), float(c)) for a, b, c in zip(nx, ny, cf)]


def gauss_sources(count, shape, seed):
    """Centres (x_p, y_p) uniform over a 2D grid, phases U[0, 2 pi) and unit
    normal amplitudes for `count` Gaussian-envelope current sources."""
    rng = np.random.default_rng(seed)
    nx, ny = int(shape[0]), int(shape[1])
    cxy = np.stack([rng.uniform(0, nx, count), rng.uniform(0, ny, count)], axis=1)
    phases = rng.uniform(0.0, 2.0 * math.pi, count)
    theta = rng.standard_normal(count)
    return cxy, phases, theta
