"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

None of these compare the oracle with itself: each checks a closed form the
paper prints, a conservation law it proves, a value it prints, a textbook
special case, or a second derivation (the per-wavevector symbols of Sec. 2).
"""
import math

import numpy as np
import pytest
import scipy.linalg

from oracle import core, spectral
from paper_1907_13088_gb300 import synth
from tests.conftest import golden


def _rel(a, b):
    return float(np.linalg.norm(np.ravel(a - b)) / max(np.linalg.norm(np.ravel(b)), 1e-300))


def _mode_coeff(field2d, mx, my):
    return np.fft.fft2(field2d)[my, mx]


def _omega_by_recurrence(p, E, B, comp, which, mx, my, steps=3):
    """Frequency of a single spatial mode from three consecutive steps: a
    sequence c+ z^n + c- z^-n obeys f[n+1] + f[n-1] = 2 cos(omega dt) f[n]."""
    seq = []
    for _ in range(steps):
        f = (E if which == "E" else B)[comp, 0]
        seq.append(_mode_coeff(f, mx, my))
        E, B, rc, _ = core.step(p, E, B, None, 1)
        assert rc == core.OK
    cosw = ((seq[2] + seq[0]) / (2 * seq[1])).real
    return math.acos(cosw) / p.time_step()


def _tm_mode(p, mx, my):
    nx, ny = p.shape
    E = np.zeros(p.array_shape)
    B = np.zeros(p.array_shape)
    ii = np.arange(nx)[None, :]
    jj = np.arange(ny)[:, None]
    E[2, 0] = np.cos(2 * np.pi * (mx * ii / nx + my * jj / ny))
    return E, B


# --------------------------------------------------------------------------
# two derivations agree: stencils (Sec. 2 operators) vs Fourier symbols
# --------------------------------------------------------------------------

@pytest.mark.parametrize("shape,courant,m,passes", [
    ((16, 12), 0.5, 4, 3), ((9, 7), 0.9, 2, 1), ((8, 6, 5), 0.5, 4, 1), ((6, 5, 7), 0.95, 3, 0),
    ((20,), 0.7, 5, 2)])
def test_stencil_matches_spectral(shape, courant, m, passes):
    p = core.Params(shape=shape, courant=courant, m=m, filter_passes=passes)
    E, B, J = synth.random_fields(shape, seed=11)
    E1, B1, rc, _ = core.step(p, E, B, J, nsteps=3)
    E2, B2 = spectral.step(p, E, B, J, nsteps=3)
    assert rc == core.OK
    assert _rel(E1, E2) < 1e-13 and _rel(B1, B2) < 1e-13


def test_coefficients_match_spectral_bitwise():
    for f32 in (False, True):
        for lumped in (False, True):
            p = core.Params(shape=(8, 8, 8), d=(1.0, 0.7, 1.3), courant=0.61, lumped=lumped, coef_f32=f32)
            a = core.coefficients(p)
            b = spectral.coefficients(p)
            assert a == b


# --------------------------------------------------------------------------
# dispersion relation, Eq. dispersion-em-F-2d / -3d (converged iteration)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("courant", [0.1, 0.5, 0.7, 1.0])
@pytest.mark.parametrize("mode", [(1, 0), (5, 3), (3, 7), (8, 8), (12, 4)])
def test_tm_dispersion_converged(courant, mode):
    p = core.Params(shape=(32, 24), courant=courant, residual=True, tol=1e-15, m_max=4000)
    mx, my = mode
    my = my % 24
    E, B = _tm_mode(p, mx, my)
    w = _omega_by_recurrence(p, E, B, 2, "E", mx, my)
    kv = (2 * np.pi * mx / 32, 2 * np.pi * my / 24)
    assert abs(w - spectral.omega_converged(p, kv)) / w < 1e-11


@pytest.mark.parametrize("courant", [0.5, 1.0])
@pytest.mark.parametrize("mode", [(2, 1), (6, 5), (11, 3)])
def test_te_dispersion_converged(courant, mode):
    """The TE polarisation (E_x, E_y, B_z) obeys the same relation (the
    determinant of the vacuum dielectric tensor has a double EM root)."""
    p = core.Params(shape=(24, 20), courant=courant, residual=True, tol=1e-15, m_max=4000)
    mx, my = mode
    E = np.zeros(p.array_shape)
    B = np.zeros(p.array_shape)
    ii = np.arange(24)[None, :] + 0.5
    jj = np.arange(20)[:, None] + 0.5
    B[2, 0] = np.cos(2 * np.pi * (mx * ii / 24 + my * jj / 20))
    w = _omega_by_recurrence(p, E, B, 2, "B", mx, my)
    kv = (2 * np.pi * mx / 24, 2 * np.pi * my / 20)
    assert abs(w - spectral.omega_converged(p, kv)) / w < 1e-11


def test_3d_dispersion_converged():
    p = core.Params(shape=(12, 10, 8), d=(1.0, 0.8, 1.2), courant=0.8, residual=True, tol=1e-15, m_max=4000)
    mx, my, mz = 2, 3, 1
    E = np.zeros(p.array_shape)
    B = np.zeros(p.array_shape)
    k = np.arange(8)[:, None, None]
    j = np.arange(10)[None, :, None]
    i = np.arange(12)[None, None, :]
    E[1] = np.cos(2 * np.pi * (mx * i / 12 + my * (j + 0.5) / 10 + mz * k / 8))
    E[2] = 0.3 * np.sin(2 * np.pi * (mx * i / 12 + my * j / 10 + mz * (k + 0.5) / 8))
    seq = []
    for _ in range(3):
        seq.append([np.fft.fftn(B[c])[mz, my, mx] for c in range(3)])
        E, B, rc, _ = core.step(p, E, B, None, 1)
    kv = (2 * np.pi * mx / (12 * 1.0), 2 * np.pi * my / (10 * 0.8), 2 * np.pi * mz / (8 * 1.2))
    # every component of B: a wrong term may move only a curl-free part of E,
    # which a single component of curl E can miss
    for c in range(3):
        f0, f1, f2 = (seq[n][c] for n in range(3))
        w = math.acos(((f0 + f2) / (2 * f1)).real) / p.time_step()
        assert abs(w - spectral.omega_converged(p, kv)) / w < 1e-11, c


def test_plane_wave_sum_phase_advance_200_steps():
    """Config-1-like run: 8 TM plane waves on 64x64, dt = 0.5 dt_CFL, 200 steps,
    residual mode 1e-13.  Every mode's complex amplitude must rotate by the
    closed-form omega (counter-propagating parts separated by two samples)."""
    p = core.Params(shape=(64, 64), courant=0.5, residual=True, tol=1e-13, m_max=2000)
    E, B, modes = synth.tm_plane_waves((64, 64), p.time_step(), seed=1907001)
    E, B, rc, _ = core.step(p, E, B, None, 198)
    assert rc == core.OK
    seq = []
    for _ in range(3):
        seq.append(np.fft.fft2(E[2, 0]))
        E, B, rc, _ = core.step(p, E, B, None, 1)
    for mx, my, _, _ in modes:
        kv = (2 * np.pi * mx / 64, 2 * np.pi * my / 64)
        c = [s[my % 64, mx % 64] for s in seq]
        w = math.acos(((c[0] + c[2]) / (2 * c[1])).real) / p.time_step()
        assert abs(w - spectral.omega_converged(p, kv)) / w < 1e-10


# --------------------------------------------------------------------------
# truncated iteration (App. D) and the printed Fig. 2(a) values
# --------------------------------------------------------------------------

@pytest.mark.parametrize("courant,m", [(0.5, 4), (0.9, 4), (1.0, 20), (0.3, 1), (0.7, 0)])
@pytest.mark.parametrize("mode", [(5, 3), (12, 9), (16, 12)])
def test_tm_dispersion_fixed_m(courant, m, mode):
    p = core.Params(shape=(32, 24), courant=courant, m=m)
    mx, my = mode
    E, B = _tm_mode(p, mx, my)
    w = _omega_by_recurrence(p, E, B, 2, "E", mx, my)
    kv = (2 * np.pi * mx / 32, 2 * np.pi * my / 24)
    assert abs(w - spectral.omega_fixed_m_tm(p, kv, m)) / w < 1e-11


def test_fig2a_printed_error():
    """Fig. 2(a): after m = 20 sweeps at dt = dt_CFL, dx = dy, the error of the
    dispersion relation, |[w_m]^2/[w_inf]^2 - 1| ~ |lambda_3|^{m+1}
    (Eq. dispersion_error), peaks at 2e-4 at the Brillouin-zone corner and is
    below 1e-16 near k = 0.  Checked three ways: the A-matrix eigenvalues over
    the zone, and the stencil oracle's measured frequency at the corner."""
    g = golden("fig2a_dispersion_error.txt")
    m = int(g["m"])
    p = core.Params(shape=(16, 16), courant=g["courant"], m=m)
    ks = np.linspace(-np.pi, np.pi, 65)
    worst, worst_k = 0.0, None
    for kx in ks:
        for ky in ks:
            lam = np.max(np.abs(np.linalg.eigvalsh(spectral.A_matrix(p, (kx, ky, 0.0))[:3, :3])))
            err = lam ** (m + 1)
            if err > worst:
                worst, worst_k = err, (kx, ky)
    printed = g["max_error"]
    assert abs(worst - printed) < 0.5 * 10 ** (math.floor(math.log10(printed)))  # 1 printed digit
    assert abs(abs(worst_k[0]) - np.pi) < 1e-12 and abs(abs(worst_k[1]) - np.pi) < 1e-12
    # near k = 0
    lam0 = np.max(np.abs(np.linalg.eigvalsh(spectral.A_matrix(p, (0.05, 0.05, 0.0)))))
    assert lam0 ** (m + 1) < g["small_k_error_below"]
    # the stencil oracle at the corner mode: ratio of squared bracket frequencies
    E, B = _tm_mode(p, 8, 8)
    wm = _omega_by_recurrence(p, E, B, 2, "E", 8, 8)
    dt = p.time_step()
    winf = spectral.omega_converged(p, (np.pi, np.pi))
    br = lambda w: (math.sin(w * dt / 2) / (dt / 2)) ** 2
    err = abs(br(wm) / br(winf) - 1.0)
    assert abs(err - (2.0 / 3.0) ** (m + 1)) < 1e-12
    assert abs(err - printed) < 0.5e-4


def test_step_matrix_unit_modulus_fixed_m():
    """Fixed m = 4 stays neutrally stable (all |eig T(k)| = 1) below dt_CFL for
    dx = dy (lambda >= 0), while dt beyond dt_CFL grows.  (At exactly dt_CFL the
    zone corner is a double root z = -1, a Jordan block, as for Yee.)"""
    for courant in (0.3, 0.5, 0.9, 0.99):
        p = core.Params(shape=(8, 8), courant=courant, m=4)
        for kx in np.linspace(0.1, np.pi, 9):
            for ky in np.linspace(0.0, np.pi, 9):
                ev = np.linalg.eigvals(spectral.step_matrix(p, (kx, ky, 0.0)))
                assert np.max(np.abs(ev)) < 1 + 1e-9
    p = core.Params(shape=(8, 8), courant=1.02, residual=True)
    ev = np.linalg.eigvals(spectral.step_matrix(p, (np.pi, np.pi, 0.0), exact=True))
    assert np.max(np.abs(ev)) > 1.01


# --------------------------------------------------------------------------
# CFL limit, superluminal phase speed, small-k expansion (Sec. 2.1, App. B)
# --------------------------------------------------------------------------

def test_cfl_and_superluminal():
    for d in ((1.0, 1.0), (1.0, 0.5), (0.7, 1.3)):
        p = core.Params(shape=(8, 8), d=d + (1.0,), courant=1.0)
        assert abs(core.dt_cfl(p) - 1.0 / math.sqrt(1 / d[0] ** 2 + 1 / d[1] ** 2)) < 1e-15
        # superluminous "in a large range of k including k = 0" (Sec. 1, Sec. 2.1):
        # over the whole zone for dt <= dt_CFL/2, and for |k d| <= 2.5 up to dt_CFL
        for courant in (0.1, 0.5, 0.7, 1.0):
            p.courant = courant
            for kx in np.linspace(0.01, np.pi / d[0], 17):
                for ky in np.linspace(0.0, np.pi / d[1], 17):
                    if courant > 0.5 and math.hypot(kx * d[0], ky * d[1]) > 2.5:
                        continue
                    w = spectral.omega_converged(p, (kx, ky))
                    assert w / math.hypot(kx, ky) >= p.c * (1 - 1e-13)
    # luminous on the diagonal at dt_CFL for dx = dy (Sec. 2.1)
    p = core.Params(shape=(8, 8), courant=1.0)
    for t in np.linspace(0.05, np.pi, 12):
        assert abs(spectral.omega_converged(p, (t, t)) / (math.sqrt(2) * t) - 1) < 1e-12
    # ... and superluminous off it
    assert spectral.omega_converged(p, (1.0, 0.3)) / math.hypot(1.0, 0.3) > 1 + 1e-4


def test_small_k_expansion():
    """Eq. phase-speed-2d / -3d: the leading correction of omega/k."""
    for dims, d, courant in ((2, (1.0, 0.6, 1.0), 0.5), (3, (1.0, 0.9, 1.2), 0.8), (2, (1.0, 1.0, 1.0), 0.3)):
        p = core.Params(shape=(8,) * dims, d=d, courant=courant)
        direction = np.array([0.8, 0.5, 0.33])[:dims]
        direction /= np.linalg.norm(direction)
        for kn in (3e-3, 1e-2):
            kv = tuple(kn * direction)
            w = spectral.omega_converged(p, kv)
            exact = w / kn / p.c - 1
            pred = spectral.phase_speed_expansion(p, kv) / p.c - 1
            assert exact > 0 and abs(exact / pred - 1) < 20 * kn ** 2


# --------------------------------------------------------------------------
# Yee limit (Sec. 2: lumping the averaging operators)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("mode", [(3, 2), (9, 10), (16, 1)])
def test_lumped_is_yee(mode):
    p = core.Params(shape=(32, 24), courant=0.8, lumped=True, m=4)
    mx, my = mode
    E, B = _tm_mode(p, mx, my % 24)
    w = _omega_by_recurrence(p, E, B, 2, "E", mx, my % 24)
    kv = (2 * np.pi * mx / 32, 2 * np.pi * (my % 24) / 24)
    assert abs(w - spectral.omega_yee(p, kv)) / w < 1e-12


# --------------------------------------------------------------------------
# conservation laws (App. A) and discrete energy
# --------------------------------------------------------------------------

def test_div_b_conserved_any_m():
    for shape, m in (((20, 18), 4), ((8, 7, 6), 2)):
        p = core.Params(shape=shape, courant=0.7, m=m, filter_passes=1)
        E, B, J = synth.random_fields(shape, seed=5)
        d0 = core.div_b(p, B)
        E1, B1, _, _ = core.step(p, E, B, J, nsteps=15)
        assert np.max(np.abs(core.div_b(p, B1) - d0)) < 1e-12 * max(1.0, np.max(np.abs(d0)))


def test_gauss_conserved_converged_not_fixed():
    """Eq. gauss_E holds when the solve converges and j is divergence-free
    (charge-conserving, rho constant); a fixed m leaves a small violation
    -Dbar.(A^{m+1} dE') per step, which is why the conservation pin runs the
    converged solve."""
    shape = (24, 20)
    E, B, _ = synth.random_fields(shape, seed=7)
    J = synth.solenoidal_current(shape, seed=8, width=2.0, rms=0.1, dtype=np.float64)
    p = core.Params(shape=shape, courant=0.6, residual=True, tol=1e-15, m_max=5000, filter_passes=2)
    g0 = core.gauss_e(p, E)
    E1, _, rc, _ = core.step(p, E, B, J, nsteps=10)
    assert rc == core.OK
    assert np.max(np.abs(core.gauss_e(p, E1) - g0)) < 1e-11
    pf = core.Params(shape=shape, courant=0.6, m=2, filter_passes=2)
    E2, _, _, _ = core.step(pf, E, B, J, nsteps=10)
    assert np.max(np.abs(core.gauss_e(pf, E2) - g0)) > 1e-6
    py = core.Params(shape=shape, courant=0.6, lumped=True, filter_passes=2)
    E3, _, _, _ = core.step(py, E, B, J, nsteps=10)
    assert np.max(np.abs(core.gauss_e(py, E3) - core.gauss_e(py, E))) < 1e-11


def test_energy_conserved_and_balanced():
    """W = sum[E.(1-A)E + B^{n-1/2}.S B^{n+1/2}] dV/8pi is exactly conserved by
    the converged vacuum step, and changes by -4 pi dt sum (E^{n+1}+E^n).j_f
    dV/8pi with a current (derived from the symmetry of A and S)."""
    shape = (16, 14)
    E, B, J = synth.random_fields(shape, seed=9)
    p = core.Params(shape=shape, courant=0.8, residual=True, tol=1e-15, m_max=5000)
    w0, _ = core.energy(p, E, B)
    E1, B1, _, _ = core.step(p, E, B, None, nsteps=40)
    w1, _ = core.energy(p, E1, B1)
    assert abs(w1 - w0) / w0 < 1e-12
    pj = core.Params(shape=shape, courant=0.8, residual=True, tol=1e-15, m_max=5000, filter_passes=1)
    Jf = core.filter(pj, J, 1)
    w0, _ = core.energy(pj, E, B)
    E1, B1, _, _ = core.step(pj, E, B, J, nsteps=1)
    w1, _ = core.energy(pj, E1, B1)
    pred = -4 * np.pi * pj.time_step() * np.sum((E1 + E) * Jf) / (8 * np.pi)
    assert abs((w1 - w0) - pred) < 1e-11 * abs(w0)


# --------------------------------------------------------------------------
# Algorithm 1 -> exact inverse; norms of A (App. C, App. D)
# --------------------------------------------------------------------------

def test_iteration_converges_to_exact_inverse():
    for shape, courant in (((16, 16), 0.5), ((12, 10), 1.0), ((8, 8, 8), 0.9)):
        rng = np.random.default_rng(3)
        dEp = rng.standard_normal((3,) + tuple(reversed(shape + (1,) * (3 - len(shape)))))
        p = core.Params(shape=shape, courant=courant)
        exact = spectral.exact_inverse(p, dEp)
        rho = 0.0
        kx, ky, kz = spectral.wavevectors(p)
        for a in np.ravel(kx):
            for b in np.ravel(ky):
                for c in np.ravel(kz):
                    rho = max(rho, np.max(np.abs(np.linalg.eigvalsh(spectral.A_matrix(p, (a, b, c))))))
        assert rho < 1
        for m in (0, 4, 12):
            p.m = m
            dE, rc, sw, _ = core.solve(p, dEp)
            err = _rel(dE, exact)
            assert err <= rho ** (m + 1) / (1 - rho) * 1.0001 + 1e-14
        p.residual, p.tol = True, 1e-14
        dE, rc, sw, r = core.solve(p, dEp)
        assert rc == core.OK and _rel(dE, exact) < 1e-12


def test_A_norm_bounds():
    """App. C: ||A||_inf < 1 in 2D for any dt <= dt_CFL; in 3D when
    dt <= min(d)/(sqrt(2) c).  The spectral radius is below those bounds."""
    rng = np.random.default_rng(4)
    for _ in range(20):
        d = tuple(rng.uniform(0.5, 2.0, 3))
        p2 = core.Params(shape=(4, 4), d=d, courant=rng.uniform(0.05, 1.0))
        dt = p2.time_step()
        sx, sy = (dt / d[0]) ** 2, (dt / d[1]) ** 2
        for kx in np.linspace(0, np.pi, 7):
            for ky in np.linspace(0, np.pi, 7):
                A = spectral.A_matrix(p2, (kx, ky, 0.0))
                assert abs(A[2, 2]) <= 8 / 9 - 2 / 9 * sx - 2 / 9 * sy + 1e-14
                assert np.max(np.abs(np.linalg.eigvalsh(A))) < 1
        p3 = core.Params(shape=(4, 4, 4), d=d, courant=1.0)
        p3.dt = min(min(d) / math.sqrt(2), p3.dt_cfl())
        for kv in rng.uniform(-np.pi, np.pi, (30, 3)):
            A = spectral.A_matrix(p3, tuple(kv))
            assert np.max(np.sum(np.abs(A), axis=1)) < 1
            assert np.max(np.abs(np.linalg.eigvalsh(A))) < 1


def test_1d_exact_tridiagonal():
    """1D (Sec. 2.2.3): E_x = E'_x and (1 - A_yy) = 1 - (sigma_x - 1)/6 Dbar_xx is a
    periodic tridiagonal (circulant) system; the converged iteration must equal
    its direct solution."""
    n = 40
    p = core.Params(shape=(n,), courant=0.8, residual=True, tol=1e-15, m_max=5000)
    rng = np.random.default_rng(6)
    dEp = rng.standard_normal((3, 1, 1, n))
    dE, rc, sw, _ = core.solve(p, dEp)
    assert rc == core.OK
    assert np.array_equal(dE[0], dEp[0])
    sig = p.time_step() ** 2
    a = (sig - 1.0) / 6.0
    col = np.zeros(n)
    col[0], col[1], col[-1] = 1 + 2 * a, -a, -a
    for comp in (1, 2):
        x = scipy.linalg.solve_circulant(col, dEp[comp, 0, 0])
        assert _rel(dE[comp, 0, 0], x) < 1e-13


def test_2d_polarisations_decouple():
    """Sec. 2.2.2: E_z is solved independently of (E_x, E_y)."""
    p = core.Params(shape=(16, 12), courant=0.7, m=4, filter_passes=1)
    E, B, J = synth.random_fields((16, 12), seed=2)
    E[:2] = 0
    B[2] = 0
    J[:2] = 0
    E1, B1, _, _ = core.step(p, E, B, J, nsteps=5)
    assert np.all(E1[:2] == 0) and np.all(B1[2] == 0)


# --------------------------------------------------------------------------
# low-pass filter
# --------------------------------------------------------------------------

@pytest.mark.parametrize("passes", [1, 3])
def test_filter_transfer_function(passes):
    """Binomial passes multiply a single mode by prod_i cos^{2p}(k_i d_i/2)."""
    for shape, mode in (((32, 24), (5, 7)), ((10, 8, 12), (2, 3, 5))):
        p = core.Params(shape=shape)
        nx, ny, nz = p.n3
        k = np.arange(nz)[:, None, None]
        j = np.arange(ny)[None, :, None]
        i = np.arange(nx)[None, None, :]
        mz = mode[2] if len(mode) > 2 else 0
        phase = 2 * np.pi * (mode[0] * i / nx + mode[1] * j / ny + mz * k / nz)
        f = np.cos(phase)
        out = core.filter(p, f[None], passes)[0]
        h = np.cos(np.pi * mode[0] / nx) ** 2 * np.cos(np.pi * mode[1] / ny) ** 2 * np.cos(np.pi * mz / nz) ** 2
        assert np.max(np.abs(out - h ** passes * f)) < 1e-14


def test_residual_mode_zero_source_and_noconv():
    p = core.Params(shape=(8, 8), courant=0.5, residual=True, tol=1e-14)
    dE, rc, sw, _ = core.solve(p, np.zeros(p.array_shape))
    assert rc == core.OK and sw == 0
    p.m_max, p.tol = 3, 1e-15
    rng = np.random.default_rng(1)
    _, rc, sw, _ = core.solve(p, rng.standard_normal(p.array_shape))
    assert rc == core.ENOCONV and sw == 3


def _lambda_tm(p, kx, ky):
    """Symbol of A_zz (Eqs. matrixA_1st_2d..last_2d) with Dbar_aa -> -4 sin^2(k_a d_a / 2):
    (2/3)(1 - s_x) S_x + (2/3)(1 - s_y) S_y - (4/9)(1 - s_x - s_y) S_x S_y,
    s_a = (c dt / d_a)^2, S_a = sin^2(k_a d_a / 2)."""
    dt = p.time_step()
    sx, sy = (p.c * dt / p.d[0]) ** 2, (p.c * dt / p.d[1]) ** 2
    ax, ay = math.sin(kx * p.d[0] / 2) ** 2, math.sin(ky * p.d[1] / 2) ** 2
    return 2 / 3 * (1 - sx) * ax + 2 / 3 * (1 - sy) * ay - 4 / 9 * (1 - sx - sy) * ax * ay


@pytest.mark.parametrize("shape,d,courant,mode,tol", [
    ((20, 16), (1.0, 1.0, 1.0), 0.9, (3, 5), 1e-9),
    ((24, 20), (1.0, 0.7, 1.0), 0.5, (9, 7), 1e-12),
    ((32, 32), (1.0, 1.0, 1.0), 0.3, (16, 16), 1e-11),
    ((18, 30), (0.8, 1.1, 1.0), 1.0, (2, 11), 1e-7)])
def test_residual_stop_on_one_eigenmode(shape, d, courant, mode, tol):
    """Residual mode (Sec. 2.2.1 stop rule, read as the relative L2 norm of
    the update): for dE' a single TM mode, A acts as the scalar lambda_z(k),
    the update of sweep s is lambda^s dE', so the solve stops at the first s
    with |lambda|^s <= tol and reports |lambda|^s."""
    nx, ny = shape
    p = core.Params(shape=shape, d=d, courant=courant, residual=True, tol=tol, m_max=100000)
    kx, ky = 2 * math.pi * mode[0] / (nx * d[0]), 2 * math.pi * mode[1] / (ny * d[1])
    dEp = np.zeros(p.array_shape)
    dEp[2, 0] = np.cos(2 * math.pi * (mode[0] * np.arange(nx)[None, :] / nx + mode[1] * np.arange(ny)[:, None] / ny))
    lam = abs(_lambda_tm(p, kx, ky))
    q = math.log(tol) / math.log(lam)
    assert 0.05 < q - math.floor(q) < 0.95  # the case is not at a rounding boundary
    dE, rc, sw, r = core.solve(p, dEp)
    assert rc == core.OK and sw == math.ceil(q), (sw, q)
    assert abs(r - lam ** sw) <= 1e-6 * lam ** sw + 1e-14
    np.testing.assert_allclose(dE, dEp / (1 - _lambda_tm(p, kx, ky)), rtol=0, atol=10 * tol)


@pytest.mark.parametrize("shape,kw", [((12, 10), dict(m=4, filter_passes=3)),
                                      ((6, 5, 7), dict(m=2, filter_passes=1, d=(1.0, 0.8, 1.2))),
                                      ((20,), dict(m=3)),
                                      ((9, 8), dict(residual=True, tol=1e-14))])
def test_uniform_current_closed_form(shape, kw):
    """A uniform current with no fields: every difference operator vanishes,
    so Ampere's law in Gaussian units (Sec. 2) leaves dE/dt = -4 pi j exactly,
    E^n = -4 pi n dt j and B = 0, for any m, filter or solve mode (the
    binomial filter keeps constants)."""
    p = core.Params(shape=shape, courant=0.7, **kw)
    jv = (0.3, -1.1, 0.7)
    J = np.zeros(p.array_shape)
    for c in range(3):
        J[c] = jv[c]
    E, B, rc, _ = core.step(p, np.zeros(p.array_shape), np.zeros(p.array_shape), J, 3)
    assert rc == core.OK
    for c in range(3):
        np.testing.assert_allclose(E[c], -3 * 4 * math.pi * p.time_step() * jv[c], rtol=1e-14, atol=0)
    assert np.all(B == 0)
