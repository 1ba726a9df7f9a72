"""Pins of the NCI oracle (``oracle/nci.py``): the resonance curves of Eqs.
reson1/reson2 and the growth rate of App. E, checked against what the paper
states and what the mathematics fixes, not against the oracle itself:

* Sec. 4.2: the nu = 0 curve appears exactly at dt = dt_CFL / sqrt 2; no
  |nu| >= 2 curve for dt <= dt_CFL; every crossing has |k_x| > 2.06 / dx, the
  bound reached as dt -> 0;
* every crossing lies on the converged EM branch (Eq. dispersion-em-F-2d,
  solved for omega by the spectral oracle) at omega = c |k_x'|;
* A_1' is the omega-derivative of A_1 at the crossing (finite differences of
  the undifferentiated A_1), which fixes xi_0..xi_3;
* Gamma is the largest imaginary part among the roots of A_1' dw^3 + C_1 = 0
  (numpy.roots);
* Eq. NCI-growth-rate, the paper's final closed form, gives the same Gamma;
* Gamma vanishes on the k_x axis, is even in k_y, scales as omega_p^(2/3) and
  falls with the particle-shape order.
Planted mistakes in a copy of the oracle must each fail one of these.
"""
import math
import types

import numpy as np
import pytest

from oracle import core, nci, spectral

DX = DY = 1.0
WP = 1.0 / 16.0  # Sec. 4.2 table: L_x = 16 d_e over 256 cells, omega_p dx / c = 1/16


def _crossings(mod, courant, nu, nkx=4096, dx=DX, dy=DY):
    dt = courant * mod.dt_cfl(dx, dy)
    kx = mod.kx_samples(nkx, dx)
    ky = mod.resonance_ky(kx, nu, dx, dy, dt)
    ok = ~np.isnan(ky)
    return kx[ok], ky[ok], dt


def pin_nu0_threshold(mod):
    c0 = 1.0 / math.sqrt(2.0)
    dt0 = c0 * mod.dt_cfl(DX, DY)
    # at the threshold the curve touches the zone corner k = (pi, 0)
    f = mod.resonance_function(np.array([math.pi]), np.array([0.0]), 0, DX, DY, dt0)
    assert abs(f[0]) < 1e-12, f
    assert len(_crossings(mod, c0 * (1 - 1e-3), 0)[0]) == 0
    assert len(_crossings(mod, 0.72, 0)[0]) > 0


def pin_no_second_alias(mod):
    for courant in np.linspace(0.1, 1.0, 10):
        for nu in (-2, 2):
            assert len(_crossings(mod, courant, nu, 1024)[0]) == 0, (courant, nu)
        for nu in (-1, 1):
            assert len(_crossings(mod, courant, nu, 1024)[0]) > 0, (courant, nu)


def pin_kx_bound(mod):
    lows = []
    for courant in (1e-3, 0.1, 0.5, 0.8, 1.0):
        for nu in (-1, 0, 1):
            kx, _, _ = _crossings(mod, courant, nu, 4096)
            if len(kx):
                lows.append((courant, float(np.abs(kx).min())))
    assert min(l for _, l in lows) >= 2.06, lows
    assert 2.06 <= lows[0][1] < 2.07, lows  # dt -> 0: the printed bound


def pin_on_em_branch(mod):
    for courant in (0.3, 0.9):
        p = core.Params(shape=(8, 8), courant=courant)
        for nu in (-1, 0, 1):
            kx, ky, dt = _crossings(mod, courant, nu, 512)
            if not len(kx):
                continue
            assert abs(dt - p.time_step()) < 1e-15
            om = spectral.omega_converged(p, (kx, ky))
            np.testing.assert_allclose(om, np.abs(kx + 2 * math.pi * nu / DX), rtol=1e-9)


def _sample_points(mod, courant=0.5, nkx=256):
    pts = []
    for nu in (-1, 0, 1):
        kx, ky, dt = _crossings(mod, courant, nu, nkx)
        pts += [(a, b, nu, dt) for a, b in zip(kx[::17], ky[::17])]
    return pts


def pin_a1_derivative(mod):
    def a1(om, kx, ky, dt):
        w = np.sin(om * dt / 2) / (dt / 2)
        at = (2 + np.cos(om * dt)) / 3
        ax, ay = (2 + np.cos(kx * DX)) / 3, (2 + np.cos(ky * DY)) / 3
        bx, by = np.sin(kx * DX / 2) / (DX / 2), np.sin(ky * DY / 2) / (DY / 2)
        return ax * ay * w ** 4 - at * w ** 2 * (ay * bx ** 2 + ax * by ** 2)

    for courant in (0.5, 0.9):
        for kx, ky, nu, dt in _sample_points(mod, courant):
            t = mod.growth_terms(kx, ky, nu, DX, DY, dt, WP, 1)
            om, h = t["omega"], 1e-5
            fd = (a1(om + h, kx, ky, dt) - a1(om - h, kx, ky, dt)) / (2 * h)
            assert abs(fd - t["a1p"]) <= 1e-7 * abs(t["a1p"]) + 1e-9, (kx, ky, nu, fd, t["a1p"])


def pin_cubic_roots(mod):
    for kx, ky, nu, dt in _sample_points(mod):
        t = mod.growth_terms(kx, ky, nu, DX, DY, dt, WP, 2)
        roots = np.roots([t["a1p"], 0.0, 0.0, t["c1"]])
        g = mod.growth_rate(kx, ky, nu, DX, DY, dt, WP, 2)
        assert abs(roots.imag.max() - g) <= 1e-10 * g, (roots, g)


def pin_final_form(mod):
    """Eq. NCI-growth-rate with the momentum-conserving S factors."""
    for l in (1, 2, 4):
        for kx, ky, nu, dt in _sample_points(mod, 0.7):
            kxp = kx + 2 * math.pi * nu / DX
            x0 = np.sin(kxp * dt / 2) / (dt / 2)
            x1 = np.cos(kxp * dt / 2)
            x2 = (2 + np.cos(kxp * dt)) / 3
            x3 = -dt * np.sin(kxp * dt) / 3
            ax, ay = (2 + np.cos(kx * DX)) / 3, (2 + np.cos(ky * DY)) / 3
            bx, by = np.sin(kx * DX / 2) / (DX / 2), np.sin(ky * DY / 2) / (DY / 2)
            sx = (np.sin(kxp * DX / 2) / (kxp * DX / 2)) ** (l + 1)
            sy = (np.sin(ky * DY / 2) / (ky * DY / 2)) ** (l + 1)
            num = by * ky * (ax * x0 * np.cos(kxp * dt / 2) * (-1) ** nu - x2 * bx)
            den = x0 ** 2 * ax * ay * (2 * x1 - x3 * x0 / x2)
            ref = math.sqrt(3) / 2 * abs(WP * sx * sy) ** (2 / 3) * abs(num / den) ** (1 / 3)
            g = mod.growth_rate(kx, ky, nu, DX, DY, dt, WP, l)
            assert abs(g - ref) <= 1e-11 * ref, (l, kx, ky, nu, g, ref)


def pin_shape_of_gamma(mod):
    for kx, ky, nu, dt in _sample_points(mod, 0.6):
        g = [mod.growth_rate(kx, ky, nu, DX, DY, dt, WP, l) for l in (1, 2, 4)]
        assert g[0] > g[1] > g[2] > 0, g
        assert mod.growth_rate(kx, 0.0, nu, DX, DY, dt, WP, 1) == 0.0
        gm = mod.growth_rate(kx, -ky, nu, DX, DY, dt, WP, 1)
        assert abs(gm - g[0]) <= 1e-14 * g[0]
        g2 = mod.growth_rate(kx, ky, nu, DX, DY, dt, 2 * WP, 1)
        assert abs(g2 / g[0] - 2 ** (2 / 3)) < 1e-13


PINS = [pin_nu0_threshold, pin_on_em_branch, pin_a1_derivative, pin_cubic_roots,
        pin_final_form, pin_shape_of_gamma, pin_no_second_alias, pin_kx_bound]


@pytest.mark.parametrize("pin", PINS, ids=lambda f: f.__name__)
def test_oracle_nci_pins(pin):
    pin(nci)


def test_resonance_table_and_best():
    r = nci.resonance(1024, 0.5, DX, DY, WP, 1, nu_max=2)
    assert r["ky"].shape == (5, 1024) and r["nus"] == [-2, -1, 0, 1, 2]
    assert np.all(np.isnan(r["ky"][[0, 2, 4]]))  # only nu = +-1 at dt = dt_CFL / 2
    ok = ~np.isnan(r["ky"])
    assert np.all(r["gamma"][~ok] == 0) and np.all(r["gamma"][ok] > 0)
    g, kx, ky, nu = r["best"]
    assert g == r["gamma"].max() and nu in (-1.0, 1.0)
    assert abs(nci.growth_rate(kx, ky, int(nu), DX, DY, r["dt"], WP, 1) - g) == 0.0


def test_origin_is_not_a_crossing():
    """Odd nkx samples k_x = 0, where the nu = 0 beam meets the EM mode only
    at omega = k = 0."""
    r = nci.resonance(1025, 0.9, DX, DY, WP, 1, nu_max=1)
    assert r["kx"][512] == 0.0
    assert np.isnan(r["ky"][1, 512]) and r["gamma"][1, 512] == 0.0
    assert np.all(np.isfinite(r["gamma"])) and np.isfinite(r["best"][0])


MUTANTS = {
    "time_aliased_beam": ("(np.abs(om * dt) <= math.pi)", "(np.abs(om * dt) >= 0.0)"),
    "reson_without_alpha_t": ("return x0 ** 2 / (x2 * c * c) - _bracket(kx, dx)",
                              "return x0 ** 2 / (c * c) - _bracket(kx, dx)"),
    "xi1_sign": ("x1 = np.cos(omega * dt / 2.0)", "x1 = -np.cos(omega * dt / 2.0)"),
    "xi3_weight": ("x3 = -dt * np.sin(omega * dt) / 3.0", "x3 = -dt * np.sin(omega * dt) / 6.0"),
    "qxy_sign": ("(s_ey * x0 - s_bz * bx * c)", "(s_ey * x0 + s_bz * bx * c)"),
    "shape_unaliased": ("ss = shape_factor(kxp, dx, l)", "ss = shape_factor(kx, dx, l)"),
    "lost_sqrt3": ("return math.sqrt(3.0) / 2.0 * np.cbrt", "return 0.5 * np.cbrt"),
    "alias_sign_dropped": ("sign = -1.0 if (int(nu) % 2) else 1.0", "sign = 1.0"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistakes_are_caught(name):
    with open(nci.__file__) as f:
        src = f.read()
    old, new = MUTANTS[name]
    assert src.count(old) == 1, name
    mod = types.ModuleType(f"nci_mutant_{name}")
    exec(compile(src.replace(old, new), mod.__name__, "exec"), mod.__dict__)
    for pin in PINS:
        try:
            pin(mod)
        except AssertionError:
            return
    pytest.fail(f"mutation {name} passed every pin")
