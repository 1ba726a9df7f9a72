"""Plant plausible mistakes in the oracle's C source and check that the
independent pins (closed-form dispersion, conservation laws, filter transfer
function, the per-wavevector symbols in 1D and 3D, a uniform current's
closed-form response, the closed-form residual-stop sweep count) catch every
one of them.  The mutated
copies are compiled to a temporary directory; the oracle under test is not
touched."""
import math

import numpy as np
import pytest
import scipy.linalg

from oracle import core, spectral
from paper_1907_13088_gb300 import synth

MUTATIONS = {
    "cross_sign": ("co[ORC_BXY] = -(k[0] * k[1]) / 6.0;", "co[ORC_BXY] = (k[0] * k[1]) / 6.0;"),
    "drop_axy": ("co[ORC_AXY] = (s[0] + s[1] - 1.0) / 36.0;", "co[ORC_AXY] = 0.0;"),
    "alpha_weight": ("co[ORC_C6] = 1.0 / 6.0;", "co[ORC_C6] = 1.0 / 4.0;"),
    "faraday_direction": ("dbar(&s, Ez, d, 1, 1); axpy(&s, -co[ORC_KY], d, Bx);",
                          "dbar(&s, Ez, d, 1, 0); axpy(&s, -co[ORC_KY], d, Bx);"),
    "source_direction": ("alpha(&s, co[ORC_C6], Bz, ab, t, 2); dbar(&s, ab, d, 1, 0); axpy(&s, co[ORC_KY], d, ex);",
                         "alpha(&s, co[ORC_C6], Bz, ab, t, 2); dbar(&s, ab, d, 1, 1); axpy(&s, co[ORC_KY], d, ex);"),
    "transposed_operand": ("add_cross(&s, co[ORC_BXY], c6, y, ox, 0, 1, 2, t1, t2);",
                           "add_cross(&s, co[ORC_BXY], c6, x, ox, 0, 1, 2, t1, t2);"),
    "extra_sweep": ("for (int it = 0; it < p->m; ++it) {", "for (int it = 0; it <= p->m; ++it) {"),
    "skewed_filter": ("0.25 * at(&s, g, i, j, k, a, -1) + 0.5 * at(&s, g, i, j, k, a, 0) +\n                                0.25 * at(&s, g, i, j, k, a, 1);",
                      "0.2 * at(&s, g, i, j, k, a, -1) + 0.5 * at(&s, g, i, j, k, a, 0) +\n                                0.3 * at(&s, g, i, j, k, a, 1);"),
    "alpha_axis": ("alpha(&s, co[ORC_C6], Bx, ab, t, 0); dbar(&s, ab, d, 1, 0); axpy(&s, -co[ORC_KY], d, ez);",
                   "alpha(&s, co[ORC_C6], Bx, ab, t, 1); dbar(&s, ab, d, 1, 0); axpy(&s, -co[ORC_KY], d, ez);"),
    # terms that only a 3D grid exercises
    "cross_yz_operand": ("add_cross(&s, co[ORC_BYZ], c6, z, oy, 1, 2, 0, t1, t2);",
                         "add_cross(&s, co[ORC_BYZ], c6, x, oy, 1, 2, 0, t1, t2);"),
    "cross_zx_average_axis": ("add_cross(&s, co[ORC_BZX], c6, x, oz, 2, 0, 1, t1, t2);",
                              "add_cross(&s, co[ORC_BZX], c6, x, oz, 2, 0, 2, t1, t2);"),
    "ayz_weight": ("co[ORC_AYZ] = (s[1] + s[2] - 1.0) / 36.0;", "co[ORC_AYZ] = (s[1] + s[2] - 1.0) / 18.0;"),
    "diag_y_weights_swapped": ("add_diag(&s, co[ORC_AZ], co[ORC_AX], co[ORC_AZX], y, oy, 2, 0, t1, t2);",
                               "add_diag(&s, co[ORC_AX], co[ORC_AZ], co[ORC_AZX], y, oy, 2, 0, t1, t2);"),
    "byz_coefficient": ("co[ORC_BYZ] = -(k[1] * k[2]) / 6.0;", "co[ORC_BYZ] = -(k[1] * k[1]) / 6.0;"),
    "source_z_sign": ("alpha(&s, co[ORC_C6], By, ab, t, 1); dbar(&s, ab, d, 2, 0); axpy(&s, -co[ORC_KZ], d, ex);",
                      "alpha(&s, co[ORC_C6], By, ab, t, 1); dbar(&s, ab, d, 2, 0); axpy(&s, co[ORC_KZ], d, ex);"),
    "faraday_z_direction": ("dbar(&s, Ey, d, 2, 1); axpy(&s, co[ORC_KZ], d, Bx);",
                            "dbar(&s, Ey, d, 2, 0); axpy(&s, co[ORC_KZ], d, Bx);"),
    # the current's factor 4 pi dt (Gaussian units) and the residual stop
    "current_factor": ("co[ORC_Q] = (4.0 * M_PI) * p->dt;", "co[ORC_Q] = (2.0 * M_PI) * p->dt;"),
    "residual_squared": ("                r = sqrt(dd) / nrm;", "                r = dd / (nrm * nrm);"),
}


def _omega(p, E, B, comp, which, sel):
    seq = []
    for _ in range(3):
        f = E if which == "E" else B
        seq.append(np.fft.fftn(f[comp])[sel])
        E, B, _, _ = core.step(p, E, B, None, 1)
    return math.acos(max(-1.0, min(1.0, ((seq[0] + seq[2]) / (2 * seq[1])).real))) / p.time_step()


def _battery():
    """Returns the names of the pins that fail."""
    bad = []
    # TM fixed m (App. D reading) and converged
    for courant, m, resid in ((0.9, 4, False), (0.6, 0, True)):
        p = core.Params(shape=(20, 16), courant=courant, m=m, residual=resid, tol=1e-15, m_max=3000)
        E = np.zeros(p.array_shape)
        B = np.zeros(p.array_shape)
        mx, my = 3, 5
        E[2, 0] = np.cos(2 * np.pi * (mx * np.arange(20)[None, :] / 20 + my * np.arange(16)[:, None] / 16))
        w = _omega(p, E, B, 2, "E", (0, my, mx))
        kv = (2 * np.pi * mx / 20, 2 * np.pi * my / 16)
        ref = spectral.omega_converged(p, kv) if resid else spectral.omega_fixed_m_tm(p, kv, m)
        if not abs(w - ref) / ref < 1e-10:
            bad.append(f"tm_{courant}")
    # TE converged
    p = core.Params(shape=(20, 16), courant=0.8, residual=True, tol=1e-15, m_max=3000)
    E = np.zeros(p.array_shape)
    B = np.zeros(p.array_shape)
    B[2, 0] = np.cos(2 * np.pi * (4 * (np.arange(20)[None, :] + .5) / 20 + 3 * (np.arange(16)[:, None] + .5) / 16))
    w = _omega(p, E, B, 2, "B", (0, 3, 4))
    ref = spectral.omega_converged(p, (2 * np.pi * 4 / 20, 2 * np.pi * 3 / 16))
    if not abs(w - ref) / ref < 1e-10:
        bad.append("te")
    # conservation with a divergence-free current, converged (App. A)
    E, B, _ = synth.random_fields((14, 12), seed=3)
    J = synth.solenoidal_current((14, 12), seed=4, width=2.0, rms=0.1, dtype=np.float64)
    p = core.Params(shape=(14, 12), courant=0.6, residual=True, tol=1e-15, m_max=5000, filter_passes=1)
    g0, d0 = core.gauss_e(p, E), core.div_b(p, B)
    w0, _ = core.energy(p, E, B)
    E1, B1, _, _ = core.step(p, E, B, J, 3)
    if np.max(np.abs(core.gauss_e(p, E1) - g0)) > 1e-10:
        bad.append("gauss")
    if np.max(np.abs(core.div_b(p, B1) - d0)) > 1e-10:
        bad.append("divb")
    pv = core.Params(shape=(14, 12), courant=0.6, residual=True, tol=1e-15, m_max=5000)
    E2, B2, _, _ = core.step(pv, E, B, None, 3)
    w2, _ = core.energy(pv, E2, B2)
    if abs(w2 - w0) / w0 > 1e-11:
        bad.append("energy")
    # filter transfer function
    pf = core.Params(shape=(16, 12))
    f = np.cos(2 * np.pi * (3 * np.arange(16)[None, :] / 16 + 2 * np.arange(12)[:, None] / 12))[None, None]
    out = core.filter(pf, f, 2)
    h = (np.cos(np.pi * 3 / 16) ** 2 * np.cos(np.pi * 2 / 12) ** 2) ** 2
    if np.max(np.abs(out - h * f)) > 1e-13:
        bad.append("filter")
    # 3D with unequal spacings and 1D: stencils against the per-wavevector symbols
    for shape, d in (((8, 6, 5), (1.0, 0.8, 1.2)), ((20,), (1.0, 1.0, 1.0))):
        p = core.Params(shape=shape, d=d, courant=0.8, m=3, filter_passes=1)
        E, B, J = synth.random_fields(shape, seed=12)
        E1, B1, _, _ = core.step(p, E, B, J, 2)
        E2, B2 = spectral.step(p, E, B, J, 2)
        if _rel(E1, E2) > 1e-13 or _rel(B1, B2) > 1e-13:
            bad.append(f"spectral_{len(shape)}d")
    # 3D converged scheme: a mode with all three k components and unequal
    # spacings advances at the omega of Eq. dispersion-em-F-3d, seen in every
    # B component (a mistake may move only a curl-free part of E, which one
    # component of curl E can miss)
    p = core.Params(shape=(12, 10, 8), d=(1.0, 0.8, 1.2), courant=0.8, residual=True, tol=1e-15, m_max=4000)
    k3 = np.arange(8)[:, None, None]
    j3 = np.arange(10)[None, :, None]
    i3 = np.arange(12)[None, None, :]
    E = np.zeros(p.array_shape)
    E[1] = np.cos(2 * np.pi * (2 * i3 / 12 + 3 * (j3 + 0.5) / 10 + k3 / 8))
    E[2] = 0.3 * np.sin(2 * np.pi * (2 * i3 / 12 + 3 * j3 / 10 + (k3 + 0.5) / 8))
    B = np.zeros(p.array_shape)
    seq = []
    for _ in range(3):
        seq.append([np.fft.fftn(B[c])[1, 3, 2] for c in range(3)])
        E, B, _, _ = core.step(p, E, B, None, 1)
    ref = spectral.omega_converged(p, (2 * np.pi * 2 / 12, 2 * np.pi * 3 / 8, 2 * np.pi / 9.6))
    for c in range(3):
        f0, f1, f2 = (seq[n][c] for n in range(3))
        w = math.acos(max(-1.0, min(1.0, ((f0 + f2) / (2 * f1)).real))) / p.time_step()
        if not abs(w - ref) / ref < 1e-10:
            bad.append("dispersion_3d")
            break
    # a uniform current drives a uniform field at -4 pi j per unit time, B stays 0
    p = core.Params(shape=(6, 5, 7), d=(1.0, 0.8, 1.2), courant=0.7, m=2, filter_passes=1)
    J = np.zeros(p.array_shape)
    jv = (0.3, -1.1, 0.7)
    for c in range(3):
        J[c] = jv[c]
    E1, B1, _, _ = core.step(p, np.zeros(p.array_shape), np.zeros(p.array_shape), J, 3)
    ref = np.stack([np.full(p.array_shape[1:], -12.0 * math.pi * p.time_step() * v) for v in jv])
    if np.max(np.abs(E1 - ref)) > 1e-13 or np.max(np.abs(B1)) > 0:
        bad.append("uniform_current")
    # residual stop on a single TM eigenmode: the update after s sweeps is lambda^s
    p = core.Params(shape=(20, 16), courant=0.9, residual=True, tol=1e-9, m_max=1000)
    dEp = np.zeros(p.array_shape)
    dEp[2, 0] = np.cos(2 * np.pi * (3 * np.arange(20)[None, :] / 20 + 5 * np.arange(16)[:, None] / 16))
    _, _, sw, _ = core.solve(p, dEp)
    if sw != 20:  # ceil(ln 1e-9 / ln lambda_z), lambda_z = 0.34396 (Eqs. matrixA_1st_2d..last_2d)
        bad.append("sweep_count")
    return bad


def _rel(a, b):
    return float(np.linalg.norm(np.ravel(a - b)) / max(np.linalg.norm(np.ravel(b)), 1e-300))


def test_unmutated_battery_passes():
    assert _battery() == []


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_mutation_is_caught(name, tmp_path):
    old, new = MUTATIONS[name]
    src = core.source_text()
    assert src.count(old) == 1, f"mutation anchor for {name} not found exactly once"
    lib = core.compile_variant(src.replace(old, new), str(tmp_path / "libmut.so"))
    with core.using_library(lib):
        failed = _battery()
    assert failed, f"mutation {name} was not caught by any pin"
