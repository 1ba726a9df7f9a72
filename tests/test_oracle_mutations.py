"""Plant plausible mistakes in the oracle's C source and check that the
independent pins (closed-form dispersion, conservation laws, filter transfer
function, textbook tridiagonal solve) catch every one of them.  The mutated
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
    return bad


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
