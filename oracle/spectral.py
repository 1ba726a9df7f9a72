"""Spectral (per-wavevector) form of the step and the paper's closed forms.

TEST INFRASTRUCTURE ONLY (see ``oracle/core.py``).

In the per-component *physical-position* Fourier basis every operator of the
scheme is a scalar: with s_i = sin(k_i d_i / 2),
  Dbar_i -> 2 i s_i, D_i -> i [k]_i, [k]_i = 2 s_i / d_i (Eq. braket_k),
  alpha_i -> 1 - (2/3) s_i^2 (Eq. alphax),
so A (Eqs. matrixA_1st..matrixA_last) becomes a real symmetric 3x3 matrix per
k and one full step a 6x6 matrix T(k).  This is a second, independent
derivation of the stencil oracle in ``fmx_oracle.c``; the two must agree to
round-off on periodic grids.  numpy's FFT is used as a library primitive.
"""
from __future__ import annotations

import math

import numpy as np

# staggering offsets (in cells) of each stored component, Sec. 2 variable list
E_OFF = ((0.5, 0.0, 0.0), (0.0, 0.5, 0.0), (0.0, 0.0, 0.5))
B_OFF = ((0.0, 0.5, 0.5), (0.5, 0.0, 0.5), (0.5, 0.5, 0.0))


def coefficients(p) -> dict:
    """The step's scalar factors, computed here in numpy from the problem
    (kept separate from the C oracle on purpose)."""
    dt = p.time_step()
    cdt = p.c * dt
    d = [float(p.d[a]) if a < len(p.d) else 1.0 for a in range(3)]
    k = [cdt / d[a] for a in range(3)]
    s = [k[a] * k[a] for a in range(3)]
    co = {"kx": k[0], "ky": k[1], "kz": k[2], "q": 4.0 * math.pi * dt}
    if p.lumped:
        co.update({n: 0.0 for n in ("c6", "ax", "ay", "az", "ayz", "azx", "axy", "byz", "bzx", "bxy")})
    else:
        co.update({
            "c6": 1.0 / 6.0,
            "ax": (s[0] - 1.0) / 6.0, "ay": (s[1] - 1.0) / 6.0, "az": (s[2] - 1.0) / 6.0,
            "ayz": (s[1] + s[2] - 1.0) / 36.0, "azx": (s[2] + s[0] - 1.0) / 36.0,
            "axy": (s[0] + s[1] - 1.0) / 36.0,
            "byz": -(k[1] * k[2]) / 6.0, "bzx": -(k[2] * k[0]) / 6.0, "bxy": -(k[0] * k[1]) / 6.0,
        })
    if p.coef_f32:
        co = {n: float(np.float32(v)) for n, v in co.items()}
    return co


def wavevectors(p):
    """k_i d_i on the DFT grid of the problem, broadcastable to (nz, ny, nx)."""
    nx, ny, nz = p.n3
    kx = 2 * np.pi * np.fft.fftfreq(nx)[None, None, :]
    ky = 2 * np.pi * np.fft.fftfreq(ny)[None, :, None]
    kz = 2 * np.pi * np.fft.fftfreq(nz)[:, None, None]
    return kx, ky, kz


def symbols(p, kd=None):
    """Per-k symbols: returns (dbar[3], alpha[3], A[3][3]) as complex arrays.
    ``kd`` = (kx dx, ky dy, kz dz) arrays; default the problem's DFT grid."""
    co = coefficients(p)
    if kd is None:
        kd = wavevectors(p)
    active = [a < p.dims for a in range(3)]
    s = [np.sin(np.asarray(kd[a], dtype=float) / 2.0) if active[a] else np.zeros(1) for a in range(3)]
    db = [2j * s[a] for a in range(3)]
    dd = [-4.0 * s[a] ** 2 for a in range(3)]  # Dbar_aa
    al = [1.0 + co["c6"] * dd[a] for a in range(3)]
    ad = (co["ax"], co["ay"], co["az"])
    apair = {(1, 2): co["ayz"], (2, 0): co["azx"], (0, 1): co["axy"]}
    bpair = {(1, 2): co["byz"], (2, 0): co["bzx"], (0, 1): co["bxy"]}
    A = [[None] * 3 for _ in range(3)]
    for i in range(3):
        j, k = (i + 1) % 3, (i + 2) % 3
        A[i][i] = ad[j] * dd[j] + ad[k] * dd[k] + apair[(j, k)] * dd[j] * dd[k]
    for (i, j), b in bpair.items():
        k = 3 - i - j
        v = b * db[i] * db[j] * (1.0 + co["c6"] * dd[k])
        A[i][j] = v
        A[j][i] = v
    return db, al, A


def _to_phys(p, f, offs):
    kx, ky, kz = wavevectors(p)
    out = np.empty(f.shape, dtype=complex)
    for c in range(3):
        ph = np.exp(-1j * (kx * offs[c][0] + ky * offs[c][1] + kz * offs[c][2]))
        out[c] = np.fft.fftn(f[c]) * ph
    return out


def _from_phys(p, F, offs):
    kx, ky, kz = wavevectors(p)
    out = np.empty(F.shape, dtype=float)
    for c in range(3):
        ph = np.exp(1j * (kx * offs[c][0] + ky * offs[c][1] + kz * offs[c][2]))
        out[c] = np.fft.ifftn(F[c] * ph).real
    return out


def _matvec(M, v):
    return np.stack([sum(M[i][j] * v[j] for j in range(3)) for i in range(3)])


def _poly_sum(A, v, m):
    """sum_{s=0}^{m} A^s v (Algorithm 1 with m sweeps, unrolled)."""
    acc = v.copy()
    term = v.copy()
    for _ in range(m):
        term = _matvec(A, term)
        acc = acc + term
    return acc


def _solve3(A, v):
    """(1 - A)^{-1} v per k (the converged iteration)."""
    shp = np.broadcast(*[A[i][j] for i in range(3) for j in range(3)], v[0]).shape
    M = np.zeros(shp + (3, 3), dtype=complex)
    for i in range(3):
        for j in range(3):
            M[..., i, j] = (1.0 if i == j else 0.0) - np.broadcast_to(A[i][j], shp)
    rhs = np.stack([np.broadcast_to(v[i], shp) for i in range(3)], axis=-1)
    x = np.linalg.solve(M, rhs[..., None])[..., 0]
    return np.moveaxis(x, -1, 0)


def step(p, E, B, J=None, nsteps=1, exact=False):
    """Spectral twin of the stencil oracle's step (fixed m, or the exact
    inverse of (1 - A) when exact=True).  Filter target CURRENT only."""
    co = coefficients(p)
    db, al, A = symbols(p)
    Ef = _to_phys(p, np.asarray(E, float).reshape(p.array_shape), E_OFF)
    Bf = _to_phys(p, np.asarray(B, float).reshape(p.array_shape), B_OFF)
    if J is not None:
        Jf = _to_phys(p, np.asarray(J, float).reshape(p.array_shape), E_OFF)
        if p.filter_passes > 0:
            F = 1.0
            for a in range(p.dims):
                F = F * (1.0 + 0.25 * (db[a] ** 2)) ** p.filter_passes  # (1/2 + cos/2) per pass
            Jf = Jf * F
    kx, ky, kz = co["kx"], co["ky"], co["kz"]
    for _ in range(nsteps):
        SB = [al[0] * Bf[0], al[1] * Bf[1], al[2] * Bf[2]]
        dEp = np.stack([ky * db[1] * SB[2] - kz * db[2] * SB[1],
                        kz * db[2] * SB[0] - kx * db[0] * SB[2],
                        kx * db[0] * SB[1] - ky * db[1] * SB[0]])
        if J is not None:
            dEp = dEp - co["q"] * Jf
        dE = _solve3(A, dEp) if exact else _poly_sum(A, dEp, p.m)
        Ef = Ef + dE
        Bf = Bf - np.stack([ky * db[1] * Ef[2] - kz * db[2] * Ef[1],
                            kz * db[2] * Ef[0] - kx * db[0] * Ef[2],
                            kx * db[0] * Ef[1] - ky * db[1] * Ef[0]])
    return _from_phys(p, Ef, E_OFF), _from_phys(p, Bf, B_OFF)


def exact_inverse(p, dEp):
    """(1 - A)^{-1} dEp on the periodic grid, by a per-k 3x3 solve."""
    _, _, A = symbols(p)
    F = _to_phys(p, np.asarray(dEp, float).reshape(p.array_shape), E_OFF)
    return _from_phys(p, _solve3(A, F), E_OFF)


def a_interval(p, samples=33, widen=0.01):
    """Interval [lo, hi] holding the eigenvalues of A for the Chebyshev mode:
    the extreme eigenvalues of the real symmetric 3x3 symbol over s_i^2 =
    j / (samples - 1), j = 0 .. samples - 1, on every active axis (s_i =
    sin(k_i d_i / 2); the signs of the s_i do not change the eigenvalues),
    widened by widen * (1 - hi) at both ends."""
    g = np.linspace(0.0, 1.0, samples)
    axes = [g if a < p.dims else np.zeros(1) for a in range(3)]
    S = np.stack(np.meshgrid(*axes, indexing="ij"), -1).reshape(-1, 3)
    kd = tuple(2.0 * np.arcsin(np.sqrt(S[:, a])) for a in range(3))
    _, _, A = symbols(p, kd)
    n = S.shape[0]
    M = np.empty((n, 3, 3))
    for i in range(3):
        for j in range(3):
            M[:, i, j] = np.broadcast_to(np.real(np.asarray(A[i][j])), (n,))
    w = np.linalg.eigvalsh(M)
    lo, hi = float(w.min()), float(w.max())
    return lo - widen * (1.0 - hi), hi + widen * (1.0 - hi)


def chebyshev_error_poly(t, m, lo, hi):
    """Chebyshev semi-iteration's error polynomial P_m(t) = T_m((theta - t) /
    delta) / T_m(theta / delta) for M = 1 - A with spectrum in [1 - hi, 1 - lo]
    (theta, delta: centre and half-width); T_m evaluated as cos(m acos x) or
    cosh(m acosh |x|) sign(x)^m."""
    al, be = 1.0 - hi, 1.0 - lo
    theta, delta = 0.5 * (be + al), 0.5 * (be - al)

    def T(x):
        x = np.asarray(x, dtype=float)
        inside = np.abs(x) <= 1.0
        out = np.empty_like(x)
        out[inside] = np.cos(m * np.arccos(x[inside]))
        xo = x[~inside]
        out[~inside] = np.cosh(m * np.arccosh(np.abs(xo))) * np.sign(xo) ** m
        return out

    return T((theta - np.asarray(t, dtype=float)) / delta) / T(np.array([theta / delta]))[0]


def A_matrix(p, kd):
    """Real symmetric 3x3 symbol of A at one wavevector kd = (kx dx, ky dy, kz dz)."""
    _, _, A = symbols(p, tuple(np.array([v]) for v in kd))
    return np.array([[complex(np.ravel(A[i][j])[0]).real for j in range(3)] for i in range(3)])


def step_matrix(p, kd, exact=False):
    """6x6 one-step matrix T(k) acting on (E, B) in the physical basis."""
    co = coefficients(p)
    db, al, A = symbols(p, tuple(np.array([v]) for v in kd))
    db = [complex(np.ravel(x)[0]) for x in db]
    al = [complex(np.ravel(x)[0]) for x in al]
    Am = np.array([[complex(np.ravel(A[i][j])[0]) for j in range(3)] for i in range(3)])
    kk = (co["kx"], co["ky"], co["kz"])
    d = [kk[a] * db[a] for a in range(3)]  # c dt D_a
    K = np.array([[0, -d[2], d[1]], [d[2], 0, -d[0]], [-d[1], d[0], 0]], dtype=complex)  # curl
    G = K @ np.diag(al)
    P = np.linalg.inv(np.eye(3) - Am) if exact else sum(np.linalg.matrix_power(Am, s) for s in range(p.m + 1))
    T = np.zeros((6, 6), dtype=complex)
    T[:3, :3] = np.eye(3)
    T[:3, 3:] = P @ G
    T[3:, :3] = -K
    T[3:, 3:] = np.eye(3) - K @ P @ G
    return T


# ---------------------------------------------------------------------------
# closed forms
# ---------------------------------------------------------------------------

def G(theta):
    """Eq. G: G(theta) = sin^2 theta / (1 - (2/3) sin^2 theta)."""
    s2 = np.sin(theta) ** 2
    return s2 / (1.0 - 2.0 / 3.0 * s2)


def omega_converged(p, kvec):
    """omega from Eq. dispersion-em-F-3d (2D: Eq. dispersion-em-F-2d):
    G(omega dt/2)/(c dt)^2 = sum_i G(k_i d_i/2)/d_i^2, solved for omega."""
    dt = p.time_step()
    R = 0.0
    for a in range(p.dims):
        R = R + G(kvec[a] * p.d[a] / 2.0) / p.d[a] ** 2
    R = R * (p.c * dt) ** 2
    s2 = R / (1.0 + 2.0 / 3.0 * R)  # invert G: sin^2 = G/(1 + 2G/3)
    return 2.0 * np.arcsin(np.sqrt(s2)) / dt


def omega_yee(p, kvec):
    """Textbook Yee dispersion: sin^2(omega dt/2) = (c dt)^2 sum sin^2(k_i d_i/2)/d_i^2."""
    dt = p.time_step()
    s2 = 0.0
    for a in range(p.dims):
        s2 = s2 + np.sin(kvec[a] * p.d[a] / 2.0) ** 2 / p.d[a] ** 2
    s2 = s2 * (p.c * dt) ** 2
    return 2.0 * np.arcsin(np.sqrt(s2)) / dt


def lambda_tm(p, kvec):
    """A_zz symbol in 2D (Eq. matrixA_1st_2d block for E_z)."""
    dt = p.time_step()
    sx2 = np.sin(kvec[0] * p.d[0] / 2.0) ** 2
    sy2 = np.sin(kvec[1] * p.d[1] / 2.0) ** 2
    sgx = (p.c * dt / p.d[0]) ** 2
    sgy = (p.c * dt / p.d[1]) ** 2
    return (2.0 / 3.0) * (1 - sgx) * sx2 + (2.0 / 3.0) * (1 - sgy) * sy2 - (4.0 / 9.0) * (1 - sgx - sgy) * sx2 * sy2


def omega_fixed_m_tm(p, kvec, m):
    """2D TM mode after m sweeps.  Reading of App. D: from Eq.
    derive_convergence_3 the truncated solve multiplies the converged
    increment by (1 - lambda^{m+1}), so sin^2(omega_m dt/2)
    = (1 - lambda^{m+1}) sin^2(omega_inf dt/2) (the printed Eq. 9 has the
    factor on the other side; both agree to first order in lambda^{m+1})."""
    dt = p.time_step()
    w = omega_converged(p, kvec)
    lam = lambda_tm(p, kvec)
    s2 = (1.0 - lam ** (m + 1)) * np.sin(w * dt / 2.0) ** 2
    return 2.0 * np.arcsin(np.sqrt(s2)) / dt


def phase_speed_expansion(p, kvec):
    """Eq. phase-speed-3d / phase-speed-2d: omega/k ~ c [1 + (1/24)
    (sum k_i^4 d_i^2 / k^2 - k^2 c^2 dt^2)]."""
    dt = p.time_step()
    k2 = sum(kvec[a] ** 2 for a in range(p.dims))
    q4 = sum(kvec[a] ** 4 * p.d[a] ** 2 for a in range(p.dims))
    return p.c * (1.0 + (q4 / k2 - k2 * p.c ** 2 * dt ** 2) / 24.0)
