"""Oracle pins of the Chebyshev-accelerated solve (the next-row iteration mode:
Chebyshev semi-iteration for (1 - A) dE = dE' on the spectral interval of A).

The result of m sweeps is pinned, wavevector by wavevector, against the
closed-form Chebyshev error polynomial applied to the exact inverse's error:
x_m = x* + P_m(M)(dE' - x*), M = 1 - A, x* = M^{-1} dE', evaluated with the
per-k symbol of A (a second derivation, spectral.py) and an eigendecomposition.
Residual mode must land on the exact inverse, in fewer sweeps than Algorithm 1.
"""
import numpy as np
import pytest

from oracle import core, spectral
from paper_1907_13088_gb300 import synth
from tests.helpers import rel_l2

E_OFF = spectral.E_OFF


def _per_k_expected(p, b, m):
    """x* + P_m(M)(b - x*) per wavevector, back in real space."""
    _, _, A = spectral.symbols(p)
    B = spectral._to_phys(p, b, E_OFF)
    shp = B.shape[1:]
    Mk = np.zeros(shp + (3, 3))
    for i in range(3):
        for j in range(3):
            Mk[..., i, j] = (1.0 if i == j else 0.0) - np.broadcast_to(np.real(A[i][j]), shp)
    lo, hi = spectral.a_interval(p)
    w, V = np.linalg.eigh(Mk)
    # x* = V diag(1/w) V^T b;  x_m = x* + V diag(P_m(w)) V^T (b - x*) = V diag(1/w + P_m(w)(1 - 1/w)) V^T b
    Pm = spectral.chebyshev_error_poly(w.ravel(), m, lo, hi).reshape(w.shape)
    g = 1.0 / w + Pm * (1.0 - 1.0 / w)
    bk = np.moveaxis(B, 0, -1)[..., None]
    xk = V @ (g[..., None] * (np.swapaxes(V, -1, -2) @ bk))
    return spectral._from_phys(p, np.moveaxis(xk[..., 0], -1, 0), E_OFF)


@pytest.mark.parametrize("shape,courant", [((16, 12), 0.5), ((16, 12), 0.95), ((8, 6, 5), 0.6), ((24,), 0.9)])
@pytest.mark.parametrize("m", [1, 2, 5, 9])
def test_chebyshev_matches_error_polynomial_per_k(shape, courant, m):
    p = core.Params(shape=shape, courant=courant, m=m, cheb=True)
    b = synth.random_fields(shape, seed=70 + m)[0]
    x, rc, sweeps, _ = core.solve(p, b)
    assert rc == 0
    assert sweeps == m
    ref = _per_k_expected(p, b, m)
    assert rel_l2(x, ref) < 1e-12, rel_l2(x, ref)


@pytest.mark.parametrize("shape,courant", [((32, 32), 0.5), ((10, 8, 6), 0.5), ((32, 32), 0.99)])
def test_chebyshev_residual_reaches_exact_inverse_faster(shape, courant):
    b = synth.random_fields(shape, seed=80)[0]
    pc = core.Params(shape=shape, courant=courant, residual=True, tol=1e-13, cheb=True)
    pj = core.Params(shape=shape, courant=courant, residual=True, tol=1e-13)
    xc, rc, nc, _ = core.solve(pc, b)
    assert rc == 0
    xj, rcj, nj, _ = core.solve(pj, b)
    exact = spectral.exact_inverse(pc, b)
    assert rel_l2(xc, exact) < 1e-11 and rel_l2(xj, exact) < 1e-11
    # rate: ((sqrt(kappa) - 1) / (sqrt(kappa) + 1)) per sweep against lambda_max for Algorithm 1
    lo, hi = spectral.a_interval(pc)
    kappa = (1.0 - lo) / (1.0 - hi)
    q = (np.sqrt(kappa) - 1.0) / (np.sqrt(kappa) + 1.0)
    assert nc <= int(np.ceil(np.log(2.0 / 1e-13) / np.log(1.0 / q))) + 2
    assert nc < 0.6 * nj, (nc, nj)


def test_interval_holds_the_grid_spectrum():
    """The sampled, widened interval contains every eigenvalue of A on a grid."""
    for shape, cf in (((32, 32), 0.5), ((12, 10, 8), 0.7), ((64,), 0.3)):
        p = core.Params(shape=shape, courant=cf)
        lo, hi = spectral.a_interval(p)
        _, _, A = spectral.symbols(p)
        shp = np.broadcast(*[np.asarray(A[i][j]) for i in range(3) for j in range(3)]).shape
        M = np.zeros(shp + (3, 3))
        for i in range(3):
            for j in range(3):
                M[..., i, j] = np.broadcast_to(np.real(A[i][j]), shp)
        w = np.linalg.eigvalsh(M)
        assert w.min() >= lo and w.max() <= hi and hi < 1.0


@pytest.mark.parametrize("shape,courant,d", [((64, 64), 0.5, (1.0, 1.0, 1.0)), ((16, 16, 16), 0.5, (1.0, 1.0, 1.0)),
                                             ((40,), 0.9, (1.0, 1.0, 1.0)), ((20, 12, 8), 0.7, (1.0, 0.8, 1.2))])
def test_library_interval_matches_oracle(shape, courant, d):
    """fmx_cheb_interval (the library's own sampling and eigenvalues, host
    code: no GPU needed) against the oracle's interval."""
    import ctypes
    from paper_1907_13088_gb300 import fmx
    p = fmx.make_params(shape, courant=courant, d=d, iter_mode=fmx.FMX_ITER_CHEB_FIXED, precision=fmx.FMX_F64)
    h = ctypes.c_void_p()
    fmx.check(fmx.fmx_create(ctypes.byref(p), ctypes.byref(h), None), "fmx_create")
    try:
        lo, hi = ctypes.c_double(), ctypes.c_double()
        fmx.check(fmx.fmx_cheb_interval(h, ctypes.byref(lo), ctypes.byref(hi)), "fmx_cheb_interval")
    finally:
        fmx.fmx_destroy(h)
    olo, ohi = spectral.a_interval(core.Params(shape=shape, courant=courant, d=d))
    assert abs(lo.value - olo) < 1e-13 and abs(hi.value - ohi) < 1e-13


CHEB_MUTATIONS = {
    "rho_recurrence": ("const double rho_new = 1.0 / (2.0 * sig - rho);",
                       "const double rho_new = 1.0 / (sig - rho);"),
    "first_step_scale": ("c2 = 1.0 / theta;", "c2 = 1.0 / delta;"),
    "momentum_weight": ("c1 = rho_new * rho;", "c1 = rho_new;"),
    "step_weight": ("c2 = 2.0 * rho_new / delta;", "c2 = rho_new / delta;"),
    # the interval of A taken for that of M = 1 - A (swapping the interval's
    # ends is no mistake: delta and every rho change sign together and the
    # recurrence's coefficients stay the same)
    "interval_of_A": ("const double al = 1.0 - p->cheb_hi, be = 1.0 - p->cheb_lo;",
                      "const double al = p->cheb_lo, be = p->cheb_hi;"),
}


@pytest.mark.parametrize("name", sorted(CHEB_MUTATIONS))
def test_chebyshev_planted_mistake_is_caught(name, tmp_path):
    """A plausible mistake in the C recurrence must break the per-wavevector
    error-polynomial pin (the mutated copy is compiled to a temporary
    directory; the oracle under test is not touched)."""
    old, new = CHEB_MUTATIONS[name]
    src = core.source_text()
    assert src.count(old) == 1, name
    lib = core.compile_variant(src.replace(old, new), str(tmp_path / "libmut.so"))
    caught = False
    with core.using_library(lib):
        for shape, courant in (((16, 12), 0.5), ((8, 6, 5), 0.6)):
            for m in (2, 5):
                p = core.Params(shape=shape, courant=courant, m=m, cheb=True)
                b = synth.random_fields(shape, seed=70 + m)[0]
                x, rc, sweeps, _ = core.solve(p, b)
                if rc != 0 or not np.all(np.isfinite(x)) or rel_l2(x, _per_k_expected(p, b, m)) >= 1e-12:
                    caught = True
    assert caught, f"mutation {name} passed the error-polynomial pin"
