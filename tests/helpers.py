"""Shared test helpers: run the CUDA path through the C ABI and the oracle on
the same seeded inputs, and compare per field component."""
import numpy as np

COMP = ("Ex", "Ey", "Ez", "Bx", "By", "Bz")


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b.ravel())
    if nb == 0.0:
        return float(np.max(np.abs(a))) if a.size else 0.0
    return float(np.linalg.norm((a - b).ravel()) / nb)


def per_component(E_gpu, B_gpu, E_ref, B_ref):
    out = {}
    for c in range(3):
        out[COMP[c]] = rel_l2(E_gpu[c], E_ref[c])
        out[COMP[3 + c]] = rel_l2(B_gpu[c], B_ref[c])
    return out


def assert_parity(E_gpu, B_gpu, E_ref, B_ref, tol, what=""):
    errs = per_component(E_gpu, B_gpu, E_ref, B_ref)
    bad = {k: v for k, v in errs.items() if not v <= tol}
    assert not bad, f"{what}: relative L2 above {tol}: {bad} (all: {errs})"
    return errs


def oracle_params(shape, **kw):
    from oracle import core
    return core.Params(shape=tuple(shape), **kw)


def periodic_window(a, center, size):
    """(3, 1, ny, nx) -> (3, 1, size, size) periodic window whose cell
    (size//2, size//2) is `center` = (j, i)."""
    j0 = center[0] - size // 2
    i0 = center[1] - size // 2
    ny, nx = a.shape[-2:]
    rows = np.arange(j0, j0 + size) % ny
    cols = np.arange(i0, i0 + size) % nx
    return a[..., rows[:, None], cols[None, :]]
