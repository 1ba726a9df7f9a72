"""GPU NCI tools (fmx_nci_resonance, Sec. 3 and App. E) against the oracle.

The kernel solves Eq. reson1 for k_y in closed form (inverting G) and
evaluates the paper's final Eq. NCI-growth-rate; the oracle bisects Eq.
reson1 and follows the steps of App. E.  Both in FP64.  Tolerances: k_y and
Gamma to 1e-12 in relative L2 over the crossings of each alias (the bar of
the FP64 step); pointwise, k_y to 1e-12 / dy absolute and Gamma at the GPU's
crossing to 1e-10 relative (Gamma passes through zeros of its numerator,
where a relative error of a few ulp of the terms is amplified).  The crossing
masks must agree except where the oracle's resonance function at an end of
[0, pi/dy] is within 1e-12 of zero (a tangency the two orders of rounding may
place on either side)."""
import math

import numpy as np
import pytest

from oracle import nci

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fmx():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1907_13088_gb300 import build
    build.build()
    from paper_1907_13088_gb300 import fmx as m
    return m


def _rel_l2(a, b):
    n = np.linalg.norm(b)
    return np.linalg.norm(a - b) / n if n > 0 else np.linalg.norm(a - b)


CASES = [
    dict(dx=1.0, dy=1.0, c=1.0, courant=0.5, omega_p=1 / 16, shape_order=1, nu_max=1, nkx=4096),
    dict(dx=1.0, dy=1.0, c=1.0, courant=0.9, omega_p=1 / 16, shape_order=2, nu_max=2, nkx=4097),
    dict(dx=1.0, dy=1.0, c=1.0, courant=1.0, omega_p=1 / 16, shape_order=4, nu_max=1, nkx=1025),
    dict(dx=1.0, dy=0.7, c=1.0, courant=0.72, omega_p=0.2, shape_order=1, nu_max=2, nkx=3001),
    dict(dx=0.5, dy=1.3, c=2.0, courant=0.1, omega_p=0.05, shape_order=0, nu_max=3, nkx=2048),
    dict(dx=1.0, dy=1.0, c=1.0, courant=0.3, omega_p=1 / 16, shape_order=1, nu_max=0, nkx=512),  # no crossing
    dict(dx=1.0, dy=1.0, c=1.0, courant=0.8, omega_p=1 / 16, shape_order=1, nu_max=1, nkx=1),
    dict(dx=1.0, dy=1.0, c=1.0, courant=0.8, omega_p=1 / 16, shape_order=1, nu_max=1, nkx=7),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"dy{c['dy']}-C{c['courant']}-l{c['shape_order']}-nu{c['nu_max']}-n{c['nkx']}")
def test_nci_resonance_matches_oracle(fmx, case):
    g = fmx.nci_resonance(**case)
    r = nci.resonance(case["nkx"], case["courant"], case["dx"], case["dy"], case["omega_p"], case["shape_order"],
                      nu_max=case["nu_max"], c=case["c"])
    kx = g["kx"].cpu().numpy()
    assert np.array_equal(kx, r["kx"])
    ky, gam = g["ky"].cpu().numpy(), g["gamma"].cpu().numpy()
    dx, dy, dt = case["dx"], case["dy"], r["dt"]
    for row, nu in enumerate(r["nus"]):
        mg, mo = ~np.isnan(ky[row]), ~np.isnan(r["ky"][row])
        diff = np.nonzero(mg != mo)[0]
        if len(diff):
            f0 = nci.resonance_function(kx[diff], np.zeros(len(diff)), nu, dx, dy, dt, case["c"])
            f1 = nci.resonance_function(kx[diff], np.full(len(diff), math.pi / dy), nu, dx, dy, dt, case["c"])
            assert np.all(np.minimum(np.abs(f0), np.abs(f1)) < 1e-12), (nu, diff)
        assert np.all(gam[row][~mg] == 0.0)
        both = mg & mo
        if not both.any():
            continue
        assert _rel_l2(ky[row, both], r["ky"][row, both]) <= 1e-12
        assert np.max(np.abs(ky[row, both] - r["ky"][row, both])) <= 1e-12 / dy
        assert _rel_l2(gam[row, both], r["gamma"][row, both]) <= 1e-12
        at_gpu = nci.growth_rate(kx[both], ky[row, both], nu, dx, dy, dt, case["omega_p"], case["shape_order"],
                                 case["c"])
        assert np.all(np.abs(gam[row, both] - at_gpu) <= 1e-10 * at_gpu), nu
    gmax, bkx, bky, bnu = g["best"]
    omax = r["best"][0]
    if omax == 0.0:
        assert gmax == 0.0 and all(math.isnan(v) for v in (bkx, bky, bnu))
        return
    assert abs(gmax - omax) <= 1e-12 * omax
    # the GPU's argmax is a crossing whose oracle growth rate is the maximum (ties may pick either mirror)
    row = int(bnu) + case["nu_max"]
    i = int(np.argmin(np.abs(kx - bkx)))
    assert kx[i] == bkx and ky[row, i] == bky and gam[row, i] == gmax
    at = nci.growth_rate(np.array([bkx]), np.array([bky]), int(bnu), dx, dy, dt, case["omega_p"],
                         case["shape_order"], case["c"])[0]
    assert at >= omax * (1 - 1e-12)
    assert i + row * case["nkx"] == int(np.argmax(gam))  # lowest flat index among equal maxima


def test_nci_sec42_statements_on_gpu(fmx):
    """Sec. 4.2 through the GPU tool: nu = 0 only above dt_CFL / sqrt 2, no
    |nu| = 2 crossing, |k_x| > 2.06 / dx, and a fastest mode that a higher
    particle-shape order slows."""
    lows, peaks = [], {}
    for courant in (0.001, 0.3, 0.7, 0.75, 1.0):
        out = fmx.nci_resonance(courant=courant, nu_max=2, nkx=8192, shape_order=1)
        ky = out["ky"].cpu().numpy()
        kx = out["kx"].cpu().numpy()
        assert np.all(np.isnan(ky[0])) and np.all(np.isnan(ky[4]))
        assert np.isnan(ky[2]).all() == (courant < 1 / math.sqrt(2))
        lows.append(np.abs(np.broadcast_to(kx, ky.shape)[~np.isnan(ky)]).min())
        peaks[courant] = [fmx.nci_resonance(courant=courant, nkx=8192, shape_order=l)["best"][0] for l in (1, 2, 4)]
    assert min(lows) >= 2.06 and lows[0] < 2.07
    for courant, p in peaks.items():
        assert p[0] > p[1] > p[2] > 0, (courant, p)
