"""NCI tools of Sec. 3 and App. E on the GPU (fmx_nci_resonance).

For the drifting pair plasma of Sec. 4.2 (v -> c along x, dx = dy, omega_p
dx / c = 1/16: L_x = 16 d_e over 256 cells) and dt / dt_CFL = 0.1 .. 1.0, the
resonance curves of Eqs. reson1/reson2 give the smallest |k_x| reached by
each alias nu, and Eq. NCI-growth-rate along them the fastest-growing mode
for B-spline particle shapes of order 1, 2 and 4.

    python -m paper_1907_13088_gb300.nci [--nkx 8192] [--omega-p 0.0625]
"""
from __future__ import annotations

import argparse

import numpy as np

from . import fmx


def scan(courants, omega_p=1.0 / 16.0, orders=(1, 2, 4), nkx=8192, nu_max=1, dx=1.0, dy=1.0, c=1.0):
    """Per dt / dt_CFL: min |k_x| of each alias's curve (None if it has no
    crossing) and (Gamma_max, k_x, k_y, nu) of the fastest mode per shape order."""
    rows = []
    for courant in courants:
        out = {"courant": float(courant), "min_kx": {}, "best": {}}
        for l in orders:
            r = fmx.nci_resonance(dx=dx, dy=dy, c=c, courant=courant, omega_p=omega_p, shape_order=l,
                                  nu_max=nu_max, nkx=nkx)
            out["best"][l] = r["best"]
            if not out["min_kx"]:
                ky = r["ky"].cpu().numpy()
                kx = np.abs(r["kx"].cpu().numpy())
                for j, nu in enumerate(r["nus"]):
                    ok = ~np.isnan(ky[j])
                    out["min_kx"][nu] = float(kx[ok].min()) if ok.any() else None
        rows.append(out)
    return rows


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--nkx", type=int, default=8192)
    ap.add_argument("--omega-p", type=float, default=1.0 / 16.0)
    a = ap.parse_args(argv)
    rows = scan(np.round(np.arange(1, 11) * 0.1, 10), a.omega_p, nkx=a.nkx)
    print("dt/dt_CFL  min|kx| nu=0   nu=+-1    Gamma_max/omega_p (l=1, 2, 4)   fastest (kx, ky, nu) for l=1")
    for r in rows:
        m0, m1 = r["min_kx"].get(0), r["min_kx"].get(1)
        g = [r["best"][l][0] / a.omega_p for l in (1, 2, 4)]
        b = r["best"][1]
        print(f"  {r['courant']:4.1f}     {'   -   ' if m0 is None else f'{m0:7.4f}'}   "
              f"{'   -   ' if m1 is None else f'{m1:7.4f}'}   {g[0]:8.4f} {g[1]:8.4f} {g[2]:8.4f}      "
              f"({b[1]:.4f}, {b[2]:.4f}, {int(b[3]):+d})")


if __name__ == "__main__":
    main()
