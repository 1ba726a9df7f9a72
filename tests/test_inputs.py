"""The seeded synthetic inputs follow the recipes they are documented with
(mode support, normalisation, divergence, draw ranges); no GPU needed."""
import math

import numpy as np

from paper_1907_13088_gb300 import synth


def _mode_norm_2d(nx, ny):
    mx = np.fft.fftfreq(nx, 1.0 / nx)[None, :]
    my = np.fft.fftfreq(ny, 1.0 / ny)[:, None]
    return np.sqrt(mx * mx + my * my)


def test_power_law_fields_support_rms_and_slope():
    nx, ny, kmax = 256, 192, 24
    E, B = synth.power_law_fields((nx, ny), kmax, seed=1, dtype=np.float64)
    nrm = _mode_norm_2d(nx, ny)
    outside = (nrm < 1.0) | (nrm > kmax)
    shells = np.arange(2, kmax + 1)
    for F in (E, B):
        assert abs(math.sqrt(np.mean(F * F)) - 1.0) < 1e-12  # unit RMS over the three components
        for f in F:
            f = f[0]
            P = np.abs(np.fft.fft2(f)) ** 2
            assert P[outside].max() < 1e-10 * P.max()  # only 1 <= |n| <= k_max
            # shell-averaged power falls as |n|^-2 (random phases: on average)
            mean = np.array([P[(nrm >= r - 0.5) & (nrm < r + 0.5)].mean() for r in shells])
            slope = np.polyfit(np.log(shells), np.log(mean), 1)[0]
            assert abs(slope + 2.0) < 0.25, slope


def _fwd_div(B, d):
    """Forward-difference divergence on the periodic grid (arrays (3, nz, ny, nx))."""
    div = np.zeros(B.shape[1:])
    for a, axis in ((0, 2), (1, 1), (2, 0)):
        if B.shape[1 + axis] > 1:
            div += (np.roll(B[a], -1, axis=axis) - B[a]) / d[a]
    return div


def test_power_law_fields_are_divergence_free():
    """E = C^T psi_E has zero backward divergence, B = C psi_B zero forward
    divergence (the divergence of the Faraday update), to round-off."""
    for shape, d in (((64, 48), (1.0, 1.0, 1.0)), ((16, 12, 10), (1.0, 0.8, 1.2))):
        E, B = synth.power_law_fields(shape, 6, seed=3, dtype=np.float64, d=d)
        assert np.abs(_back_div(E, d)).max() < 1e-12 * np.abs(E).max()
        assert np.abs(_fwd_div(B, d)).max() < 1e-12 * np.abs(B).max()


def _back_div(J, d):
    """Backward-difference divergence on the periodic grid (arrays (3, nz, ny, nx))."""
    div = np.zeros(J.shape[1:])
    for a, axis in ((0, 2), (1, 1), (2, 0)):
        if J.shape[1 + axis] > 1:
            div += (J[a] - np.roll(J[a], 1, axis=axis)) / d[a]
    return div


def test_solenoidal_current_is_divergence_free_with_the_stated_rms():
    for shape, d in (((64, 48), (1.0, 1.0, 1.0)), ((16, 12, 10), (1.0, 0.8, 1.2))):
        J = synth.solenoidal_current(shape, seed=3, width=2.0, rms=1e-2, dtype=np.float64, d=d)
        assert abs(math.sqrt(np.mean(J * J)) - 1e-2) < 1e-15
        div = _back_div(J, d)
        assert np.max(np.abs(div)) < 1e-13 * np.max(np.abs(J)), np.max(np.abs(div))


def test_tm_plane_waves_modes_and_polarisation():
    n, dt = 64, 0.5 / math.sqrt(2.0)
    E, B, modes = synth.tm_plane_waves((n, n), dt, seed=1907001)
    assert len(modes) == 8
    vecs = [(mx, my) for mx, my, _, _ in modes]
    assert len(set(vecs)) == 8
    for mx, my in vecs:
        assert 1 <= mx * mx + my * my <= 64
        assert (-mx, -my) not in vecs  # never a mode and its negative
    assert np.all(E[:2] == 0) and np.all(B[2] == 0)  # E_z, B_x, B_y only
    Ez, Bx, By = (np.fft.fft2(f[0]) for f in (E[2], B[0], B[1]))
    support = np.zeros((n, n), dtype=bool)
    for mx, my in vecs:
        support[my % n, mx % n] = support[-my % n, -mx % n] = True
    assert np.abs(Ez[~support]).max() < 1e-9 * np.abs(Ez).max()
    for mx, my, a, _ in modes:
        kx, ky = 2 * math.pi * mx / n, 2 * math.pi * my / n
        k = math.hypot(kx, ky)
        ez, bx, by = Ez[my % n, mx % n], Bx[my % n, mx % n], By[my % n, mx % n]
        # B = k_hat x E: staggering and the half step shift phases only
        assert abs(abs(ez) - abs(a) * n * n / 2) < 1e-9 * n * n
        assert abs(abs(bx) - abs(ky) / k * abs(ez)) < 1e-9 * abs(ez)
        assert abs(abs(by) - abs(kx) / k * abs(ez)) < 1e-9 * abs(ez)


def test_batch_sizes_and_sources_draw_ranges():
    sizes = synth.batch_sizes(256, 1907004)
    assert len(sizes) == 256
    sides = np.array([s[:2] for s in sizes])
    cf = np.array([s[2] for s in sizes])
    assert sides.min() >= 64 and sides.max() <= 1024
    assert cf.min() >= 0.3 and cf.max() <= 0.9
    # log-uniform per side: the median side near sqrt(64 * 1024) = 256
    assert 200 < np.median(sides) < 330
    assert synth.batch_sizes(256, 1907004) == sizes  # seeded
    cxy, phases, theta = synth.gauss_sources(64, (1024, 1024), 1907005)
    assert cxy.shape == (64, 2) and np.all((cxy >= 0) & (cxy < 1024))
    assert np.all((phases >= 0) & (phases < 2 * math.pi))
    assert theta.shape == (64,) and abs(theta.mean()) < 0.5
