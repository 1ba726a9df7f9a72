"""Pins of the oracle's adjoint step against its forward step: the
dot-product identity <T d, y> = <d, T^T y> (T the linear step acting on
(E, B, j)) to round-off, and central finite differences of a quadratic loss
through several steps."""
import numpy as np
import pytest

from oracle import core
from paper_1907_13088_gb300 import synth


@pytest.mark.parametrize("d", [(1.0, 1.0, 1.0), (1.0, 0.8, 1.2)])
@pytest.mark.parametrize("shape,m,passes", [((16, 12), 4, 3), ((9, 7), 2, 1), ((6, 5, 4), 3, 1), ((20,), 4, 0)])
def test_dot_product_identity(shape, m, passes, d):
    p = core.Params(shape=shape, courant=0.7, m=m, filter_passes=passes, d=d)
    dE, dB, dJ = synth.random_fields(shape, seed=31)
    yE, yB, _ = synth.random_fields(shape, seed=32)
    E1, B1, _, _ = core.step(p, dE, dB, dJ, 1)
    lhs = np.sum(E1 * yE) + np.sum(B1 * yB)
    Eb, Bb, jb = core.adjoint_step(p, yE, yB)
    rhs = np.sum(dE * Eb) + np.sum(dB * Bb) + np.sum(dJ * jb)
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), 1.0)


def test_finite_differences_through_steps():
    """L = 1/2 |window of E^N, B^N|^2 with j = theta * G; dL/dtheta from
    N adjoint steps against central differences."""
    shape, N = (24, 20), 6
    p = core.Params(shape=shape, courant=0.5, m=4, filter_passes=2)
    E0, B0, _ = synth.random_fields(shape, seed=33)
    G = np.zeros(p.array_shape)
    G[2] = synth.random_fields(shape, seed=34)[0][0]
    mask = np.zeros(p.array_shape)
    mask[:, :, 5:15, 4:12] = 1.0

    def loss(theta):
        E, B, _, _ = core.step(p, E0, B0, theta * G, N)
        return 0.5 * np.sum((E * mask) ** 2) + 0.5 * np.sum((B * mask) ** 2)

    theta = 0.7
    E, B, _, _ = core.step(p, E0, B0, theta * G, N)
    Eb, Bb = E * mask, B * mask
    grad = 0.0
    for _ in range(N):
        Eb, Bb, jb = core.adjoint_step(p, Eb, Bb)
        grad += np.sum(jb * G)
    eps = 1e-3
    fd = (loss(theta + eps) - loss(theta - eps)) / (2 * eps)
    assert abs(grad - fd) <= 1e-8 * max(abs(fd), 1.0)  # loss is quadratic: FD exact up to round-off


ADJ_MUTATIONS = {
    "curl_sign": ("for (long c = 0; c < n3; ++c) u[c] = Ebar[c] - u[c];",
                  "for (long c = 0; c < n3; ++c) u[c] = Ebar[c] + u[c];"),
    "z_difference_direction": ("dbar(&s, Bx, d, 2, 0); axpy(&s, co[ORC_KZ], d, u + n);",
                               "dbar(&s, Bx, d, 2, 1); axpy(&s, co[ORC_KZ], d, u + n);"),
    "alpha_axis": ("alpha(&s, co[ORC_C6], ta, sa, tmp, a);", "alpha(&s, co[ORC_C6], ta, sa, tmp, (a + 1) % 3);"),
    "e_passes_solved_value": ("memcpy(Ebar, u, sizeof(double) * n3);", "memcpy(Ebar, w, sizeof(double) * n3);"),
    "current_unfiltered": ("if (p->filter_target == ORC_FILTER_CURRENT && p->filter_passes > 0) orc_filter(p, jbar, 3, "
                           "p->filter_passes);",
                           "if (0) orc_filter(p, jbar, 3, p->filter_passes);"),
}


@pytest.mark.parametrize("name", sorted(ADJ_MUTATIONS))
def test_adjoint_planted_mistake_is_caught(name, tmp_path):
    """A plausible mistake in the C adjoint step (the forward step untouched)
    must break the dot-product identity; the mutated copy is compiled to a
    temporary directory."""
    old, new = ADJ_MUTATIONS[name]
    src = core.source_text()
    assert src.count(old) == 1, name
    lib = core.compile_variant(src.replace(old, new), str(tmp_path / "libmut.so"))
    with core.using_library(lib):
        for shape, m, passes in (((16, 12), 4, 3), ((6, 5, 4), 3, 1)):
            p = core.Params(shape=shape, courant=0.7, m=m, filter_passes=passes, d=(1.0, 0.8, 1.2))
            dE, dB, dJ = synth.random_fields(shape, seed=31)
            yE, yB, _ = synth.random_fields(shape, seed=32)
            E1, B1, _, _ = core.step(p, dE, dB, dJ, 1)
            lhs = np.sum(E1 * yE) + np.sum(B1 * yB)
            Eb, Bb, jb = core.adjoint_step(p, yE, yB)
            rhs = np.sum(dE * Eb) + np.sum(dB * Bb) + np.sum(dJ * jb)
            if abs(lhs - rhs) > 1e-12 * max(abs(lhs), 1.0):
                return
    pytest.fail(f"mutation {name} kept the dot-product identity")
