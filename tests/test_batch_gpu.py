"""Batched step (many independent 2D grids, one persistent launch per step
and kind of tile, graph-replayed) against the FP64 oracle per grid and
against the single-grid path; the tile row extent picked by the autotuner
must not change any result.  The grids (odd and even n_x) run on the
column-pair TE/TM tiles."""
import numpy as np
import pytest

from oracle import core
from paper_1907_13088_gb300 import synth
from tests.helpers import assert_parity, rel_l2

pytestmark = pytest.mark.gpu
TOL32 = 1e-5


@pytest.fixture(scope="module")
def fmx():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1907_13088_gb300 import build
    build.build()
    from paper_1907_13088_gb300 import fmx as m
    return m


SHAPES = [(64, 64), (65, 97), (300, 71), (128, 257), (37, 512), (1024, 40), (255, 255), (96, 33)]
COURANT = [0.3, 0.9, 0.5, 0.75, 0.42, 0.61, 0.88, 0.33]


def _fields(shape, seed):
    kmax = max(2, min(shape) // 8)
    return synth.power_law_fields(shape, kmax, seed, dtype=np.float32)


@pytest.mark.parametrize("nsteps", [1, 6, 9])
def test_batch_matches_oracle_and_single_grid(fmx, nsteps):
    b = fmx.Batch(SHAPES, COURANT, m=4)
    inputs = [_fields(sh, 1907040 + i) for i, sh in enumerate(SHAPES)]
    for i, (E, B) in enumerate(inputs):
        b.set_fields(i, E, B)
    b.step(nsteps)
    for i, (sh, cf) in enumerate(zip(SHAPES, COURANT)):
        Eg, Bg = b.get_fields(i)
        E, B = inputs[i]
        Eo, Bo, rc, _ = core.step(core.Params(shape=sh, courant=cf, m=4, coef_f32=True), E.astype(np.float64),
                                  B.astype(np.float64), None, nsteps)
        assert_parity(Eg, Bg, Eo, Bo, TOL32, f"batch grid {i} {sh}")
        g = fmx.Grid(sh, with_current=False, precision=0, m=4, courant=cf, engine=fmx.FMX_ENGINE_FUSED)
        g.set_fields(E, B)
        g.step(nsteps)
        Es, Bs, _ = g.get_fields()
        assert rel_l2(Eg, Es) < TOL32 and rel_l2(Bg, Bs) < TOL32
    assert b.launches == nsteps


@pytest.mark.parametrize("m", [0, 1, 2, 4])
def test_batch_column_pair_tiles_every_m(fmx, m):
    """One launch per step on the column-pair tiles, every instantiated m,
    grids from 1 to 1024 columns, odd and even (one tile narrower than a
    strip, several strips, seam strips of odd n_x, rows below the warm-up
    depth)."""
    shapes = [(64, 64), (300, 71), (128, 257), (1024, 40), (97, 33), (1, 5), (259, 3), (511, 512)]
    cfs = [0.3, 0.5, 0.75, 0.61, 0.33, 0.9, 0.45, 0.8]
    b = fmx.Batch(shapes, cfs, m=m)
    inputs = [_fields(sh, 1907140 + i) for i, sh in enumerate(shapes)]
    for i, (E, B) in enumerate(inputs):
        b.set_fields(i, E, B)
    nsteps = 5
    b.step(nsteps)
    for i, (sh, cf) in enumerate(zip(shapes, cfs)):
        Eg, Bg = b.get_fields(i)
        E, B = inputs[i]
        Eo, Bo, rc, _ = core.step(core.Params(shape=sh, courant=cf, m=m, coef_f32=True), E.astype(np.float64),
                                  B.astype(np.float64), None, nsteps)
        assert_parity(Eg, Bg, Eo, Bo, TOL32, f"pair batch m={m} grid {i} {sh}")
    assert b.launches == nsteps


def test_batch_tile_rows_do_not_change_results(fmx):
    inputs = [_fields(sh, 1907060 + i) for i, sh in enumerate(SHAPES)]
    results = []
    for rows in (0, 32, 100, 4096):
        b = fmx.Batch(SHAPES, COURANT, m=4)
        b.set_rows(rows)
        for i, (E, B) in enumerate(inputs):
            b.set_fields(i, E, B)
        b.step(5)
        results.append([b.get_fields(i) for i in range(len(SHAPES))])
    for other in results[1:]:
        for (E0, B0), (E1, B1) in zip(results[0], other):
            assert np.array_equal(E0, E1) and np.array_equal(B0, B1)


def test_batch_tune_then_step(fmx):
    b = fmx.Batch(SHAPES, COURANT, m=4)
    chosen = b.tune(trial_steps=4)
    assert chosen in (0, 1024, 512, 384, 256, 192, 128, 96, 64, 32)
    assert b.tiles()["narrow_rule"] in (0, 1, 2)
    inputs = [_fields(sh, 1907080 + i) for i, sh in enumerate(SHAPES)]
    for i, (E, B) in enumerate(inputs):
        b.set_fields(i, E, B)
    b.step(4)
    for i, (sh, cf) in enumerate(zip(SHAPES, COURANT)):
        Eg, Bg = b.get_fields(i)
        E, B = inputs[i]
        Eo, Bo, _, _ = core.step(core.Params(shape=sh, courant=cf, m=4, coef_f32=True), E.astype(np.float64),
                                 B.astype(np.float64), None, 4)
        assert_parity(Eg, Bg, Eo, Bo, TOL32, f"tuned batch grid {i}")


def test_batch_with_current(fmx):
    shapes, cfs = SHAPES[:4], COURANT[:4]
    b = fmx.Batch(shapes, cfs, m=4, filter_passes=3, with_current=True)
    for i, sh in enumerate(shapes):
        E, B = _fields(sh, 1907090 + i)
        J = synth.solenoidal_current(sh, 1907095 + i, width=3.0, rms=1e-2)
        b.set_fields(i, E, B)
        b.set_current(i, J)
        b.step(0)
    b.step(5)
    for i, (sh, cf) in enumerate(zip(shapes, cfs)):
        E, B = _fields(sh, 1907090 + i)
        J = synth.solenoidal_current(sh, 1907095 + i, width=3.0, rms=1e-2)
        Eg, Bg = b.get_fields(i)
        Eo, Bo, _, _ = core.step(core.Params(shape=sh, courant=cf, m=4, filter_passes=3, coef_f32=True),
                                 E.astype(np.float64), B.astype(np.float64), J.astype(np.float64), 5)
        assert_parity(Eg, Bg, Eo, Bo, TOL32, f"batch+current grid {i}")


def test_batch_failed_rebuild_unbinds(fmx):
    """A work list that outgrows the workspace (one row per segment: 161
    tiles, where the workspace holds the 32-row bound of 21) is refused before
    anything is uploaded or launched, and leaves the batch unbound: the next
    step reports FMX_ESTATE."""
    b = fmx.Batch(SHAPES[:2], COURANT[:2], m=4)
    n0 = b.launches
    with pytest.raises(fmx.FmxError) as ei:
        b.set_rows(1)
    assert ei.value.status == fmx.FMX_EINVAL
    with pytest.raises(fmx.FmxError) as ei:
        b.step(1)
    assert ei.value.status == fmx.FMX_ESTATE
    assert b.launches == n0
    b.close()


@pytest.mark.parametrize("rule", [0, 1, 2])
@pytest.mark.parametrize("with_j", [False, True])
def test_batch_tile_rules_match_oracle(fmx, rule, with_j):
    """Wide tiles only (0), narrow tiles where they compute fewer columns (1)
    and narrow tiles everywhere (2; two independent tiles per CTA on named
    barriers, including the seam tiles of odd n_x): the same results, every
    grid against the oracle, with and without a filtered current."""
    kw = dict(m=4, filter_passes=3, with_current=True) if with_j else dict(m=4)
    b = fmx.Batch(SHAPES, COURANT, **kw)
    b.set_tiles(rule)
    t = b.tiles()
    assert t["narrow_rule"] == rule
    if rule == 0:
        assert t["narrow"] == 0
    if rule == 2:
        assert t["wide"] == 0 and t["narrow"] > 0
    inputs = [_fields(sh, 1907060 + i) for i, sh in enumerate(SHAPES)]
    currents = [synth.solenoidal_current(sh, 1907070 + i, width=4.0, rms=1e-2) for i, sh in enumerate(SHAPES)]
    for i, (E, B) in enumerate(inputs):
        b.set_fields(i, E, B)
        if with_j:
            b.set_current(i, currents[i])
    nsteps = 5
    b.step(nsteps)
    for i, (sh, cf) in enumerate(zip(SHAPES, COURANT)):
        Eg, Bg = b.get_fields(i)
        E, B = inputs[i]
        J = currents[i].astype(np.float64) if with_j else None
        Eo, Bo, rc, _ = core.step(core.Params(shape=sh, courant=cf, m=4, filter_passes=3 if with_j else 0,
                                              coef_f32=True), E.astype(np.float64), B.astype(np.float64), J, nsteps)
        assert_parity(Eg, Bg, Eo, Bo, TOL32, f"rule {rule} grid {i} {sh}")


def test_batch_tune_caches_its_choice(fmx):
    """A second batch of the same grids takes the tuned choice from the
    process cache, without trial steps (its step counter does not move)."""
    b = fmx.Batch(SHAPES, COURANT, m=4)
    rows = b.tune(trial_steps=4)
    first = b.tiles()
    b2 = fmx.Batch(SHAPES, COURANT, m=4)
    rows2 = b2.tune(trial_steps=4)
    assert rows2 == rows and b2.tiles()["narrow_rule"] == first["narrow_rule"]
    assert b2.launches == 0, "the cached choice needs no trial steps"
