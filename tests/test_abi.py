"""Host-side checks of the C ABI: the library loads, exports every entry
point of include/fmx.h, validates its parameters, and uses exactly the
coefficients the oracle derives independently (no GPU needed)."""
import math
import os
import re

import numpy as np
import pytest

from oracle import core
from paper_1907_13088_gb300 import build as fbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def fmx():
    fbuild.build()
    from paper_1907_13088_gb300 import fmx as m
    return m


def _declared():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        with open(os.path.join(ROOT, "include", h)) as f:
            txt = f.read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        names += re.findall(r"\b(fmx_[a-z0-9_]+)\s*\(", txt)
    return sorted(set(names))


def test_exports_every_declared_symbol(fmx):
    import ctypes
    lib = ctypes.CDLL(fmx.LIB_PATH)
    declared = _declared()
    assert len(declared) >= 18
    for name in declared:
        assert hasattr(lib, name), f"{name} declared in include/ but not exported"
    assert set(declared) <= set(fmx.ABI_SIGNATURES)


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("case", [
    dict(shape=(64, 64), courant=0.5), dict(shape=(4096, 4096), courant=0.5),
    dict(shape=(33, 17, 9), d=(1.0, 0.7, 1.3), courant=0.61), dict(shape=(100,), courant=0.9),
    dict(shape=(20, 30), d=(0.5, 2.0, 1.0), courant=1.0), dict(shape=(8, 8), courant=0.3, lumped=True)])
def test_coefficients_bitwise_equal_oracle(fmx, prec, case):
    case = dict(case)
    lumped = case.pop("lumped", False)
    p = fmx.make_params(case["shape"], d=case.get("d", (1.0, 1.0, 1.0)), courant=case["courant"],
                        precision=prec, lumped=lumped, engine=fmx.FMX_ENGINE_STAGED)
    got = fmx.coefficients_of(p)
    o = core.Params(shape=case["shape"], d=case.get("d", (1.0, 1.0, 1.0)), courant=case["courant"],
                    lumped=lumped, coef_f32=(prec == 0))
    want = np.array([core.coefficients(o)[n] for n in core.COEF_NAMES])
    assert np.array_equal(got, want), (got, want)
    # and the time step is the oracle's dt = courant * dt_CFL
    h = __import__("ctypes").c_void_p()
    fmx.check(fmx.fmx_create(__import__("ctypes").byref(p), __import__("ctypes").byref(h), None))
    assert fmx.fmx_time_step(h) == o.time_step()
    fmx.fmx_destroy(h)


def test_validation_codes(fmx):
    ok = fmx.make_params((16, 16), courant=0.5)
    assert fmx.create_status(ok) == (fmx.FMX_OK, 0)
    # Eq. dt_cfl_3d: above the limit -> FMX_ECFL
    bad = fmx.make_params((16, 16), dt=1.0 / math.sqrt(2) * 1.001)
    assert fmx.create_status(bad)[0] == fmx.FMX_ECFL
    assert fmx.create_status(fmx.make_params((16, 16), dt=1.0 / math.sqrt(2)))[0] == fmx.FMX_OK
    assert fmx.create_status(fmx.make_params((16, 16), courant=1.2))[0] == fmx.FMX_ECFL
    # 3D non-cubic with dt > min(d)/(sqrt(2) c): App. C bound not guaranteed -> warning
    s, w = fmx.create_status(fmx.make_params((8, 8, 8), d=(1.0, 1.0, 0.3), courant=0.99))
    assert s == fmx.FMX_OK and w & fmx.FMX_WARN_ANORM
    s, w = fmx.create_status(fmx.make_params((8, 8, 8), courant=0.99))
    assert s == fmx.FMX_OK and w == 0
    p = fmx.make_params((16, 16))
    p.dims = 4
    assert fmx.create_status(p)[0] == fmx.FMX_EINVAL
    p = fmx.make_params((16, 16))
    p.n[2] = 3
    assert fmx.create_status(p)[0] == fmx.FMX_EINVAL
    assert fmx.create_status(fmx.make_params((16, 16), pitch=17))[0] == fmx.FMX_EINVAL
    # extents whose product would overflow the size arithmetic: one field array is capped at 2^40 bytes
    assert fmx.create_status(fmx.make_params((1 << 30, 1 << 30, 1 << 30)))[0] == fmx.FMX_EINVAL
    assert fmx.fmx_field_bytes(__import__("ctypes").byref(fmx.make_params((1 << 30, 1 << 30, 1 << 30)))) == 0
    assert fmx.create_status(fmx.make_params((8192, 8192, 8192)))[0] == fmx.FMX_EINVAL  # 2^41 bytes in FP32
    assert fmx.create_status(fmx.make_params((8192, 8192, 4096)))[0] == fmx.FMX_OK  # 2^40 bytes
    assert fmx.create_status(fmx.make_params((1 << 30, 1 << 10), precision=1))[0] == fmx.FMX_EINVAL
    # launch limits of the one-thread-per-cell kernels: (n_x/32, n_y/8, n_z) blocks, y and z <= 65535
    S = fmx.FMX_ENGINE_STAGED
    assert fmx.create_status(fmx.make_params((4, 524280), engine=S))[0] == fmx.FMX_OK
    assert fmx.create_status(fmx.make_params((4, 524281), engine=S))[0] == fmx.FMX_EUNSUPPORTED
    assert fmx.create_status(fmx.make_params((4, 524281), iter_mode=1))[0] == fmx.FMX_EUNSUPPORTED  # AUTO -> staged
    assert fmx.create_status(fmx.make_params((4, 524281), m=4))[0] == fmx.FMX_OK  # AUTO -> fused, 1D launch grid
    assert fmx.create_status(fmx.make_params((2, 2, 65535), m=4))[0] == fmx.FMX_OK
    assert fmx.create_status(fmx.make_params((2, 2, 65536), m=4))[0] == fmx.FMX_EUNSUPPORTED
    assert fmx.create_status(fmx.make_params((16, 16), iter_mode=1, tol=0.0))[0] == fmx.FMX_EINVAL
    assert fmx.create_status(fmx.make_params((16, 16), m=-1))[0] == fmx.FMX_EINVAL
    # the fused engine covers 2D fixed sweeps only
    assert fmx.create_status(fmx.make_params((16, 16, 16), engine=fmx.FMX_ENGINE_FUSED))[0] == fmx.FMX_EUNSUPPORTED
    assert fmx.create_status(fmx.make_params((16, 16), iter_mode=1, engine=fmx.FMX_ENGINE_FUSED))[0] == \
        fmx.FMX_EUNSUPPORTED
    assert fmx.create_status(fmx.make_params((16, 16), engine=fmx.FMX_ENGINE_FUSED, m=4, filter_passes=3))[0] == \
        fmx.FMX_OK
    # the resident engine: small grids, Algorithm 1 (fixed m or residual), no field filter
    R = fmx.FMX_ENGINE_RESIDENT
    assert fmx.create_status(fmx.make_params((64, 64), iter_mode=1, precision=1, engine=R))[0] == fmx.FMX_OK
    assert fmx.create_status(fmx.make_params((16, 16, 16), m=4, engine=R))[0] == fmx.FMX_OK
    assert fmx.create_status(fmx.make_params((1024, 1024), iter_mode=1, engine=R))[0] == fmx.FMX_EUNSUPPORTED
    assert fmx.create_status(fmx.make_params((64, 64), iter_mode=3, engine=R))[0] == fmx.FMX_EUNSUPPORTED
    assert fmx.create_status(fmx.make_params((64, 64), filter_passes=1, filter_target=fmx.FMX_FILTER_FIELDS,
                                             engine=R))[0] == fmx.FMX_EUNSUPPORTED
    assert fmx.create_status(fmx.make_params((16, 16), engine=4))[0] == fmx.FMX_EINVAL
    # the copy calls check `where` before anything else about the grid
    import ctypes as _ct
    h0 = _ct.c_void_p()
    assert fmx.fmx_create(_ct.byref(fmx.make_params((16, 16))), _ct.byref(h0), None) == fmx.FMX_OK
    ptrs = (_ct.c_void_p * 9)()
    for where in (-1, 2, 7):
        assert fmx.fmx_set_fields(h0, fmx.FMX_E, ptrs, where) == fmx.FMX_EINVAL
        assert fmx.fmx_set_current(h0, ptrs, where) == fmx.FMX_EINVAL
        assert fmx.fmx_get_fields(h0, fmx.FMX_E, ptrs, where) == fmx.FMX_EINVAL
    for where in (fmx.FMX_HOST, fmx.FMX_DEVICE):  # valid: the next check is the unbound grid
        assert fmx.fmx_set_fields(h0, fmx.FMX_E, ptrs, where) == fmx.FMX_ESTATE
        assert fmx.fmx_get_fields(h0, fmx.FMX_E, ptrs, where) == fmx.FMX_ESTATE
    fmx.fmx_destroy(h0)
    # per-grid kernel options (host only)
    import ctypes
    h = ctypes.c_void_p()
    q = fmx.make_params((32, 32, 32), m=4)
    assert fmx.fmx_create(ctypes.byref(q), ctypes.byref(h), None) == fmx.FMX_OK
    assert fmx.fmx_get_option(h, fmx.FMX_OPT_SWEEPS_PER_PASS) == 1
    assert fmx.fmx_set_option(h, fmx.FMX_OPT_SWEEPS_PER_PASS, 2) == fmx.FMX_OK
    assert fmx.fmx_get_option(h, fmx.FMX_OPT_SWEEPS_PER_PASS) == 2
    assert fmx.fmx_set_option(h, fmx.FMX_OPT_SWEEPS_PER_PASS, 3) == fmx.FMX_EINVAL
    assert fmx.fmx_set_option(h, 99, 1) == fmx.FMX_EINVAL and fmx.fmx_get_option(h, 99) == -1
    assert fmx.fmx_get_option(h, fmx.FMX_OPT_WAIT_LIMIT_US) == 1000000
    assert fmx.fmx_set_option(h, fmx.FMX_OPT_WAIT_LIMIT_US, 0) == fmx.FMX_EINVAL
    assert fmx.fmx_set_option(h, fmx.FMX_OPT_WAIT_LIMIT_US, 5000) == fmx.FMX_OK
    assert fmx.fmx_get_option(h, fmx.FMX_OPT_WAIT_LIMIT_US) == 5000
    assert fmx.fmx_set_option(h, fmx.FMX_OPT_SELFTEST_LOST_ARRIVAL, 2) == fmx.FMX_EINVAL
    assert fmx.fmx_get_option(h, fmx.FMX_OPT_SELFTEST_LOST_ARRIVAL) == 0
    assert fmx.fmx_get_option(h, fmx.FMX_OPT_RESIDENT_CLUSTERS) == 0  # no launch yet
    assert fmx.fmx_set_option(h, fmx.FMX_OPT_RESIDENT_CLUSTERS, 2) == fmx.FMX_EINVAL  # read only
    assert fmx.fmx_get_option(h, fmx.FMX_OPT_SEGMENT_ROWS) == 0  # automatic
    assert fmx.fmx_set_option(h, fmx.FMX_OPT_SEGMENT_ROWS, -1) == fmx.FMX_EINVAL
    assert fmx.fmx_set_option(h, fmx.FMX_OPT_SEGMENT_ROWS, 64) == fmx.FMX_OK
    assert fmx.fmx_get_option(h, fmx.FMX_OPT_SEGMENT_ROWS) == 64
    fmx.fmx_destroy(h)
    # the FMA-rate measurement refuses bad arguments before any device work
    out = ctypes.c_double(0.0)
    assert fmx.fmx_fma_peak(7, None, ctypes.byref(out)) == fmx.FMX_EINVAL
    assert fmx.fmx_fma_peak(fmx.FMX_F64, None, None) == fmx.FMX_EINVAL
    assert b"CFL" in fmx.fmx_strerror(fmx.FMX_ECFL)


def test_sizes(fmx):
    import ctypes
    p = fmx.make_params((4099, 31), precision=0)
    assert fmx.fmx_field_bytes(ctypes.byref(p)) == 4100 * 31 * 4
    p = fmx.make_params((4099, 31), precision=1)
    assert fmx.fmx_field_bytes(ctypes.byref(p)) == 4100 * 31 * 8
    p = fmx.make_params((10, 6, 5), precision=0, pitch=16)
    assert fmx.fmx_field_bytes(ctypes.byref(p)) == 16 * 6 * 5 * 4
    staged = fmx.make_params((1000, 1000), engine=fmx.FMX_ENGINE_STAGED)
    fused = fmx.make_params((1000, 1000), engine=fmx.FMX_ENGINE_FUSED)
    fb = fmx.fmx_field_bytes(ctypes.byref(staged))
    assert fmx.fmx_workspace_bytes(ctypes.byref(staged)) >= 13 * fb
    assert fmx.fmx_workspace_bytes(ctypes.byref(fused)) < 2 * fb
    res = fmx.make_params((100, 100), iter_mode=1, engine=fmx.FMX_ENGINE_RESIDENT)
    sta = fmx.make_params((100, 100), iter_mode=1, engine=fmx.FMX_ENGINE_STAGED)
    assert fmx.fmx_workspace_bytes(ctypes.byref(res)) == fmx.fmx_workspace_bytes(ctypes.byref(sta))
    bad = fmx.make_params((16, 16), courant=2.0)
    assert fmx.fmx_workspace_bytes(ctypes.byref(bad)) == 0


def test_batch_validation(fmx):
    import ctypes
    stream = ctypes.c_void_p(0x1)  # any non-NULL handle: create does no device work
    good = [fmx.make_params((64, 40), courant=0.5, stream=stream), fmx.make_params((33, 70), courant=0.9, stream=stream)]
    arr = (fmx.fmx_params * 2)(*good)
    h = ctypes.c_void_p()
    assert fmx.fmx_batch_create(arr, 2, ctypes.byref(h)) == fmx.FMX_OK
    wb = fmx.fmx_batch_workspace_bytes(h)
    assert wb > 0
    # not bound yet: every call that needs the buffers refuses without device work
    assert fmx.fmx_batch_items(h) == 0 and fmx.fmx_batch_launch_count(h) == 0
    assert fmx.fmx_batch_step(h, 1) == fmx.FMX_ESTATE
    assert fmx.fmx_batch_set_rows(h, 64) == fmx.FMX_ESTATE
    assert fmx.fmx_batch_tune(h, 4, None) == fmx.FMX_ESTATE
    ptrs = (ctypes.c_void_p * 6)()
    assert fmx.fmx_batch_get_fields(h, 0, fmx.FMX_E, ptrs, fmx.FMX_HOST) == fmx.FMX_ESTATE
    assert fmx.fmx_batch_set_fields(h, 0, fmx.FMX_E, ptrs, fmx.FMX_HOST) == fmx.FMX_ESTATE
    assert fmx.fmx_batch_get_fields(h, 2, fmx.FMX_E, ptrs, fmx.FMX_HOST) == fmx.FMX_EINVAL  # no grid 2
    assert fmx.fmx_batch_get_fields(h, 0, fmx.FMX_E, ptrs, 5) == fmx.FMX_EINVAL  # where
    assert fmx.fmx_batch_set_fields(h, 0, fmx.FMX_E, ptrs, -1) == fmx.FMX_EINVAL
    # bind's argument checks come before any device work (the pointers are
    # never dereferenced on these paths)
    bufs = (fmx.fmx_buffers * 2)()
    fake = ctypes.c_void_p(1 << 20)
    assert fmx.fmx_batch_bind(h, bufs, ctypes.c_void_p(256 + 16), wb) == fmx.FMX_EINVAL  # misaligned workspace
    assert fmx.fmx_batch_bind(h, bufs, fake, wb - 1) == fmx.FMX_EINVAL  # too small
    assert fmx.fmx_batch_bind(h, bufs, fake, wb) == fmx.FMX_EINVAL  # NULL field buffers
    assert fmx.fmx_batch_step(h, 1) == fmx.FMX_ESTATE  # a failed bind leaves it unbound
    fmx.fmx_batch_destroy(h)
    assert fmx.fmx_batch_create(arr, 0, ctypes.byref(h)) == fmx.FMX_EINVAL
    bad = [fmx.make_params((64, 40), courant=0.5, stream=stream), fmx.make_params((33, 70), m=3, stream=stream)]
    assert fmx.fmx_batch_create((fmx.fmx_params * 2)(*bad), 2, ctypes.byref(h)) == fmx.FMX_EINVAL
    nostream = [fmx.make_params((64, 40), courant=0.5)]
    assert fmx.fmx_batch_create((fmx.fmx_params * 1)(*nostream), 1, ctypes.byref(h)) == fmx.FMX_EINVAL
    cfl = [fmx.make_params((64, 40), courant=1.5, stream=stream)]
    assert fmx.fmx_batch_create((fmx.fmx_params * 1)(*cfl), 1, ctypes.byref(h)) == fmx.FMX_ECFL
    f64 = [fmx.make_params((64, 40), precision=1, stream=stream)]
    assert fmx.fmx_batch_create((fmx.fmx_params * 1)(*f64), 1, ctypes.byref(h)) == fmx.FMX_EINVAL
    for kw in (dict(iter_mode=fmx.FMX_ITER_RESIDUAL), dict(filter_passes=1, filter_target=fmx.FMX_FILTER_FIELDS)):
        one = [fmx.make_params((64, 40), stream=stream, **kw)]
        assert fmx.fmx_batch_create((fmx.fmx_params * 1)(*one), 1, ctypes.byref(h)) == fmx.FMX_EINVAL, kw
    three_d = [fmx.make_params((16, 16, 16), stream=stream)]
    assert fmx.fmx_batch_create((fmx.fmx_params * 1)(*three_d), 1, ctypes.byref(h)) == fmx.FMX_EINVAL


def test_nci_rejects_bad_parameters_before_any_device_work(fmx):
    """fmx_nci_resonance validates on the host and returns FMX_EINVAL before it
    enqueues anything (the output pointers are never touched here; the test
    only runs where there is no GPU)."""
    import ctypes
    import torch
    if torch.cuda.is_available():
        pytest.skip("host-only check")
    for bad in (dict(courant=0.0), dict(courant=1.01), dict(dx=-1.0), dict(dy=float("inf")), dict(c=0.0),
                dict(nkx=0), dict(nkx=(1 << 26) + 1), dict(nu_max=-1), dict(nu_max=65), dict(shape_order=-1),
                dict(shape_order=17), dict(omega_p=float("nan")), dict(omega_p=-1.0)):
        p = fmx.nci_params(**bad)
        assert fmx.fmx_nci_resonance(ctypes.byref(p), None, 16, 16, None, None) == fmx.FMX_EINVAL, bad
        assert b"fmx_nci_resonance" in fmx.fmx_last_error()
    p = fmx.nci_params()
    assert fmx.fmx_nci_resonance(ctypes.byref(p), None, None, 16, None, None) == fmx.FMX_EINVAL
    assert fmx.fmx_nci_resonance(None, None, 16, 16, None, None) == fmx.FMX_EINVAL


def test_current_profile_needs_a_bound_grid(fmx):
    """fmx_set_current_profile checks its handle on the host: NULL grid ->
    FMX_EINVAL, a grid not yet bound -> FMX_ESTATE (no device work)."""
    import ctypes
    p = fmx.make_params((16, 16), courant=0.5)
    h = ctypes.c_void_p()
    fmx.check(fmx.fmx_create(ctypes.byref(p), ctypes.byref(h), None))
    try:
        t = (ctypes.c_double * 2)(1.0, 0.5)
        assert fmx.fmx_set_current_profile(None, t, 2) == fmx.FMX_EINVAL
        assert fmx.fmx_set_current_profile(h, t, 2) == fmx.FMX_ESTATE
    finally:
        fmx.fmx_destroy(h)


def test_resource_report_kernel_names():
    """The ptxas resource report names kernels by their short name with
    template arguments (enum casts and anonymous namespaces dropped)."""
    from paper_1907_13088_gb300.build import _short
    assert _short("(anonymous namespace)::k_nci_best((anonymous namespace)::NciCoef, double const*, double*)") \
        == "k_nci_best"
    assert _short("void fmx::pol2d::k_pol2d<(fmx::pol2d::Pol)0, 4, 3, true, 128>(fmx::Fused2dArgs<float>, "
                  "fmx::Geo, fmx::pol2d::Coef2, int, int, int)") == "k_pol2d<0, 4, 3, true, 128>"
    assert _short("void fmx::(anonymous namespace)::k3_sweep2<true>(fmx::Geo, float const*)") == "k3_sweep2<true>"
