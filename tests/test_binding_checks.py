"""Host-side checks of the Python binding: a field component's size, dtype,
layout and device are checked before its pointer reaches the library (which
copies a fixed number of elements and trusts the pointer).  No GPU needed:
CUDA tensors are stood in for by an object with a tensor's attributes."""
import ctypes
import types

import numpy as np
import pytest

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def fmx():
    from paper_1907_13088_gb300 import build

    build.build()
    from paper_1907_13088_gb300 import fmx as m

    return m


class FakeCudaTensor:
    """The attributes component_ptr reads from a CUDA tensor."""

    __module__ = "torch.fake"

    def __init__(self, n, dtype=torch.float32, index=0, contiguous=True):
        self.n, self.dtype, self._contig = n, dtype, contiguous
        self.is_cuda = True
        self.device = types.SimpleNamespace(type="cuda", index=index)

    def numel(self):
        return self.n

    def is_contiguous(self):
        return self._contig

    def contiguous(self):
        return self if self._contig else FakeCudaTensor(self.n, self.dtype, self.device.index)

    def data_ptr(self):
        return 0x7F0000000000


CELLS = 6 * 5


def test_numpy_input_is_converted(fmx):
    a = np.arange(CELLS, dtype=np.float64).reshape(1, 5, 6)[:, :, ::1]
    p, keep, where = fmx.component_ptr(a, CELLS, np.float32)
    assert where == fmx.FMX_HOST
    assert keep.dtype == np.float32 and keep.flags.c_contiguous and p == keep.ctypes.data
    np.testing.assert_array_equal(keep.ravel(), np.arange(CELLS, dtype=np.float32))
    # a strided view is copied into a contiguous array
    b = np.arange(2 * CELLS, dtype=np.float32)[::2]
    _, keep, _ = fmx.component_ptr(b, CELLS, np.float32)
    assert keep.flags.c_contiguous and keep[1] == 2.0


@pytest.mark.parametrize("n", [CELLS - 1, CELLS + 1, 0])
def test_wrong_size_is_rejected(fmx, n):
    with pytest.raises(ValueError):
        fmx.component_ptr(np.zeros(n, np.float32), CELLS, np.float32)
    with pytest.raises(ValueError):
        fmx.component_ptr(np.zeros(n, np.float32), CELLS, np.float32, out=True)
    with pytest.raises(ValueError):
        fmx.component_ptr(FakeCudaTensor(n), CELLS, np.float32, torch.float32, 0)


def test_host_outputs_are_not_converted(fmx):
    ok = np.zeros(CELLS, np.float64)
    p, keep, where = fmx.component_ptr(ok, CELLS, np.float64, out=True)
    assert keep is ok and p == ok.ctypes.data and where == fmx.FMX_HOST
    with pytest.raises(TypeError):  # another dtype: the library would write past it or garble it
        fmx.component_ptr(np.zeros(CELLS, np.float32), CELLS, np.float64, out=True)
    with pytest.raises(TypeError):  # strided
        fmx.component_ptr(np.zeros(2 * CELLS, np.float64)[::2], CELLS, np.float64, out=True)
    ro = np.zeros(CELLS, np.float64)
    ro.flags.writeable = False
    with pytest.raises(TypeError):
        fmx.component_ptr(ro, CELLS, np.float64, out=True)


def test_device_tensors(fmx):
    p, _, where = fmx.component_ptr(FakeCudaTensor(CELLS), CELLS, np.float32, torch.float32, 0)
    assert where == fmx.FMX_DEVICE and p == 0x7F0000000000
    with pytest.raises(TypeError):  # dtype
        fmx.component_ptr(FakeCudaTensor(CELLS, torch.float64), CELLS, np.float32, torch.float32, 0)
    with pytest.raises(ValueError):  # another device
        fmx.component_ptr(FakeCudaTensor(CELLS, index=1), CELLS, np.float32, torch.float32, 0)
    with pytest.raises(TypeError):  # an output must be written in place
        fmx.component_ptr(FakeCudaTensor(CELLS, contiguous=False), CELLS, np.float32, torch.float32, 0, out=True)
    # an input is made contiguous first
    fmx.component_ptr(FakeCudaTensor(CELLS, contiguous=False), CELLS, np.float32, torch.float32, 0)


def test_host_tensors_and_other_objects_are_rejected(fmx):
    with pytest.raises(TypeError):  # a CPU tensor's pointer is not device memory
        fmx.component_ptr(torch.zeros(CELLS), CELLS, np.float32, torch.float32, 0)
    with pytest.raises(TypeError):
        fmx.component_ptr([0.0] * CELLS, CELLS, np.float32)


def test_pointer_arrays(fmx):
    a = np.zeros(CELLS, np.float32)
    ptrs, keep, where = fmx.component_ptrs([a, None, a], CELLS, np.float32)
    assert isinstance(ptrs, ctypes.Array) and len(ptrs) == 3 and ptrs[1] is None
    assert ptrs[0] == a.ctypes.data and len(keep) == 2 and where == fmx.FMX_HOST
    assert fmx.component_ptrs([None, None], CELLS, np.float32)[2] == fmx.FMX_HOST
    with pytest.raises(TypeError):  # host and device components in one call
        fmx.component_ptrs([a, FakeCudaTensor(CELLS)], CELLS, np.float32, torch.float32, 0)


def _host_grid(fmx, monkeypatch, shape=(6, 5), f64=False):
    """A Grid whose library calls are replaced by recorders (no device)."""
    g = object.__new__(fmx.Grid)
    g.torch = torch
    g.shape = shape
    nx, ny, nz = shape + (1,) * (3 - len(shape))
    g.array_shape = (3, nz, ny, nx)
    g.cells = nx * ny * nz
    g.np_dtype = np.float64 if f64 else np.float32
    g.dtype = torch.float64 if f64 else torch.float32
    g._dev_index = 0
    g.handle = None
    calls = []

    def rec(name, writer=None):
        def f(*args):
            calls.append((name, args))
            if writer:
                writer(*args)
            return fmx.FMX_OK
        monkeypatch.setattr(fmx, name, f)

    def fill(h, mask, ptrs, where):  # component c of the grid holds the value c
        for c in range(9):
            if mask & (1 << c):
                src = np.full(g.cells, c, g.np_dtype)
                ctypes.memmove(ptrs[c], src.ctypes.data, src.nbytes)

    rec("fmx_set_fields")
    rec("fmx_set_current")
    rec("fmx_get_fields", fill)
    rec("fmx_step_host")
    return g, calls


def test_grid_methods_pass_checked_pointers(fmx, monkeypatch):
    g, calls = _host_grid(fmx, monkeypatch)
    E = np.random.default_rng(0).standard_normal((3, 1, 5, 6))
    g.set_fields(E, None)
    name, (h, mask, ptrs, where) = calls[-1]
    assert name == "fmx_set_fields" and mask == fmx.FMX_E and where == fmx.FMX_HOST
    got = np.ctypeslib.as_array(ctypes.cast(ptrs[1], ctypes.POINTER(ctypes.c_float)), (g.cells,))
    np.testing.assert_array_equal(got, E[1].ravel().astype(np.float32))
    with pytest.raises(ValueError):
        g.set_fields(np.zeros((3, 1, 5, 5)), None)  # a column short
    with pytest.raises(ValueError):
        g.set_current(np.zeros((2, 1, 5, 6)))
    with pytest.raises(TypeError):
        g.set_fields(E, torch.zeros((3, 1, 5, 6)))  # a CPU tensor
    n = len(calls)
    # read-back into a fresh array, into host_out, and a rejected host_out
    Eg, Bg, Jg = g.get_fields(fmx.FMX_E | fmx.FMX_J)
    assert Bg is None and Eg.shape == (3, 1, 5, 6) and Jg.shape == (3, 1, 5, 6)
    assert [int(Eg[c, 0, 0, 0]) for c in range(3)] == [0, 1, 2] and int(Jg[2].max()) == 8
    host = np.zeros((9, 1, 5, 6), np.float32)
    Eh, _, _ = g.get_fields(fmx.FMX_E, host_out=host)
    assert Eh.base is host and host[2].min() == 2.0
    with pytest.raises(TypeError):
        g.get_fields(host_out=np.zeros((9, 1, 5, 6), np.float64))
    with pytest.raises(ValueError):
        g.get_fields(host_out=np.zeros((6, 1, 5, 6), np.float32))
    with pytest.raises(TypeError):
        g.get_fields(out=np.zeros((9, 1, 5, 6), np.float32))  # out= is for device tensors
    assert len(calls) == n + 2


def test_step_host_checks(fmx, monkeypatch):
    g, calls = _host_grid(fmx, monkeypatch, f64=True)
    inp = np.zeros((9, 1, 5, 6))
    out = np.zeros((6, 1, 5, 6))
    g.step_host([(inp, out), (inp[:6], None)])
    name, (h, recs, count) = calls[-1]
    assert name == "fmx_step_host" and count == 2
    assert [recs[0].inp[c] for c in range(9)] == [inp[c].ctypes.data for c in range(9)]
    assert [recs[0].out[c] for c in range(6)] == [out[c].ctypes.data for c in range(6)]
    assert recs[1].inp[6] is None and recs[1].out[0] is None
    for bad in [(inp.astype(np.float32), out), (inp, out[:, :, :, :5].copy()), (inp[:, :, :, ::2], out),
                (inp[:7], out), (inp, out[:5])]:
        with pytest.raises((TypeError, ValueError)):
            g.step_host([bad])
    ro = out.copy()
    ro.flags.writeable = False
    with pytest.raises(TypeError):
        g.step_host([(inp, ro)])
    assert calls[-1][1][2] == 2  # no rejected call reached the library
