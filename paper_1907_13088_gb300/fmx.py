"""Python binding of the fmx C ABI (``include/fmx.h``).

Argument marshalling only: every step of the field advance runs in the CUDA
kernels of ``_build/libfmx.so``.  The functions below carry the C names and
take plain integers, floats and pointers; ``Grid`` is a convenience wrapper
that allocates the device buffers the library borrows with PyTorch (device
memory and streams are the only things PyTorch provides here).

Importing this module never falls back to anything: if the shared library is
missing or fails to load, the import raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libfmx.so")

# status codes
FMX_OK, FMX_EINVAL, FMX_ECFL, FMX_ENOCONV, FMX_ECUDA, FMX_ETIMEOUT, FMX_ESTATE, FMX_EUNSUPPORTED = range(8)
FMX_F32, FMX_F64 = 0, 1
FMX_ITER_FIXED, FMX_ITER_RESIDUAL, FMX_ITER_CHEB_FIXED, FMX_ITER_CHEB_RESIDUAL = 0, 1, 2, 3
FMX_FILTER_NONE, FMX_FILTER_CURRENT, FMX_FILTER_FIELDS = 0, 1, 2
FMX_ENGINE_AUTO, FMX_ENGINE_STAGED, FMX_ENGINE_FUSED, FMX_ENGINE_RESIDENT = 0, 1, 2, 3
FMX_HOST, FMX_DEVICE = 0, 1
FMX_EX, FMX_EY, FMX_EZ, FMX_BX, FMX_BY, FMX_BZ, FMX_JX, FMX_JY, FMX_JZ = (1 << i for i in range(9))
FMX_E, FMX_B, FMX_J = 7, 7 << 3, 7 << 6
FMX_WARN_ANORM = 1
FMX_NCOEF = 14


class fmx_params(ctypes.Structure):
    _fields_ = [("dims", ctypes.c_int), ("n", ctypes.c_int64 * 3), ("d", ctypes.c_double * 3),
                ("c", ctypes.c_double), ("dt", ctypes.c_double), ("courant", ctypes.c_double),
                ("precision", ctypes.c_int), ("iter_mode", ctypes.c_int), ("m", ctypes.c_int),
                ("tol", ctypes.c_double), ("m_max", ctypes.c_int), ("filter_passes", ctypes.c_int),
                ("filter_target", ctypes.c_int), ("lumped", ctypes.c_int), ("engine", ctypes.c_int),
                ("pitch", ctypes.c_int64), ("stream", ctypes.c_void_p)]


class fmx_buffers(ctypes.Structure):
    _fields_ = [("E", (ctypes.c_void_p * 3) * 2), ("B", (ctypes.c_void_p * 3) * 2), ("J", ctypes.c_void_p * 3),
                ("work", ctypes.c_void_p), ("work_bytes", ctypes.c_size_t)]


class fmx_kernel_stat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 48), ("launches", ctypes.c_int64), ("total_ms", ctypes.c_double),
                ("bytes_per_launch", ctypes.c_double)]


class fmx_host_step(ctypes.Structure):
    _fields_ = [("inp", ctypes.c_void_p * 9), ("out", ctypes.c_void_p * 6)]


class fmx_nci_params(ctypes.Structure):
    _fields_ = [("dx", ctypes.c_double), ("dy", ctypes.c_double), ("c", ctypes.c_double),
                ("courant", ctypes.c_double), ("omega_p", ctypes.c_double), ("shape_order", ctypes.c_int),
                ("nu_max", ctypes.c_int), ("nkx", ctypes.c_int)]


class fmx_diag(ctypes.Structure):
    _fields_ = [("w_scheme", ctypes.c_double), ("w_plain", ctypes.c_double), ("divb_max", ctypes.c_double),
                ("divb_l2", ctypes.c_double), ("gauss_max", ctypes.c_double), ("gauss_l2", ctypes.c_double),
                ("last_resid", ctypes.c_double), ("last_sweeps", ctypes.c_int), ("total_sweeps", ctypes.c_int64),
                ("steps", ctypes.c_int64)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"fmx CUDA library not built ({LIB_PATH}); run paper_1907_13088_gb300.build")
    lib = ctypes.CDLL(LIB_PATH)
    P = ctypes.POINTER(fmx_params)
    G = ctypes.c_void_p
    vpp = ctypes.POINTER(ctypes.c_void_p)
    sig = {
        "fmx_create": (ctypes.c_int, [P, ctypes.POINTER(G), ctypes.POINTER(ctypes.c_int)]),
        "fmx_field_bytes": (ctypes.c_size_t, [P]),
        "fmx_workspace_bytes": (ctypes.c_size_t, [P]),
        "fmx_bind": (ctypes.c_int, [G, ctypes.POINTER(fmx_buffers)]),
        "fmx_set_fields": (ctypes.c_int, [G, ctypes.c_uint, vpp, ctypes.c_int]),
        "fmx_set_current": (ctypes.c_int, [G, vpp, ctypes.c_int]),
        "fmx_set_current_profile": (ctypes.c_int, [G, ctypes.POINTER(ctypes.c_double), ctypes.c_int]),
        "fmx_step": (ctypes.c_int, [G, ctypes.c_int]),
        "fmx_filter": (ctypes.c_int, [G, ctypes.c_uint, ctypes.c_int]),
        "fmx_get_fields": (ctypes.c_int, [G, ctypes.c_uint, vpp, ctypes.c_int]),
        "fmx_diagnostics": (ctypes.c_int, [G, ctypes.POINTER(fmx_diag)]),
        "fmx_sync": (ctypes.c_int, [G]),
        "fmx_coefficients": (ctypes.c_int, [G, ctypes.POINTER(ctypes.c_double), ctypes.c_int]),
        "fmx_time_step": (ctypes.c_double, [G]),
        "fmx_field_ptr": (ctypes.c_void_p, [G, ctypes.c_int]),
        "fmx_launch_count": (ctypes.c_int64, [G]),
        "fmx_destroy": (None, [G]),
        "fmx_strerror": (ctypes.c_char_p, [ctypes.c_int]),
        "fmx_last_error": (ctypes.c_char_p, []),
        "fmx_step_static": (ctypes.c_int, [P, vpp, vpp, vpp, ctypes.c_int]),
        "fmx_profile_enable": (ctypes.c_int, [G, ctypes.c_int]),
        "fmx_adjoint_workspace_bytes": (ctypes.c_size_t, [P]),
        "fmx_adjoint_step": (ctypes.c_int, [G, vpp, vpp, vpp, ctypes.c_void_p, ctypes.c_size_t]),
        "fmx_gauss_source": (ctypes.c_int, [G, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                            ctypes.POINTER(ctypes.c_double), ctypes.c_double]),
        "fmx_gauss_project": (ctypes.c_int, [G, ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.c_double,
                                             ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)]),
        "fmx_gauss_accumulate": (ctypes.c_int, [G, ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.c_double,
                                                ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_int]),
        "fmx_gauss_accumulated": (ctypes.c_int, [G, ctypes.c_int, ctypes.POINTER(ctypes.c_double)]),
        "fmx_cheb_interval": (ctypes.c_int, [G, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]),
        "fmx_gauss_setup": (ctypes.c_int, [G, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                           ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                           ctypes.c_double, ctypes.c_double]),
        "fmx_gauss_run": (ctypes.c_int, [G, ctypes.c_int64, ctypes.c_int]),
        "fmx_gauss_adjoint_run": (ctypes.c_int, [G, ctypes.c_int64, ctypes.c_int, vpp, vpp, vpp, ctypes.c_void_p,
                                                 ctypes.c_size_t, ctypes.c_int]),
        "fmx_batch_create": (ctypes.c_int, [P, ctypes.c_int, ctypes.POINTER(G)]),
        "fmx_batch_workspace_bytes": (ctypes.c_size_t, [G]),
        "fmx_batch_bind": (ctypes.c_int, [G, ctypes.POINTER(fmx_buffers), ctypes.c_void_p, ctypes.c_size_t]),
        "fmx_batch_set_fields": (ctypes.c_int, [G, ctypes.c_int, ctypes.c_uint, vpp, ctypes.c_int]),
        "fmx_batch_get_fields": (ctypes.c_int, [G, ctypes.c_int, ctypes.c_uint, vpp, ctypes.c_int]),
        "fmx_batch_set_rows": (ctypes.c_int, [G, ctypes.c_int]),
        "fmx_batch_tune": (ctypes.c_int, [G, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
        "fmx_batch_set_tiles": (ctypes.c_int, [G, ctypes.c_int]),
        "fmx_batch_grid_width": (ctypes.c_int, [G, ctypes.c_int]),
        "fmx_batch_tiles": (ctypes.c_int, [G] + [ctypes.POINTER(ctypes.c_int)] * 5),
        "fmx_batch_step": (ctypes.c_int, [G, ctypes.c_int]),
        "fmx_batch_items": (ctypes.c_int, [G]),
        "fmx_batch_launch_count": (ctypes.c_int64, [G]),
        "fmx_batch_destroy": (None, [G]),
        "fmx_profile_read": (ctypes.c_int, [G, ctypes.POINTER(fmx_kernel_stat), ctypes.c_int,
                                            ctypes.POINTER(ctypes.c_int)]),
        "fmx_nci_resonance": (ctypes.c_int, [ctypes.POINTER(fmx_nci_params), ctypes.c_void_p, ctypes.c_void_p,
                                             ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
        "fmx_fma_peak": (ctypes.c_int, [ctypes.c_int, ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)]),
        "fmx_step_host": (ctypes.c_int, [G, ctypes.POINTER(fmx_host_step), ctypes.c_int]),
        "fmx_set_option": (ctypes.c_int, [G, ctypes.c_int, ctypes.c_int]),
        "fmx_get_option": (ctypes.c_int, [G, ctypes.c_int]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib, sig


_lib, ABI_SIGNATURES = _load()

fmx_create = _lib.fmx_create
fmx_field_bytes = _lib.fmx_field_bytes
fmx_workspace_bytes = _lib.fmx_workspace_bytes
fmx_bind = _lib.fmx_bind
fmx_set_fields = _lib.fmx_set_fields
fmx_set_current = _lib.fmx_set_current
fmx_set_current_profile = _lib.fmx_set_current_profile
fmx_step = _lib.fmx_step
fmx_filter = _lib.fmx_filter
fmx_get_fields = _lib.fmx_get_fields
fmx_diagnostics = _lib.fmx_diagnostics
fmx_sync = _lib.fmx_sync
fmx_coefficients = _lib.fmx_coefficients
fmx_time_step = _lib.fmx_time_step
fmx_field_ptr = _lib.fmx_field_ptr
fmx_launch_count = _lib.fmx_launch_count
fmx_destroy = _lib.fmx_destroy
fmx_strerror = _lib.fmx_strerror
fmx_last_error = _lib.fmx_last_error
fmx_step_static = _lib.fmx_step_static
fmx_profile_enable = _lib.fmx_profile_enable
fmx_adjoint_workspace_bytes = _lib.fmx_adjoint_workspace_bytes
fmx_adjoint_step = _lib.fmx_adjoint_step
fmx_gauss_source = _lib.fmx_gauss_source
fmx_gauss_project = _lib.fmx_gauss_project
fmx_gauss_accumulate = _lib.fmx_gauss_accumulate
fmx_gauss_accumulated = _lib.fmx_gauss_accumulated
fmx_cheb_interval = _lib.fmx_cheb_interval
fmx_gauss_setup = _lib.fmx_gauss_setup
fmx_gauss_run = _lib.fmx_gauss_run
fmx_gauss_adjoint_run = _lib.fmx_gauss_adjoint_run
fmx_batch_create = _lib.fmx_batch_create
fmx_batch_workspace_bytes = _lib.fmx_batch_workspace_bytes
fmx_batch_bind = _lib.fmx_batch_bind
fmx_batch_set_fields = _lib.fmx_batch_set_fields
fmx_batch_get_fields = _lib.fmx_batch_get_fields
fmx_batch_set_rows = _lib.fmx_batch_set_rows
fmx_batch_tune = _lib.fmx_batch_tune
fmx_batch_step = _lib.fmx_batch_step
fmx_batch_set_tiles = _lib.fmx_batch_set_tiles
fmx_batch_tiles = _lib.fmx_batch_tiles
fmx_batch_grid_width = _lib.fmx_batch_grid_width
fmx_batch_items = _lib.fmx_batch_items
fmx_batch_launch_count = _lib.fmx_batch_launch_count
fmx_batch_destroy = _lib.fmx_batch_destroy
fmx_profile_read = _lib.fmx_profile_read
fmx_nci_resonance = _lib.fmx_nci_resonance
fmx_fma_peak = _lib.fmx_fma_peak
fmx_step_host = _lib.fmx_step_host
fmx_set_option = _lib.fmx_set_option
fmx_get_option = _lib.fmx_get_option
FMX_OPT_SWEEPS_PER_PASS, FMX_OPT_WAIT_LIMIT_US, FMX_OPT_SELFTEST_LOST_ARRIVAL, FMX_OPT_RESIDENT_CLUSTERS = 1, 2, 3, 4
FMX_OPT_SEGMENT_ROWS = 5
FMX_STATIC_SCRATCH_BYTES = 4 << 20


class FmxError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = fmx_last_error().decode(errors="replace")
        super().__init__(f"{where}: {fmx_strerror(status).decode()} ({status}): {msg}")


def check(status: int, where: str = "fmx") -> None:
    if status != FMX_OK:
        raise FmxError(status, where)


def make_params(shape, d=(1.0, 1.0, 1.0), c=1.0, dt=0.0, courant=0.5, precision=FMX_F32, iter_mode=FMX_ITER_FIXED,
                m=4, tol=1e-13, m_max=10000, filter_passes=0, filter_target=FMX_FILTER_CURRENT, lumped=False,
                engine=FMX_ENGINE_AUTO, pitch=0, stream=None) -> fmx_params:
    """fmx_params for a grid of ``shape`` = (nx,), (nx, ny) or (nx, ny, nz)."""
    p = fmx_params()
    p.dims = len(shape)
    n3 = tuple(shape) + (1,) * (3 - len(shape))
    for a in range(3):
        p.n[a] = int(n3[a])
        p.d[a] = float(d[a]) if a < len(d) else 1.0
    p.c, p.dt, p.courant = float(c), float(dt or 0.0), float(courant)
    p.precision, p.iter_mode, p.m = int(precision), int(iter_mode), int(m)
    p.tol, p.m_max = float(tol), int(m_max)
    p.filter_passes, p.filter_target, p.lumped = int(filter_passes), int(filter_target), int(bool(lumped))
    p.engine, p.pitch = int(engine), int(pitch)
    p.stream = stream
    return p


def _is_tensor(a) -> bool:
    return type(a).__module__.startswith("torch") and hasattr(a, "data_ptr")


def component_ptr(a, cells, np_dtype, torch_dtype=None, dev_index=None, out=False):
    """Checks one field component before its pointer goes to the library and
    returns (pointer, keep-alive object, FMX_HOST or FMX_DEVICE).

    The library copies exactly ``cells`` elements of the grid's precision per
    component and trusts the pointer, so a short array, another dtype, a
    strided view or a tensor on another device would make it read or write
    past the buffer.  A numpy input is converted (a contiguous copy of the
    grid's dtype); a numpy output must already be a C-contiguous, writeable
    array of that dtype.  A torch tensor must be a CUDA tensor of the grid's
    dtype on device ``dev_index`` (None: any CUDA device), contiguous when it
    receives data; an input is made contiguous.  Raises TypeError or
    ValueError; nothing is copied here."""
    if isinstance(a, np.ndarray):
        if out:
            if a.dtype != np.dtype(np_dtype) or not a.flags.c_contiguous or not a.flags.writeable:
                raise TypeError(f"host output must be a writeable C-contiguous {np.dtype(np_dtype)} array "
                                f"(got {a.dtype}, contiguous={a.flags.c_contiguous}, writeable={a.flags.writeable})")
        else:
            a = np.ascontiguousarray(a, dtype=np_dtype)
        if a.size != cells:
            raise ValueError(f"a field component has {a.size} elements, the grid {cells}")
        return a.ctypes.data, a, FMX_HOST
    if _is_tensor(a):
        if not a.is_cuda:
            raise TypeError("torch tensors must be CUDA tensors on the grid's device (pass numpy arrays for host data)")
        if dev_index is not None and a.device.index != dev_index:
            raise ValueError(f"tensor on cuda:{a.device.index}, the grid on cuda:{dev_index}")
        if torch_dtype is not None and a.dtype != torch_dtype:
            raise TypeError(f"tensor of {a.dtype}, the grid stores {torch_dtype}")
        if out and not a.is_contiguous():
            raise TypeError("an output tensor must be contiguous")
        if a.numel() != cells:
            raise ValueError(f"a field component has {a.numel()} elements, the grid {cells}")
        a = a.contiguous()
        return a.data_ptr(), a, FMX_DEVICE
    raise TypeError(f"a field component must be a numpy array or a CUDA tensor (got {type(a).__name__})")


def component_ptrs(arrays, cells, np_dtype, torch_dtype=None, dev_index=None, out=False):
    """component_ptr over a list (None entries stay NULL): returns (ctypes
    pointer array, keep-alive list, FMX_HOST or FMX_DEVICE).  Host and device
    components cannot be mixed in one call."""
    ptrs = (ctypes.c_void_p * len(arrays))()
    keep, where = [], set()
    for i, a in enumerate(arrays):
        if a is None:
            ptrs[i] = None
            continue
        p, k, w = component_ptr(a, cells, np_dtype, torch_dtype, dev_index, out)
        ptrs[i] = p
        keep.append(k)
        where.add(w)
    if len(where) > 1:
        raise TypeError("host arrays and device tensors cannot be mixed in one call")
    return ptrs, keep, (where.pop() if where else FMX_HOST)


class Grid:
    """A field-advance grid whose device buffers are PyTorch tensors.

    Fields are exchanged as arrays of shape (3, nz, ny, nx) (numpy on the
    host or torch tensors on the device) at the staggered positions
    documented in fmx.h.
    """

    def __init__(self, shape, device="cuda", with_current=True, **kw):
        import torch

        self.torch = torch
        self.shape = tuple(shape)
        self.device = torch.device(device)
        stream = kw.pop("stream", None)
        if stream is None:
            stream = torch.cuda.current_stream(self.device)
        self.stream = stream
        kw.setdefault("precision", FMX_F32)
        self.params = make_params(shape, stream=ctypes.c_void_p(stream.cuda_stream), **kw)
        self.dtype = torch.float64 if self.params.precision == FMX_F64 else torch.float32
        self.np_dtype = np.float64 if self.params.precision == FMX_F64 else np.float32
        h = ctypes.c_void_p()
        warn = ctypes.c_int(0)
        check(fmx_create(ctypes.byref(self.params), ctypes.byref(h), ctypes.byref(warn)), "fmx_create")
        self.handle = h
        self.warnings = warn.value
        fb = fmx_field_bytes(ctypes.byref(self.params))
        wb = fmx_workspace_bytes(ctypes.byref(self.params))
        esz = 8 if self.params.precision == FMX_F64 else 4
        nfield = (fb + 255) // 256 * 256 // esz
        ncomp = 12 + (3 if with_current else 0)
        # one slab for every field component, each at a 256-byte boundary
        self._slab = torch.zeros(ncomp * nfield, dtype=self.dtype, device=self.device)
        self._work = torch.zeros((wb + 511) // 256 * 256, dtype=torch.uint8, device=self.device)
        base = self._slab.data_ptr()
        wbase = (self._work.data_ptr() + 255) // 256 * 256
        ptr = lambda i: base + i * nfield * esz
        b = fmx_buffers()
        for s in range(2):
            for c in range(3):
                b.E[s][c] = ptr(s * 6 + c)
                b.B[s][c] = ptr(s * 6 + 3 + c)
        for c in range(3):
            b.J[c] = ptr(12 + c) if with_current else None
        b.work = wbase
        b.work_bytes = wb
        self.buffers = b
        check(fmx_bind(self.handle, ctypes.byref(b)), "fmx_bind")
        nx, ny, nz = self.shape + (1,) * (3 - len(self.shape))
        self.array_shape = (3, nz, ny, nx)
        self.cells = nx * ny * nz
        self._dev_index = self._slab.device.index

    # -- lifetime --------------------------------------------------------
    def close(self):
        if getattr(self, "handle", None):
            fmx_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- copies ----------------------------------------------------------
    def _ptr_array(self, arrays, out=False):
        """Checked pointers of field components (component_ptrs with this
        grid's size, dtype and device)."""
        return component_ptrs(arrays, self.cells, self.np_dtype, self.dtype, self._dev_index, out)

    def set_fields(self, E=None, B=None):
        arrs = [None] * 6
        mask = 0
        for k, F in enumerate((E, B)):
            if F is None:
                continue
            if len(F) != 3:
                raise ValueError(f"{'EB'[k]} must have 3 components (got {len(F)})")
            for c in range(3):
                arrs[3 * k + c] = F[c]
                mask |= 1 << (3 * k + c)
        ptrs, keep, where = self._ptr_array(arrs)
        check(fmx_set_fields(self.handle, mask, ptrs, where), "fmx_set_fields")
        del keep

    def set_current(self, J):
        if len(J) != 3:
            raise ValueError(f"J must have 3 components (got {len(J)})")
        ptrs, keep, where = self._ptr_array([J[0], J[1], J[2]])
        check(fmx_set_current(self.handle, ptrs, where), "fmx_set_current")
        del keep

    def set_current_profile(self, table):
        """j^{n+1/2} = table[k] * J for the next len(table) steps (fmx_set_current_profile)."""
        t = np.ascontiguousarray(table, dtype=np.float64)
        check(fmx_set_current_profile(self.handle, t.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), int(t.size)),
              "fmx_set_current_profile")

    def get_fields(self, mask=FMX_E | FMX_B, out=None, host_out=None):
        """Copies the components in mask to host numpy arrays (``host_out``
        when given, e.g. pinned memory, shape (9, nz, ny, nx)) or into the
        given device tensors ``out`` of that shape.  Returns E, B, J arrays of
        shape (3, nz, ny, nx) (None where not requested)."""
        nz, ny, nx = self.array_shape[1:]
        res = out if out is not None else (host_out if host_out is not None else
                                           np.zeros((9, nz, ny, nx), dtype=self.np_dtype))
        if len(res) != 9:
            raise ValueError(f"the output holds {len(res)} components, not 9 (E, B, J)")
        if out is not None and not _is_tensor(out):
            raise TypeError("out must be a CUDA tensor (host arrays go to host_out)")
        if out is None and not isinstance(res, np.ndarray):
            raise TypeError("host_out must be a numpy array")
        ptrs, keep, where = self._ptr_array([res[c] if mask & (1 << c) else None for c in range(9)], out=True)
        check(fmx_get_fields(self.handle, mask, ptrs, FMX_DEVICE if out is not None else FMX_HOST), "fmx_get_fields")
        del keep
        E = res[0:3] if mask & FMX_E else None
        B = res[3:6] if mask & FMX_B else None
        J = res[6:9] if mask & FMX_J else None
        return E, B, J

    # -- work ------------------------------------------------------------
    def step(self, nsteps=1):
        check(fmx_step(self.handle, int(nsteps)), "fmx_step")

    def set_option(self, option, value):
        check(fmx_set_option(self.handle, int(option), int(value)), "fmx_set_option")

    def get_option(self, option) -> int:
        return int(fmx_get_option(self.handle, int(option)))

    def step_host(self, steps):
        """fmx_step_host: ``steps`` is a list of (inputs, outputs), inputs a
        (9 or 6, nz, ny, nx) host array (E, B and optionally J; pinned memory
        lets the copies overlap), outputs a (6, nz, ny, nx) host array or
        None.  One step per entry; returns when every output is written."""
        recs = (fmx_host_step * len(steps))()
        keep = []
        for i, (inp, out) in enumerate(steps):
            # the library reads and writes these arrays in place: no conversion
            if not isinstance(inp, np.ndarray) or len(inp) not in (6, 9):
                raise ValueError(f"step {i}: inputs must be a host array of 6 or 9 components")
            if out is not None and (not isinstance(out, np.ndarray) or len(out) != 6):
                raise ValueError(f"step {i}: outputs must be a host array of 6 components or None")
            for arr in (inp,) + ((out,) if out is not None else ()):
                if arr.dtype != np.dtype(self.np_dtype) or not arr.flags.c_contiguous:
                    raise TypeError(f"step {i}: host arrays must be C-contiguous {np.dtype(self.np_dtype)}")
                if arr[0].size != self.cells:
                    raise ValueError(f"step {i}: {arr[0].size} elements per component, the grid {self.cells}")
            if out is not None and not out.flags.writeable:
                raise TypeError(f"step {i}: the output array is read-only")
            for c in range(9):
                recs[i].inp[c] = inp[c].ctypes.data if c < len(inp) else None
            for c in range(6):
                recs[i].out[c] = out[c].ctypes.data if out is not None else None
            keep.append((inp, out))
        check(fmx_step_host(self.handle, recs, len(steps)), "fmx_step_host")
        del keep

    def filter(self, mask, passes):
        check(fmx_filter(self.handle, int(mask), int(passes)), "fmx_filter")

    def sync(self):
        check(fmx_sync(self.handle), "fmx_sync")

    def diagnostics(self) -> dict:
        d = fmx_diag()
        check(fmx_diagnostics(self.handle, ctypes.byref(d)), "fmx_diagnostics")
        return {k: getattr(d, k) for k, _ in fmx_diag._fields_}

    def coefficients(self) -> np.ndarray:
        out = (ctypes.c_double * FMX_NCOEF)()
        check(fmx_coefficients(self.handle, out, FMX_NCOEF), "fmx_coefficients")
        return np.array(out[:])

    def profile(self, enable: bool):
        check(fmx_profile_enable(self.handle, int(bool(enable))), "fmx_profile_enable")

    def profile_read(self) -> list:
        arr = (fmx_kernel_stat * 4)()
        n = ctypes.c_int(0)
        check(fmx_profile_read(self.handle, arr, 4, ctypes.byref(n)), "fmx_profile_read")
        return [{"name": arr[i].name.decode(), "launches": arr[i].launches, "total_ms": arr[i].total_ms,
                 "bytes_per_launch": arr[i].bytes_per_launch} for i in range(n.value)]

    @property
    def dt(self) -> float:
        return fmx_time_step(self.handle)

    @property
    def launches(self) -> int:
        return int(fmx_launch_count(self.handle))

    def field_tensor(self, c: int):
        """Zero-copy torch view of component c (0..5 E/B current state, 6..8 J),
        shape (nz, ny, pitch)."""
        ptr = fmx_field_ptr(self.handle, c)
        if not ptr:
            return None
        base = self._slab.data_ptr()
        esz = self._slab.element_size()
        off = (ptr - base) // esz
        nx, ny, nz = self.shape + (1,) * (3 - len(self.shape))
        pitch = self.params.pitch or (nx + (16 // esz) - 1) // (16 // esz) * (16 // esz)
        return self._slab[off:off + pitch * ny * nz].view(nz, ny, pitch)


def coefficients_of(params: fmx_params) -> np.ndarray:
    """Coefficients of a parameter set (host only; creates and frees a handle)."""
    h = ctypes.c_void_p()
    check(fmx_create(ctypes.byref(params), ctypes.byref(h), None), "fmx_create")
    try:
        out = (ctypes.c_double * FMX_NCOEF)()
        check(fmx_coefficients(h, out, FMX_NCOEF), "fmx_coefficients")
        return np.array(out[:])
    finally:
        fmx_destroy(h)


def create_status(params: fmx_params):
    """Returns (status, warnings) of fmx_create for a parameter set (host only)."""
    h = ctypes.c_void_p()
    w = ctypes.c_int(0)
    s = fmx_create(ctypes.byref(params), ctypes.byref(h), ctypes.byref(w))
    if s == FMX_OK:
        fmx_destroy(h)
    return s, w.value


class Batch:
    """Many independent 2D FP32 grids advanced together (fmx_batch_*): one
    persistent launch per step, replayed from captured CUDA graphs.  Device
    buffers are PyTorch tensors; the batch runs on a stream of its own."""

    def __init__(self, shapes, courants, m=4, filter_passes=0, with_current=False, device="cuda", d=(1.0, 1.0)):
        import torch

        self.torch = torch
        self.device = torch.device(device)
        self.stream = torch.cuda.Stream(self.device)
        self.n = len(shapes)
        self.shapes = [tuple(int(v) for v in sh) for sh in shapes]
        params = (fmx_params * self.n)()
        for i, (sh, cf) in enumerate(zip(self.shapes, courants)):
            params[i] = make_params(sh, d=tuple(d) + (1.0,), courant=float(cf), precision=FMX_F32, m=m,
                                    filter_passes=filter_passes,
                                    filter_target=FMX_FILTER_CURRENT if with_current else FMX_FILTER_NONE,
                                    stream=ctypes.c_void_p(self.stream.cuda_stream))
        self.params = params
        h = ctypes.c_void_p()
        check(fmx_batch_create(params, self.n, ctypes.byref(h)), "fmx_batch_create")
        self.handle = h
        # one slab: per grid 12 state arrays (+3 current), each at a 256-byte boundary
        self.pitch = [(sh[0] + 3) // 4 * 4 for sh in self.shapes]
        sizes = [(p * sh[1] + 63) // 64 * 64 for p, sh in zip(self.pitch, self.shapes)]
        ncomp = 12 + (3 if with_current else 0)
        offs, tot = [], 0
        for sz in sizes:
            offs.append(tot)
            tot += ncomp * sz
        self._slab = torch.zeros(tot, dtype=torch.float32, device=self.device)
        base = self._slab.data_ptr()
        bufs = (fmx_buffers * self.n)()
        for i in range(self.n):
            ptr = lambda k: base + 4 * (offs[i] + k * sizes[i])
            for s_ in range(2):
                for c in range(3):
                    bufs[i].E[s_][c] = ptr(s_ * 6 + c)
                    bufs[i].B[s_][c] = ptr(s_ * 6 + 3 + c)
            for c in range(3):
                bufs[i].J[c] = ptr(12 + c) if with_current else None
        self._offs, self._sizes = offs, sizes
        wb = fmx_batch_workspace_bytes(self.handle)
        self._work = torch.zeros(wb + 256, dtype=torch.uint8, device=self.device)
        wbase = (self._work.data_ptr() + 255) // 256 * 256
        self.bufs = bufs
        torch.cuda.synchronize()
        check(fmx_batch_bind(self.handle, bufs, wbase, wb), "fmx_batch_bind")

    def close(self):
        if getattr(self, "handle", None):
            fmx_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_fields(self, i, E, B):
        nx, ny = self.shapes[i]
        if len(E) != 3 or len(B) != 3:
            raise ValueError("E and B must have 3 components each")
        keep = [np.ascontiguousarray(F[c], dtype=np.float32) for F in (E, B) for c in range(3)]
        if any(k.size != nx * ny for k in keep):
            raise ValueError(f"grid {i} has {nx * ny} cells per component")
        ptrs = (ctypes.c_void_p * 6)(*[k.ctypes.data for k in keep])
        check(fmx_batch_set_fields(self.handle, i, FMX_E | FMX_B, ptrs, FMX_HOST), "fmx_batch_set_fields")

    def set_current(self, i, J):
        """Writes grid i's current buffers directly (device copy on the batch stream)."""
        nx, ny = self.shapes[i]
        with self.torch.cuda.stream(self.stream):
            for c in range(3):
                o = self._offs[i] + (12 + c) * self._sizes[i]
                view = self._slab[o:o + self.pitch[i] * ny].view(ny, self.pitch[i])
                view[:, :nx].copy_(self.torch.from_numpy(np.ascontiguousarray(J[c][0], dtype=np.float32)))
        self.stream.synchronize()

    def get_fields(self, i):
        nx, ny = self.shapes[i]
        host = np.zeros((6, 1, ny, nx), dtype=np.float32)
        ptrs = (ctypes.c_void_p * 6)(*[host[c].ctypes.data for c in range(6)])
        check(fmx_batch_get_fields(self.handle, i, FMX_E | FMX_B, ptrs, FMX_HOST), "fmx_batch_get_fields")
        return host[:3], host[3:]

    def set_rows(self, rows):
        check(fmx_batch_set_rows(self.handle, int(rows)), "fmx_batch_set_rows")

    def set_tiles(self, narrow_rule):
        check(fmx_batch_set_tiles(self.handle, int(narrow_rule)), "fmx_batch_set_tiles")

    def tiles(self) -> dict:
        v = [ctypes.c_int(0) for _ in range(5)]
        check(fmx_batch_tiles(self.handle, *[ctypes.byref(x) for x in v]), "fmx_batch_tiles")
        return dict(zip(("wide", "narrow", "single", "rows", "narrow_rule"), (x.value for x in v)))

    def grid_width(self, i) -> int:
        """Columns one tile of grid i writes (fmx_batch_grid_width)."""
        return int(fmx_batch_grid_width(self.handle, int(i)))

    def tune(self, trial_steps=20) -> int:
        chosen = ctypes.c_int(0)
        check(fmx_batch_tune(self.handle, int(trial_steps), ctypes.byref(chosen)), "fmx_batch_tune")
        return chosen.value

    def step(self, nsteps=1):
        check(fmx_batch_step(self.handle, int(nsteps)), "fmx_batch_step")

    def sync(self):
        self.stream.synchronize()

    @property
    def items(self) -> int:
        return int(fmx_batch_items(self.handle))

    @property
    def launches(self) -> int:
        return int(fmx_batch_launch_count(self.handle))


def nci_params(dx=1.0, dy=1.0, c=1.0, courant=0.5, omega_p=1.0 / 16.0, shape_order=1, nu_max=1, nkx=4096):
    p = fmx_nci_params()
    p.dx, p.dy, p.c, p.courant, p.omega_p = float(dx), float(dy), float(c), float(courant), float(omega_p)
    p.shape_order, p.nu_max, p.nkx = int(shape_order), int(nu_max), int(nkx)
    return p


def nci_resonance(device="cuda", stream=None, **kw):
    """fmx_nci_resonance on torch buffers: returns dict kx [nkx], ky and gamma
    [2 nu_max + 1, nkx] (device tensors, FP64), best = (Gamma_max, k_x, k_y,
    nu) and nus.  Keyword arguments as ``nci_params``; enqueued on
    ``stream`` (default: torch's current stream) and synchronised."""
    import torch

    p = nci_params(**kw)
    dev = torch.device(device)
    if stream is None:
        stream = torch.cuda.current_stream(dev)
    rows = 2 * p.nu_max + 1
    kx = torch.empty(p.nkx, dtype=torch.float64, device=dev)
    ky = torch.empty((rows, p.nkx), dtype=torch.float64, device=dev)
    gamma = torch.empty((rows, p.nkx), dtype=torch.float64, device=dev)
    best = torch.empty(4, dtype=torch.float64, device=dev)
    check(fmx_nci_resonance(ctypes.byref(p), kx.data_ptr(), ky.data_ptr(), gamma.data_ptr(), best.data_ptr(),
                            ctypes.c_void_p(stream.cuda_stream)), "fmx_nci_resonance")
    stream.synchronize()
    return dict(kx=kx, ky=ky, gamma=gamma, best=tuple(best.tolist()), nus=list(range(-p.nu_max, p.nu_max + 1)))


def fma_peak(precision=FMX_F32, stream=None) -> float:
    """Measured FMA rate of the current device (flops/s) in FP32 or FP64
    (fmx_fma_peak), on `stream` (a torch stream; default: the current one)."""
    import torch
    stream = stream or torch.cuda.current_stream()
    out = ctypes.c_double(0.0)
    check(fmx_fma_peak(int(precision), ctypes.c_void_p(stream.cuda_stream), ctypes.byref(out)), "fmx_fma_peak")
    return out.value
