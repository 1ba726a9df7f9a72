"""ctypes front end of the FP64 C oracle (``fmx_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``.  The product package never imports
it.  Arrays are numpy float64 of shape ``(3, nz, ny, nx)`` (x fastest), one
plane per component, at the Yee positions of the variable list in Sec. 2 of
the paper.
"""
from __future__ import annotations

import contextlib
import ctypes
import dataclasses
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fmx_oracle.c")
_HDR = os.path.join(_HERE, "fmx_oracle.h")
_LIB = os.path.join(_HERE, "_build", "libfmx_oracle.so")
_lock = threading.Lock()
_lib = None

FILTER_NONE, FILTER_CURRENT, FILTER_FIELDS = 0, 1, 2
OK, ENOCONV = 0, 3
COEF_NAMES = ("kx", "ky", "kz", "q", "c6", "ax", "ay", "az", "ayz", "azx", "axy", "byz", "bzx", "bxy")


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (C, -O2, OpenMP, no FMA contraction)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    fresh = os.path.exists(_LIB) and all(
        os.path.getmtime(_LIB) >= os.path.getmtime(f) for f in (_SRC, _HDR))
    if fresh and not force:
        return _LIB
    tmp = _LIB + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off", "-std=gnu11",
           _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


class _Params(ctypes.Structure):
    _fields_ = [("dims", ctypes.c_int), ("n", ctypes.c_long * 3), ("d", ctypes.c_double * 3),
                ("c", ctypes.c_double), ("dt", ctypes.c_double), ("m", ctypes.c_int),
                ("residual", ctypes.c_int), ("tol", ctypes.c_double), ("m_max", ctypes.c_int),
                ("filter_passes", ctypes.c_int), ("filter_target", ctypes.c_int),
                ("lumped", ctypes.c_int), ("coef_f32", ctypes.c_int), ("cheb", ctypes.c_int),
                ("cheb_lo", ctypes.c_double), ("cheb_hi", ctypes.c_double)]


class _Stats(ctypes.Structure):
    _fields_ = [("last_sweeps", ctypes.c_int), ("total_sweeps", ctypes.c_int),
                ("last_resid", ctypes.c_double)]


def _configure(lib):
    P = ctypes.POINTER(_Params)
    dp = ctypes.POINTER(ctypes.c_double)
    lib.orc_threads.argtypes = [ctypes.c_int]
    lib.orc_threads.restype = ctypes.c_int
    lib.orc_dt_cfl.argtypes = [P]
    lib.orc_dt_cfl.restype = ctypes.c_double
    lib.orc_coefficients.argtypes = [P, dp]
    lib.orc_filter.argtypes = [P, dp, ctypes.c_int, ctypes.c_int]
    lib.orc_source.argtypes = [P, dp, dp, dp]
    lib.orc_apply_A.argtypes = [P, dp, dp]
    lib.orc_solve.argtypes = [P, dp, dp, ctypes.POINTER(ctypes.c_int), dp]
    lib.orc_solve.restype = ctypes.c_int
    lib.orc_faraday.argtypes = [P, dp, dp]
    lib.orc_step.argtypes = [P, dp, dp, dp, ctypes.c_int, ctypes.POINTER(_Stats)]
    lib.orc_step.restype = ctypes.c_int
    lib.orc_div_b.argtypes = [P, dp, dp]
    lib.orc_gauss_e.argtypes = [P, dp, dp]
    lib.orc_energy.argtypes = [P, dp, dp, dp, dp]
    lib.orc_adjoint_step.argtypes = [P, dp, dp, dp]
    lib.orc_adjoint_step.restype = ctypes.c_int
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _configure(ctypes.CDLL(build()))
    return _lib


@contextlib.contextmanager
def using_library(path: str):
    """Temporarily route every call to another build of the oracle source
    (the mutation tests compile deliberately broken copies)."""
    global _lib
    prev = _load()
    with _lock:
        _lib = _configure(ctypes.CDLL(path))
    try:
        yield
    finally:
        with _lock:
            _lib = prev


def compile_variant(source_text: str, out_path: str) -> str:
    """Compile a (modified) copy of the oracle source to out_path."""
    d = os.path.dirname(out_path)
    src = os.path.join(d, "variant.c")
    with open(src, "w") as f:
        f.write(source_text)
    subprocess.run(["gcc", "-O1", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off", "-std=gnu11",
                    "-I", _HERE, src, "-o", out_path, "-lm"], check=True)
    return out_path


def source_text() -> str:
    with open(_SRC) as f:
        return f.read()


@dataclasses.dataclass
class Params:
    """Problem description for the oracle.

    ``shape`` is (nx,), (nx, ny) or (nx, ny, nz); its length is the number of
    active axes.  ``dt`` wins over ``courant`` (the fraction of dt_CFL,
    Eq. dt_cfl_3d and its 2D form) when it is given."""
    shape: tuple
    d: tuple = (1.0, 1.0, 1.0)
    c: float = 1.0
    dt: float | None = None
    courant: float = 0.5
    m: int = 4
    residual: bool = False
    tol: float = 1e-13
    m_max: int = 10000
    filter_passes: int = 0
    filter_target: int = FILTER_CURRENT
    lumped: bool = False
    coef_f32: bool = False
    cheb: bool = False  # Chebyshev acceleration of the solve (spectral.a_interval)

    @property
    def dims(self) -> int:
        return len(self.shape)

    @property
    def n3(self) -> tuple:
        s = tuple(self.shape) + (1,) * (3 - len(self.shape))
        return s

    @property
    def array_shape(self) -> tuple:
        nx, ny, nz = self.n3
        return (3, nz, ny, nx)

    def dt_cfl(self) -> float:
        s = 0.0
        for a in range(self.dims):
            s += 1.0 / (self.d[a] * self.d[a])
        return 1.0 / (self.c * math.sqrt(s))

    def time_step(self) -> float:
        return float(self.dt) if self.dt is not None else self.courant * self.dt_cfl()

    def _c(self) -> _Params:
        p = _Params()
        p.dims = self.dims
        for a in range(3):
            p.n[a] = self.n3[a]
            p.d[a] = float(self.d[a]) if a < len(self.d) else 1.0
        p.c = self.c
        p.dt = self.time_step()
        p.m = self.m
        p.residual = int(self.residual)
        p.tol = self.tol
        p.m_max = self.m_max
        p.filter_passes = self.filter_passes
        p.filter_target = self.filter_target
        p.lumped = int(self.lumped)
        p.coef_f32 = int(self.coef_f32)
        p.cheb = int(self.cheb)
        if self.cheb:
            from . import spectral
            p.cheb_lo, p.cheb_hi = spectral.a_interval(self)
        return p


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _field(p: Params, a, name: str) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if a.shape != p.array_shape:
        a = a.reshape(p.array_shape)
    return a.copy()


def threads(n: int = 0) -> int:
    return _load().orc_threads(int(n))


def dt_cfl(p: Params) -> float:
    cp = p._c()
    return _load().orc_dt_cfl(ctypes.byref(cp))


def coefficients(p: Params) -> dict:
    out = np.zeros(len(COEF_NAMES))
    cp = p._c()
    _load().orc_coefficients(ctypes.byref(cp), _dp(out))
    return dict(zip(COEF_NAMES, out.tolist()))


def filter(p: Params, f: np.ndarray, passes: int) -> np.ndarray:
    f = np.ascontiguousarray(np.array(f, dtype=np.float64))
    ncomp = f.size // int(np.prod(p.n3))
    cp = p._c()
    _load().orc_filter(ctypes.byref(cp), _dp(f), ncomp, passes)
    return f


def source(p: Params, B, J=None) -> np.ndarray:
    B = _field(p, B, "B")
    Jc = _field(p, J, "J") if J is not None else None
    out = np.zeros(p.array_shape)
    cp = p._c()
    _load().orc_source(ctypes.byref(cp), _dp(B), _dp(Jc) if Jc is not None else None, _dp(out))
    return out


def apply_A(p: Params, dE) -> np.ndarray:
    dE = _field(p, dE, "dE")
    out = np.zeros(p.array_shape)
    cp = p._c()
    _load().orc_apply_A(ctypes.byref(cp), _dp(dE), _dp(out))
    return out


def solve(p: Params, dEp):
    dEp = _field(p, dEp, "dEp")
    out = np.zeros(p.array_shape)
    sw = ctypes.c_int(0)
    r = ctypes.c_double(0.0)
    cp = p._c()
    rc = _load().orc_solve(ctypes.byref(cp), _dp(dEp), _dp(out), ctypes.byref(sw), ctypes.byref(r))
    return out, rc, sw.value, r.value


def faraday(p: Params, E, B) -> np.ndarray:
    E = _field(p, E, "E")
    B = _field(p, B, "B")
    cp = p._c()
    _load().orc_faraday(ctypes.byref(cp), _dp(E), _dp(B))
    return B


def step(p: Params, E, B, J=None, nsteps: int = 1):
    """Advance (E^n, B^{n+1/2}) by nsteps.  Returns (E, B, rc, stats)."""
    E = _field(p, E, "E")
    B = _field(p, B, "B")
    Jc = _field(p, J, "J") if J is not None else None
    st = _Stats()
    cp = p._c()
    rc = _load().orc_step(ctypes.byref(cp), _dp(E), _dp(B), _dp(Jc) if Jc is not None else None,
                          int(nsteps), ctypes.byref(st))
    return E, B, rc, {"last_sweeps": st.last_sweeps, "total_sweeps": st.total_sweeps,
                      "last_resid": st.last_resid}


def div_b(p: Params, B) -> np.ndarray:
    B = _field(p, B, "B")
    out = np.zeros(p.array_shape[1:])
    cp = p._c()
    _load().orc_div_b(ctypes.byref(cp), _dp(B), _dp(out))
    return out


def gauss_e(p: Params, E) -> np.ndarray:
    E = _field(p, E, "E")
    out = np.zeros(p.array_shape[1:])
    cp = p._c()
    _load().orc_gauss_e(ctypes.byref(cp), _dp(E), _dp(out))
    return out


def energy(p: Params, E, B):
    E = _field(p, E, "E")
    B = _field(p, B, "B")
    ws = ctypes.c_double(0.0)
    wp = ctypes.c_double(0.0)
    cp = p._c()
    _load().orc_energy(ctypes.byref(cp), _dp(E), _dp(B), ctypes.byref(ws), ctypes.byref(wp))
    return ws.value, wp.value


def adjoint_step(p: Params, Ebar, Bbar):
    """One adjoint step: returns (dL/dE^n, dL/dB^{n+1/2}, dL/dj) from
    dL/d(E^{n+1}, B^{n+3/2}).  Fixed m only."""
    Eb = _field(p, Ebar, "Ebar")
    Bb = _field(p, Bbar, "Bbar")
    jb = np.zeros(p.array_shape)
    cp = p._c()
    rc = _load().orc_adjoint_step(ctypes.byref(cp), _dp(Eb), _dp(Bb), _dp(jb))
    if rc != 0:
        raise ValueError("the oracle adjoint covers fixed m without field filtering")
    return Eb, Bb, jb
