"""Differentiable field advance driven by a Gaussian-envelope current.

j_z^{n+1/2}(r) = sum_p theta_p sin(omega0 (n + 1/2) dt + phi_p) G_p(r),
G_p(r) = exp(-|r - c_p|^2 / (2 w^2)), on a 2D periodic grid.  The forward
pass runs N steps through the C ABI (fmx_gauss_run: source synthesis from
theta and the phases on the device, then the step); the backward pass runs N
adjoint steps (fmx_gauss_adjoint_run: fmx_adjoint_step, the hand-written
transpose of the step, then the projection of dL/dj_z on the G_p, weighted
and accumulated on the device).

Checkpointing: the forward keeps the state every `checkpoint_every` steps,
O(N / K) states, and the backward walks the segments in reverse.  The step
is linear and does not depend on the state, so its adjoint needs no forward
state; with recompute=True the backward re-runs each segment forward from its
checkpoint and checks that it lands exactly on the next checkpoint, which is
where a state-dependent step would take its linearisation point.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import fmx


class GaussSourceRun:
    def __init__(self, shape, cxy, phases, nsteps, width=8.0, omega0=0.2, m=4, passes=3, courant=0.5,
                 precision=fmx.FMX_F32, checkpoint_every=50, engine=fmx.FMX_ENGINE_AUTO):
        import torch

        self.torch = torch
        self.shape = tuple(int(v) for v in shape)
        self.cxy = np.ascontiguousarray(np.asarray(cxy, dtype=np.float64))
        self.phases = np.asarray(phases, dtype=np.float64)
        self.np_ = len(self.phases)
        self.nsteps = int(nsteps)
        self.width = float(width)
        self.omega0 = float(omega0)
        self.K = max(1, int(checkpoint_every))
        self.grid = fmx.Grid(self.shape, precision=precision, m=m, filter_passes=passes, courant=courant,
                             engine=engine)
        g = self.grid
        self.dt = g.dt
        nx, ny = self.shape
        esz = 8 if precision == fmx.FMX_F64 else 4
        q = 16 // esz
        self.pitch = (nx + q - 1) // q * q
        dev = g.device
        wb = fmx.fmx_adjoint_workspace_bytes(ctypes.byref(g.params))
        self._awork = torch.zeros(wb + 256, dtype=torch.uint8, device=dev)
        self._awork_ptr = (self._awork.data_ptr() + 255) // 256 * 256
        self._awork_bytes = wb
        self.Ebar = torch.zeros((3, ny, self.pitch), dtype=g.dtype, device=dev)
        self.Bbar = torch.zeros_like(self.Ebar)
        self.jbar = torch.zeros_like(self.Ebar)
        self.launches = 0

    # ------------------------------------------------------------------
    def _state(self):
        out = self.torch.empty((9, 1) + self.shape[::-1], dtype=self.grid.dtype, device=self.grid.device)
        E, B, _ = self.grid.get_fields(fmx.FMX_E | fmx.FMX_B, out=out)
        return E[:, 0].clone(), B[:, 0].clone()

    def _setup(self, theta):
        th = np.ascontiguousarray(np.asarray(theta, dtype=np.float64))
        dp = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        fmx.check(fmx.fmx_gauss_setup(self.grid.handle, self.np_, dp(self.cxy), dp(th),
                                      dp(np.ascontiguousarray(self.phases)), self.width, self.omega0),
                  "fmx_gauss_setup")

    def forward(self, theta, E0, B0):
        """E0, B0: device tensors (3, ny, nx).  Returns (E^N, B^N) and keeps
        the checkpoints (state before steps 0, K, 2K, ...).  Each segment of
        K steps is one fmx_gauss_run call (source synthesis and step on the
        device, no host synchronisation inside)."""
        g = self.grid
        g.set_fields(E0.reshape((3, 1) + E0.shape[1:]), B0.reshape((3, 1) + B0.shape[1:]))
        self._setup(theta)
        self.checkpoints = {}
        l0 = g.launches
        for n in range(0, self.nsteps, self.K):
            self.checkpoints[n] = self._state()
            k = min(self.K, self.nsteps - n)
            fmx.check(fmx.fmx_gauss_run(g.handle, n, k), "fmx_gauss_run")
        self.launches += g.launches - l0
        return self._state()

    def backward(self, theta, gE, gB, recompute=False):
        """gE, gB = dL/d(E^N, B^N) (device tensors (3, ny, nx)).  Returns
        dL/dtheta (numpy), dL/dE^0, dL/dB^0 (device tensors)."""
        nx, ny = self.shape
        g = self.grid
        self.Ebar.zero_()
        self.Bbar.zero_()
        self.Ebar[:, :, :nx].copy_(gE)
        self.Bbar[:, :, :nx].copy_(gB)
        grad = np.zeros(self.np_)
        self._setup(theta)
        vp = lambda t: (ctypes.c_void_p * 3)(*[t[c].data_ptr() for c in range(3)])
        starts = sorted(self.checkpoints)
        l0 = g.launches
        for si in range(len(starts) - 1, -1, -1):
            s0 = starts[si]
            s1 = starts[si + 1] if si + 1 < len(starts) else self.nsteps
            if recompute:
                E, B = self.checkpoints[s0]
                g.set_fields(E.reshape((3, 1, ny, nx)), B.reshape((3, 1, ny, nx)))
                fmx.check(fmx.fmx_gauss_run(g.handle, s0, s1 - s0), "fmx_gauss_run")
                if s1 in self.checkpoints:
                    E1, B1 = self._state()
                    assert self.torch.equal(E1, self.checkpoints[s1][0]) and \
                        self.torch.equal(B1, self.checkpoints[s1][1]), "recomputed segment left its checkpoint"
            fmx.check(fmx.fmx_gauss_adjoint_run(g.handle, s0, s1 - s0, vp(self.Ebar), vp(self.Bbar), vp(self.jbar),
                                                self._awork_ptr, self._awork_bytes, int(si == len(starts) - 1)),
                      "fmx_gauss_adjoint_run")
        if starts:
            fmx.check(fmx.fmx_gauss_accumulated(g.handle, self.np_, grad.ctypes.data_as(ctypes.POINTER(ctypes.c_double))),
                      "fmx_gauss_accumulated")
        self.launches += g.launches - l0
        return grad, self.Ebar[:, :, :nx].clone(), self.Bbar[:, :, :nx].clone()


def make_function():
    """torch.autograd.Function: (theta, E0, B0) -> (E^N, B^N) through a GaussSourceRun."""
    import torch

    class FieldRun(torch.autograd.Function):
        @staticmethod
        def forward(ctx, theta, E0, B0, run, recompute):
            th = theta.detach().cpu().numpy().astype(np.float64)
            EN, BN = run.forward(th, E0.detach(), B0.detach())
            ctx.run, ctx.theta, ctx.recompute = run, th, recompute
            ctx.theta_meta = (theta.dtype, theta.device)
            return EN, BN

        @staticmethod
        def backward(ctx, gE, gB):
            grad, gE0, gB0 = ctx.run.backward(ctx.theta, gE.contiguous(), gB.contiguous(), ctx.recompute)
            # dL/dtheta is accumulated in FP64 on the host; autograd wants it
            # with theta's own dtype and device
            dtype, device = ctx.theta_meta
            return torch.from_numpy(grad).to(dtype=dtype, device=device), gE0, gB0, None, None

    return FieldRun
