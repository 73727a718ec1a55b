"""torch.autograd binding of the hand-written RLBM adjoint.

``CalibrationRun`` owns a Lattice with a per-cell relaxation-time field and
an Adjoint; ``shear_loss`` returns L = 1/2 sum |u(T) - u_target|^2 as a torch
scalar whose backward runs the checkpointed adjoint kernels and returns
gradients for the tau field and the initial velocity.  All arrays are float64
CUDA tensors of shape (ny, nx).
"""
from __future__ import annotations

import torch

from .rlbm import Adjoint, Lattice


class CalibrationRun:
    def __init__(self, nx, ny, nsteps, checkpoint_every=100, precision="fp32", stream="onlattice", lam=0.0,
                 m=0.0, order=2):
        self.nx, self.ny, self.nsteps = nx, ny, nsteps
        self.lat = Lattice(nx, ny, m=m, order=order, tau_mode="field", precision=precision, stream=stream,
                           lam=lam, cuda_stream=torch.cuda.current_stream().cuda_stream)
        self.adj = Adjoint(self.lat, nsteps, checkpoint_every)

    def close(self):
        self.adj.close()
        self.lat.close()


class _ShearLoss(torch.autograd.Function):
    @staticmethod
    def forward(ctx, tau, ux0, uy0, n0, T0, ux_t, uy_t, run):
        run.lat.set_tau_field(tau.detach().contiguous())
        run.adj.forward(n0.contiguous(), ux0.detach().contiguous(), uy0.detach().contiguous(), T0.contiguous())
        f = {k: torch.empty_like(n0) for k in ("n", "ux", "uy", "T", "eps")}
        run.lat.moments(out=f)
        ctx.run = run
        ctx.save_for_backward(ux_t, uy_t)
        return 0.5 * ((f["ux"] - ux_t) ** 2 + (f["uy"] - uy_t) ** 2).sum()

    @staticmethod
    def backward(ctx, gout):
        ux_t, uy_t = ctx.saved_tensors
        run = ctx.run
        out = {"loss": torch.zeros(1, dtype=torch.float64, device=ux_t.device),
               "tau": torch.empty_like(ux_t), "ux0": torch.empty_like(ux_t), "uy0": torch.empty_like(ux_t)}
        run.adj.backward(ux_t.contiguous(), uy_t.contiguous(), out=out)
        return gout * out["tau"], gout * out["ux0"], gout * out["uy0"], None, None, None, None, None


def shear_loss(run, tau, ux0, uy0, n0, T0, ux_t, uy_t):
    """L(tau, u0) with gradients through the hand-written adjoint."""
    return _ShearLoss.apply(tau, ux0, uy0, n0, T0, ux_t, uy_t, run)
