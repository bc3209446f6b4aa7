"""torch.autograd.Function over the library's hand-written adjoint.

``scalar_loss(h, T0, U, V, W, nsteps, checkpoint_every, wnu, wvar)`` sets the
coarse velocity and the initial scalar on handle ``h``, runs ``nsteps`` steps
with checkpoints every ``checkpoint_every`` steps, and returns the loss
    L = sum_s wnu[s] Nu_bot(T^s) + wvar[s] Var(T^s)
as a 0-d FP64 CUDA tensor.  ``L.backward()`` calls the adjoint sweep of the
CUDA library and delivers dL/dT0 (dense) and dL/dU, dL/dV, dL/dW (coarse).
Every step of the computation runs in libmr.so; this module only marshals.
"""
from __future__ import annotations

import torch

from . import mr


class _ScalarLoss(torch.autograd.Function):
    @staticmethod
    def forward(ctx, T0, U, V, W, h, nsteps, checkpoint_every, wnu, wvar):
        mr.mr_refine_velocity(h, U.detach().contiguous(), V.detach().contiguous(), W.detach().contiguous())
        mr.mr_set_scalar(h, T0.detach().contiguous())
        loss = mr.mr_adjoint_forward(h, nsteps, checkpoint_every, wnu, wvar)
        ctx.h = h
        ctx.meta = (T0.shape, T0.dtype, U.shape, V.shape, W.shape, T0.device)
        return torch.tensor(loss, dtype=torch.float64, device=T0.device)

    @staticmethod
    def backward(ctx, gout):
        tshape, tdtype, ushape, vshape, wshape, device = ctx.meta
        gT0 = torch.empty(tshape, dtype=tdtype, device=device)
        gU = torch.empty(ushape, dtype=torch.float64, device=device)
        gV = torch.empty(vshape, dtype=torch.float64, device=device)
        gW = torch.empty(wshape, dtype=torch.float64, device=device)
        mr.mr_adjoint_backward(ctx.h, float(gout), gT0, gU, gV, gW)
        return gT0, gU, gV, gW, None, None, None, None, None


def scalar_loss(h, T0, U, V, W, nsteps, checkpoint_every, wnu=None, wvar=None):
    return _ScalarLoss.apply(T0, U, V, W, h, nsteps, checkpoint_every, wnu, wvar)
