"""torch.autograd.Function over libptycho's loss and exact adjoint.

F(O, P) = sum_i sum_k (sqrt(I_i[k]) - |G(P, O)_i[k]|)^2   (Eq. 1)

The forward call evaluates F and both gradients in one pass of the library
(the adjoint needs the forward waves, which the library keeps in its own
workspace); backward scales the stored gradients by the incoming scalar.  The
library's gradient convention dF/dRe + i dF/dIm is PyTorch's, so the values
pass through unchanged.
"""
from __future__ import annotations

import torch

from .api import Plan, potential_grad, potential_to_transmission


class PtychoLoss(torch.autograd.Function):
    @staticmethod
    def forward(ctx, obj: torch.Tensor, probe: torch.Tensor, plan: Plan, pos: torch.Tensor,
                meas: torch.Tensor):
        need_o, need_p = ctx.needs_input_grad[0], ctx.needs_input_grad[1]
        loss, gO, gP = plan.loss_grad(pos, probe.detach(), obj.detach(), meas,
                                      want_obj=need_o, want_probe=need_p)
        ctx.save_for_backward(*(t for t in (gO, gP) if t is not None))
        ctx.has = (gO is not None, gP is not None)
        return loss

    @staticmethod
    def backward(ctx, grad_out):
        saved = list(ctx.saved_tensors)
        gO = saved.pop(0) if ctx.has[0] else None
        gP = saved.pop(0) if ctx.has[1] else None
        s = grad_out.to(torch.float32)
        return (gO * s if gO is not None else None, gP * s if gP is not None else None, None, None, None)


def ptycho_loss(obj: torch.Tensor, probe: torch.Tensor, plan: Plan, pos: torch.Tensor,
                meas: torch.Tensor) -> torch.Tensor:
    """Differentiable amplitude loss of Eq. 1 (float64 scalar)."""
    return PtychoLoss.apply(obj, probe, plan, pos, meas)


class PtychoLossPotential(torch.autograd.Function):
    """F as a function of the real potential V (O = exp(i sigma V)) and the probe."""

    @staticmethod
    def forward(ctx, V: torch.Tensor, probe: torch.Tensor, plan: Plan, pos: torch.Tensor, meas: torch.Tensor,
                sigma: float):
        O = potential_to_transmission(V.detach(), sigma)
        loss, gO, gP = plan.loss_grad(pos, probe.detach(), O, meas, want_obj=ctx.needs_input_grad[0],
                                      want_probe=ctx.needs_input_grad[1])
        gV = potential_grad(O, gO, sigma) if gO is not None else None
        ctx.save_for_backward(*(t for t in (gV, gP) if t is not None))
        ctx.has = (gV is not None, gP is not None)
        return loss

    @staticmethod
    def backward(ctx, grad_out):
        saved = list(ctx.saved_tensors)
        gV = saved.pop(0) if ctx.has[0] else None
        gP = saved.pop(0) if ctx.has[1] else None
        s = grad_out.to(torch.float32)
        return (gV * s if gV is not None else None, gP * s if gP is not None else None, None, None, None, None)


def ptycho_loss_potential(V, probe, plan, pos, meas, sigma: float = 1.0):
    """Differentiable loss of Eq. 1 in terms of the real potential V."""
    return PtychoLossPotential.apply(V, probe, plan, pos, meas, sigma)
