"""torch.autograd.Function over the evaluation and its adjoint.

Forward: u = bem_eval(theta, xy).  Backward: d(loss)/d(theta) = bem_vjp(xy,
dloss/du), the reverse-mode adjoint of Sec. 3.2 (kernel values recomputed,
no samples x panels matrix stored).  Gradients flow to theta only; sample
positions are data.
"""
from __future__ import annotations

import torch

from . import BEM


class BemEval(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta: torch.Tensor, xy: torch.Tensor, model: BEM):
        th = theta.detach().to(torch.float64).contiguous()
        model.set_params(th)
        out = model.eval(xy)
        ctx.model = model
        ctx.save_for_backward(th, xy)
        return out

    @staticmethod
    def backward(ctx, grad_out):
        th, xy = ctx.saved_tensors
        m = ctx.model
        m.set_params(th)                       # the parameters of the forward call
        g = m.vjp(xy, grad_out.to(m.dtype).contiguous())
        return g.to(th.dtype), None, None


def bem_eval(theta: torch.Tensor, xy: torch.Tensor, model: BEM) -> torch.Tensor:
    """Differentiable colours [n, 3] of the handle parameters theta at xy."""
    return BemEval.apply(theta, xy, model)
