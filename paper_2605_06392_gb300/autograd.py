"""``torch.autograd.Function`` around the hand-written adjoint.

Forward runs the value-only evaluation (both factorisations, the mode, f;
Eq. 1) and leaves the factors in the model.  Backward runs the reverse pass
of Eq. 6 in the library: the two selected inversions overwrite those
factors in place with the fused Phase A / C traces, Phase B comes from the
stencil quadratic forms of the forward, and the result is scaled by the
incoming gradient.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from ._capi import check, lib


class InlaFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta: torch.Tensor, model):
        th = theta.detach().to("cpu", torch.float64).contiguous().numpy()
        f = model.value(th)
        ctx.model = model
        ctx.theta = th.copy()
        ctx.token = getattr(model, "_eval_token", 0) + 1
        model._eval_token = ctx.token
        return theta.new_tensor(f, dtype=torch.float64)

    @staticmethod
    def backward(ctx, grad_out):
        model = ctx.model
        g = np.zeros(model.d)
        if getattr(model, "_eval_token", None) == ctx.token:
            code = lib().inla_backward(model.handle, g.ctypes.data_as(C.POINTER(C.c_double)), 1,
                                       C.c_void_p(torch.cuda.current_stream().cuda_stream))
            check(code, "inla_backward")
            model._eval_token = None          # the factors were consumed
        else:
            # another evaluation overwrote the factors: redo value and gradient
            _, g = model.value_and_grad(ctx.theta)
        grad = torch.from_numpy(g).to(grad_out.device, torch.float64)
        return grad_out * grad, None


def inla_objective(theta: torch.Tensor, model) -> torch.Tensor:
    """f(theta) as a differentiable scalar (FP64)."""
    return InlaFn.apply(theta, model)
