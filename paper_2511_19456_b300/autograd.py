"""torch.autograd.Function over the C-ABI: forward = |M|^2 (qed_eval_grad keeps
the gradient), backward = grad_out * d|M|^2/dk_j.

The gradient flows to the 3-momentum components (px, py, pz) of the outgoing
photons (slots 3..k+2) with their energies on shell, E_j = |k_j|; every other
entry of the momenta tensor gets a zero gradient.
"""
from __future__ import annotations

import torch


class QedM2(torch.autograd.Function):
    @staticmethod
    def forward(ctx, momenta, plan):
        if momenta.requires_grad:
            out, grad = plan.eval_grad(momenta.detach().contiguous())
            ctx.save_for_backward(grad)
        else:
            out = plan.eval(momenta.contiguous())
            ctx.save_for_backward(None)
        ctx.k = plan.k
        return out

    @staticmethod
    def backward(ctx, grad_out):
        (grad,) = ctx.saved_tensors
        full = torch.zeros((grad.shape[0], ctx.k + 3, 4), dtype=grad.dtype, device=grad.device)
        full[:, 3:, 1:] = grad_out[:, None, None] * grad
        return full, None


def m2(momenta, plan):
    """|M|^2 per point, differentiable with respect to the outgoing photons' 3-momenta."""
    return QedM2.apply(momenta, plan)
