"""The sliding-step criterion as a differentiable torch function.

C(mu) = 1/2 |y - Phi mu|^2 + lambda sum_n w_n (Eq. 4) of the atom parameters
[m (N x 3) | sigma (N) | d (N) | w (N)] (the 6N variables of the local descent,
step 4 of Algorithm 1 and step 2b of Algorithm 2).  The gradient is the
library's hand-written adjoint (Section 2: "grad C is computed analytically").

forward computes the loss only (render, blur, residual); backward recomputes
the rendered atom field and runs the transposed blur and the per-atom adjoint
sums.  Nothing per atom (and no volume) is kept between the two passes: the
saved state is the 6N parameters.
"""

from __future__ import annotations

import torch

from . import AtomSet, Plan


class SlideLoss(torch.autograd.Function):
    @staticmethod
    def forward(ctx, params: torch.Tensor, y: torch.Tensor, plan: Plan, lam: float):
        if params.dim() != 1 or params.numel() % 6 or not params.is_cuda:
            raise ValueError("params must be a CUDA vector of 6N entries [m | sigma | d | w]")
        atoms = AtomSet.from_params(params.detach(), device=params.device)
        loss, _, _ = plan.slide_loss_grad(y, atoms, lam, want_grad=False)
        ctx.save_for_backward(params.detach())
        ctx.plan, ctx.y, ctx.lam = plan, y, lam
        return loss[0].to(params.dtype)

    @staticmethod
    def backward(ctx, gout):
        (params,) = ctx.saved_tensors
        atoms = AtomSet.from_params(params, device=params.device)
        _, grad, _ = ctx.plan.slide_loss_grad(ctx.y, atoms, ctx.lam)
        return (gout * grad).to(params.dtype), None, None, None


def slide_loss(params: torch.Tensor, y: torch.Tensor, plan: Plan, lam: float) -> torch.Tensor:
    """Differentiable sliding-step criterion C(params) (a 0-dim tensor)."""
    return SlideLoss.apply(params, y, plan, lam)
