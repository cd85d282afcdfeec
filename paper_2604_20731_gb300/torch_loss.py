"""The CRVPINN robust loss as a differentiable PyTorch function.

LOSS(theta) = RES^T G^-1 RES (Sec. 5, Eqs. 25-28) for the collocation
coefficients the solver holds (set them with `update_coefficients()` from the
current saturation).  The forward and the gradient both run in the library's
kernels:
- the network forward, the residual and the Gram solve compute the loss;
- the adjoint stencil gives dLOSS/du = 2 A z;
- the hand-written network backward pulls that back to dLOSS/dtheta.

This module only moves theta in and the loss and gradient out.  Loading theta
resets the context's own Adam state, which an external optimiser does not use.
"""
from __future__ import annotations

import torch


class CrvpinnLoss(torch.autograd.Function):
    """forward(theta, solver) -> LOSS; backward -> grad_out * dLOSS/dtheta."""

    @staticmethod
    def forward(ctx, theta: torch.Tensor, solver) -> torch.Tensor:
        if theta.dim() != 1 or theta.numel() != solver.nparams:
            raise ValueError(f"theta must be a vector of {solver.nparams} parameters")
        solver.set_theta(theta.detach().to("cpu", torch.float64).numpy())
        loss = solver.loss_grad()
        grad = torch.as_tensor(solver.get("GRAD"), dtype=theta.dtype, device=theta.device)
        ctx.save_for_backward(grad)
        return torch.tensor(loss, dtype=theta.dtype, device=theta.device)

    @staticmethod
    def backward(ctx, grad_out: torch.Tensor):
        (grad,) = ctx.saved_tensors
        return grad_out * grad, None


def crvpinn_loss(solver, theta: torch.Tensor) -> torch.Tensor:
    """LOSS(theta) with the hand-written adjoint as its gradient."""
    return CrvpinnLoss.apply(theta, solver)
