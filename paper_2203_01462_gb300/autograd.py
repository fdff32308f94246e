"""``torch.autograd.Function`` from the design densities rho to W~.

forward runs set_design + forward (checkpointing the fields as configured);
backward runs the adjoint solve, whose sensitivities (Eq. 25) and chain rule
(Eq. 27) give dW~/drho, and scales it by the incoming gradient.

W~ of Eq. (24) is tiny in SI units (~1e-32 for the 2048^2 workload) and its
per-node derivatives smaller still, below the FP32 range.  ``scale``
multiplies W~ and, in FP64 before the cast to rho's dtype, its gradient;
optimizers normally pass 1 / W~(rho0).

The adjoint needs the forward run of the same design and damping.  If the
solver ran another forward in between (two objectives evaluated before the
first backward, as in a line search), backward first runs the forward again
at the saved design, so the gradient always belongs to its own objective.
"""
from __future__ import annotations

import torch

from .binding import Solver


class FdtdObjective(torch.autograd.Function):
    @staticmethod
    def forward(ctx, rho: torch.Tensor, solver: Solver, sigma_max: float = 0.0, gamma_scale: float = 1.0,
                scale: float = 1.0):
        solver.set_design(rho.detach())
        solver.set_damping(sigma_max, gamma_scale)
        W = solver.forward().clone().reshape(()) * scale
        ctx.solver = solver
        ctx.generation = solver.generation
        ctx.rho = rho.detach().clone()
        ctx.damping = (sigma_max, gamma_scale)
        ctx.shape = rho.shape
        ctx.dtype = rho.dtype
        ctx.scale = scale
        return W

    @staticmethod
    def backward(ctx, gW: torch.Tensor):
        s: Solver = ctx.solver
        if s.generation != ctx.generation:
            s.set_design(ctx.rho)
            s.set_damping(*ctx.damping)
            s.forward()
            ctx.generation = s.generation
        s.adjoint()
        g = s.gradient()
        g = (g * (gW.to(g.dtype) * ctx.scale)).to(ctx.dtype).reshape(ctx.shape)
        return g, None, None, None, None


def objective(rho: torch.Tensor, solver: Solver, sigma_max: float = 0.0, gamma_scale: float = 1.0,
              scale: float = 1.0):
    """scale * W~(rho) as a differentiable FP64 scalar."""
    return FdtdObjective.apply(rho, solver, sigma_max, gamma_scale, scale)
