"""Design-optimization loop around the CUDA path (Sec. 3.2, Eq. 28).

The paper maximises W~ over 0 < rho < 1 with GCMMA, inner / outer loops, a
grayness stop zeta < 0.5 % and a final threshold at 0.5.  This driver keeps
the problem, the artificial-damping continuation, zeta and the threshold, and
replaces GCMMA by a projected, normalised gradient-ascent step with a move
limit (``fdtd_ascent_step``).  Every array operation runs in the library's
kernels; Python only sequences the calls.
"""
from __future__ import annotations

import dataclasses
import math
import time

import torch

from .binding import Solver


def damping_schedule(k: int, start: float = 10.0, iters: int = 50) -> float:
    """Collision-rate factor: start x decaying geometrically to 1 over ``iters`` iterations."""
    if iters <= 0 or k >= iters:
        return 1.0
    return start ** (1.0 - k / iters)


@dataclasses.dataclass
class History:
    W: list = dataclasses.field(default_factory=list)
    zeta: list = dataclasses.field(default_factory=list)
    gamma_scale: list = dataclasses.field(default_factory=list)
    kind: list = dataclasses.field(default_factory=list)   # "adjoint" or "surrogate"
    seconds: list = dataclasses.field(default_factory=list)


def gradient_step(s: Solver, rho: torch.Tensor, sigma_max: float, gamma_scale: float):
    """One FDTD evaluation: W~ (FP64 scalar tensor), dW~/drho (FP64), zeta."""
    W, g = s.evaluate(rho, sigma_max, gamma_scale)
    zeta = s.grayness()
    return W, g, zeta


def optimize(s: Solver, rho0, iters: int, move: float = 0.05, sigma_max: float = 0.0,
             damping_start: float = 10.0, damping_iters: int = 50, zeta_stop: float = 0.005,
             move_decay: float = 0.98) -> tuple[torch.Tensor, History]:
    """Plain adjoint loop: every iteration runs forward + adjoint + gradient
    and one ascent step.  Stops after ``iters`` iterations or when zeta falls
    below ``zeta_stop``.  Returns the final (unthresholded) design and the
    history."""
    rho = torch.as_tensor(rho0, device=s.device).to(s.real).contiguous().clone()
    h = History()
    t0 = time.perf_counter()
    for k in range(iters):
        gs = damping_schedule(k, damping_start, damping_iters)
        W, g, zeta = gradient_step(s, rho, sigma_max, gs)
        s.ascent_step(rho, g, move * move_decay ** k)
        h.W.append(float(W.item()))
        h.zeta.append(float(zeta.item()))
        h.gamma_scale.append(gs)
        h.kind.append("adjoint")
        h.seconds.append(time.perf_counter() - t0)
        if h.zeta[-1] < zeta_stop:
            break
    return rho, h


def final_design(s: Solver, rho: torch.Tensor, level: float = 0.5):
    """Threshold the design (the paper's last step) and evaluate it without damping."""
    r = rho.clone()
    s.threshold(r, level)
    s.set_design(r)
    s.set_damping(0.0, 1.0)
    W = s.forward().clone()
    s.sync()
    return r, float(W.item())
