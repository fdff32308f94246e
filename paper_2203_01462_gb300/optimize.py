"""Design-optimization loops around the CUDA path (Sec. 3.2, Eq. 28).

The paper maximises W~ over 0 < rho < 1 with GCMMA.  A subproblem ends once
at least 12 iterations have run and the norm of the first-order optimality
residual has fallen by 70 %; the optimization ends when the grayness zeta
falls below 0.5 % or after 600 iterations; the design is then thresholded at
0.5.  The artificial damping is temporary (Sec. 2.2).

* ``optimize_gcmma`` follows that structure: one subproblem per damping level
  (a geometric continuation from x10 to x1), each solved by GCMMA iterations
  whose per-variable work runs in ``fdtd_mma_asymptotes`` / ``fdtd_mma_solve``;
  each inner GCMMA iteration costs one forward solve, each accepted point one
  adjoint.  It can write and resume from a checkpoint file.
* ``optimize`` is the simpler loop used by the surrogate comparison: one
  projected, normalised gradient-ascent step (``fdtd_ascent_step``) per
  forward + adjoint, with the damping decaying every iteration.

Every array operation runs in the library's kernels; Python only sequences
the calls and makes the scalar decisions.
"""
from __future__ import annotations

import dataclasses
import math
import os
import time

import numpy as np

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


def damping_levels(start: float = 10.0, stages: int = 6) -> list:
    """Damping factors of the continuation: ``start`` decaying geometrically to 1 in ``stages`` levels."""
    if stages <= 1:
        return [1.0]
    return [start ** (1.0 - j / (stages - 1)) for j in range(stages)]


def filter_widths(start_fwhm: float = 5.0, end_fwhm: float = 2.0, stages: int = 6) -> list:
    """Gaussian widths sigma (cells) of a filter continuation: the full width
    at half maximum shrinking geometrically from ``start_fwhm`` to
    ``end_fwhm`` over ``stages`` stages (sigma = FWHM / (2 sqrt(2 ln 2)))."""
    c = 2.0 * math.sqrt(2.0 * math.log(2.0))
    if stages <= 1:
        return [end_fwhm / c]
    return [start_fwhm * (end_fwhm / start_fwhm) ** (j / (stages - 1)) / c for j in range(stages)]


@dataclasses.dataclass
class GcmmaHistory:
    W: list = dataclasses.field(default_factory=list)          # W~ at each accepted outer iterate
    zeta: list = dataclasses.field(default_factory=list)
    opt_norm: list = dataclasses.field(default_factory=list)   # first-order optimality residual
    gamma_scale: list = dataclasses.field(default_factory=list)
    stage: list = dataclasses.field(default_factory=list)
    inner: list = dataclasses.field(default_factory=list)      # forward solves spent by the inner loop
    stop: str = ""


_FIELDS = ("W", "zeta", "opt_norm", "gamma_scale", "stage", "inner")


def _save(path, **kw):
    tmp = path + ".tmp.npz"
    np.savez(tmp, **kw)
    os.replace(tmp, path)


def optimize_gcmma(s: Solver, rho0=None, max_iters: int = 600, levels=None, sigma_max: float = 0.0,
                   move: float = 0.5, min_inner: int = 12, norm_drop: float = 0.7, zeta_stop: float = 0.005,
                   max_inner: int = 10, tol: float = 1e-10, checkpoint: str | None = None,
                   checkpoint_every: int = 1, resume: str | None = None, fixed=None, fixed_value: float = 1.0,
                   symmetry: int | None = None, widths=None):
    """GCMMA loop of Sec. 3.2 with the damping continuation.

    Stage j solves max W~ at damping factor ``levels[j]`` with GCMMA from the
    current design.  Stage j ends after at least ``min_inner`` iterations once
    the optimality residual is at most (1 - norm_drop) of its value at the
    stage's first iterate; the last stage runs until the grayness falls below
    ``zeta_stop`` or ``max_iters`` outer iterations have run in total.  Every
    outer iteration: asymptotes, then inner iterations (subproblem solve +
    forward) that raise rho0 until the approximation is conservative
    (f~(y) >= f(y) - tol, f = -W~/W~(x)), then the adjoint at the accepted
    design.  W~ therefore never decreases within a stage.

    ``checkpoint``: file written every ``checkpoint_every`` outer iterations
    (design, MMA state, gradient, counters, history); ``resume``: such a file
    to continue from (the same workload and settings).

    ``fixed``: boolean mask of design variables held at ``fixed_value`` (the
    paper's fixed metal blocks); ``symmetry``: an axis across whose design
    mid-plane the design stays mirror-symmetric (gradients are
    mirror-averaged).  Variables with a zero gradient do not move under MMA,
    so both constraints hold exactly.

    ``widths``: filter continuation, one Gaussian width (cells) per stage
    (``filter_widths``), set with the damping level at every stage change;
    None keeps the context's filter.  Returns (rho, history)."""
    t = torch
    levels = list(damping_levels() if levels is None else levels)
    if widths is not None and len(widths) != len(levels):
        raise ValueError("one filter width per damping level")

    def set_stage_filter(j):
        if widths is not None:
            s.set_filter_width(widths[j])
    n = s.n_design
    h = GcmmaHistory()
    mask = None
    if fixed is not None:
        mask = t.as_tensor(np.asarray(fixed, dtype=np.uint8).reshape(-1), device=s.device).contiguous()

    def constrain(g):
        if mask is not None:
            s.fix_design(mask, grad=g)
        if symmetry is not None:
            s.mirror_average(g, symmetry)
        return g

    def evaluate(r, gs):
        Wt, g = s.evaluate(r, sigma_max, gs)
        return float(Wt.item()), constrain(g)

    if resume is not None:
        z = np.load(resume)
        rho = t.as_tensor(z["rho"], device=s.device).to(s.real).contiguous()
        state = t.as_tensor(z["state"], device=s.device).contiguous()
        g = t.as_tensor(z["g"], device=s.device).contiguous()
        W = float(z["W"])
        k, kk, stage, it_stage = (int(v) for v in z["counters"])
        norm0 = float(z["norm0"])
        for f in _FIELDS:
            getattr(h, f).extend(z["h_" + f].tolist())
        set_stage_filter(stage)
        s.set_design(rho)
        s.set_damping(sigma_max, levels[stage])
    else:
        rho = t.as_tensor(rho0, device=s.device).to(s.real).contiguous().reshape(-1).clone()
        if mask is not None:
            s.fix_design(mask, rho=rho, value=fixed_value)
        if symmetry is not None:
            s.mirror_average(rho, symmetry)
        state = s.mma_state()
        k = kk = stage = it_stage = 0
        norm0 = 0.0
        set_stage_filter(0)
        W, g = evaluate(rho, levels[0])
    y = t.empty_like(rho)
    while True:
        gs = levels[stage]
        zeta = float(s.grayness().item())
        sums = s.mma_asymptotes(rho, g, state, kk).cpu().numpy()
        norm = math.sqrt(float(sums[1]))
        if it_stage == 0:
            norm0 = norm
        if stage + 1 < len(levels) and it_stage >= min_inner and norm <= (1.0 - norm_drop) * norm0:
            # subproblem solved: next damping level (and filter width), a
            # fresh GCMMA run from this design
            stage += 1
            it_stage = kk = 0
            set_stage_filter(stage)
            W, g = evaluate(rho, levels[stage])
            continue
        h.W.append(W)
        h.zeta.append(zeta)
        h.opt_norm.append(norm)
        h.gamma_scale.append(gs)
        h.stage.append(stage)
        if zeta < zeta_stop:
            h.stop = "zeta"
            break
        if k >= max_iters:
            h.stop = "max_iters"
            break
        scale = 1.0 / W
        raa0 = max(1e-6, 0.1 * scale * float(sums[0]) / n)
        for inner in range(max_inner):
            sd = s.mma_solve(state, g, scale, raa0, move, y)
            s.set_design(y)
            Wy = float(s.forward().item())
            change, d = (float(v) for v in sd.cpu().numpy())
            f_y, f_a = -scale * Wy, -1.0 + change
            if f_a >= f_y - tol or d <= 0.0:
                break
            raa0 = min(1.1 * (raa0 + (f_y - f_a) / d), 10.0 * raa0)
        h.inner.append(inner + 1)
        rho.copy_(y)
        W = Wy
        s.adjoint()
        g = constrain(s.gradient())
        k += 1
        kk += 1
        it_stage += 1
        if checkpoint is not None and k % checkpoint_every == 0:
            _save(checkpoint, rho=rho.cpu().numpy(), state=state.cpu().numpy(), g=g.cpu().numpy(), W=W,
                  counters=np.array([k, kk, stage, it_stage]), norm0=norm0,
                  **{"h_" + f: np.asarray(getattr(h, f)) for f in _FIELDS})
    s.sync()
    return rho, h
