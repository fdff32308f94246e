"""Surrogate-assisted design optimization.

A plain adjoint loop spends one forward + adjoint FDTD solve per design step.
Here the U-Net surrogate (``surrogate.UNet``) predicts the sensitivity map
from (rho, damping level) and takes ``inner`` cheap steps after every full
solve.  The full solve stays the reference: it checks the previous surrogate
steps (if W~ fell, the design returns to the last checked one and that round's
surrogate steps are skipped), it supplies a new training pair, and the
network is fine-tuned on the pairs collected so far.

Training targets are gradients normalised by their largest magnitude; the
ascent step (``fdtd_ascent_step``) normalises its direction the same way.

With ``correct=True`` (default) the network is used as a correction model
around the last checked design rho_j: the step direction is
g(rho_j) + N(rho) - N(rho_j), the exact normalised gradient of the last full
solve plus the change the network predicts, so that the network's absolute
errors largely cancel.
"""
from __future__ import annotations

import dataclasses
import math
import time

import numpy as np
import torch

from .binding import Solver
from .optimize import History, damping_schedule
from .surrogate import UNet


def design_map(s: Solver, rho: torch.Tensor) -> torch.Tensor:
    """rho of the design box as an H x W map (y rows, x columns)."""
    w = s.w
    H = w["design_hi"][1] - w["design_lo"][1]
    W = w["design_hi"][0] - w["design_lo"][0]
    return rho.reshape(H, W)


def net_input(rho_map: torch.Tensor, gamma_scale: float) -> torch.Tensor:
    """[2][1][H][W]: rho and the damping level log10(gamma_scale) as a constant map."""
    lvl = torch.full_like(rho_map, math.log10(gamma_scale))
    return torch.stack([rho_map, lvl]).unsqueeze(1).float().contiguous()


def normalised(g: torch.Tensor) -> torch.Tensor:
    """g over its largest magnitude (g itself when it is zero), without a host
    synchronisation."""
    m = g.abs().max()
    return (g / torch.where(m > 0, m, torch.ones_like(m))).float()


@dataclasses.dataclass
class Pairs:
    x: list = dataclasses.field(default_factory=list)   # [2][1][H][W] inputs
    t: list = dataclasses.field(default_factory=list)   # [1][1][H][W] targets

    def add(self, x, t):
        self.x.append(x)
        self.t.append(t)

    def __len__(self):
        return len(self.x)


def collect_pairs(s: Solver, rho0_list, iters: int, move: float = 0.05, sigma_max: float = 0.0,
                  damping_start: float = 10.0, damping_iters: int = 50, pairs: Pairs | None = None) -> Pairs:
    """(rho, damping level) -> normalised gradient pairs along plain adjoint
    optimization trajectories started from each design in rho0_list."""
    pairs = pairs or Pairs()
    for rho0 in rho0_list:
        rho = torch.as_tensor(rho0, device=s.device).to(s.real).contiguous().clone()
        for k in range(iters):
            gs = damping_schedule(k, damping_start, damping_iters)
            W, g = s.evaluate(rho, sigma_max, gs)
            m = design_map(s, rho)
            pairs.add(net_input(m, gs), normalised(design_map(s, g)).unsqueeze(0).unsqueeze(0).contiguous())
            s.ascent_step(rho, g, move)
    return pairs


def collect_pairs_concurrent(w: dict, rho0_list, iters: int, move: float = 0.05, sigma_max: float = 0.0,
                             damping_start: float = 10.0, damping_iters: int = 50, pairs: Pairs | None = None,
                             width: int = 16, steps_per_launch: int | None = None) -> Pairs:
    """collect_pairs with the trajectories run side by side: up to ``width``
    solvers of workload ``w``, each on its own CUDA stream, take one design
    step each per round, so that the launches of several small-grid
    trajectories (one partial wave of blocks each) share the GPU.  Every
    trajectory computes exactly what collect_pairs computes (same kernels,
    same inputs); the pairs are kept in trajectory order.  steps_per_launch
    (None: the library's default) sets the solvers' steps per launch: side
    by side, one launch per step shares the GPU better than temporally
    blocked launches, which each hold about a hundred SMs."""
    pairs = pairs or Pairs()
    for b0 in range(0, len(rho0_list), width):
        group = list(rho0_list[b0:b0 + width])
        solvers = [Solver(w, stream=torch.cuda.Stream()) for _ in group]
        if steps_per_launch is not None:
            for s in solvers:
                s.set_steps_per_launch(steps_per_launch)
        per = [Pairs() for _ in group]
        rhos = []
        for s, rho0 in zip(solvers, group):
            with torch.cuda.stream(s.stream):
                rhos.append(torch.as_tensor(rho0, device=s.device).to(s.real).contiguous().clone())
        for k in range(iters):
            gs = damping_schedule(k, damping_start, damping_iters)
            for s, rho, pp in zip(solvers, rhos, per):
                with torch.cuda.stream(s.stream):
                    W, g = s.evaluate(rho, sigma_max, gs)
                    m = design_map(s, rho)
                    pp.add(net_input(m, gs), normalised(design_map(s, g)).unsqueeze(0).unsqueeze(0).contiguous())
                    s.ascent_step(rho, g, move)
        torch.cuda.synchronize()
        for pp in per:
            pairs.x += pp.x
            pairs.t += pp.t
        for s in solvers:
            s.close()
    return pairs


class Trainer:
    def __init__(self, H: int, W: int, base: int = 24, batch: int = 8, seed: int = 0, lr: float = 1e-3,
                 precision: str = "bf16"):
        self.net = UNet(base=base, batch=batch, H=H, W=W, seed=seed, precision=precision)
        self.pred = self.net.sibling(1)
        self.batch, self.lr = batch, lr
        self.rng = np.random.default_rng(seed)

    def fit(self, pairs: Pairs, steps: int) -> float:
        loss = float("nan")
        B = self.batch
        for _ in range(steps):
            idx = self.rng.choice(len(pairs), B, replace=len(pairs) < B)
            x = torch.cat([pairs.x[i] for i in idx], dim=1)
            t = torch.cat([pairs.t[i] for i in idx], dim=1)
            loss = self.net.train_step(x, t, self.lr)
        return float(loss.item()) if steps else loss

    def predict(self, rho_map: torch.Tensor, gamma_scale: float) -> torch.Tensor:
        return self.pred.forward(net_input(rho_map, gamma_scale))[0, 0]


def surrogate_optimize(s: Solver, tr: Trainer, rho0, updates: int, inner: int = 4, move: float = 0.05,
                       sigma_max: float = 0.0, damping_start: float = 10.0, damping_iters: int = 50,
                       pairs: Pairs | None = None, fit_steps: int = 2,
                       target_W: float | None = None, correct: bool = True) -> tuple[torch.Tensor, History, dict]:
    """Up to ``updates`` design steps: each round is one full solve +
    ascent step, then ``inner`` surrogate steps.  Stops early once the W~ of a full
    solve reaches ``target_W``.  Returns the design, the history and counters
    (full solves, surrogate steps, rejected rounds)."""
    rho = torch.as_tensor(rho0, device=s.device).to(s.real).contiguous().clone()
    pairs = pairs if pairs is not None else Pairs()
    h = History()
    stats = dict(solves=0, surrogate_steps=0, rejected=0)
    t0 = time.perf_counter()
    k = 0
    last_W, last_rho, last_g = None, None, None
    skip = False
    while k < updates:
        gs = damping_schedule(k, damping_start, damping_iters)
        W, g = s.evaluate(rho, sigma_max, gs)
        stats["solves"] += 1
        Wv = float(W.item())
        if last_W is not None and Wv < last_W and not skip:
            # the surrogate steps made things worse: back to the checked design
            rho.copy_(last_rho)
            W, g, Wv = None, last_g, last_W
            stats["rejected"] += 1
            skip = True
        else:
            skip = False
            m = design_map(s, rho)
            pairs.add(net_input(m, gs), normalised(design_map(s, g)).unsqueeze(0).unsqueeze(0).contiguous())
            if fit_steps:
                tr.fit(pairs, fit_steps)
        last_W, last_rho, last_g = Wv, rho.clone(), g
        if target_W is not None and Wv >= target_W:
            h.W.append(Wv)
            h.gamma_scale.append(gs)
            h.kind.append("adjoint")
            h.seconds.append(time.perf_counter() - t0)
            break
        g_n = normalised(g).reshape(-1)
        base_pred = tr.predict(design_map(s, rho).float(), gs).reshape(-1).clone() if correct and not skip else None
        s.ascent_step(rho, g, move)
        h.W.append(Wv)
        h.gamma_scale.append(gs)
        h.kind.append("adjoint")
        h.seconds.append(time.perf_counter() - t0)
        k += 1
        if skip:
            continue
        for _ in range(inner):
            if k >= updates:
                break
            gs = damping_schedule(k, damping_start, damping_iters)
            pred = tr.predict(design_map(s, rho).float(), gs).reshape(-1)
            ghat = (g_n + (pred - base_pred)) if correct else pred
            s.ascent_step(rho, ghat.double().contiguous(), move)
            stats["surrogate_steps"] += 1
            h.W.append(float("nan"))
            h.gamma_scale.append(gs)
            h.kind.append("surrogate")
            h.seconds.append(time.perf_counter() - t0)
            k += 1
    torch.cuda.synchronize()
    return rho, h, stats
