"""What the trained surrogate gains over the plain adjoint loop.

On the 256^2-design workload (316^2 grid, 4000 steps), a U-Net pretrained on
(rho, gradient) pairs from plain optimization trajectories drives the
surrogate-assisted loop (one full forward + adjoint solve, then four
surrogate steps, per round).  It must reach the plain loop's final objective
(within 1 %) in less wall time than the plain loop took."""

import numpy as np
import pytest

from paper_2203_01462_gb300 import inputs as I

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

def test_surrogate_loop_matches_plain_objective_in_less_time(save_report):
    import time
    import torch
    from paper_2203_01462_gb300.binding import Solver
    from paper_2203_01462_gb300.optimize import optimize
    from paper_2203_01462_gb300.surrogate_loop import Trainer, collect_pairs, surrogate_optimize
    w = I.cfg_2d_316()
    s = Solver(w)
    rho0s = [I.zero_gap(w, 0.02 * I.rho_uniform(w, 200 + k)) for k in range(4)]
    pairs = collect_pairs(s, rho0s, iters=15, move=0.05, damping_start=1.0, damping_iters=0)
    tr = Trainer(256, 256, base=24, batch=8, seed=0, lr=1e-3)
    tr.fit(pairs, 200)
    rho_start = I.zero_gap(w, np.zeros(I.design_shape(w)))
    torch.cuda.synchronize()
    t = time.perf_counter()
    _, hp = optimize(s, rho_start, iters=30, move=0.05, zeta_stop=0.0, damping_start=1.0, damping_iters=0,
                     move_decay=1.0)
    torch.cuda.synchronize()
    plain_s = time.perf_counter() - t
    target = hp.W[-1]
    t = time.perf_counter()
    _, hs, st = surrogate_optimize(s, tr, rho_start, updates=90, inner=4, move=0.05, damping_start=1.0,
                                   damping_iters=0, pairs=pairs, fit_steps=0, target_W=0.99 * target)
    torch.cuda.synchronize()
    sur_s = time.perf_counter() - t
    Ws = [x for x in hs.W if x == x]
    rep = dict(plain_s=plain_s, plain_updates=30, plain_W=target, sur_s=sur_s, sur_updates=len(hs.W),
               sur_W=Ws[-1], **st)
    save_report("surrogate_loop.json", rep)
    assert Ws[-1] >= 0.99 * target, rep
    assert sur_s < 0.9 * plain_s, rep
    assert st["solves"] < 30
