"""Optimization-loop kernels and driver: zeta against the oracle, the ascent
step and the threshold against numpy, and an optimization run whose
objective rises (the paper reports a monotonically increasing objective)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2203_01462_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def medium(real="f32"):
    w = I.workload_2d(150, 140, dx=10e-9, nsteps=900, npml=10, design=(90, 80), gap=(3, 3), real=real,
                      filter_radius=3, filter_fwhm=3.0, src_offset=5)
    w.update(I.pulse(800e-9, 200e12))
    return w


def test_grayness_matches_oracle():
    import torch
    from paper_2203_01462_gb300.binding import Solver
    w = medium("f64")
    rho = I.rho_uniform(w, 51)
    s = Solver(w)
    s.set_design(rho)
    z = float(s.grayness().item())
    assert abs(z - O.grayness(w, rho)) <= 1e-12


def test_ascent_and_threshold_kernels():
    import torch
    from paper_2203_01462_gb300.binding import Solver
    w = medium("f32")
    s = Solver(w)
    rng = np.random.default_rng(52)
    rho = rng.random(s.n_design).astype(np.float32)
    g = rng.standard_normal(s.n_design)
    r = torch.tensor(rho, device="cuda")
    gt = torch.tensor(g, device="cuda")
    s.ascent_step(r, gt, 0.1)
    ref = np.clip(rho.astype(np.float64) + 0.1 * g / np.abs(g).max(), 0.0, 1.0).astype(np.float32)
    np.testing.assert_array_equal(r.cpu().numpy(), ref)
    s.threshold(r, 0.5)
    np.testing.assert_array_equal(r.cpu().numpy(), (ref >= 0.5).astype(np.float32))


def test_plain_optimization_raises_the_objective():
    from paper_2203_01462_gb300.binding import Solver
    from paper_2203_01462_gb300.optimize import final_design, optimize
    w = medium("f32")
    s = Solver(w)
    rho0 = I.zero_gap(w, np.full(I.design_shape(w), 0.5))
    rho, h = optimize(s, rho0, iters=12, move=0.1, damping_start=1.0, damping_iters=0)
    W = np.array(h.W)
    assert W[-1] > 2.0 * W[0]
    assert np.sum(np.diff(W) > 0) >= len(W) - 3
    _, Wbin = final_design(s, rho)
    assert Wbin > 0
