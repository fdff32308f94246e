"""Degenerate and edge cases of the method through the C ABI, against the
oracle: an empty gap (W~ = 0 and a zero gradient), very short runs,
checkpoint intervals that do not divide the step count or exceed it,
binary densities (the artificial conductivity vanishes), and a design box
that spans the whole interior up to the absorbing layers."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2203_01462_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def l2rel(a, b):
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / nb) if nb > 0 else float(np.linalg.norm(a))


def small(nsteps=300, **kw):
    w = I.small_2d(nx=41, ny=37, nsteps=nsteps, dx=20e-9, npml=6, design=kw.pop("design", (17, 15)), real="f64",
                   **kw)
    w.update(I.pulse(800e-9, 300e12))
    return w


def run(w, rho, smax=5e5, gs=2.0):
    from paper_2203_01462_gb300.binding import Solver
    s = Solver(w)
    W, g = s.evaluate(rho, smax, gs)
    s.sync()
    return float(W.item()), g.cpu().numpy()


def test_empty_gap_gives_zero_objective_and_gradient():
    w = small()
    w["gap_lo"], w["gap_hi"] = [20, 18, 0], [20, 18, 1]
    rho = I.rho_uniform(w, 61)
    W, g = run(w, rho)
    assert W == 0.0 and O.objective(w, rho, 5e5, 2.0) == 0.0
    assert np.all(g == 0.0)


@pytest.mark.parametrize("nsteps,snap", [(1, 0), (1, 4), (23, 7), (23, 30), (64, 64)])
def test_short_runs_and_ragged_checkpoints(nsteps, snap):
    w = small(nsteps=nsteps, snapshot_every=snap)
    # the gap next to the source row so that a few steps already reach it
    w["gap_lo"], w["gap_hi"] = [19, 9, 0], [22, 11, 1]
    w["design_lo"], w["design_hi"] = [12, 8, 0], [29, 16, 1]
    rho = I.rho_uniform(w, 62)
    W, g = run(w, rho)
    ref = O.gradient(w, rho, 5e5, 2.0)
    assert abs(W - ref["W"]) <= 1e-10 * abs(ref["W"]) + 1e-300
    assert l2rel(g, ref["grad"]) <= 1e-9


def test_binary_design_sigma_term_vanishes():
    w = small()
    rho = I.zero_gap(w, (np.random.default_rng(63).random(I.design_shape(w)) > 0.5).astype(float))
    W1, g1 = run(w, rho, smax=5e5)
    W0, _ = run(w, rho, smax=0.0)
    assert W1 == W0  # sigma_i = rho (1 - rho) sigma_max is exactly zero
    ref = O.gradient(w, rho, 5e5, 2.0)
    assert abs(W1 - ref["W"]) <= 1e-10 * abs(ref["W"])
    assert l2rel(g1, ref["grad"]) <= 1e-9


@pytest.mark.parametrize("mode", ["tmz", "inplane", "3d"])
def test_design_box_spanning_the_interior(mode):
    if mode == "tmz":
        w = small(nsteps=200)
        w["design_lo"], w["design_hi"] = [6, 6, 0], [35, 31, 1]
    elif mode == "inplane":
        w = I.workload_2d_inplane(41, 37, dx=20e-9, nsteps=200, npml=6, design=(17, 15), gap=(3, 3), real="f64",
                                  src_offset=2)
        w.update(I.pulse(800e-9, 300e12))
        w["design_lo"], w["design_hi"] = [6, 9, 0], [34, 30, 1]
    else:
        w = I.workload_3d(21, 19, 23, dx=20e-9, nsteps=120, npml=4, design=(9, 7, 6), gap=(2, 2, 2), real="f64",
                          source="dipole")
        w.update(I.pulse(800e-9, 300e12))
        w["design_lo"], w["design_hi"] = [4, 4, 4], [17, 15, 19]
    rho = I.rho_uniform(w, 64)
    W, g = run(w, rho)
    ref = O.gradient(w, rho, 5e5, 2.0)
    assert abs(W - ref["W"]) <= 1e-10 * abs(ref["W"])
    assert l2rel(g, ref["grad"]) <= 1e-9
