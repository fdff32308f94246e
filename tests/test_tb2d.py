"""Temporally blocked 2D E_z steps (several steps per launch on tiles with a
halo in shared memory; fdtd_set_steps_per_launch on a 2D E_z context),
through the C ABI.

The blocked kernel runs the launch-per-step kernel's generic per-node
arithmetic, so it is held to the same bars against the FP64 oracle (FP64:
W 1e-10, gap history 1e-10, gradient 1e-9; FP32: W 1e-4, gradient 1e-3) and
to FP32 rounding against the launch-per-step path.  The tile side is the
smallest from 16 to 32 whose tiles fit one wave of blocks: 16 on the small
grids, 27 on the surrogate workload's 316^2, 32 (several waves) on a
520 x 500 grid.  Cases: grids ragged against the tiles, a grid smaller than
one tile plus its halo, a filtered design, a checkpointed run (blocked
forward and recompute, paired adjoint launches), step counts that do not
divide the run, the three tile sides, and the stability guard's early
stop."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2203_01462_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def solver(w, steps):
    from paper_2203_01462_gb300.binding import Solver
    s = Solver(w)
    s.set_steps_per_launch(steps)
    return s


def l2rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def small(real, nx=41, ny=37, nsteps=400, **kw):
    w = I.small_2d(nx=nx, ny=ny, nsteps=nsteps, dx=20e-9, npml=6, design=kw.pop("design", (17, 15)), real=real, **kw)
    w.update(I.pulse(800e-9, 300e12))
    return w


@pytest.mark.parametrize("nx,ny,steps", [(41, 37, 8), (150, 140, 8), (23, 19, 3), (150, 140, 5)])
def test_fp64_blocked_matches_oracle(nx, ny, steps):
    w = small("f64", nx=nx, ny=ny, design=(17, 15) if nx < 100 else (60, 50))
    if nx < 30:
        w = small("f64", nx=nx, ny=ny, design=(9, 7))
    rho = I.rho_uniform(w, 61)
    ref = O.gradient(w, rho, 5e5, 2.0)
    gh_ref = O.forward(w, rho, 5e5, 2.0, record_gap=True)["gap_hist"]
    s = solver(w, steps)
    W, g = s.evaluate(rho, 5e5, 2.0)
    s.sync()
    assert abs(float(W.item()) - ref["W"]) <= 1e-10 * abs(ref["W"])
    gh = s.gap_history().cpu().numpy()
    assert np.max(np.abs(gh - gh_ref)) <= 1e-10 * np.max(np.abs(gh_ref))
    assert l2rel(g.cpu().numpy(), ref["grad"]) <= 1e-9


@pytest.mark.parametrize("snap", [0, 16])
def test_fp32_filtered_blocked_matches_oracle(snap):
    w = small("f32", nx=90, ny=83, design=(40, 36), filter_radius=3, filter_fwhm=3.0, snapshot_every=snap)
    rho = I.rho_uniform(w, 62)
    ref = O.gradient(w, rho, 5e5, 3.0)
    s = solver(w, 8)
    W, g = s.evaluate(rho, 5e5, 3.0)
    s.sync()
    assert abs(float(W.item()) - ref["W"]) <= 1e-4 * abs(ref["W"])
    assert l2rel(g.cpu().numpy(), ref["grad"]) <= 1e-3


def test_blocked_agrees_with_launch_per_step_on_the_surrogate_grid():
    """316^2 (the surrogate workload), 600 steps, a near-empty design (as the
    surrogate's starts): the two paths agree to FP32 rounding, and the
    blocked path takes about 1/8 of the launches."""
    w = I.cfg_2d_316(nsteps=600)
    rho = 0.02 * I.rho_uniform(w, 63)
    out = []
    for steps in (1, 8):
        s = solver(w, steps)
        s.set_graphs(0)
        l0 = s.info().launches
        W, g = s.evaluate(rho, 0.0, 2.0)
        s.sync()
        out.append((float(W.item()), g.cpu().numpy(), s.info().launches - l0))
    (W0, g0, n0), (W1, g1, n1) = out
    assert abs(W1 - W0) <= 1e-5 * abs(W0)
    assert l2rel(g1, g0) <= 1e-4
    assert n1 * 6 < n0, (n1, n0)


def test_blocked_guard_stops_early():
    from paper_2203_01462_gb300.binding import FdtdError
    N = 20000
    w = small("f32", nsteps=N)
    s = solver(w, 8)
    s.set_graphs(0)  # plain launches: the host loop itself stops (a replayed graph reports at fdtd_sync)
    s.set_design(I.rho_uniform(w, 64))
    s.set_damping(0.0, 1.0)
    s.set_stability_guard(64, 1e-30)
    c0 = s.info().cell_updates
    with pytest.raises(FdtdError) as e:
        s.forward()
    assert e.value.status == 5  # FDTD_EUNSTABLE
    assert (s.info().cell_updates - c0) // s.info().n_cells < N // 2


def test_blocked_repeat_and_graph_replay_are_bit_identical():
    w = small("f32", nsteps=300)
    rho = I.rho_uniform(w, 65)
    s = solver(w, 8)
    s.set_graphs(0)
    W0, g0 = s.evaluate(rho, 5e5, 2.0)
    W0, g0 = float(W0.item()), g0.cpu().numpy().copy()
    s.set_graphs(1)
    for _ in range(2):
        W, g = s.evaluate(rho, 5e5, 2.0)
        assert float(W.item()) == W0 and np.array_equal(g.cpu().numpy(), g0)


def test_blocked_multi_wave_grid_matches_oracle():
    """A grid of more tiles than SMs even at the largest tile side (520 x 500:
    17 x 16 tiles of 32, several waves), ragged against the tile: the blocked
    path, asked for explicitly, and the launch-per-step path (mostly its
    interior vector branch here) both meet the FP32 bars against the FP64
    oracle."""
    w = small("f32", nx=520, ny=500, nsteps=900, design=(60, 50))
    rho = I.rho_uniform(w, 66)
    ref = O.gradient(w, rho, 5e5, 2.0)
    assert ref["W"] > 0 and np.linalg.norm(ref["grad"]) > 0  # the pulse has reached the gap
    for steps in (1, 8):
        s = solver(w, steps)
        W, g = s.evaluate(rho, 5e5, 2.0)
        s.sync()
        assert abs(float(W.item()) - ref["W"]) <= 1e-4 * abs(ref["W"]), (steps, float(W.item()), ref["W"])
        assert l2rel(g.cpu().numpy(), ref["grad"]) <= 1e-3, steps
