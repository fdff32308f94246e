"""Several in-plane steps per cooperative launch (opt-in).

With fdtd_set_steps_per_launch(n > 1) the in-plane 2D mode runs a run of
steps as one cooperative launch whose half steps are separated by grid-wide
barriers.  The per-node arithmetic is the same as with one launch per half
step, so the results must be bit-identical whatever the number of steps per
launch, and the oracle parity of the default path carries over.  The bounded
wait the barrier relies on must give up and report FDTD_ETIMEOUT when
nothing sets its flag.
"""
import numpy as np
import pytest

from paper_2203_01462_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def inplane_case(real="f32", snapshot_every=16, nsteps=300, nx=97, ny=70):
    w = I.workload_2d_inplane(nx, ny, dx=20e-9, nsteps=nsteps, npml=8, design=(41, 31), gap=(3, 3), real=real,
                              material=I.SILVER, src_offset=2, snapshot_every=snapshot_every)
    w.update(I.pulse(800e-9, 300e12))
    return w


@pytest.mark.parametrize("real,snap", [("f32", 16), ("f64", 0), ("f32", 0)])
def test_results_do_not_depend_on_steps_per_launch(real, snap):
    """97 x 70 nodes (4 x 3 tiles, ragged), silver, damping: W, the gap
    history and the gradient with 1 step per launch, 64, and 7 (runs that
    end off the checkpoint and guard grid) are bit-identical."""
    from paper_2203_01462_gb300.binding import Solver
    w = inplane_case(real, snap)
    rho = I.rho_uniform(w, 61)
    out = []
    for spl in (1, 64, 7):
        s = Solver(w)
        s.set_stability_guard(0)  # runs of 7 steps then really end off the checkpoint grid
        s.set_steps_per_launch(spl)
        W, g = s.evaluate(rho, 5e5, 3.0)
        gh = s.gap_history()
        s.sync()
        out.append((float(W.item()), g.cpu().numpy(), gh.cpu().numpy(), s.info().launches))
    for W, g, gh, _ in out[1:]:
        assert W == out[0][0]
        np.testing.assert_array_equal(g, out[0][1])
        np.testing.assert_array_equal(gh, out[0][2])
    assert out[1][3] * 10 < out[0][3]  # far fewer launches (runs of at most 16 steps here)


def test_paper_geometry_uses_one_launch_per_run_of_steps():
    """On the paper's 491^2 geometry (200 nm box) 64 forward steps take one
    step launch when asked for, and two launches per step by default."""
    from paper_2203_01462_gb300.binding import Solver
    w = I.cfg_2d_inplane_paper(200.0, nsteps=128, snapshot_every=64)
    s = Solver(w)
    s.set_steps_per_launch(64)
    s.set_design(I.rho_uniform(w, 1))
    l0 = s.info().launches
    s.forward()
    s.sync()
    fwd = s.info().launches - l0
    assert fwd < 20, fwd  # 2 runs of 64 steps + checkpoints, zeroing, objective
    s.set_steps_per_launch(1)
    l0 = s.info().launches
    s.forward()
    s.sync()
    assert s.info().launches - l0 > 256


def test_bounded_wait_gives_up_and_reports_timeout():
    """A wait on a flag that nothing sets, limited to 2e6 clock cycles
    (about a millisecond): it must return, record ERR_TIMEOUT and raise the
    abort word, which the library reports as FDTD_ETIMEOUT; the context of
    the device stays usable afterwards."""
    import torch
    from paper_2203_01462_gb300.binding import selftest_bounded_wait
    assert selftest_bounded_wait(2_000_000) == 6
    assert selftest_bounded_wait(20_000_000) == 6
    x = torch.ones(1024, device="cuda")
    assert float(x.sum().item()) == 1024.0
