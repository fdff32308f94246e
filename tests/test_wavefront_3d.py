"""3D wavefront launches (several time steps per persistent launch) against
the two-launch form of the same step, through the C ABI.

Every node runs the same arithmetic in both forms, only the order in which
the z slabs are visited differs, so W~, the gap history and the gradient
must agree bit for bit.  The cases cover a ragged grid (x not a multiple of
the 32-node tile, odd nz so the last slab holds one plane), the plane wave
(its face corrections are folded into the wavefront tiles), the dipole,
checkpointed and full-history adjoints, FP32 and FP64, and every count of
steps per launch up to the maximum, including counts that do not divide
the checkpoint interval.  The forms are also checked against the FP64
oracle on a case where the wavefront launch holds several jobs per slab."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2203_01462_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def solver(w):
    from paper_2203_01462_gb300.binding import Solver
    return Solver(w)


def run(w, rho, wave, sigma=5e5, gs=2.0):
    s = solver(w)
    s.set_wavefront(wave)
    c0 = s.info().launches
    W, g = s.evaluate(rho, sigma, gs)
    s.sync()
    return float(W.item()), g.cpu().numpy().copy(), s.gap_history().cpu().numpy().copy(), s.info().launches - c0


def tfsf_case(real, nx=45, ny=22, nz=33, nsteps=150, snap=0, **kw):
    w = I.workload_3d(nx, ny, nz, dx=20e-9, nsteps=nsteps, npml=4, design=(11, 7, 6), gap=(2, 2, 2),
                      source="tfsf", substrate=True, real=real, tf_margin=1, snapshot_every=snap, **kw)
    w.update(I.pulse(800e-9, 300e12))
    return w


def dipole_case(real, nx=70, ny=27, nz=29, nsteps=120, snap=0, **kw):
    w = I.workload_3d(nx, ny, nz, dx=20e-9, nsteps=nsteps, npml=5, design=(20, 9, 8), gap=(2, 2, 2),
                      source="dipole", real=real, snapshot_every=snap, **kw)
    w.update(I.pulse(800e-9, 300e12))
    return w


@pytest.mark.parametrize("real", ["f32", "f64"])
@pytest.mark.parametrize("make,snap", [(tfsf_case, 0), (tfsf_case, 12), (dipole_case, 0), (dipole_case, 10)])
def test_wavefront_is_bit_identical_to_two_launches(real, make, snap):
    w = make(real, snap=snap)
    rho = I.rho_uniform(w, 41)
    W0, g0, h0, n0 = run(w, rho, 0)
    assert np.isfinite(W0) and W0 > 0
    for wave in (1, 2, 3, 8):
        W, g, h, n = run(w, rho, wave)
        assert W == W0, (wave, W, W0)
        assert np.array_equal(h, h0), wave
        assert np.array_equal(g, g0), wave
        assert n < n0, (wave, n, n0)


def test_wavefront_launch_count_follows_steps_per_launch():
    """Full history, no guard stop: one launch per `wave` steps in each pass
    (forward, adjoint) against two per step (dipole) in the default form."""
    w = dipole_case("f32", nsteps=96)
    rho = I.rho_uniform(w, 42)
    _, _, _, n0 = run(w, rho, 0)
    _, _, _, n1 = run(w, rho, 1)
    _, _, _, n4 = run(w, rho, 4)
    # the wavefront adds one counter reset per pass
    assert n0 - n1 == 2 * 96 * 2 - 2 * 96 - 2
    assert n1 - n4 == 2 * 96 - 2 * 24


def test_wavefront_matches_oracle_on_many_slabs():
    """FP64, plane wave, checkpoints every 7 steps, four steps per launch:
    the wavefront path against the oracle itself."""
    w = tfsf_case("f64", nx=24, ny=20, nz=41, nsteps=110, snap=7)
    rho = I.rho_uniform(w, 43)
    ref = O.gradient(w, rho, 5e5, 2.0)
    W, g, h, _ = run(w, rho, 4)
    assert abs(W - ref["W"]) <= 1e-10 * abs(ref["W"])
    gh_ref = O.forward(w, rho, 5e5, 2.0, record_gap=True)["gap_hist"]
    assert np.max(np.abs(h - gh_ref)) <= 1e-10 * np.max(np.abs(gh_ref))
    assert float(np.linalg.norm(g - ref["grad"]) / np.linalg.norm(ref["grad"])) <= 1e-9


def test_wavefront_setting_is_validated():
    from paper_2203_01462_gb300.binding import FdtdError
    w = dipole_case("f32", nsteps=10)
    s = solver(w)
    for bad in (-1, 9):
        with pytest.raises(FdtdError):
            s.set_wavefront(bad)
    w2 = I.small_2d(nx=41, ny=37, npml=6, design=(17, 15), real="f32")
    with pytest.raises(FdtdError):
        solver(w2).set_wavefront(2)


def test_wavefront_with_the_stability_guard():
    """Guard every 20 steps: runs end on multiples of 20 (launches of up to 8
    steps) and the result is still bit-identical; a bound below the fields
    stops a long forward early with FDTD_EUNSTABLE."""
    from paper_2203_01462_gb300.binding import FdtdError
    w = dipole_case("f32", nsteps=100)
    rho = I.rho_uniform(w, 44)
    W0, g0, _, _ = run(w, rho, 0)
    s = solver(w)
    s.set_wavefront(8)
    s.set_stability_guard(20, 0.0)
    W, g = s.evaluate(rho, 5e5, 2.0)
    s.sync()
    assert float(W.item()) == W0 and np.array_equal(g.cpu().numpy(), g0)
    N = 6000
    w = dipole_case("f32", nsteps=N)
    s = solver(w)
    s.set_wavefront(8)
    s.set_design(rho)
    s.set_damping(0.0, 1.0)
    s.set_stability_guard(20, 1e-30)
    c0 = s.info().cell_updates
    with pytest.raises(FdtdError) as e:
        s.forward()
    assert e.value.status == 5  # FDTD_EUNSTABLE
    steps = (s.info().cell_updates - c0) // s.info().n_cells
    assert steps < N // 2, steps
