"""The forward solve's stability guard, made to trip from the host.

The guard reads the whole solver state every `every` forward steps and flags
a word that is not finite or above a bound.  No stable configuration comes
near the automatic bound, so these tests trip it in two host-made ways: a
bound set far below the run's real fields, and an FP32 source amplitude
(1e38) whose fields pass the automatic bound's FP32 cap.  They check that fdtd_forward stops enqueuing
steps early and returns FDTD_EUNSTABLE with plain launches, that fdtd_sync
reports it when the pass replays as a CUDA graph, that the context then
gives the normal results again, and that the checks change no result.
"""
import numpy as np
import pytest

from paper_2203_01462_gb300 import inputs as I

pytestmark = pytest.mark.gpu

EUNSTABLE = 5


def small(real="f64", nsteps=20000, **kw):
    w = I.small_2d(nx=41, ny=37, nsteps=nsteps, dx=20e-9, npml=6, design=(17, 15), real=real, **kw)
    w.update(I.pulse(800e-9, 300e12))
    return w


def solver(w, graphs=0):
    from paper_2203_01462_gb300.binding import Solver
    s = Solver(w)
    s.set_graphs(graphs)
    return s


def test_guard_changes_no_result():
    w = small(nsteps=600, snapshot_every=16)
    rho = I.rho_uniform(w, 3)
    out = []
    for every in (0, 1, 256):
        s = solver(w)
        s.set_stability_guard(every)
        W, g = s.evaluate(rho, 5e5, 2.0)
        s.sync()
        out.append((float(W.item()), g.cpu().numpy()))
    for W, g in out[1:]:
        assert W == out[0][0]
        np.testing.assert_array_equal(g, out[0][1])


def test_low_bound_stops_the_forward_early():
    from paper_2203_01462_gb300.binding import FdtdError
    N = 20000
    w = small(nsteps=N)
    rho = I.rho_uniform(w, 4)
    s = solver(w)
    s.set_design(rho)
    s.set_damping(0.0, 1.0)
    s.set_stability_guard(64, 1e-30)  # any field the source makes exceeds it
    c0 = s.info().cell_updates
    with pytest.raises(FdtdError) as e:
        s.forward()
    assert e.value.status == EUNSTABLE
    steps = (s.info().cell_updates - c0) // s.info().n_cells
    assert steps < N // 2, steps  # stopped enqueuing long before step N
    with pytest.raises(FdtdError) as e:
        s.adjoint()  # no forward run to take the adjoint of
    assert e.value.status == 4
    # the error word was cleared: the same context runs normally again
    s.set_stability_guard(256, 0.0)
    W = s.forward().clone()
    s.adjoint()
    s.sync()
    ref = solver(w)
    Wr, _ = ref.evaluate(rho)
    ref.sync()
    assert float(W.item()) == float(Wr.item())


def test_graph_replay_reports_at_sync():
    from paper_2203_01462_gb300.binding import FdtdError
    w = small(nsteps=400)
    rho = I.rho_uniform(w, 5)
    s = solver(w, graphs=1)
    s.set_design(rho)
    s.set_stability_guard(64, 1e-30)
    s.forward()  # the whole pass is one graph launch: nothing to stop early
    with pytest.raises(FdtdError) as e:
        s.sync()
    assert e.value.status == EUNSTABLE
    s.set_stability_guard(256, 0.0)  # drops the captured pass
    W, _ = s.evaluate(rho)
    s.sync()
    assert np.isfinite(float(W.item())) and float(W.item()) > 0


def test_fp32_overflow_is_caught_with_the_automatic_bound():
    """A 1e38 source amplitude: the pulse's field (about src_amp / 2) passes
    the FP32 cap of the automatic bound (1e37) for a few tens of steps before
    the CPML absorbs it, so the checks run every 16 steps."""
    from paper_2203_01462_gb300.binding import FdtdError
    N = 20000
    w = small(real="f32", nsteps=N, src_amp=1e38)
    s = solver(w)
    s.set_stability_guard(16, 0.0)
    s.set_design(I.rho_uniform(w, 6))
    c0 = s.info().cell_updates
    with pytest.raises(FdtdError) as e:
        s.forward()
    assert e.value.status == EUNSTABLE
    assert (s.info().cell_updates - c0) // s.info().n_cells < N // 2


@pytest.mark.parametrize("mode", ["inplane", "3d"])
def test_guard_in_the_other_modes(mode):
    from paper_2203_01462_gb300.binding import FdtdError
    N = 8000
    if mode == "inplane":
        w = I.workload_2d_inplane(41, 37, dx=20e-9, nsteps=N, npml=6, design=(17, 15), gap=(3, 3), real="f32",
                                  src_offset=2)
    else:
        w = I.workload_3d(21, 19, 23, dx=20e-9, nsteps=N, npml=4, design=(9, 7, 6), gap=(2, 2, 2), real="f32")
    w.update(I.pulse(800e-9, 300e12))
    s = solver(w)
    s.set_design(I.rho_uniform(w, 7))
    s.set_stability_guard(32, 1e-30)
    c0 = s.info().cell_updates
    with pytest.raises(FdtdError) as e:
        s.forward()
    assert e.value.status == EUNSTABLE
    assert (s.info().cell_updates - c0) // s.info().n_cells < N // 2
    s.set_stability_guard(256, 0.0)
    s.forward()
    s.sync()
