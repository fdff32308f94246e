"""CUDA-graph replay of whole forward / adjoint passes gives bit-identical
results to plain launches, across design and damping changes, in every
solver mode."""
import numpy as np
import pytest

from paper_2203_01462_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _modes():
    w2 = I.small_2d(nx=41, ny=37, nsteps=300, dx=20e-9, npml=6, design=(17, 14), real="f32", snapshot_every=16)
    w2.update(I.pulse(800e-9, 300e12))
    wp = I.workload_2d_inplane(41, 37, dx=20e-9, nsteps=300, npml=6, design=(17, 14), gap=(3, 2), real="f32",
                               src_offset=2, snapshot_every=16)
    wp.update(I.pulse(800e-9, 300e12))
    w3 = I.workload_3d(21, 19, 23, dx=20e-9, nsteps=160, npml=4, design=(9, 7, 6), gap=(2, 2, 2), real="f32",
                       source="dipole", snapshot_every=16)
    w3.update(I.pulse(800e-9, 300e12))
    return {"tmz": w2, "inplane": wp, "3d": w3}


@pytest.mark.parametrize("mode", ["tmz", "inplane", "3d"])
def test_graph_replay_is_bit_identical(mode):
    from paper_2203_01462_gb300.binding import Solver
    w = _modes()[mode]
    plain, graph = Solver(w), Solver(w)
    plain.set_graphs(0)
    graph.set_graphs(1)
    for seed, smax, gs in ((1, 0.0, 1.0), (2, 5e5, 3.0), (3, 2e5, 1.5)):
        rho = I.rho_uniform(w, seed)
        Wp, gp = plain.evaluate(rho, smax, gs)
        Wg, gg = graph.evaluate(rho, smax, gs)
        plain.sync()
        graph.sync()
        assert float(Wp.item()) == float(Wg.item())
        assert np.array_equal(gp.cpu().numpy(), gg.cpu().numpy())
    ip, ig = plain.info(), graph.info()
    assert ip.launches == ig.launches and ip.cell_updates == ig.cell_updates


def test_l2_residency_changes_nothing():
    """The L2 access-policy windows change where the state is cached, not what
    is computed: W and the gradient are bit-identical with and without."""
    from paper_2203_01462_gb300.binding import Solver
    w = _modes()["tmz"]
    plain, held = Solver(w), Solver(w)
    held.set_l2_residency(0.3)
    try:
        for seed in (4, 5):
            rho = I.rho_uniform(w, seed)
            Wp, gp = plain.evaluate(rho, 2e5, 2.0)
            Wh, gh = held.evaluate(rho, 2e5, 2.0)
            plain.sync()
            held.sync()
            assert float(Wp.item()) == float(Wh.item())
            assert np.array_equal(gp.cpu().numpy(), gh.cpu().numpy())
    finally:
        held.set_l2_residency(0.0)  # release the set-aside for the tests that follow
