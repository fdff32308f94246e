"""3D plane wave by total-field / scattered-field injection: CUDA path vs the
FP64 oracle, through the C ABI.

The library tabulates the incident column on the device at create and adds
the face corrections after each half step; the oracle converts every
neighbour sample that crosses the box boundary.  FP64 agrees to round-off
(W, the gap history, the gradient); FP32 within 1e-4 (W) and 1e-3
(gradient, L2-relative).  Checkpointed runs recompute the injected forward
field segment by segment."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2203_01462_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def case(real, nx=21, ny=19, nz=31, npml=4, design=(9, 7, 6), nsteps=240, material=None, tf_margin=1, **kw):
    w = I.workload_3d(nx, ny, nz, dx=20e-9, nsteps=nsteps, npml=npml, design=design, gap=(2, 2, 2),
                      source="tfsf", substrate=True, material=material, real=real, tf_margin=tf_margin, **kw)
    w.update(I.pulse(800e-9, 300e12))
    return w


def l2rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def solver(w):
    from paper_2203_01462_gb300.binding import Solver
    return Solver(w)


@pytest.mark.parametrize("snap,material", [(0, "gold"), (9, "silver")])
def test_fp64_plane_wave_matches_oracle(snap, material):
    w = case("f64", material=I.SILVER if material == "silver" else I.GOLD, snapshot_every=snap)
    rho = I.rho_uniform(w, 31)
    ref = O.gradient(w, rho, 5e5, 2.0)
    gh_ref = O.forward(w, rho, 5e5, 2.0, record_gap=True)["gap_hist"]
    s = solver(w)
    W, g = s.evaluate(rho, 5e5, 2.0)
    s.sync()
    assert abs(float(W.item()) - ref["W"]) <= 1e-10 * abs(ref["W"])
    gh = s.gap_history().cpu().numpy()
    assert np.max(np.abs(gh - gh_ref)) <= 1e-10 * np.max(np.abs(gh_ref))
    assert l2rel(g.cpu().numpy(), ref["grad"]) <= 1e-9


def test_fp32_plane_wave_interior_tiles_match_oracle():
    """80 x 34 x 40 nodes: the box faces cross tiles that are clear of the
    CPML (vector paths) as well as ragged edge tiles; FP32 checkpoints."""
    w = case("f32", nx=80, ny=34, nz=40, design=(26, 12, 10), nsteps=260, tf_margin=2, snapshot_every=16)
    rho = I.rho_uniform(w, 32)
    ref = O.gradient(w, rho, 5e5, 3.0)
    s = solver(w)
    W, g = s.evaluate(rho, 5e5, 3.0)
    s.sync()
    assert abs(float(W.item()) - ref["W"]) <= 1e-4 * abs(ref["W"])
    assert l2rel(g.cpu().numpy(), ref["grad"]) <= 1e-3


def test_plane_wave_graph_replay_and_repeat_are_bit_identical():
    """The incident table is made once at create: a second evaluation, and
    one replayed from CUDA graphs, give the same bits."""
    w = case("f32", snapshot_every=8)
    rho = I.rho_uniform(w, 33)
    s = solver(w)
    s.set_graphs(0)
    W0, g0 = s.evaluate(rho, 0.0, 1.0)
    W0, g0 = float(W0.item()), g0.cpu().numpy().copy()
    W1, g1 = s.evaluate(rho, 0.0, 1.0)
    assert float(W1.item()) == W0 and np.array_equal(g1.cpu().numpy(), g0)
    s.set_graphs(1)
    for _ in range(2):
        W2, g2 = s.evaluate(rho, 0.0, 1.0)
        assert float(W2.item()) == W0 and np.array_equal(g2.cpu().numpy(), g0)


def test_cfg256_code_path_on_a_64_cube_crop():
    """The 256^3 workload's code path (FP32, substrate, plane wave, BF16
    checkpoints every 32 with segment recompute, dx = 5 nm, 12-cell CPML, box
    4 nodes inside it) on a 64^3 grid, against the oracle.  The gradient
    bound is the one stated for BF16 checkpoints."""
    w = I.workload_3d(64, 64, 64, dx=5e-9, nsteps=700, npml=12, design=(20, 20, 12), gap=(4, 4, 4),
                      source="tfsf", tf_margin=4, substrate=True, snapshot_every=32, snapshot_dtype="bf16")
    w.update(I.pulse(800e-9, 300e12))
    rho = I.rho_uniform(w, 34)
    O.set_threads(16)
    try:
        ref = O.gradient(w, rho, 0.0, 10.0)
    finally:
        O.set_threads(1)
    s = solver(w)
    W, g = s.evaluate(rho, 0.0, 10.0)
    s.sync()
    assert abs(float(W.item()) - ref["W"]) <= 1e-4 * abs(ref["W"])
    assert l2rel(g.cpu().numpy(), ref["grad"]) <= 3e-3
