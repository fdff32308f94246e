"""2D mode with E in plane (Ex, Ey, Hz, per-edge design; the paper's 2D
"TM" case) against the FP64 oracle, element by element, through the C ABI.
Tolerances as for the other modes: FP64 W 1e-10, gap history 1e-10,
gradient 1e-9 L2; FP32 W 1e-4 and gradient 1e-3 L2."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2203_01462_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def case(real="f64", npml=6, material=None, nsteps=400, **kw):
    w = I.workload_2d_inplane(kw.pop("nx", 41), kw.pop("ny", 37), dx=20e-9, nsteps=nsteps, npml=npml,
                              design=kw.pop("design", (17, 15)), gap=kw.pop("gap", (3, 3)), real=real,
                              material=material, src_offset=2, **kw)
    w.update(I.pulse(800e-9, 300e12))
    if npml == 0:
        w["src_lo"], w["src_hi"] = [1, 3, 0], [w["nx"] - 2, 4, 1]
    return w


def l2rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def solver(w):
    from paper_2203_01462_gb300.binding import Solver
    return Solver(w)


@pytest.mark.parametrize("snap", [0, 7])
@pytest.mark.parametrize("npml,material", [(6, "gold"), (6, "silver"), (0, "gold")])
def test_fp64_inplane_matches_oracle(snap, npml, material):
    w = case("f64", npml=npml, material=I.SILVER if material == "silver" else I.GOLD, snapshot_every=snap)
    rho = I.rho_uniform(w, 41)
    smax, gs = 5e5, 2.0
    ref = O.gradient(w, rho, smax, gs)
    gh_ref = O.forward(w, rho, smax, gs, record_gap=True)["gap_hist"]
    s = solver(w)
    assert s.n_design == rho.size and s.n_gap == gh_ref.shape[1]
    W, g = s.evaluate(rho, smax, gs)
    s.sync()
    assert abs(float(W.item()) - ref["W"]) <= 1e-10 * abs(ref["W"])
    gh = s.gap_history().cpu().numpy()
    assert np.max(np.abs(gh - gh_ref)) <= 1e-10 * np.max(np.abs(gh_ref))
    g = g.cpu().numpy()
    assert l2rel(g, ref["grad"]) <= 1e-9
    assert np.all(g[I.gap_edge_mask(w)] == 0.0)


@pytest.mark.parametrize("snap,dtype,tol", [(16, "f32", 1e-3), (16, "f16", 1e-3)])
def test_fp32_inplane_matches_oracle(snap, dtype, tol):
    w = case("f32", nx=70, ny=58, design=(30, 24), gap=(4, 4), nsteps=600, snapshot_every=snap,
             snapshot_dtype=dtype)
    rho = I.rho_uniform(w, 42)
    ref = O.gradient(w, rho, 5e5, 3.0)
    s = solver(w)
    W, g = s.evaluate(rho, 5e5, 3.0)
    s.sync()
    assert abs(float(W.item()) - ref["W"]) <= 1e-4 * abs(ref["W"])
    assert l2rel(g.cpu().numpy(), ref["grad"]) <= tol


def test_inplane_sinc_hanning_bowtie_fp64():
    w = case("f64", nsteps=500)
    w.update(I.sinc_hanning(center_m=500e-9, rel_bandwidth=0.5, lobes=4))
    rho = 0.05 + 0.9 * I.rho_bowtie(w)
    rho = I.zero_gap(w, rho)
    ref = O.gradient(w, rho, 0.0, 1.0)
    s = solver(w)
    W, g = s.evaluate(rho, 0.0, 1.0)
    s.sync()
    assert abs(float(W.item()) - ref["W"]) <= 1e-10 * abs(ref["W"])
    assert l2rel(g.cpu().numpy(), ref["grad"]) <= 1e-9


def test_paper_geometry_design_counts():
    """The library's per-edge design vector for the paper's 100 nm and 200 nm
    boxes: M_d - M_g = 79 560 and 319 960 free design variables."""
    for d, free in ((100.0, 79560), (200.0, 319960)):
        s = solver(I.cfg_2d_inplane_paper(d, nsteps=10))
        assert s.n_design - s.n_gap == free


def test_inplane_grayness_and_gcmma_raise_the_objective():
    from paper_2203_01462_gb300.optimize import optimize_gcmma
    w = case("f32", nx=70, ny=58, design=(30, 24), gap=(4, 4), nsteps=600)
    s = solver(w)
    rho0 = I.zero_gap(w, np.full(I.n_design(w), 0.5))
    s.set_design(rho0)
    z = float(s.grayness().item())
    assert z == pytest.approx(1.0, rel=1e-6)
    rho, h = optimize_gcmma(s, rho0, max_iters=6, levels=[1.0], zeta_stop=0.0, move=0.2)
    assert h.W[-1] > h.W[0]
    assert np.all(np.diff(h.W) >= -2e-10 * h.W[0])
