"""3D CUDA path vs the FP64 oracle, through the C ABI.

Grids are small and ragged against the 32 x 4 x 2 thread blocks; every CPML
slab, the design box, the gap and the source are exercised.  FP64 fields
agree with the oracle to round-off; FP32 within 1e-4 (W) and 1e-3
(gradient, L2-relative)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2203_01462_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def case3d(real="f64", source="dipole", npml=4, material=None, nsteps=220, **kw):
    w = I.workload_3d(kw.pop("nx", 21), kw.pop("ny", 19), kw.pop("nz", 23), dx=20e-9, nsteps=nsteps, npml=npml,
                      design=kw.pop("design", (9, 7, 6)), gap=(2, 2, 2), source=source, material=material,
                      real=real, **kw)
    w.update(I.pulse(800e-9, 300e12))
    return w


def l2rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def solver(w):
    from paper_2203_01462_gb300.binding import Solver
    return Solver(w)


@pytest.mark.parametrize("snap", [0, 9])
@pytest.mark.parametrize("source,material", [("dipole", "gold"), ("sheet", "silver")])
def test_fp64_3d_matches_oracle(snap, source, material):
    w = case3d("f64", source, material=I.SILVER if material == "silver" else I.GOLD, snapshot_every=snap)
    rho = I.rho_uniform(w, 21)
    ref = O.gradient(w, rho, 5e5, 2.0)
    gh_ref = O.forward(w, rho, 5e5, 2.0, record_gap=True)["gap_hist"]
    s = solver(w)
    W, g = s.evaluate(rho, 5e5, 2.0)
    s.sync()
    assert abs(float(W.item()) - ref["W"]) <= 1e-10 * abs(ref["W"])
    gh = s.gap_history().cpu().numpy()
    assert np.max(np.abs(gh - gh_ref)) <= 1e-10 * np.max(np.abs(gh_ref))
    assert l2rel(g.cpu().numpy(), ref["grad"]) <= 1e-9


def test_fp32_3d_substrate_sheet_matches_oracle():
    w = case3d("f32", "sheet", substrate=True, snapshot_every=16, nx=26, ny=24, nz=30, npml=6,
               design=(10, 9, 6), nsteps=300)
    rho = I.rho_uniform(w, 22)
    ref = O.gradient(w, rho, 5e5, 1.0)
    s = solver(w)
    W, g = s.evaluate(rho, 5e5, 1.0)
    s.sync()
    assert abs(float(W.item()) - ref["W"]) <= 1e-4 * abs(ref["W"])
    assert l2rel(g.cpu().numpy(), ref["grad"]) <= 1e-3


def test_fp32_3d_dipole_run_host():
    w = case3d("f32", "dipole", snapshot_every=0)
    rho = I.rho_uniform(w, 23)
    ref = O.gradient(w, rho)
    s = solver(w)
    Wh, gh = s.run_host(rho.astype(np.float32))
    assert abs(Wh - ref["W"]) <= 1e-4 * abs(ref["W"])
    assert l2rel(gh, ref["grad"]) <= 1e-3


@pytest.mark.parametrize("real,source", [("f64", "sheet"), ("f32", "dipole")])
def test_3d_interior_tiles_match_oracle(real, source):
    """80 x 34 x 34 nodes, 4-cell CPML: some 32 x 8 x 4 tiles are clear of the
    CPML (vector kernels) and hold design, gap and source nodes."""
    w = case3d(real, source, npml=4, nx=80, ny=34, nz=34, design=(26, 12, 10), nsteps=200, snapshot_every=16,
               substrate=(source == "sheet"))
    rho = I.rho_uniform(w, 24)
    ref = O.gradient(w, rho, 5e5, 3.0)
    s = solver(w)
    W, g = s.evaluate(rho, 5e5, 3.0)
    s.sync()
    tol_w, tol_g = (1e-10, 1e-9) if real == "f64" else (1e-4, 1e-3)
    assert abs(float(W.item()) - ref["W"]) <= tol_w * abs(ref["W"])
    assert l2rel(g.cpu().numpy(), ref["grad"]) <= tol_g


@pytest.mark.slow
def test_cfg512_code_path_on_a_64_cube_crop():
    """The 512 x 512 x 384 configuration's code path (z-dipole in the gap, two
    bands 650-750 and 850-950 nm, FP16 per-slab checkpoints with segment
    recompute, FP32 fields) on a 64^3 crop: 64^3 nodes, 12-cell CPML, 32 x 32 x 24
    design box, 4400 steps (the two-band pulse peaks near step 3860), against the
    FP64 oracle."""
    big = I.cfg_3d_512()
    w = I.workload_3d(64, 64, 64, dx=5e-9, nsteps=4400, npml=12, design=(32, 32, 24), gap=(4, 4, 4),
                      source="dipole", snapshot_every=100, snapshot_dtype="f16")
    for key in ("nbands", "f0", "tau", "t0"):
        w[key] = big[key]
    rho = I.rho_uniform(w, 25)
    O.set_threads(16)
    ref = O.gradient(w, rho, 0.0, 1.0)
    O.set_threads(1)
    s = solver(w)
    W, g = s.evaluate(rho)
    s.sync()
    assert abs(float(W.item()) - ref["W"]) <= 1e-4 * abs(ref["W"])
    assert l2rel(g.cpu().numpy(), ref["grad"]) <= 1e-3


def test_sinc_hanning_dipole_3d_matches_oracle():
    """The paper's sinc-Hanning excitation on the 3D dipole source."""
    w = case3d("f64", "dipole", nsteps=260)
    w.update(I.sinc_hanning(center_m=500e-9, rel_bandwidth=0.5, lobes=4))
    rho = I.rho_uniform(w, 29)
    ref = O.gradient(w, rho, 0.0, 1.0)
    s = solver(w)
    W, g = s.evaluate(rho, 0.0, 1.0)
    s.sync()
    assert abs(float(W.item()) - ref["W"]) <= 1e-10 * abs(ref["W"])
    assert l2rel(g.cpu().numpy(), ref["grad"]) <= 1e-9
