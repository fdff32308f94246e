"""CUDA path vs the FP64 oracle, element by element, through the C ABI.

Small cases are ragged against the kernel's 128 x 4 node tiles (a partial
tile in x, ten tile rows in y) and so run the scalar edge path; the 160^2
workload is the full FP64 parity configuration.  Grids large enough for the
float4 interior path are in test_parity_2d_vector.py.  Tolerances: FP64 fields
agree with the oracle to round-off (W 1e-10 relative, gradient 1e-9
L2-relative); FP32 fields within 1e-4 on W and 1e-3 L2-relative on the
gradient.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2203_01462_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def fast_case(real="f64", **kw):
    """41 x 37 nodes (ragged against 128 x 4 tiles), 6-cell CPML, coarse dx
    and a broadband pulse so that a few hundred steps see it."""
    w = I.small_2d(nx=kw.pop("nx", 41), ny=kw.pop("ny", 37), nsteps=kw.pop("nsteps", 400), dx=20e-9,
                   npml=kw.pop("npml", 6), design=kw.pop("design", (17, 15)), real=real, **kw)
    w.update(I.pulse(800e-9, 300e12))
    return w


def l2rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def solver(w):
    from paper_2203_01462_gb300.binding import Solver
    return Solver(w)


@pytest.mark.parametrize("snap", [0, 7])
@pytest.mark.parametrize("material", ["gold", "silver"])
def test_fp64_small_matches_oracle(snap, material):
    w = fast_case("f64", snapshot_every=snap, material=I.SILVER if material == "silver" else I.GOLD)
    rho = I.rho_uniform(w, 11)
    smax, gs = 5e5, 2.0
    ref = O.gradient(w, rho, smax, gs)
    gh_ref = O.forward(w, rho, smax, gs, record_gap=True)["gap_hist"]
    s = solver(w)
    W, g = s.evaluate(rho, smax, gs)
    s.sync()
    W = float(W.item())
    assert abs(W - ref["W"]) <= 1e-10 * abs(ref["W"])
    gh = s.gap_history().cpu().numpy()
    assert np.max(np.abs(gh - gh_ref)) <= 1e-10 * np.max(np.abs(gh_ref))
    g = g.cpu().numpy()
    assert l2rel(g, ref["grad"]) <= 1e-9


def test_fp32_small_matches_oracle():
    w = fast_case("f32", snapshot_every=16)
    rho = I.rho_uniform(w, 12)
    ref = O.gradient(w, rho, 5e5, 3.0)
    s = solver(w)
    W, g = s.evaluate(rho, 5e5, 3.0)
    s.sync()
    assert abs(float(W.item()) - ref["W"]) <= 1e-4 * abs(ref["W"])
    assert l2rel(g.cpu().numpy(), ref["grad"]) <= 1e-3


def test_fp32_filtered_medium_matches_oracle():
    """Gaussian filter (radius 5, FWHM 5) on a 90 x 80 design box, 1200 steps."""
    w = I.workload_2d(150, 140, dx=10e-9, nsteps=1200, npml=10, design=(90, 80), gap=(3, 3), real="f32",
                      filter_radius=5, filter_fwhm=5.0, snapshot_every=64, src_offset=5)
    w.update(I.pulse(800e-9, 200e12))
    rho = I.rho_uniform(w, 13)
    ref = O.gradient(w, rho, 5e5, 10.0)
    s = solver(w)
    W, g = s.evaluate(rho, 5e5, 10.0)
    s.sync()
    assert abs(float(W.item()) - ref["W"]) <= 1e-4 * abs(ref["W"])
    assert l2rel(g.cpu().numpy(), ref["grad"]) <= 1e-3


def test_cfg_160_fp64_full_matches_oracle():
    """The 160^2 FP64 parity workload: forward, adjoint and gradient."""
    w = I.cfg_2d_160()
    rho = I.rho_uniform(w, 1)
    ref = O.gradient(w, rho, 0.0, 1.0)
    s = solver(w)
    W, g = s.evaluate(rho)
    s.sync()
    assert abs(float(W.item()) - ref["W"]) <= 1e-10 * abs(ref["W"])
    assert l2rel(g.cpu().numpy(), ref["grad"]) <= 1e-9


def test_run_host_matches_device_path():
    w = fast_case("f32")
    rho = I.rho_uniform(w, 14)
    s = solver(w)
    Wd, gd = s.evaluate(rho)
    s.sync()
    Wh, gh = s.run_host(rho.astype(np.float32))
    assert Wh == float(Wd.item())
    np.testing.assert_array_equal(gh, gd.cpu().numpy())


def test_density_out_of_range_is_rejected():
    from paper_2203_01462_gb300.binding import FdtdError
    w = fast_case("f32")
    s = solver(w)
    rho = I.rho_uniform(w, 15)
    rho[3, 4] = 1.5
    with pytest.raises(FdtdError) as e:
        s.set_design(rho)
    assert e.value.status == 7
    s.set_design(I.rho_uniform(w, 15))  # context still usable
    s.forward()
    s.sync()


def test_call_order_is_enforced():
    from paper_2203_01462_gb300.binding import FdtdError
    s = solver(fast_case("f32"))
    with pytest.raises(FdtdError) as e:
        s.forward()
    assert e.value.status == 4
    s.set_design(I.rho_uniform(s.w, 1))
    with pytest.raises(FdtdError) as e:
        s.adjoint()
    assert e.value.status == 4


def test_autograd_matches_oracle_gradient():
    import torch
    from paper_2203_01462_gb300.autograd import objective
    w = fast_case("f64", snapshot_every=9)
    rho = I.rho_uniform(w, 16)
    ref = O.gradient(w, rho, 1e5, 1.0)
    s = solver(w)
    r = torch.tensor(rho, device="cuda", requires_grad=True)
    W = objective(r, s, 1e5, 1.0)
    (3.0 * W).backward()
    assert abs(W.item() - ref["W"]) <= 1e-10 * abs(ref["W"])
    assert l2rel(r.grad.cpu().numpy().reshape(-1), 3.0 * ref["grad"]) <= 1e-9


@pytest.mark.parametrize("real", ["f64", "f32"])
def test_sinc_hanning_excitation_matches_oracle(real):
    """The paper's truncated, Hanning-smoothed sinc excitation (Sec. 2),
    20 % bandwidth around 600 THz, against the oracle."""
    w = fast_case(real, snapshot_every=9 if real == "f32" else 0, nsteps=500)
    w.update(I.sinc_hanning(center_m=500e-9, rel_bandwidth=0.5, lobes=4))
    rho = I.rho_uniform(w, 17)
    ref = O.gradient(w, rho, 0.0, 1.0)
    s = solver(w)
    W, g = s.evaluate(rho, 0.0, 1.0)
    s.sync()
    tol_w, tol_g = (1e-10, 1e-9) if real == "f64" else (1e-4, 1e-3)
    assert abs(float(W.item()) - ref["W"]) <= tol_w * abs(ref["W"])
    assert l2rel(g.cpu().numpy(), ref["grad"]) <= tol_g
