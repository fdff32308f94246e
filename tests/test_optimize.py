"""Optimization-loop kernels and driver: zeta against the oracle, the ascent
step and the threshold against numpy, and an optimization run whose
objective rises (the paper reports a monotonically increasing objective)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2203_01462_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def medium(real="f32"):
    w = I.workload_2d(150, 140, dx=10e-9, nsteps=900, npml=10, design=(90, 80), gap=(3, 3), real=real,
                      filter_radius=3, filter_fwhm=3.0, src_offset=5)
    w.update(I.pulse(800e-9, 200e12))
    return w


def test_grayness_matches_oracle():
    import torch
    from paper_2203_01462_gb300.binding import Solver
    w = medium("f64")
    rho = I.rho_uniform(w, 51)
    s = Solver(w)
    s.set_design(rho)
    z = float(s.grayness().item())
    assert abs(z - O.grayness(w, rho)) <= 1e-12


def test_ascent_and_threshold_kernels():
    import torch
    from paper_2203_01462_gb300.binding import Solver
    w = medium("f32")
    s = Solver(w)
    rng = np.random.default_rng(52)
    rho = rng.random(s.n_design).astype(np.float32)
    g = rng.standard_normal(s.n_design)
    r = torch.tensor(rho, device="cuda")
    gt = torch.tensor(g, device="cuda")
    s.ascent_step(r, gt, 0.1)
    ref = np.clip(rho.astype(np.float64) + 0.1 * g / np.abs(g).max(), 0.0, 1.0).astype(np.float32)
    np.testing.assert_array_equal(r.cpu().numpy(), ref)
    s.threshold(r, 0.5)
    np.testing.assert_array_equal(r.cpu().numpy(), (ref >= 0.5).astype(np.float32))


def test_plain_optimization_raises_the_objective():
    from paper_2203_01462_gb300.binding import Solver
    from paper_2203_01462_gb300.optimize import final_design, optimize
    w = medium("f32")
    s = Solver(w)
    rho0 = I.zero_gap(w, np.full(I.design_shape(w), 0.5))
    rho, h = optimize(s, rho0, iters=12, move=0.1, damping_start=1.0, damping_iters=0)
    W = np.array(h.W)
    assert W[-1] > 2.0 * W[0]
    assert np.sum(np.diff(W) > 0) >= len(W) - 3
    _, Wbin = final_design(s, rho)
    assert Wbin > 0


@pytest.mark.parametrize("real", ["f64", "f32"])
@pytest.mark.parametrize("k", [0, 1, 5])
def test_mma_kernels_match_oracle(real, k):
    import torch
    from oracle import mma_oracle as M
    from paper_2203_01462_gb300.binding import Solver
    w = medium(real)
    s = Solver(w)
    n = s.n_design
    npt = np.float64 if real == "f64" else np.float32
    rng = np.random.default_rng(60 + k)
    x = rng.random(n).astype(npt)
    x[rng.random(n) < 0.05] = 0.0
    x[rng.random(n) < 0.05] = 1.0
    g = rng.standard_normal(n) * 1e-30
    g[rng.random(n) < 0.03] = 0.0
    x1 = rng.random(n)
    x2 = rng.random(n)
    L0 = x1 - rng.uniform(0.01, 1.0, n)
    U0 = x1 + rng.uniform(0.01, 1.0, n)
    state = torch.tensor(np.concatenate([x1, x2, L0, U0]), device="cuda")
    xt = torch.tensor(x, device="cuda")
    gt = torch.tensor(g, device="cuda")
    sums = s.mma_asymptotes(xt, gt, state, k).cpu().numpy()
    xd = x.astype(np.float64)
    L, U = M.asymptotes(xd, x1, x2, L0, U0, k)
    st = state.cpu().numpy()
    np.testing.assert_array_equal(st[:n], xd)
    np.testing.assert_array_equal(st[n:2 * n], x1)
    np.testing.assert_allclose(st[2 * n:3 * n], L, rtol=0, atol=4e-15)
    np.testing.assert_allclose(st[3 * n:], U, rtol=0, atol=4e-15)
    assert sums[0] == pytest.approx(np.sum(np.abs(g)), rel=1e-12)
    assert sums[1] == pytest.approx(M.optimality_norm(xd, g) ** 2, rel=1e-12)
    scale, raa0, move = 3e29, 1e-3, 0.3
    out = torch.empty(n, dtype=xt.dtype, device="cuda")
    sd = s.mma_solve(state, gt, scale, raa0, move, out).cpu().numpy()
    y, p, q = M.subproblem(xd, -scale * g, L, U, raa0, move)
    y = y.astype(npt)
    got = out.cpu().numpy()
    if real == "f64":
        np.testing.assert_allclose(got, y, rtol=0, atol=1e-14)
    else:
        # the FP64 minimiser may differ in its last bits, so the FP32 rounding may differ by one ulp
        assert np.max(np.abs(got.astype(np.float64) - y)) <= 2 ** -24 * 1.0001
        assert np.mean(got != y) < 1e-3
    yd = got.astype(np.float64)
    assert np.array_equal(got[g == 0], x[g == 0])
    assert sd[0] == pytest.approx(M.approx_change(xd, yd, p, q, L, U), rel=1e-10)
    assert sd[1] == pytest.approx(M.d_term(xd, yd, L, U), rel=1e-10)


def test_gcmma_on_the_device_is_monotone_and_resumes_exactly(tmp_path):
    from paper_2203_01462_gb300.binding import Solver
    from paper_2203_01462_gb300.optimize import optimize_gcmma
    w = medium("f32")
    s = Solver(w)
    rho0 = I.zero_gap(w, np.full(I.design_shape(w), 0.3))
    kw = dict(levels=[3.0, 1.0], min_inner=2, norm_drop=0.5, zeta_stop=0.0, move=0.2)
    r_full, h = optimize_gcmma(s, rho0, max_iters=8, **kw)
    W = np.array(h.W)
    st = np.array(h.stage)
    assert W[-1] > 1.5 * W[0]
    for j in set(st.tolist()):
        wj = W[st == j]
        assert np.all(np.diff(wj) >= -2e-10 * wj[0])
    ck = str(tmp_path / "gcmma.npz")
    optimize_gcmma(Solver(w), rho0, max_iters=4, checkpoint=ck, **kw)
    r_res, h_res = optimize_gcmma(Solver(w), None, max_iters=8, resume=ck, **kw)
    assert np.array_equal(r_full.cpu().numpy(), r_res.cpu().numpy())
    assert h.W == h_res.W and h.inner == h_res.inner


def test_filter_width_change_matches_oracle():
    """fdtd_set_filter_width: after narrowing the filter of a context, W~ and
    the gradient (F^T with the new width) match the oracle run with that
    width (FP64); the design has to be set again after the change."""
    from paper_2203_01462_gb300.binding import FdtdError, Solver
    w = medium("f64")
    rho = I.rho_uniform(w, 53)
    s = Solver(w)
    s.evaluate(rho, 5e5, 2.0)
    s.set_filter_width(0.7)
    with pytest.raises(FdtdError) as e:
        s.forward()
    assert e.value.status == 4
    W, g = s.evaluate(rho, 5e5, 2.0)
    s.sync()
    ref = O.gradient(dict(w, filter_sigma=0.7), rho, 5e5, 2.0)
    assert abs(float(W.item()) - ref["W"]) <= 1e-10 * abs(ref["W"])
    gg = g.cpu().numpy()
    assert np.linalg.norm(gg - ref["grad"]) <= 1e-9 * np.linalg.norm(ref["grad"])


def test_gcmma_with_filter_continuation_ends_on_the_last_width():
    """GCMMA through two damping stages with the filter narrowing from FWHM 3
    to 1.5 cells: the objective the driver reports for its final design is
    the oracle's W~ of that design with the last filter width and damping."""
    import torch
    from paper_2203_01462_gb300.binding import Solver
    from paper_2203_01462_gb300.optimize import filter_widths, optimize_gcmma
    w = medium("f64")
    s = Solver(w)
    rho0 = I.zero_gap(w, np.full(I.design_shape(w), 0.3))
    widths = filter_widths(3.0, 1.5, 2)
    rho, h = optimize_gcmma(s, rho0, max_iters=8, levels=[3.0, 1.0], min_inner=2, norm_drop=-1e9, zeta_stop=0.0,
                            widths=widths)
    assert 1 in h.stage
    ref = O.forward(dict(w, filter_sigma=widths[-1]), rho.cpu().numpy(), 0.0, 1.0)["W"]
    assert abs(h.W[-1] - ref) <= 1e-9 * abs(ref)
