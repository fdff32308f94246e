"""Host logic of the GCMMA driver (stages, stopping rules, checkpoint /
resume) on the CPU, with a stand-in solver whose objective is a smooth toy
function and whose per-variable MMA steps are the oracle's."""
import numpy as np
import pytest
import torch

from oracle import mma_oracle as M
from paper_2203_01462_gb300.optimize import damping_levels, optimize_gcmma


class ToySolver:
    """W(rho) = exp(-sum a (rho - c)^2 / n) * (1 + 1/gamma_scale); the gap (first entry) has g = 0."""

    def __init__(self, n=40, seed=0, binary=False):
        rng = np.random.default_rng(seed)
        self.n_design = n
        self.device = torch.device("cpu")
        self.real = torch.float32
        self.c = (rng.random(n) > 0.5).astype(float) if binary else rng.uniform(0.1, 0.9, n)
        self.a = rng.uniform(0.5, 3.0, n)
        self.gs = 1.0
        self.rho = None
        self.forwards = 0
        self.adjoints = 0

    def _W(self, r):
        return float(np.exp(-np.sum(self.a * (r - self.c) ** 2) / self.n_design) * (1 + 1 / self.gs))

    def set_design(self, rho):
        self.rho = rho.detach().cpu().numpy().astype(np.float64).reshape(-1).copy()

    def set_damping(self, sigma_max, gamma_scale):
        self.gs = gamma_scale

    def forward(self):
        self.forwards += 1
        return torch.tensor([self._W(self.rho)], dtype=torch.float64)

    def adjoint(self):
        self.adjoints += 1

    def gradient(self):
        r = self.rho
        g = self._W(r) * (-2 * self.a * (r - self.c) / self.n_design)
        g[0] = 0.0
        return torch.tensor(g)

    def evaluate(self, rho, sigma_max, gamma_scale):
        self.set_design(rho)
        self.set_damping(sigma_max, gamma_scale)
        W = self.forward()
        self.adjoint()
        return W, self.gradient()

    def grayness(self):
        r = self.rho[1:]
        return torch.tensor([4 * np.sum(r * (1 - r)) / r.size])

    def sync(self):
        pass

    def mma_state(self):
        return torch.zeros(4 * self.n_design, dtype=torch.float64)

    def mma_asymptotes(self, rho, g, state, k):
        n = self.n_design
        st = state.numpy()
        x = rho.numpy().astype(np.float64)
        gg = g.numpy()
        L, U = M.asymptotes(x, st[:n], st[n:2 * n], st[2 * n:3 * n], st[3 * n:], k)
        st[n:2 * n] = st[:n]
        st[:n] = x
        st[2 * n:3 * n] = L
        st[3 * n:] = U
        return torch.tensor([np.sum(np.abs(gg)), M.optimality_norm(x, gg) ** 2])

    def mma_solve(self, state, g, scale, raa0, move, out):
        n = self.n_design
        st = state.numpy()
        x, L, U = st[:n], st[2 * n:3 * n], st[3 * n:]
        y, p, q = M.subproblem(x, -scale * g.numpy(), L, U, raa0, move)
        y = y.astype(np.float32).astype(np.float64)
        out.copy_(torch.tensor(y, dtype=torch.float32))
        return torch.tensor([M.approx_change(x, y, p, q, L, U), M.d_term(x, y, L, U)])


def test_damping_levels():
    lv = damping_levels(10.0, 6)
    assert lv[0] == 10.0 and lv[-1] == 1.0 and len(lv) == 6
    assert np.allclose(np.diff(np.log10(lv)), -0.2)


def test_monotone_within_stages_and_stage_rule():
    s = ToySolver()
    rho, h = optimize_gcmma(s, np.full(40, 0.5), max_iters=60, levels=[4.0, 1.0], min_inner=3, norm_drop=0.7,
                            zeta_stop=0.0)
    assert h.stop == "max_iters"
    st = np.array(h.stage)
    assert set(st.tolist()) == {0, 1}
    first1 = int(np.argmax(st == 1))
    assert first1 >= 3  # at least min_inner iterations in stage 0
    n0 = np.array(h.opt_norm)[:first1]
    # stage 0 ended at the first iterate (from the 3rd on) with norm <= 0.3 of the stage's first norm
    assert np.all(n0[3:] > 0.3 * n0[0])
    W = np.array(h.W)
    for j in (0, 1):
        w = W[st == j]
        assert np.all(np.diff(w) >= -2e-10 * w[0])  # the driver accepts f~(y) >= f(y) - 1e-10
    np.testing.assert_allclose(rho.numpy()[1:], s.c[1:], atol=1e-4)
    assert rho.numpy()[0] == np.float32(0.5)  # the gap entry never moves


def test_zeta_stop_on_a_binary_optimum():
    s = ToySolver(binary=True, seed=3)
    rho, h = optimize_gcmma(s, np.full(40, 0.5), max_iters=200, levels=[1.0], zeta_stop=0.005)
    assert h.stop == "zeta"
    assert h.zeta[-1] < 0.005 <= h.zeta[-2]


def test_checkpoint_resume_is_exact(tmp_path):
    ck = str(tmp_path / "ck.npz")
    kw = dict(levels=[4.0, 1.0], min_inner=3, zeta_stop=0.0)
    s1 = ToySolver(seed=5)
    r_full, h_full = optimize_gcmma(s1, np.full(40, 0.3), max_iters=14, **kw)
    s2 = ToySolver(seed=5)
    optimize_gcmma(s2, np.full(40, 0.3), max_iters=7, checkpoint=ck, **kw)
    s3 = ToySolver(seed=5)
    r_res, h_res = optimize_gcmma(s3, None, max_iters=14, resume=ck, **kw)
    assert np.array_equal(r_full.numpy(), r_res.numpy())
    assert h_full.W == h_res.W and h_full.stage == h_res.stage and h_full.inner == h_res.inner


def test_filter_widths_schedule():
    """FWHM shrinking geometrically from 5 to 2 cells over 4 stages, as
    Gaussian sigma = FWHM / 2.3548."""
    from paper_2203_01462_gb300.optimize import filter_widths
    w = filter_widths(5.0, 2.0, 4)
    c = 2.0 * np.sqrt(2.0 * np.log(2.0))
    assert len(w) == 4
    assert w[0] == pytest.approx(5.0 / c) and w[-1] == pytest.approx(2.0 / c)
    r = [w[k + 1] / w[k] for k in range(3)]
    assert np.allclose(r, r[0]) and r[0] < 1.0
    assert filter_widths(5.0, 2.0, 1) == [pytest.approx(2.0 / c)]


def test_filter_continuation_is_set_with_each_stage():
    """With widths, the driver sets the stage's filter width before the
    stage's first evaluation, and at resume; the number of widths must match
    the number of damping levels."""
    class Recording(ToySolver):
        def __init__(self):
            super().__init__()
            self.widths = []
            self.events = []

        def set_filter_width(self, sigma):
            self.widths.append(sigma)
            self.events.append(("filter", sigma))

        def set_damping(self, sigma_max, gamma_scale):
            super().set_damping(sigma_max, gamma_scale)
            self.events.append(("damping", gamma_scale))

    s = Recording()
    rho, h = optimize_gcmma(s, np.full(40, 0.5), max_iters=60, levels=[4.0, 2.0, 1.0], min_inner=3, norm_drop=0.7,
                            widths=[2.0, 1.5, 1.0], zeta_stop=0.0)
    stages = sorted(set(h.stage))
    assert stages == [0, 1, 2]
    assert s.widths == [2.0, 1.5, 1.0]
    # each width comes right before the evaluation at its damping level
    for sigma, gs in zip([2.0, 1.5, 1.0], [4.0, 2.0, 1.0]):
        k = s.events.index(("filter", sigma))
        assert s.events[k + 1] == ("damping", gs)
    with pytest.raises(ValueError):
        optimize_gcmma(Recording(), np.full(40, 0.5), max_iters=2, levels=[4.0, 1.0], widths=[1.0])
