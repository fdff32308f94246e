"""Pins of the MMA / GCMMA oracle (the design update of Sec. 3.2) against
what the mathematics fixes: the closed-form subproblem minimiser against a
brute-force search, convergence to the known minimiser of separable and
non-separable test functions, the monotone decrease that conservativeness
guarantees, and the first-order optimality residual at a known optimum."""
import numpy as np
import pytest

from oracle import mma_oracle as M


def test_subproblem_closed_form_is_the_box_minimiser():
    rng = np.random.default_rng(1)
    n = 400
    x = rng.random(n)
    df = rng.standard_normal(n) * np.where(rng.random(n) < 0.1, 100.0, 1.0)
    L = x - rng.uniform(0.01, 2.0, n)
    U = x + rng.uniform(0.01, 2.0, n)
    raa0 = 1e-3
    y, p, q = M.subproblem(x, df, L, U, raa0, move=0.3)
    alpha, beta = M.bounds(x, L, U, 0.3)
    for j in range(n):
        t = np.linspace(alpha[j], beta[j], 20001)
        v = p[j] / (U[j] - t) + q[j] / (t - L[j])
        tb = t[np.argmin(v)]
        assert abs(y[j] - tb) <= (beta[j] - alpha[j]) / 20000 + 1e-12
        # first-order agreement: the approximation's derivative at x is df
        g = p[j] / (U[j] - x[j]) ** 2 - q[j] / (x[j] - L[j]) ** 2
        assert abs(g - df[j]) <= 1e-12 * max(1.0, abs(df[j]))
    # a zero gradient entry (a gap node) stays where it is
    gap = np.zeros(5)
    y0, _, _ = M.subproblem(np.full(5, 0.3), gap, np.full(5, -0.2), np.full(5, 0.8), 1e-3, 0.5)
    assert np.array_equal(y0, np.full(5, 0.3))


@pytest.mark.parametrize("c", [np.array([0.2, 0.5, 0.9, 0.37]), np.array([-0.4, 1.3, 0.61, 1.0])])
def test_separable_quadratic_converges_to_projection(c):
    a = np.array([1.0, 3.0, 0.5, 10.0])
    f = lambda x: float(np.sum(a * (x - c) ** 2))
    g = lambda x: 2 * a * (x - c)
    x, h = M.gcmma_minimize(f, g, np.full(4, 0.5), iters=60)
    np.testing.assert_allclose(x, np.clip(c, 0, 1), atol=1e-6)
    fs = [e["f"] for e in h]
    assert all(b <= a_ + 1e-15 for a_, b in zip([f(np.full(4, 0.5))] + fs, fs))


def test_rosenbrock_in_the_unit_box():
    # Rosenbrock in x = 2u - 0.5: minimiser x = (1, 1), i.e. u = (0.75, 0.75); non-convex valley
    def f(u):
        x = 2 * u - 0.5
        return float(100 * (x[1] - x[0] ** 2) ** 2 + (1 - x[0]) ** 2)

    def g(u):
        x = 2 * u - 0.5
        return 2 * np.array([-400 * x[0] * (x[1] - x[0] ** 2) - 2 * (1 - x[0]), 200 * (x[1] - x[0] ** 2)])

    u, h = M.gcmma_minimize(f, g, np.array([0.1, 0.9]), iters=400, max_inner=50)
    np.testing.assert_allclose(u, [0.75, 0.75], atol=2e-3)
    fs = [f(np.array([0.1, 0.9]))] + [e["f"] for e in h]
    assert np.all(np.diff(fs) <= 1e-12), "GCMMA must decrease f monotonically"
    assert any(e["inner"] > 1 for e in h), "the conservative inner loop must have been exercised"


def test_every_accepted_point_is_conservative():
    rng = np.random.default_rng(3)
    A = rng.standard_normal((30, 30))
    Q = A @ A.T / 30 + np.eye(30)
    b = rng.standard_normal(30)
    f = lambda x: float(0.5 * x @ Q @ x - b @ x + 0.3 * np.sum(np.sin(7 * x)))
    g = lambda x: Q @ x - b + 2.1 * np.cos(7 * x)
    _, h = M.gcmma_minimize(f, g, np.full(30, 0.5), iters=40, max_inner=60)
    for e in h:
        assert e["f_approx"] >= e["f"]


def test_float32_storage_keeps_monotone_decrease():
    c = np.linspace(0.05, 0.95, 64)
    f = lambda x: float(np.sum((x - c) ** 2 * (1 + c)))
    g = lambda x: 2 * (x - c) * (1 + c)
    x, h = M.gcmma_minimize(f, g, np.zeros(64), iters=40, store=np.float32)
    assert np.all(np.diff([e["f"] for e in h]) <= 1e-12)
    np.testing.assert_allclose(x, c, atol=1e-6)


def test_optimality_norm():
    # at the box maximiser of W = -sum (x - c)^2 with c outside the box the residual is zero
    c = np.array([-0.5, 0.3, 1.7])
    x = np.clip(c, 0, 1)
    assert M.optimality_norm(x, -2 * (x - c)) == 0.0
    # interior point: the plain gradient norm
    x = np.array([0.2, 0.4, 0.6])
    gr = -2 * (x - c)
    assert M.optimality_norm(x, gr) == pytest.approx(np.linalg.norm(gr), rel=1e-15)
