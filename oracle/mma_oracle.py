"""Method of moving asymptotes (MMA) with the conservative inner loop of GCMMA,
for a problem whose only constraints are the bounds 0 <= x <= 1, in FP64 numpy.

Test infrastructure: only the tests, the smoke check and the CPU baseline of
the benchmark use this module; the product path never imports it.

The paper updates its design variables with GCMMA (Sec. 3.2, the design
problem of Eq. 28 has no constraint besides 0 < rho < 1).  This module states
the method from Svanberg's publications:

* K. Svanberg, "The method of moving asymptotes - a new method for structural
  optimization", Int. J. Numer. Meth. Eng. 24 (1987) 359-373: moving
  asymptotes L < x < U and the separable convex approximation
      f~(y) = f(x) + sum_j [p_j/(U_j - y_j) + q_j/(y_j - L_j)]
                   - sum_j [p_j/(U_j - x_j) + q_j/(x_j - L_j)];
* K. Svanberg, "A class of globally convergent optimization methods based on
  conservative convex separable approximations", SIAM J. Optim. 12 (2002)
  555-573: the positive term rho0 in p and q, the inner loop that raises
  rho0 until f~ over-estimates f at the new point (conservative), and hence a
  monotone decrease of f.

Here f is minimised; a caller that maximises W passes f = -s W and its
gradient.  With bounds only, the subproblem min f~ over alpha <= y <= beta is
separable and each coordinate has a closed-form minimiser.

Parameters (Svanberg's usual choices): initial asymptote distance 0.5 of the
box, factors 0.7 (coordinate oscillates) / 1.2 (monotone) / 1.0, distance
kept within [0.01, 10] of the box, alpha and beta at least 0.1 of the way
from the asymptote to x and within `move` of x, the 1.001 / 0.001 split of
the gradient in p and q, rho0 started at 0.1 mean |df| (at least 1e-6) and
raised by min(1.1 (rho0 + delta), 10 rho0).

Where a gradient entry is exactly zero the coordinate is left unchanged (such
entries are the gap nodes, which are not design variables).
"""
from __future__ import annotations

import numpy as np

ASY_INIT = 0.5
ASY_DEC = 0.7
ASY_INC = 1.2
ASY_MIN = 0.01
ASY_MAX = 10.0
ALBEFA = 0.1
RAA0_EPS = 1e-6


def asymptotes(x, x1, x2, L, U, k):
    """L^k, U^k from x^k, x^{k-1}, x^{k-2} and the previous asymptotes (1987, Sec. 3)."""
    x = np.asarray(x, np.float64)
    if k < 2:
        return x - ASY_INIT, x + ASY_INIT
    t = (x - x1) * (x1 - x2)
    fac = np.where(t < 0, ASY_DEC, np.where(t > 0, ASY_INC, 1.0))
    L = x - fac * (x1 - L)
    U = x + fac * (U - x1)
    L = np.clip(L, x - ASY_MAX, x - ASY_MIN)
    U = np.clip(U, x + ASY_MIN, x + ASY_MAX)
    return L, U


def bounds(x, L, U, move):
    """Subproblem box alpha <= y <= beta."""
    alpha = np.maximum(np.maximum(0.0, L + ALBEFA * (x - L)), x - move)
    beta = np.minimum(np.minimum(1.0, U - ALBEFA * (U - x)), x + move)
    return alpha, beta


def pq(x, df, L, U, raa0):
    """Coefficients of the conservative convex separable approximation (2002, Eq. 3.3 form)."""
    pos, neg = np.maximum(df, 0.0), np.maximum(-df, 0.0)
    p = (U - x) ** 2 * (1.001 * pos + 0.001 * neg + raa0)
    q = (x - L) ** 2 * (0.001 * pos + 1.001 * neg + raa0)
    return p, q


def subproblem(x, df, L, U, raa0, move):
    """argmin over alpha <= y <= beta of sum_j p_j/(U_j - y_j) + q_j/(y_j - L_j).

    Each term is convex on (L, U); its stationary point solves
    p/(U-y)^2 = q/(y-L)^2, i.e. y = (sqrt(p) L + sqrt(q) U)/(sqrt(p) + sqrt(q)),
    and the box minimiser is that point clipped to [alpha, beta]."""
    x = np.asarray(x, np.float64)
    p, q = pq(x, df, L, U, raa0)
    alpha, beta = bounds(x, L, U, move)
    sp, sq = np.sqrt(p), np.sqrt(q)
    y = np.clip((sp * L + sq * U) / (sp + sq), alpha, beta)
    y = np.where(df == 0.0, x, y)
    return y, p, q


def approx_change(x, y, p, q, L, U):
    """f~(y) - f(x), written with 1/(U-y) - 1/(U-x) = (y-x)/((U-y)(U-x)) and
    1/(y-L) - 1/(x-L) = (x-y)/((y-L)(x-L)) so that it is exactly 0 at y = x."""
    return float(np.sum(p * (y - x) / ((U - y) * (U - x)) + q * (x - y) / ((y - L) * (x - L))))


def d_term(x, y, L, U):
    """d(y) = sum_j (U_j - L_j)(y_j - x_j)^2 / ((U_j - y_j)(y_j - L_j)) for the box [0, 1] (2002, Sec. 4)."""
    return float(np.sum((U - L) * (y - x) ** 2 / ((U - y) * (y - L))))


def raa0_initial(df):
    return max(RAA0_EPS, 0.1 * float(np.mean(np.abs(df))))


def raa0_raise(raa0, f_new, f_approx, d):
    """rho0 for the next inner iteration when f~(y) < f(y) (not conservative)."""
    delta = (f_new - f_approx) / d
    return min(1.1 * (raa0 + delta), 10.0 * raa0)


def optimality_norm(x, g_ascent):
    """2-norm of the first-order optimality residual of max W over [0,1]^M:
    the gradient with the entries removed where a bound is active and the
    gradient points out of the box."""
    x = np.asarray(x, np.float64)
    r = np.where(((x <= 0.0) & (g_ascent < 0)) | ((x >= 1.0) & (g_ascent > 0)), 0.0, g_ascent)
    return float(np.sqrt(np.sum(r * r)))


def gcmma_minimize(f, grad, x0, iters, move=0.5, max_inner=15, tol=0.0, store=np.float64):
    """Minimise f over [0,1]^n.  f(x) -> float, grad(x) -> array.  `store` is
    the type x is kept in between iterations (float32 mirrors a FP32 design).
    Returns (x, history) with history a list of dicts (f, inner, raa0)."""
    x = np.asarray(x0, store).astype(np.float64)
    x1 = x.copy()
    x2 = x.copy()
    L = np.zeros_like(x)
    U = np.ones_like(x)
    fx = f(x)
    hist = []
    for k in range(iters):
        df = np.asarray(grad(x), np.float64)
        L, U = asymptotes(x, x1, x2, L, U, k)
        x2, x1 = x1, x.copy()
        raa0 = raa0_initial(df)
        for inner in range(max_inner):
            y, p, q = subproblem(x, df, L, U, raa0, move)
            y = y.astype(store).astype(np.float64)
            fy = f(y)
            fa = fx + approx_change(x, y, p, q, L, U)
            if fa + tol >= fy:
                break
            raa0 = raa0_raise(raa0, fy, fa, d_term(x, y, L, U))
        hist.append(dict(f=fy, f_approx=fa, inner=inner + 1, raa0=raa0))
        x, fx = y, fy
    return x, hist
