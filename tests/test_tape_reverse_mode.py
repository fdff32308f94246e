"""The paper's adjoint gradient (Eq. 20, 25, 27; the C oracle) against the
exact discrete gradient from reverse-mode differentiation of an independent
FP64 forward (oracle/tape_oracle.py).  With the trapezoidal Drude
discretisation the adjoint recipe is the exact derivative of the discrete
objective, so the two agree to round-off, far tighter than the paper's
"more than 4 digits" against finite differences."""
import numpy as np
import pytest

from oracle import oracle as O
from oracle import tape_oracle as T
from paper_2203_01462_gb300 import inputs as I


def _case(npml, material=None):
    w = I.small_2d(nx=30, ny=28, nsteps=300, dx=20e-9, npml=npml, design=(12, 10), real="f64",
                   material=material)
    w.update(I.pulse(800e-9, 300e12))
    if npml == 0:
        w["src_lo"], w["src_hi"] = [1, 3, 0], [29, 4, 1]
    return w


@pytest.mark.parametrize("npml,material,smax,gs", [(4, "gold", 5e5, 3.0), (0, "silver", 2e5, 1.0),
                                                  (4, "silver", 0.0, 10.0)])
def test_adjoint_equals_exact_discrete_gradient(npml, material, smax, gs):
    w = _case(npml, I.SILVER if material == "silver" else I.GOLD)
    rho = I.zero_gap(w, I.rho_uniform(w, 9) * 0.8 + 0.1).reshape(-1)
    Wt, gt = T.gradient_tm(w, rho, smax, gs)
    ref = O.gradient(w, rho, smax, gs)
    # the two forwards are independent statements of the same scheme
    assert abs(Wt - ref["W"]) <= 1e-12 * abs(ref["W"])
    err = np.linalg.norm(ref["grad"] - gt) / np.linalg.norm(gt)
    assert err <= 1e-12, err  # observed <= 7e-15
