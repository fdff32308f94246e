"""The three terms of Eq. (25) one at a time, against the oracle's terms.

``fdtd_set_sensitivity_terms`` makes the adjoint accumulate a single term;
the library then returns F^T of that term times its chain-rule factor
(Eq. 27).  The oracle reports the Eq. (25a-c) sensitivities themselves, so
the expected values are (psi - psi_s) dW/dpsi_i, (eps_inf - eps_s)
dW/deps_i and dsigma_i/drho~ dW/dsigma_i, through F^T.  Silver (eps_inf != 1)
keeps every term non-zero.  FP64: each term to 1e-9 L2-relative, and the
three add up to the full gradient."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2203_01462_gb300 import inputs as I

pytestmark = pytest.mark.gpu

SMAX, GS = 5e5, 2.0


def l2rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def expected_terms(w, rho):
    ref = O.gradient(w, rho, SMAX, GS, parts=True)
    psi = w["omega_p"] ** 2
    rt = O.filt(w, rho) if w.get("filter_radius", 0) else np.asarray(rho, dtype=np.float64).reshape(-1)
    dsdr = SMAX * (1.0 - 2.0 * rt) * (4.0 if w.get("sigma_form", 0) else 1.0)
    parts = {1: (1.0 - w["psi_s_ratio"]) * psi * ref["g_psi"],
             2: (w["eps_inf"] - w["eps_s"]) * ref["g_eps"],
             4: dsdr * ref["g_sig"]}
    if w.get("filter_radius", 0):
        # F^T, then the gap entries zeroed, as for the full gradient
        shape = I.design_shape(w)
        parts = {k: I.zero_gap(w, O.filt(w, v, transpose=True).reshape(shape)).reshape(-1)
                 for k, v in parts.items()}
    return ref["grad"], parts


def check(w, rho):
    from paper_2203_01462_gb300.binding import Solver, TERM_ALL
    full_ref, parts = expected_terms(w, rho)
    s = Solver(w)
    got = {}
    for term in (1, 2, 4):
        s.set_sensitivity_terms(term)
        _, g = s.evaluate(rho, SMAX, GS)
        got[term] = g.cpu().numpy().copy()
        assert np.linalg.norm(parts[term]) > 1e-3 * np.linalg.norm(full_ref), term
        assert l2rel(got[term], parts[term]) <= 1e-9, term
    s.set_sensitivity_terms(TERM_ALL)
    _, g = s.evaluate(rho, SMAX, GS)
    full = g.cpu().numpy()
    assert l2rel(full, full_ref) <= 1e-9
    assert l2rel(got[1] + got[2] + got[4], full) <= 1e-12


def test_terms_2d_ez_filtered():
    w = I.small_2d(nx=41, ny=37, nsteps=400, dx=20e-9, npml=6, design=(17, 15), real="f64", material=I.SILVER,
                   filter_radius=2, filter_fwhm=2.0)
    w.update(I.pulse(800e-9, 300e12))
    check(w, I.rho_uniform(w, 51))


def test_terms_2d_inplane():
    w = I.workload_2d_inplane(41, 37, dx=20e-9, nsteps=400, npml=6, design=(17, 15), gap=(3, 3), real="f64",
                              material=I.SILVER, src_offset=2)
    w.update(I.pulse(800e-9, 300e12))
    check(w, I.rho_uniform(w, 52))


def test_terms_3d_plane_wave():
    w = I.workload_3d(21, 19, 31, dx=20e-9, nsteps=220, npml=4, design=(9, 7, 6), gap=(2, 2, 2), source="tfsf",
                      substrate=True, material=I.SILVER, real="f64", tf_margin=1)
    w.update(I.pulse(800e-9, 300e12))
    check(w, I.rho_uniform(w, 53))


def test_term_mask_is_checked():
    from paper_2203_01462_gb300.binding import FdtdError, Solver
    w = I.small_2d(nx=41, ny=37, nsteps=10, dx=20e-9, npml=6, design=(17, 15), real="f64")
    s = Solver(w)
    for bad in (0, 8, -1):
        with pytest.raises(FdtdError) as e:
            s.set_sensitivity_terms(bad)
        assert e.value.status == 1
