"""The Drude-slab reflection / transmission pin run on the GPU: a slab
between PEC plates with E in plane (the TEM mode of the plates, uniform in
x), the field sampled through the gap-spectrum monitor, against the
analytic Fresnel result with eps(w) of Eq. (1) and the interpolation of
Eq. (5)."""
import numpy as np
import pytest

from paper_2203_01462_gb300 import inputs as I

pytestmark = pytest.mark.gpu
C0 = 299792458.0
MU0 = 1.25663706212e-6
EPS0 = 1.0 / (MU0 * C0 * C0)


def _spectrum(w, rho, probe_row, freqs, smax=0.0):
    """E_x(f) on the row ``probe_row``: the first entry of a gap that is one
    full-width cell row.  A full-width gap keeps the field uniform in x; a
    single gap cell would send non-uniform fields into the x-CPML, where the
    slab's Drude metal and an alpha = 0 CPML make the scheme grow."""
    from paper_2203_01462_gb300.binding import Solver
    v = dict(w)
    v["gap_lo"], v["gap_hi"] = [0, probe_row, 0], [w["nx"] - 1, probe_row + 1, 1]
    s = Solver(v)
    s.set_design(I.zero_gap(v, rho))
    s.set_damping(smax, 1.0)
    s.forward()
    z = s.gap_spectrum(freqs).cpu().numpy()[:, 0]
    s.sync()
    return z


@pytest.mark.parametrize("rho_val,smax", [(1.0, 0.0), (0.5, 5e5)])
def test_drude_slab_fresnel_on_the_gpu(rho_val, smax):
    L, dx, nx, ny, npml = 20, 1e-9, 43, 1000, 20
    js = npml + 5
    pr, j0 = js + 60, 500
    pt = j0 + L + 60
    w = I.workload_2d_inplane(nx, ny, dx=dx, nsteps=34000, npml=npml, design=(nx - 1, 1), gap=(0, 0),
                              real="f64", snapshot_every=1000)
    w.update(psi_s_ratio=1e-12,  # the void phase is vacuum
             src_lo=[0, js, 0], src_hi=[nx - 1, js + 1, 1],
             design_lo=[0, pr, 0], design_hi=[nx - 1, pt + 1, 1])
    rho = np.zeros(I.n_design(w))
    rx, ry = I.split_edges(w, rho)  # views
    rx[j0 - pr:j0 - pr + L + 1, :] = rho_val  # L + 1 rows of E_x edges: thickness (L + 1) dx
    ry[j0 - pr:j0 - pr + L, :] = rho_val
    lam = np.linspace(600e-9, 1000e-9, 41)
    f = C0 / lam
    vac = np.zeros_like(rho)
    Rr = _spectrum(w, rho, pr, f, smax) - _spectrum(w, vac, pr, f)
    Rf = _spectrum(w, vac, pr, f)
    Tt = _spectrum(w, rho, pt, f, smax)
    Tf = _spectrum(w, vac, pt, f)
    R, T = np.abs(Rr) / np.abs(Rf), np.abs(Tt) / np.abs(Tf)
    om = 2 * np.pi * f
    psi = w["omega_p"] ** 2
    e_inf = w["eps_s"] + rho_val * (w["eps_inf"] - w["eps_s"])
    ps = w["psi_s_ratio"] * psi + rho_val * (psi - w["psi_s_ratio"] * psi)
    sg = rho_val * (1 - rho_val) * smax
    eps = e_inf - ps / (om ** 2 - 1j * om * w["gamma_p"]) - 1j * sg / (om * EPS0)
    n = np.sqrt(eps)
    n = np.where(n.imag > 0, -n, n)
    ph = np.exp(-1j * n * (om / C0) * (L + 1) * dx)
    r12 = (1 - n) / (1 + n)
    den = 1 - r12 ** 2 * ph ** 2
    Ra, Ta = np.abs(r12 * (1 - ph ** 2) / den), np.abs((1 - r12 ** 2) * ph / den)
    assert np.max(np.abs(R - Ra)) < 1e-3
    assert np.max(np.abs(T - Ta)) < 1e-3
