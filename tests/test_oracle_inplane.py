"""Pins of the oracle's 2D mode with E in plane (Ex, Ey, Hz; the paper's 2D
"TM" case, Sec. 3.2): the paper's design-variable counts, a Drude slab
against the analytic Fresnel result, energy conservation and the Yee mode
frequency of a PEC cavity, the adjoint gradient against central
differences, and the literal objective."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2203_01462_gb300 import inputs as I

C0 = 299792458.0
MU0 = 1.25663706212e-6
EPS0 = 1.0 / (MU0 * C0 * C0)


def test_paper_design_variable_counts():
    """Per-edge design variables outside the observation region: 79 560 for the
    100 x 100 nm box and 319 960 for the 200 x 200 nm box at dx = 0.5 nm."""
    assert O.free_design(I.cfg_2d_inplane_paper(100.0)) == 79560
    assert O.free_design(I.cfg_2d_inplane_paper(200.0)) == 319960


def fast_case(npml=6, nsteps=400, material=None):
    w = I.workload_2d_inplane(41, 37, dx=20e-9, nsteps=nsteps, npml=npml, design=(17, 15), gap=(3, 3),
                              material=material, src_offset=2)
    w.update(I.pulse(800e-9, 300e12))
    if npml == 0:
        w["src_lo"], w["src_hi"] = [1, 3, 0], [39, 4, 1]
    return w


def slab(rho_val, smax=0.0, gscale=1.0, L=20, dx=1e-9):
    """A Drude slab between the PEC plates x = 0 and x = (nx-1) dx: the
    E_x-polarised wave uniform in x is the TEM mode of the plates (E normal to
    them), so a uniform current sheet launches it and the x-CPML, driven by
    x-derivatives only, leaves it alone.  The slab holds L cell rows, i.e.
    L + 1 rows of E_x edges, thickness (L + 1) dx."""
    ny, npml, nx = 1000, 20, 41
    js = npml + 5
    pr, j0 = js + 60, 500
    pt = j0 + L + 60
    base = I.workload_2d_inplane(nx, ny, dx=dx, nsteps=34000, npml=npml, design=(nx - 1, L), gap=(0, 0))
    base.update(src_lo=[0, js, 0], src_hi=[nx - 1, js + 1, 1],
                design_lo=[0, j0, 0], design_hi=[nx - 1, j0 + L, 1], gap_lo=[0, 0, 0], gap_hi=[0, 0, 1])
    ref = dict(base, design_lo=[0, 0, 0], design_hi=[0, 0, 1])
    probes = [(nx // 2, pr), (nx // 2, pt)]
    a = O.forward(base, np.full(I.n_design(base), rho_val), smax, gscale, probes=probes)["probe_hist"]
    b = O.forward(ref, np.zeros(0), probes=probes)["probe_hist"]
    N = a.shape[0]
    dt = base["courant"] * dx / C0
    f = np.fft.rfftfreq(N, dt)
    Fa, Fb = np.fft.rfft(a, axis=0), np.fft.rfft(b, axis=0)
    R = np.abs(Fa[:, 0] - Fb[:, 0]) / np.abs(Fb[:, 0])
    T = np.abs(Fa[:, 1]) / np.abs(Fb[:, 1])
    lam = C0 / np.maximum(f, 1.0)
    sel = (lam > 600e-9) & (lam < 1000e-9)
    w = 2 * np.pi * f[sel]
    psi = base["omega_p"] ** 2
    psis = base["psi_s_ratio"] * psi
    e_inf = base["eps_s"] + rho_val * (base["eps_inf"] - base["eps_s"])
    ps = psis + rho_val * (psi - psis)
    sg = rho_val * (1 - rho_val) * smax
    eps = e_inf - ps / (w ** 2 - 1j * w * base["gamma_p"] * gscale) - 1j * sg / (w * EPS0)
    n = np.sqrt(eps)
    n = np.where(n.imag > 0, -n, n)
    ph = np.exp(-1j * n * (w / C0) * (L + 1) * dx)
    r12 = (1 - n) / (1 + n)
    den = 1 - r12 ** 2 * ph ** 2
    return R[sel], T[sel], np.abs(r12 * (1 - ph ** 2) / den), np.abs((1 - r12 ** 2) * ph / den)


@pytest.mark.parametrize("rho_val,smax,gscale", [(1.0, 0.0, 1.0), (0.5, 5e5, 1.0)])
def test_inplane_drude_slab_matches_fresnel(rho_val, smax, gscale):
    R, T, Ra, Ta = slab(rho_val, smax, gscale)
    assert np.max(np.abs(R - Ra)) < 1e-3
    assert np.max(np.abs(T - Ta)) < 1e-3


def test_inplane_pec_cavity_energy_conserved_and_yee_mode_frequency():
    """Lossless PEC square cavity, E in plane: the discrete energy is constant
    after the source, and the lowest mode (one half wave across the cavity)
    sits at the Yee dispersion sin(w dt/2)/(c dt) = sin(k dx/2)/dx,
    k = pi/((n-1) dx)."""
    n, dx = 24, 20e-9
    w = I.workload_2d_inplane(n, n, dx=dx, nsteps=60000, npml=0, design=(0, 0), gap=(0, 0))
    w.update(I.pulse(3200e-9, 100e12))
    w.update(src_lo=[7, 9, 0], src_hi=[8, 10, 1], design_lo=[0, 0, 0], design_hi=[0, 0, 1],
             gap_lo=[0, 0, 0], gap_hi=[0, 0, 1])
    out = O.forward(w, np.zeros(0), probes=[(5, 6)], energy=True)
    en = out["energy"]
    dt = w["courant"] * dx / C0
    quiet = int((w["t0"] + 7.0 * w["tau"]) / dt) + 1
    tail = en[quiet:]
    assert tail.max() > 0
    assert (tail.max() - tail.min()) / tail.max() < 1e-11
    p = out["probe_hist"][quiet:, 0]
    pad = 1 << 22
    F = np.abs(np.fft.rfft(p * np.hanning(p.size), pad))
    f = np.fft.rfftfreq(pad, dt)
    k = np.pi / ((n - 1) * dx)
    f_yee = 2.0 * np.arcsin(C0 * dt * np.sin(k * dx / 2) / dx) / dt / (2 * np.pi)
    f_cont = C0 * k / (2 * np.pi)
    band = (f > 0.8 * f_yee) & (f < 1.1 * f_yee)
    i = np.flatnonzero(band)[np.argmax(F[band])]
    a, b, c = np.log(F[i - 1]), np.log(F[i]), np.log(F[i + 1])
    f_pk = f[i] + 0.5 * (a - c) / (a - 2 * b + c) * (f[1] - f[0])
    assert abs(f_pk - f_yee) < 0.1 * abs(f_yee - f_cont)


@pytest.mark.parametrize("npml,material", [(0, "gold"), (6, "gold"), (6, "silver")])
def test_inplane_adjoint_gradient_matches_central_differences(npml, material):
    w = fast_case(npml=npml, material=I.SILVER if material == "silver" else I.GOLD)
    r = I.zero_gap(w, I.rho_uniform(w, 4) * 0.8 + 0.1)
    smax, gs = 5e5, 3.0
    g = O.gradient(w, r, smax, gs)["grad"]
    gap = I.gap_edge_mask(w)
    assert np.all(g[gap] == 0.0)
    rng = np.random.default_rng(2)
    nx_edges = I.edge_shapes(w["design_lo"], w["design_hi"])[0]
    nxe = nx_edges[0] * nx_edges[1]
    free = np.flatnonzero(~gap)
    idx = np.concatenate([rng.choice(free[free < nxe], 4, replace=False),
                          rng.choice(free[free >= nxe], 4, replace=False)])
    for i in idx:
        h = 1e-4
        rp, rm = r.copy(), r.copy()
        rp[i] += h
        rm[i] -= h
        fd = (O.objective(w, rp, smax, gs) - O.objective(w, rm, smax, gs)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-5 * abs(fd) + 1e-6 * np.abs(g).max()


def test_inplane_gap_edges_and_linearity():
    w = fast_case()
    r = I.rho_uniform(w, 5)
    W0 = O.objective(w, r)
    r2 = r.copy()
    r2[I.gap_edge_mask(w)] = 0.7  # gap edges are not design variables
    assert O.objective(w, r2) == W0
    w2 = dict(w, src_amp=2.0 * w["src_amp"])
    assert O.objective(w2, r) == pytest.approx(4.0 * W0, rel=1e-12)


def test_inplane_objective_literal_sum():
    """Eq. (24): W = eps_g dt dx^2 / 2 * sum over steps and gap edges of E^2."""
    w = fast_case()
    r = I.rho_uniform(w, 6)
    out = O.forward(w, r, record_gap=True)
    dt = w["courant"] * w["dx"] / C0
    assert out["gap_hist"].shape == (w["nsteps"] + 1, 3 * 4 + 4 * 3)
    assert out["W"] == pytest.approx(0.5 * w["eps_g"] * dt * w["dx"] ** 2 * np.sum(out["gap_hist"] ** 2),
                                     rel=1e-13)
