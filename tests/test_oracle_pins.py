"""Pins of the FP64 CPU oracle against physics and mathematics it must obey.

None of these compares the oracle with itself: each checks it against a
closed form (Fresnel coefficients of a Drude slab, radiation of a current
sheet, the exact Yee dispersion of a PEC cavity), a conservation law, a
library routine (scipy's Gaussian filter) or an independent differentiation
(central finite differences of the forward solve).
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2203_01462_gb300 import inputs as I

C0 = 299792458.0
MU0 = 1.25663706212e-6
EPS0 = 1.0 / (MU0 * C0 * C0)


def fast_case(npml=6, nsteps=400, **kw):
    """Small grid, coarse dx and a broadband pulse so that 400 steps see it."""
    w = I.small_2d(nx=40, ny=36, nsteps=nsteps, dx=20e-9, npml=npml, design=(16, 14), **kw)
    w.update(I.pulse(800e-9, 300e12))
    if npml == 0:
        w["src_lo"] = [1, 3, 0]
        w["src_hi"] = [39, 4, 1]
    return w


def slab(rho_val, smax=0.0, gscale=1.0, L=20, dx=1e-9):
    """Normal-incidence Drude slab in a periodic-x strip; returns the FFT
    reflection and transmission magnitudes and the analytic Fresnel ones."""
    ny, npml = 1000, 20
    js = npml + 5
    pr, j0 = js + 60, 500
    pt = j0 + L + 60
    base = I.workload_2d(4, ny, dx=dx, nsteps=34000, npml=npml, design=(4, L), gap=(0, 0))
    base.update(periodic_x=1, src_lo=[0, js, 0], src_hi=[4, js + 1, 1],
                design_lo=[0, j0, 0], design_hi=[4, j0 + L, 1],
                gap_lo=[0, 0, 0], gap_hi=[0, 0, 1])
    ref = dict(base, design_lo=[0, 0, 0], design_hi=[0, 0, 1])
    probes = [(1, pr), (1, pt)]
    a = O.forward(base, np.full(4 * L, rho_val), smax, gscale, probes=probes)["probe_hist"]
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
    # Eq. (4)/(5): interpolated Drude + artificial conductivity, e^{jwt}.
    psi = base["omega_p"] ** 2
    psis = base["psi_s_ratio"] * psi
    e_inf = base["eps_s"] + rho_val * (base["eps_inf"] - base["eps_s"])
    ps = psis + rho_val * (psi - psis)
    sg = rho_val * (1 - rho_val) * smax
    eps = e_inf - ps / (w ** 2 - 1j * w * base["gamma_p"] * gscale) - 1j * sg / (w * EPS0)
    n = np.sqrt(eps)
    n = np.where(n.imag > 0, -n, n)           # decaying into the slab
    ph = np.exp(-1j * n * (w / C0) * L * dx)
    r12 = (1 - n) / (1 + n)
    den = 1 - r12 ** 2 * ph ** 2
    return R[sel], T[sel], np.abs(r12 * (1 - ph ** 2) / den), np.abs((1 - r12 ** 2) * ph / den)


@pytest.mark.parametrize("rho_val,smax,gscale", [
    (1.0, 0.0, 1.0),      # Eq. (1): the Drude metal itself
    (0.0, 0.0, 1.0),      # Eq. (5) at rho = 0: eps_s with psi_s = psi / 100
    (0.5, 5e5, 1.0),      # Eq. (4)/(5c): halfway material plus sigma_max / 4
    (1.0, 0.0, 10.0),     # damping level: gamma x 10
])
def test_drude_slab_matches_fresnel(rho_val, smax, gscale):
    R, T, Ra, Ta = slab(rho_val, smax, gscale)
    assert np.max(np.abs(R - Ra)) < 1e-3
    assert np.max(np.abs(T - Ta)) < 1e-3


def test_sheet_current_radiates_half_eta_K():
    """A uniform current sheet K(t) in vacuum radiates E = -(eta0/2) K(t - d/c);
    with K = J_src dx = src_amp eps0 c0 g(t) this is E = -src_amp g(t - d/c) / 2."""
    dx, ny, npml = 5e-9, 800, 20
    js, D = npml + 5, 300
    w = I.workload_2d(4, ny, dx=dx, nsteps=9000, npml=npml, design=(0, 0), gap=(0, 0))
    w.update(periodic_x=1, src_lo=[0, js, 0], src_hi=[4, js + 1, 1],
             design_lo=[0, 0, 0], design_hi=[0, 0, 1], gap_lo=[0, 0, 0], gap_hi=[0, 0, 1],
             src_amp=2.0)
    e = O.forward(w, np.zeros(0), probes=[(2, js + D)])["probe_hist"][:, 0]
    dt = w["courant"] * dx / C0
    t = np.arange(e.size) * dt - D * dx / C0
    g = np.exp(-((t - w["t0"]) / w["tau"]) ** 2) * np.sin(2 * np.pi * w["f0"][0] * (t - w["t0"]))
    expect = -0.5 * w["src_amp"] * g
    assert np.max(np.abs(expect)) > 0.9
    assert np.max(np.abs(e - expect)) < 3e-3 * np.max(np.abs(expect))


def test_pec_cavity_energy_conserved_and_yee_mode_frequency():
    """Lossless PEC cavity: after the source has died out the discrete energy is
    constant, and the lowest resonance sits at the exact Yee dispersion
    sin(w dt/2)/(c dt) = sqrt(sum sin^2(k dx/2))/dx, k = pi/((n-1) dx)."""
    n, dx = 24, 20e-9
    w = I.workload_2d(n, n, dx=dx, nsteps=60000, npml=0, design=(0, 0), gap=(0, 0))
    w.update(I.pulse(1600e-9, 200e12))
    w.update(src_lo=[7, 9, 0], src_hi=[8, 10, 1], design_lo=[0, 0, 0], design_hi=[0, 0, 1],
             gap_lo=[0, 0, 0], gap_hi=[0, 0, 1])
    out = O.forward(w, np.zeros(0), probes=[(5, 6)], energy=True)
    en = out["energy"]
    dt = w["courant"] * dx / C0
    quiet = int((w["t0"] + 7.0 * w["tau"]) / dt) + 1
    tail = en[quiet:]
    assert tail.max() > 0
    assert (tail.max() - tail.min()) / tail.max() < 1e-11  # round-off over ~6e4 steps
    p = out["probe_hist"][quiet:, 0]
    pad = 1 << 22
    F = np.abs(np.fft.rfft(p * np.hanning(p.size), pad))
    f = np.fft.rfftfreq(pad, dt)
    k = np.pi / ((n - 1) * dx)
    s = np.sqrt(2.0) * np.sin(k * dx / 2) / dx
    f_yee = 2.0 * np.arcsin(C0 * dt * s) / dt / (2 * np.pi)
    f_cont = C0 * np.sqrt(2.0) * k / (2 * np.pi)
    band = (f > 0.8 * f_yee) & (f < 1.1 * f_yee)
    i = np.flatnonzero(band)[np.argmax(F[band])]
    a, b, c = np.log(F[i - 1]), np.log(F[i]), np.log(F[i + 1])
    f_pk = f[i] + 0.5 * (a - c) / (a - 2 * b + c) * (f[1] - f[0])
    assert abs(f_pk - f_yee) < 0.1 * abs(f_yee - f_cont)


def test_stable_at_courant_limit_with_drude_and_sigma():
    """S = 0.99/sqrt(2) with Drude gold, sigma and CPML: no late-time growth."""
    w = fast_case(npml=4, nsteps=40000, courant=0.99 / np.sqrt(2.0))
    r = I.rho_uniform(w, 3)
    out = O.forward(w, r, 5e5, 1.0, probes=[(20, 18), (12, 25)])
    p = np.abs(out["probe_hist"])
    peak = p.max()
    assert np.isfinite(p).all() and peak > 1e-3
    assert p[-2000:].max() < 1e-6 * peak


@pytest.mark.parametrize("npml,material", [(0, "gold"), (6, "gold"), (6, "silver")])
def test_adjoint_gradient_matches_central_differences(npml, material):
    """Eq. (25)+(27) against central differences of the forward solve; the paper
    reports agreement to more than 4 digits.  Silver (eps_inf = 4.469) exercises
    the eps_inf term of Eq. (25b), which gold (eps_inf = eps_s = 1) leaves out."""
    w = fast_case(npml=npml, material=I.SILVER if material == "silver" else I.GOLD)
    r = I.zero_gap(w, I.rho_uniform(w, 1) * 0.8 + 0.1)
    smax, gs = 5e5, 3.0
    g = O.gradient(w, r, smax, gs)["grad"]
    rf = r.reshape(-1)
    rng = np.random.default_rng(0)
    idx = rng.choice(np.flatnonzero(rf > 0), 8, replace=False)
    for i in idx:
        h = 1e-4
        rp, rm = rf.copy(), rf.copy()
        rp[i] += h
        rm[i] -= h
        fd = (O.objective(w, rp, smax, gs) - O.objective(w, rm, smax, gs)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-5 * abs(fd) + 1e-6 * np.abs(g).max()


def test_adjoint_gradient_with_filter_matches_central_differences():
    w = fast_case(filter_radius=2, filter_fwhm=2.5)
    r = I.zero_gap(w, I.rho_uniform(w, 2))
    g = O.gradient(w, r, 2e5, 1.0)["grad"]
    rf = r.reshape(-1)
    rng = np.random.default_rng(1)
    gap = I.zero_gap(w, np.ones(I.design_shape(w))).reshape(-1) == 0
    idx = rng.choice(np.flatnonzero(~gap), 6, replace=False)
    for i in idx:
        h = 1e-4
        rp, rm = rf.copy(), rf.copy()
        rp[i] += h
        rm[i] -= h
        fd = (O.objective(w, rp, 2e5) - O.objective(w, rm, 2e5)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-5 * abs(fd) + 1e-6 * np.abs(g).max()
    assert np.all(g[gap] == 0.0)


def test_linearity_source_scaling():
    """Fields are linear in the source: doubling it multiplies W and dW by 4."""
    w = fast_case()
    r = I.rho_uniform(w, 4)
    a = O.gradient(w, r, 1e5)
    b = O.gradient(dict(w, src_amp=2.0), r, 1e5)
    assert abs(b["W"] / a["W"] - 4.0) < 1e-12
    np.testing.assert_allclose(b["grad"], 4.0 * a["grad"], rtol=1e-10, atol=1e-12 * np.abs(b["grad"]).max())


def test_sigma_vanishes_at_binary_densities():
    """Eq. (5c): sigma_i = 0 for rho in {0, 1}, so sigma_max cannot matter there."""
    w = fast_case()
    r = I.zero_gap(w, (I.rho_uniform(w, 5) > 0.5).astype(float))
    assert O.objective(w, r, 0.0) == O.objective(w, r, 5e6)


def test_gap_is_fixed_vacuum():
    """The gap is not designable: its rho entries do not change W."""
    w = fast_case()
    r = I.rho_uniform(w, 6)
    q = r.copy()
    sl = tuple(slice(w["gap_lo"][a] - w["design_lo"][a], w["gap_hi"][a] - w["design_lo"][a])
               for a in (1, 0))
    q[sl] = 0.7
    assert O.objective(w, r) == O.objective(w, q)


def test_filter_against_scipy_and_transpose():
    """Interior rows equal scipy's truncated Gaussian filter; F^T is the adjoint
    of F; constants pass unchanged (edge renormalisation)."""
    from scipy.ndimage import gaussian_filter
    w = I.workload_2d(80, 80, dx=2e-9, nsteps=10, design=(40, 36), gap=(3, 3),
                      filter_radius=5, filter_fwhm=5.0)
    rng = np.random.default_rng(0)
    x = rng.random(I.design_shape(w))
    y = rng.random(I.design_shape(w))
    Fx = O.filt(w, x).reshape(x.shape)
    R, s = w["filter_radius"], w["filter_sigma"]
    ref = gaussian_filter(x, s, truncate=R / s, mode="constant")
    np.testing.assert_allclose(Fx[R:-R, R:-R], ref[R:-R, R:-R], rtol=1e-12)
    FTy = O.filt(w, y, transpose=True).reshape(y.shape)
    assert abs(np.sum(Fx * y) - np.sum(x * FTy)) < 1e-12 * np.sum(Fx * y)
    np.testing.assert_allclose(O.filt(w, np.full(x.shape, 0.3)), 0.3, rtol=1e-14)


def test_objective_literal_sum():
    """Eq. (24) for 2D: eps_g dt dx^2 / 2 times the sum of recorded gap E^2."""
    w = fast_case()
    out = O.forward(w, I.rho_uniform(w, 7), record_gap=True)
    dt = w["courant"] * w["dx"] / C0
    assert abs(out["W"] - 0.5 * w["eps_g"] * dt * w["dx"] ** 2 * np.sum(out["gap_hist"] ** 2)) \
        <= 1e-13 * out["W"]
    assert np.all(out["gap_hist"][0] == 0.0)


# ------------------------------------------------------------------ 3D

def fast_case_3d(npml=4, source="dipole", material=None, nsteps=200):
    w = I.workload_3d(20, 18, 22, dx=20e-9, nsteps=nsteps, npml=npml, design=(8, 6, 6), gap=(2, 2, 2),
                      source=source, material=material, real="f64")
    w.update(I.pulse(800e-9, 300e12))
    if npml == 0 and source == "sheet":
        w["src_lo"] = [1, 1, 3]
        w["src_hi"] = [19, 17, 4]
    return w


def test_3d_dipole_field_matches_hertzian_dipole():
    """A soft E_z current on one edge is a current element I l = J dx^3; in the
    equatorial plane its field is E_z = -(p/r^3 + p'/(c r^2) + p''/(c^2 r)) / (4 pi eps0)
    at the retarded time (near, intermediate and far terms)."""
    n, dx, D = 52, 5e-9, 13
    c = n // 2
    w = I.workload_3d(n, n, n, dx=dx, nsteps=2400, npml=8, design=(0, 0, 0), gap=(0, 0, 0), source="dipole",
                      real="f64")
    w.update(I.pulse(800e-9, 300e12))
    w.update(design_lo=[0, 0, 0], design_hi=[0, 0, 0], gap_lo=[0, 0, 0], gap_hi=[0, 0, 0],
             src_lo=[c, c, c], src_hi=[c + 1, c + 1, c + 1], src_comp=2)
    O.set_threads(8)
    e = O.forward(w, np.zeros(0), probes=[(c + D, c, c, 2), (c, c - D, c, 2)])["probe_hist"]
    O.set_threads(1)
    dt = w["courant"] * dx / C0
    r = D * dx
    tr = np.arange(e.shape[0]) * dt - r / C0

    def g(t):
        return np.exp(-((t - w["t0"]) / w["tau"]) ** 2) * np.sin(2 * np.pi * w["f0"][0] * (t - w["t0"]))

    J0 = w["src_amp"] * EPS0 * C0 / dx
    fine = np.linspace(tr.min() - 1e-15, tr.max(), 200001)
    p = dx ** 3 * J0 * np.interp(tr, fine, np.cumsum(g(fine)) * (fine[1] - fine[0]))
    pd = dx ** 3 * J0 * g(tr)
    h = 1e-20
    pdd = dx ** 3 * J0 * (g(tr + h) - g(tr - h)) / (2 * h)
    Ez = -(p / r ** 3 + pd / (C0 * r ** 2) + pdd / (C0 ** 2 * r)) / (4 * np.pi * EPS0)
    for k in range(2):
        assert np.max(np.abs(e[:, k] - Ez)) < 3e-2 * np.max(np.abs(Ez))


def test_3d_pec_cavity_energy_conserved():
    n, dx = 12, 20e-9
    w = I.workload_3d(n, n + 1, n + 2, dx=dx, nsteps=6000, npml=0, design=(0, 0, 0), gap=(0, 0, 0),
                      source="dipole", real="f64")
    w.update(I.pulse(1600e-9, 200e12))
    w.update(design_lo=[0, 0, 0], design_hi=[0, 0, 0], gap_lo=[0, 0, 0], gap_hi=[0, 0, 0],
             src_lo=[4, 5, 6], src_hi=[5, 6, 7], src_comp=1)
    en = O.forward(w, np.zeros(0), energy=True)["energy"]
    dt = w["courant"] * dx / C0
    quiet = int((w["t0"] + 7.0 * w["tau"]) / dt) + 1
    tail = en[quiet:]
    assert tail.max() > 0
    assert (tail.max() - tail.min()) / tail.max() < 1e-11


@pytest.mark.parametrize("npml,source,material", [(0, "dipole", "gold"), (4, "dipole", "silver"),
                                                  (4, "sheet", "gold"), (0, "sheet", "silver")])
def test_3d_adjoint_gradient_matches_central_differences(npml, source, material):
    """Eq. (25) summed over the three E components of each design cell, then
    Eq. (27), against central differences of the 3D forward solve."""
    w = fast_case_3d(npml, source, I.SILVER if material == "silver" else I.GOLD)
    r = I.zero_gap(w, I.rho_uniform(w, 8) * 0.8 + 0.1)
    smax, gs = 5e5, 2.0
    g = O.gradient(w, r, smax, gs)["grad"]
    rf = r.reshape(-1)
    rng = np.random.default_rng(2)
    for i in rng.choice(np.flatnonzero(rf > 0), 5, replace=False):
        h = 1e-4
        rp, rm = rf.copy(), rf.copy()
        rp[i] += h
        rm[i] -= h
        fd = (O.objective(w, rp, smax, gs) - O.objective(w, rm, smax, gs)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-5 * abs(fd) + 1e-6 * np.abs(g).max()


def test_3d_objective_literal_sum():
    """Eq. (24) in 3D: eps_g dt dx^3 / 2 times the sum over the gap of |E|^2."""
    w = fast_case_3d()
    out = O.forward(w, I.rho_uniform(w, 9), record_gap=True)
    dt = w["courant"] * w["dx"] / C0
    assert abs(out["W"] - 0.5 * w["eps_g"] * dt * w["dx"] ** 3 * np.sum(out["gap_hist"] ** 2)) <= 1e-13 * out["W"]


def test_grayness_definition():
    """Sec. 3.2: zeta = 0 for a black-and-white design, 1 for rho~ = 0.5."""
    w = fast_case()
    shape = I.design_shape(w)
    assert O.grayness(w, np.zeros(shape)) == 0.0
    assert O.grayness(w, I.zero_gap(w, np.ones(shape))) == 0.0
    assert abs(O.grayness(w, np.full(shape, 0.5)) - 1.0) < 1e-15


# ---- the paper's excitation (Sec. 2, Fig. 1c-d)

def test_sinc_hanning_spectrum_has_the_stated_bandwidth():
    """A sinc truncated after four lobes, Hanning-smoothed, on a 600 THz
    carrier: the paper states a 20 % bandwidth at half maximum.  The
    amplitude spectrum must be centred on the carrier with a half-maximum
    width of 20 % of it (the rounding of the edges keeps the half-maximum
    points at the edges of the rectangle)."""
    w = I.workload_2d(41, 37, dx=20e-9, nsteps=10)
    w.update(I.sinc_hanning(center_m=C0 / 600e12, rel_bandwidth=0.2, lobes=4))
    f0, B = 600e12, 120e12
    dt = 1e-17
    t = np.arange(0.0, 2 * w["t0"] + 50e-15, dt)
    g = O.signal(w, t)
    assert g[0] == 0.0 and g[-1] == 0.0
    nfft = 1 << 22
    spec = np.abs(np.fft.rfft(g, nfft))
    f = np.fft.rfftfreq(nfft, dt)
    band = (f > 300e12) & (f < 900e12)
    fb, sb = f[band], spec[band]
    half = sb >= 0.5 * sb.max()
    lo, hi = fb[half][0], fb[half][-1]
    assert abs(0.5 * (lo + hi) - f0) <= 0.005 * f0
    assert abs((hi - lo) - B) <= 0.03 * B
    # outside the band the rounded rectangle has fallen well below its plateau
    assert spec[(f > 0) & (f < f0 - B)].max() < 0.05 * sb.max()
    assert spec[f > f0 + B].max() < 0.05 * sb.max()


def test_sinc_hanning_envelope_zeros_and_support():
    """The envelope vanishes at the sinc zeros t0 +- m/B (m = 1 .. 3) and
    beyond t0 +- 4/B."""
    w = I.workload_2d(41, 37, dx=20e-9, nsteps=10)
    w.update(I.sinc_hanning(center_m=C0 / 600e12, rel_bandwidth=0.2, lobes=4))
    B, t0 = w["bandwidth"], w["t0"]
    # probe the envelope through the carrier's quarter period after each zero
    tq = 0.25 / w["f0"][0]
    for m in (1, 2, 3):
        for sgn in (-1, 1):
            tz = t0 + sgn * m / B
            assert abs(O.signal(w, np.array([tz]))[0]) < 1e-12
    assert O.signal(w, np.array([t0 + 4 / B + tq, t0 - 4 / B - tq])).tolist() == [0.0, 0.0]


# ---- gap spectrum (the field-enhancement monitor)

def test_gap_spectrum_equals_fft_at_bin_frequencies():
    """At f_k = k / (N dt) the spectrum reduces to dt times numpy's FFT (with
    the e^{-j w n dt} kernel of the e^{j w t} convention)."""
    w = I.small_2d(nsteps=255)
    w.update(I.pulse(800e-9, 300e12))
    dt = w["courant"] * w["dx"] / C0
    rng = np.random.default_rng(5)
    h = rng.standard_normal((256, 7))
    k = np.array([0, 1, 5, 17, 100, 128])
    z = O.gap_spectrum(w, h, k / (256 * dt))
    ref = dt * np.fft.fft(h, axis=0)[k]
    np.testing.assert_allclose(z, ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())


def test_gap_spectrum_of_a_cosine():
    """A cosine with an integer number m of periods over N samples:
    E(f_m) = dt N / 2 exactly, real, and zero at the other bins."""
    w = I.small_2d(nsteps=999)
    dt = w["courant"] * w["dx"] / C0
    N, m = 1000, 37
    n = np.arange(N)
    h = np.cos(2 * np.pi * m * n / N)[:, None]
    z = O.gap_spectrum(w, h, np.array([m, m + 3]) / (N * dt))[:, 0]
    assert z[0] == pytest.approx(dt * N / 2, rel=1e-12)
    assert abs(z[1]) <= 1e-12 * dt * N


def _cpml_reflection(npml, sigma_factor, m=3.0, Ls=(0, 20, 34, 59, 93), D=30, gap=4):
    """Spurious reflection of the CPML at oblique incidence.  A point current
    (one E_z node, broadband pulse) D nodes above the lower absorbing layer;
    probes `gap` nodes above the layer at lateral offsets Ls, i.e. incidence
    angles atan(L / (D + gap)) from 0 to 70 degrees.  The same source and
    probes in a domain 400 nodes larger on every side (whose own boundary
    echoes arrive after the window) give the reflection-free field; the
    difference is the reflected wave.  Returns (angle, peak reflected /
    peak direct at the probe, the same corrected for the 1/sqrt(r)
    spreading of the image source in the PEC wall behind the layer)."""
    def run(nx, ny, src, probes):
        w = I.workload_2d(nx, ny, dx=20e-9, nsteps=900, npml=npml, design=(2, 2), gap=(1, 1), real="f64",
                          pml_sigma_factor=sigma_factor, pml_m=m)
        w.update(I.pulse(800e-9, 300e12))
        w.update(design_lo=[nx - npml - 4, ny - npml - 4, 0], design_hi=[nx - npml - 2, ny - npml - 2, 1],
                 gap_lo=[nx - npml - 4, ny - npml - 4, 0], gap_hi=[nx - npml - 3, ny - npml - 3, 1],
                 src_lo=[src[0], src[1], 0], src_hi=[src[0] + 1, src[1] + 1, 1])
        return O.forward(w, np.zeros(I.design_shape(w)), 0.0, 1.0, probes=probes)["probe_hist"]
    ny = 2 * npml + D + 12
    nx = 2 * npml + 60 + max(Ls)
    src = (npml + 30, npml + D)
    probes = [(src[0] + L, npml + gap) for L in Ls]
    off = 400
    near = run(nx, ny, src, probes)
    far = run(nx + 2 * off, ny + 2 * off, (src[0] + off, src[1] + off), [(x + off, y + off) for x, y in probes])
    out = []
    for k, L in enumerate(Ls):
        r = np.max(np.abs(near[:, k] - far[:, k])) / np.max(np.abs(far[:, k]))
        rd, rr = np.hypot(L, D - gap), np.hypot(L, D + gap + 2 * npml)
        out.append((np.arctan(L / (D + gap)), r, r * np.sqrt(rr / rd)))
    return out


def test_cpml_reflection_at_oblique_incidence():
    """The CPML of the workloads (polynomial grading m = 3, sigma_max =
    0.8 (m + 1) / (eta0 dx), 10 cells, kappa = 1, alpha = 0) reflects at
    most 2e-3 of the incident field from normal incidence to 70 degrees,
    more at grazing than at normal incidence.  With a tenth of that
    sigma_max the layer is so weak that the continuous-medium reflection
    exp(-2 sigma_max L cos(theta) / ((m + 1) eps0 c)) = exp(-2 f npml
    cos(theta)) (f the sigma_max factor) dominates the discretisation
    floor, and the spreading-corrected reflection follows it within a
    factor 2 at every angle, whatever the grading order at fixed f.  A wrong
    sigma_max, grading normalisation or cos(theta) law fails one of these."""
    base = _cpml_reflection(10, 0.8)
    for th, r, _ in base:
        assert r <= 2e-3, (np.degrees(th), r)
    assert base[-1][1] > base[0][1]
    weak = _cpml_reflection(10, 0.08)
    for th, _, rc in weak:
        theory = np.exp(-2 * 0.08 * 10 * np.cos(th))
        assert 0.5 * theory <= rc <= 2.0 * theory, (np.degrees(th), rc, theory)
    weak2 = _cpml_reflection(10, 0.08, m=2.0)
    for (_, r3, _), (_, r2, _) in zip(weak, weak2):
        assert abs(r2 / r3 - 1.0) < 0.05
