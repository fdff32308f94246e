"""Pins of the oracle's 3D plane-wave injection (total-field / scattered-field).

The incident wave comes from a 1D column of the same scheme.  These check:
  * the scattered-field region of an empty domain stays at round-off and the
    total-field region reproduces the incident column (leakage test);
  * the column itself against closed forms: the field radiated by a current
    sheet, and the Fresnel transmission of a plane wave from the substrate
    into air;
  * the adjoint gradient (Eq. 25, 27), unchanged by a design-independent
    source, against central differences of the forward solve.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2203_01462_gb300 import inputs as I

C0 = 299792458.0
MU0 = 1.25663706212e-6
EPS0 = 1.0 / (MU0 * C0 * C0)
ETA0 = MU0 * C0


def empty_tfsf(substrate: bool, nsteps: int = 260):
    w = I.workload_3d(22, 20, 36, dx=20e-9, nsteps=nsteps, npml=4, design=(0, 0, 0), gap=(0, 0, 0),
                      source="tfsf", substrate=substrate, real="f64", tf_margin=2)
    w.update(I.pulse(800e-9, 300e12))
    # empty design and gap boxes (the substrate plane stays at the box centre)
    w.update(design_lo=[0, 0, 0], design_hi=[0, 0, 0], gap_lo=[0, 0, 0], gap_hi=[0, 0, 0])
    return w


@pytest.mark.parametrize("substrate", [False, True])
def test_empty_domain_leaks_nothing_and_carries_the_incident_wave(substrate):
    w = empty_tfsf(substrate)
    lo, hi = w["tf_lo"], w["tf_hi"]
    kin = [lo[2], (lo[2] + hi[2]) // 2, hi[2]]
    # E_x inside the box (x position i + 1/2 in [lo, hi]) at three heights
    inside = [((lo[0] + hi[0]) // 2, (lo[1] + hi[1]) // 2, k, 0) for k in kin]
    inside += [(lo[0], lo[1], kin[1], 0), (hi[0] - 1, hi[1], kin[1], 0)]
    # every component just outside each face, and further out
    outside = [(lo[0] - 1, (lo[1] + hi[1]) // 2, kin[1], c) for c in range(3)]
    outside += [(hi[0] + 1, (lo[1] + hi[1]) // 2, kin[1], c) for c in range(3)]
    outside += [((lo[0] + hi[0]) // 2, lo[1] - 1, kin[1], c) for c in range(3)]
    outside += [((lo[0] + hi[0]) // 2, hi[1] + 1, kin[1], c) for c in range(3)]
    outside += [((lo[0] + hi[0]) // 2, (lo[1] + hi[1]) // 2, lo[2] - 1, c) for c in range(3)]
    outside += [((lo[0] + hi[0]) // 2, (lo[1] + hi[1]) // 2, hi[2] + 1, c) for c in range(3)]
    O.set_threads(4)
    try:
        ph = O.forward(w, np.zeros(0), probes=inside + outside)["probe_hist"]
    finally:
        O.set_threads(1)
    Einc, _ = O.tfsf_incident(w, [p[2] for p in inside])
    scale = np.abs(Einc).max()
    assert scale > 0
    # the wave has crossed the whole box by the end of the run
    assert np.abs(Einc[:, 2]).max() > 0.1 * scale
    np.testing.assert_allclose(ph[:, :len(inside)], Einc, rtol=0, atol=1e-12 * scale)
    assert np.abs(ph[:, len(inside):]).max() <= 1e-12 * scale


def test_sheet_current_radiates_half_eta_K_in_its_medium():
    """A soft current J on one plane of thickness dx is a surface current
    K = J dx; it radiates E = -eta K / 2 each way, eta = eta0 / n of the
    medium around it (here the substrate, n = 1.5)."""
    w = I.workload_3d(8, 8, 400, dx=5e-9, nsteps=900, npml=10, design=(0, 0, 0), gap=(0, 0, 0),
                      source="tfsf", substrate=True, real="f64", tf_margin=1)
    w.update(sub_hi=400)  # the whole column is substrate
    ks = w["src_lo"][2] + 60
    E, _ = O.tfsf_incident(w, [ks])
    n = 1.5
    dt = w["courant"] * w["dx"] / C0
    delay = 60 * w["dx"] * n / C0 + 0.5 * dt
    t = np.arange(E.shape[0]) * dt - delay
    g = np.exp(-((t - w["t0"]) / w["tau"]) ** 2) * np.sin(2 * np.pi * w["f0"][0] * (t - w["t0"]))
    J0 = w["src_amp"] * EPS0 * C0 / w["dx"]
    expect = -(ETA0 / n) * J0 * w["dx"] / 2 * g
    assert np.abs(E[:, 0] - expect).max() <= 3e-2 * np.abs(expect).max()


def test_transmission_from_substrate_into_air_is_fresnel():
    """|E_t(f)| / |E_i(f)| = 2 n1 / (n1 + n2) for normal incidence from
    n1 = 1.5 into n2 = 1: the spectrum above the interface with the
    substrate, over the spectrum at the same node in all-substrate space."""
    nz, zi = 700, 300
    w = I.workload_3d(8, 8, nz, dx=10e-9, nsteps=2600, npml=12, design=(0, 0, 0), gap=(0, 0, 0),
                      source="tfsf", substrate=True, real="f64", tf_margin=1)
    w.update(I.pulse(800e-9, 150e12))
    k_up = zi + 40
    w_int = dict(w, sub_hi=zi)
    w_bulk = dict(w, sub_hi=nz)
    Et, _ = O.tfsf_incident(w_int, [k_up])
    Ei, _ = O.tfsf_incident(w_bulk, [k_up])
    dt = w["courant"] * w["dx"] / C0
    f = np.linspace(C0 / 950e-9, C0 / 650e-9, 7)
    n = np.arange(Et.shape[0])
    kern = np.exp(-2j * np.pi * np.outer(f, n) * dt)
    T = np.abs(kern @ Et[:, 0]) / np.abs(kern @ Ei[:, 0])
    np.testing.assert_allclose(T, 2 * 1.5 / 2.5, rtol=1e-2)


@pytest.mark.parametrize("material", ["gold", "silver"])
def test_adjoint_gradient_with_plane_wave_matches_central_differences(material):
    w = I.workload_3d(20, 18, 30, dx=20e-9, nsteps=200, npml=4, design=(8, 6, 6), gap=(2, 2, 2),
                      source="tfsf", substrate=True, material=I.SILVER if material == "silver" else I.GOLD,
                      real="f64", tf_margin=1)
    w.update(I.pulse(800e-9, 300e12))
    assert all(w["tf_lo"][a] < w["design_lo"][a] and w["tf_hi"][a] >= w["design_hi"][a] for a in range(3))
    r = I.zero_gap(w, I.rho_uniform(w, 8) * 0.8 + 0.1)
    smax, gs = 5e5, 2.0
    g = O.gradient(w, r, smax, gs)["grad"]
    assert np.abs(g).max() > 0
    rf = r.reshape(-1)
    rng = np.random.default_rng(3)
    for i in rng.choice(np.flatnonzero(rf > 0), 5, replace=False):
        h = 1e-4
        rp, rm = rf.copy(), rf.copy()
        rp[i] += h
        rm[i] -= h
        fd = (O.objective(w, rp, smax, gs) - O.objective(w, rm, smax, gs)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-5 * abs(fd) + 1e-6 * np.abs(g).max()
