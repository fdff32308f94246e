"""The values the paper prints (tests/golden/paper_printed_values.txt, each
with its section) against what the workloads, the oracle and the optimizer
use or produce."""
import os

import numpy as np

from oracle import oracle as O
from paper_2203_01462_gb300 import inputs as I

C0 = 299792458.0
HERE = os.path.dirname(os.path.abspath(__file__))


def golden() -> dict:
    out = {}
    for line in open(os.path.join(HERE, "golden", "paper_printed_values.txt")):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        name, value = line.split()[:2]
        out[name] = float(value)
    return out


def test_material_constants_are_the_papers():
    g = golden()
    assert I.SILVER == dict(eps_inf=g["silver_eps_inf"], omega_p=g["silver_omega_p"], gamma_p=g["silver_gamma_p"])
    w = I.cfg_2d_inplane_paper()
    assert w["psi_s_ratio"] == g["psi_s_ratio"]


def test_paper_design_counts_from_the_oracle():
    """The paper's edge counts come out of the stated geometry: dx, the box,
    the centred gap (the oracle counts the free design edges)."""
    g = golden()
    for box, count in ((g["design_box_small_m"], g["design_edges_small"]),
                       (g["design_box_large_m"], g["design_edges_large"])):
        w = I.cfg_2d_inplane_paper(design_nm=box * 1e9, nsteps=10)
        assert w["dx"] == g["dx_2d_m"]
        assert (w["gap_hi"][0] - w["gap_lo"][0]) * w["dx"] == np.float64(g["gap_box_m"])
        assert O.free_design(w) == int(count)


def test_paper_excitation_band():
    """The first 2D study's excitation: 20 % bandwidth at half maximum around
    413 nm, from the oracle's sampled signal."""
    g = golden()
    w = I.cfg_2d_inplane_paper(nsteps=10)
    assert w["lobes"] == int(g["sinc_lobes"])
    f0 = C0 / g["excitation_center_m"]
    dt = 2e-17
    t = np.arange(0.0, 2 * w["t0"] + 20e-15, dt)
    spec = np.abs(np.fft.rfft(O.signal(w, t), 1 << 21))
    f = np.fft.rfftfreq(1 << 21, dt)
    band = (f > 0.5 * f0) & (f < 1.5 * f0)
    fb, sb = f[band], spec[band]
    half = fb[sb >= 0.5 * sb.max()]
    assert abs(0.5 * (half[0] + half[-1]) - f0) <= 0.005 * f0
    assert abs((half[-1] - half[0]) / f0 - g["excitation_fwhm_rel"]) <= 0.01


def test_optimizer_stopping_rule_and_damping_are_the_papers():
    import inspect
    from paper_2203_01462_gb300 import optimize
    g = golden()
    p = inspect.signature(optimize.optimize_gcmma).parameters
    assert p["zeta_stop"].default == g["zeta_min"]
    assert p["max_iters"].default == int(g["max_iterations"])
    assert inspect.signature(optimize.final_design).parameters["level"].default == g["threshold_level"]
    assert I.SIGMA_MAX_PAPER == g["sigma_max"]
