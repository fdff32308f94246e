"""Spectral monitors of the observation domain (Sec. 3.2 results).

The paper reports the average field enhancement over the gap,
mean_g |E(w)| / |E_in(w)|, where E_in is the incident field there: the same
excitation with no structure.  ``fdtd_gap_spectrum`` computes the gap
spectra on the device from the recorded gap field; this module forms the
ratio and sets up the structure-free run."""
from __future__ import annotations

import numpy as np

from .binding import Solver


def incident_workload(w: dict) -> dict:
    """The same grid and excitation with no structure: rho = 0 and a vanishing
    Drude term for the void phase (psi_s -> 0), so the design box is plain
    background (eps_s)."""
    v = dict(w)
    v["psi_s_ratio"] = 1e-12
    return v


def magnitude(spec) -> np.ndarray:
    """|E(w)| per gap node from a gap spectrum: (nf, M_g) in 2D, the vector
    magnitude over components of (nf, 3, M_g) in 3D."""
    z = spec.detach().cpu().numpy() if hasattr(spec, "detach") else np.asarray(spec)
    if z.ndim == 3:
        return np.sqrt(np.sum(np.abs(z) ** 2, axis=1))
    return np.abs(z)


def field_enhancement(spec, spec_in) -> np.ndarray:
    """mean over the gap nodes of |E(w)| / |E_in(w)|, one value per frequency."""
    return np.mean(magnitude(spec) / magnitude(spec_in), axis=1)


def enhancement_spectrum(s: Solver, rho, freqs, s_in: Solver | None = None, sigma_max: float = 0.0,
                         gamma_scale: float = 1.0) -> np.ndarray:
    """Run the design and the structure-free reference forward, return the
    average field enhancement at ``freqs`` (Hz)."""
    if s_in is None:
        s_in = Solver(incident_workload(s.w), device=s.device)
    s.set_design(rho)
    s.set_damping(sigma_max, gamma_scale)
    s.forward()
    e = s.gap_spectrum(freqs)
    s_in.set_design(np.zeros(s_in.n_design))
    s_in.set_damping(0.0, 1.0)
    s_in.forward()
    e_in = s_in.gap_spectrum(freqs)
    s.sync()
    s_in.sync()
    return field_enhancement(e, e_in)
