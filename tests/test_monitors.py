"""Gap-spectrum monitor (the paper's field-enhancement measure) against the
oracle's DFT of its own gap history, through the C ABI."""

import numpy as np
import pytest

from oracle import oracle as O
from paper_2203_01462_gb300 import inputs as I

pytestmark = pytest.mark.gpu
C0 = 299792458.0


def _freqs():
    return np.linspace(C0 / 1100e-9, C0 / 550e-9, 41)


@pytest.mark.parametrize("real", ["f64", "f32"])
def test_gap_spectrum_2d_matches_oracle(real):
    from paper_2203_01462_gb300.binding import Solver
    w = I.small_2d(nx=41, ny=37, nsteps=600, dx=20e-9, npml=6, design=(17, 15), real=real)
    w.update(I.pulse(800e-9, 300e12))
    rho = I.rho_uniform(w, 31)
    gh = O.forward(w, rho, 0.0, 1.0, record_gap=True)["gap_hist"]
    ref = O.gap_spectrum(w, gh, _freqs())
    s = Solver(w)
    s.set_design(rho)
    s.set_damping(0.0, 1.0)
    s.forward()
    z = s.gap_spectrum(_freqs()).cpu().numpy()
    s.sync()
    tol = 1e-10 if real == "f64" else 1e-4
    assert z.shape == ref.shape
    assert np.max(np.abs(z - ref)) <= tol * np.max(np.abs(ref))


def test_gap_spectrum_3d_matches_oracle():
    from paper_2203_01462_gb300.binding import Solver
    w = I.workload_3d(21, 19, 23, dx=20e-9, nsteps=260, npml=4, design=(11, 9, 9), gap=(3, 3, 3),
                      real="f64", source="dipole")
    w.update(I.pulse(800e-9, 300e12))
    rho = I.rho_uniform(w, 32)
    gh = O.forward(w, rho, 0.0, 1.0, record_gap=True)["gap_hist"]
    ref = O.gap_spectrum(w, gh, _freqs())
    s = Solver(w)
    s.set_design(rho)
    s.set_damping(0.0, 1.0)
    s.forward()
    z = s.gap_spectrum(_freqs()).cpu().numpy()
    s.sync()
    assert z.shape == ref.shape == (41, 3, s.n_gap)
    assert np.max(np.abs(z - ref)) <= 1e-10 * np.max(np.abs(ref))


def test_field_enhancement_of_a_bowtie(save_report):
    """A gold bowtie on the 160^2 grid against the structure-free run: the
    ratio is 1 for the structure-free design itself.  With E out of plane no
    surface plasmon exists (Sec. 3, TE case), so the metal shields the gap:
    the ratio stays below 1 across the band."""
    from paper_2203_01462_gb300.binding import Solver
    from paper_2203_01462_gb300.monitors import enhancement_spectrum, incident_workload
    w = I.cfg_2d_160()
    f = np.linspace(C0 / 1000e-9, C0 / 600e-9, 21)
    s = Solver(w)
    s_in = Solver(incident_workload(w))
    same = enhancement_spectrum(s_in, np.zeros(s_in.n_design), f, s_in=Solver(incident_workload(w)))
    np.testing.assert_allclose(same, 1.0, rtol=1e-12)
    fe = enhancement_spectrum(s, I.rho_bowtie(w), f, s_in=s_in)
    save_report("bowtie_enhancement.json", dict(wavelength_nm=(C0 / f * 1e9).tolist(), enhancement=fe.tolist()))
    assert np.all(np.isfinite(fe)) and np.all(fe > 0)
    assert fe.max() < 1.0
