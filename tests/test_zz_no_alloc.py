"""fdtd_gradient_static against fdtd_gradient.

fdtd_gradient_static serves callers that cannot hand out device memory at
call time: it takes the filter-transpose intermediates from a fixed array the
library owns instead of the workspace.  Its result must equal
fdtd_gradient's on the same solver state, call after call (the fixed array
keeps the previous call's contents, which must not leak into the next)."""
import numpy as np
import pytest

from paper_2203_01462_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def filtered_2d():
    # The Gaussian filter makes the gradient go through both intermediates.
    w = I.workload_2d(150, 140, dx=10e-9, nsteps=600, npml=10, design=(90, 80), gap=(3, 3), real="f32",
                      filter_radius=5, filter_fwhm=5.0, snapshot_every=32, src_offset=5)
    w.update(I.pulse(800e-9, 200e12))
    return w


def test_gradient_static_matches_gradient_on_consecutive_calls():
    from paper_2203_01462_gb300.binding import Solver
    w = filtered_2d()
    s = Solver(w)
    for seed, smax in ((41, 5e5), (42, 0.0)):
        s.set_design(I.rho_uniform(w, seed))
        s.set_damping(smax, 2.0)
        s.forward()
        s.adjoint()
        ref = s.gradient().cpu().numpy()
        got = s.gradient_static().cpu().numpy()
        s.sync()
        assert np.linalg.norm(ref) > 0
        # Same arithmetic on the same state: within the FP64-parity tolerance
        # of the other tests (in practice bit for bit).
        assert np.linalg.norm(got - ref) <= 1e-9 * np.linalg.norm(ref)
        np.testing.assert_allclose(got, ref, rtol=1e-9, atol=1e-9 * np.abs(ref).max())


def test_gradient_static_smaller_box_after_larger_one():
    """The fixed array keeps the last call's contents: a call for a smaller
    filtered design box right after one for a larger box (and back) must
    not pick up the larger call's leftovers."""
    from paper_2203_01462_gb300.binding import Solver
    big = filtered_2d()
    small = I.workload_2d(70, 64, dx=10e-9, nsteps=400, npml=8, design=(37, 29), gap=(3, 3), real="f32",
                          filter_radius=3, filter_fwhm=3.0, snapshot_every=32, src_offset=4)
    small.update(I.pulse(800e-9, 200e12))
    runs = []
    for w, seed in ((big, 43), (small, 44), (big, 45)):
        s = Solver(w)
        s.set_design(I.rho_uniform(w, seed))
        s.set_damping(5e5, 2.0)
        s.forward()
        s.adjoint()
        ref = s.gradient().cpu().numpy()
        got = s.gradient_static().cpu().numpy()
        s.sync()
        runs.append((got, ref))
    for got, ref in runs:
        assert np.linalg.norm(ref) > 0
        assert np.linalg.norm(got - ref) <= 1e-9 * np.linalg.norm(ref)


def test_gradient_static_rejects_filtered_boxes_beyond_its_limit():
    from paper_2203_01462_gb300.binding import FdtdError, Solver
    w = I.workload_2d(1060, 1060, dx=10e-9, nsteps=2, npml=10, design=(1030, 1030), gap=(3, 3), real="f32",
                      filter_radius=5, filter_fwhm=5.0)
    s = Solver(w)
    assert s.n_design > 1048576
    s.set_design(I.rho_uniform(w, 1))
    s.forward()
    s.adjoint()
    with pytest.raises(FdtdError) as e:
        s.gradient_static()
    assert e.value.status == 1


def test_gradient_static_unlimited_where_no_scratch_is_used():
    """A 3D design box above the limit: the 3D gradient needs no
    intermediates, so the call is accepted and equals fdtd_gradient."""
    from paper_2203_01462_gb300.binding import Solver
    w = I.workload_3d(146, 146, 82, dx=10e-9, nsteps=4, npml=4, design=(130, 130, 64), gap=(2, 2, 2), real="f32")
    s = Solver(w)
    assert s.n_design > 1048576
    s.set_design(I.rho_uniform(w, 2))
    s.forward()
    s.adjoint()
    ref = s.gradient().cpu().numpy()
    got = s.gradient_static().cpu().numpy()
    s.sync()
    np.testing.assert_array_equal(got, ref)
