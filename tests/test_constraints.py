"""Design constraints of the paper's studies: mirror symmetry of the design
and fixed metal blocks beside the gap, against numpy on the same layouts,
and inside a GCMMA run."""
import numpy as np
import pytest

from paper_2203_01462_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _mirror_ref(w, v, axis):
    v = np.asarray(v, dtype=np.float64)
    if I.inplane(w):
        parts = []
        for a in I.split_edges(w, v):
            b = a[:, ::-1] if axis == 0 else a[::-1, :]
            parts.append(0.5 * (a + b))
        return np.concatenate([p.reshape(-1) for p in parts])
    a = v.reshape(I.design_shape(w))
    ax = len(a.shape) - 1 - axis  # x is the last array axis
    return (0.5 * (a + np.flip(a, axis=ax))).reshape(-1)


def _cases():
    w2 = I.small_2d(nx=41, ny=37, nsteps=10, dx=20e-9, npml=6, design=(17, 14), real="f32")
    wp = I.workload_2d_inplane(41, 37, dx=20e-9, nsteps=10, npml=6, design=(17, 14), gap=(3, 2), real="f64",
                               src_offset=2)
    w3 = I.workload_3d(21, 19, 23, dx=20e-9, nsteps=10, npml=4, design=(9, 7, 6), gap=(2, 2, 2), real="f32",
                       source="dipole")
    return [("tmz", w2, (0, 1)), ("inplane", wp, (0, 1)), ("3d", w3, (0, 1, 2))]


@pytest.mark.parametrize("name", ["tmz", "inplane", "3d"])
def test_mirror_average_matches_numpy(name):
    import torch
    from paper_2203_01462_gb300.binding import Solver
    w, axes = [(c[1], c[2]) for c in _cases() if c[0] == name][0]
    s = Solver(w)
    rng = np.random.default_rng(70)
    for axis in axes:
        v = rng.random(s.n_design)
        for dtype in (torch.float64, s.real):
            t = torch.tensor(v, dtype=dtype, device="cuda")
            s.mirror_average(t, axis)
            ref = _mirror_ref(w, t.new_tensor(v).cpu().numpy(), axis)
            got = t.cpu().numpy().astype(np.float64)
            tol = 0 if dtype == torch.float64 else 1e-7
            np.testing.assert_allclose(got, ref, rtol=0, atol=tol)
            # a second application changes nothing: the result is symmetric
            t2 = t.clone()
            s.mirror_average(t2, axis)
            assert torch.equal(t, t2)


def test_fix_design():
    import torch
    from paper_2203_01462_gb300.binding import Solver
    w = [c[1] for c in _cases() if c[0] == "inplane"][0]
    s = Solver(w)
    m = I.fixed_blocks_mask(w)
    assert m.sum() > 0 and not np.any(m & I.gap_edge_mask(w))
    rng = np.random.default_rng(71)
    rho = torch.tensor(rng.random(s.n_design), device="cuda")
    g = torch.tensor(rng.standard_normal(s.n_design), device="cuda")
    r0, g0 = rho.cpu().numpy(), g.cpu().numpy()
    s.fix_design(torch.tensor(m.astype(np.uint8), device="cuda"), rho=rho, grad=g, value=1.0)
    r1, g1 = rho.cpu().numpy(), g.cpu().numpy()
    assert np.all(r1[m] == 1.0) and np.all(g1[m] == 0.0)
    assert np.array_equal(r1[~m], r0[~m]) and np.array_equal(g1[~m], g0[~m])


def test_gcmma_with_fixed_blocks_and_symmetry():
    from paper_2203_01462_gb300.binding import Solver
    from paper_2203_01462_gb300.optimize import optimize_gcmma
    w = I.workload_2d_inplane(70, 58, dx=20e-9, nsteps=600, npml=6, design=(30, 24), gap=(4, 4), real="f32",
                              src_offset=2)
    w.update(I.pulse(800e-9, 300e12))
    s = Solver(w)
    m = I.fixed_blocks_mask(w, axis=0)
    rho0 = I.zero_gap(w, np.full(s.n_design, 0.4))
    rho, h = optimize_gcmma(s, rho0, max_iters=5, levels=[1.0], zeta_stop=0.0, move=0.2, fixed=m, symmetry=0)
    r = rho.cpu().numpy().astype(np.float64)
    assert np.all(r[m] == 1.0)
    np.testing.assert_array_equal(r, _mirror_ref(w, r, 0))
    assert h.W[-1] > h.W[0]
