"""The 2D E_z step's vector path against the FP64 oracle, through the C ABI.

The step kernel runs a 16-byte vector path on every block whose node tile
and one-node halo are clear of walls and CPML slabs, and a scalar path on
the rest.  Small grids have no such blocks, so these cases use a 530 x 303
grid on which more than half of the blocks take the vector path, with the
design box, the 3 x 3 gap and the source row inside vector tiles: the
design box starts and ends inside tiles and inside 4-node groups, its first
and last rows are not tile-aligned, and the gap straddles a 4-node group.
The library reports how many blocks of one step launch take the vector
path (fdtd_get_info), and the test recomputes that count from the tile
rule, so a later change of the tiling cannot drop the coverage silently.

Tolerances as for the other 2D parity cases: FP64 fields W 1e-10 relative,
gap history 1e-10 of its peak, gradient 1e-9 L2-relative; FP32 fields W
1e-4 relative, gradient 1e-3 L2-relative.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2203_01462_gb300 import inputs as I

pytestmark = pytest.mark.gpu

# Tile of the 2D step kernel (128 x 4 nodes): a block takes the vector path
# when nodes x0-1 .. x0+128 and y0-1 .. y0+4 avoid the walls and the CPML.
TILE_X, TILE_Y = 128, 4


def vector_block_count(w):
    nx, ny, np_ = w["nx"], w["ny"], w["npml"]
    gx, gy = -(-nx // TILE_X), -(-ny // TILE_Y)
    vec = 0
    for by in range(gy):
        for bx in range(gx):
            x0, y0 = bx * TILE_X, by * TILE_Y
            vec += (x0 - 1 >= np_ + 1 and x0 + TILE_X <= nx - np_ - 2 and
                    y0 - 1 >= np_ + 1 and y0 + TILE_Y <= ny - np_ - 2)
    return gx * gy, vec


def in_vector_tile(w, i, j):
    x0, y0 = (i // TILE_X) * TILE_X, (j // TILE_Y) * TILE_Y
    np_ = w["npml"]
    return (x0 - 1 >= np_ + 1 and x0 + TILE_X <= w["nx"] - np_ - 2 and
            y0 - 1 >= np_ + 1 and y0 + TILE_Y <= w["ny"] - np_ - 2)


def wide_case(real, *, filt=5, snapshot_every=0, material=None, nsteps=1000):
    """530 x 303 nodes, dx = 10 nm, 10-cell CPML; 251 x 61 design box at
    x 139..389, y 121..181; gap x 263..265, y 150..152; source row y = 15."""
    w = I.workload_2d(530, 303, dx=10e-9, nsteps=nsteps, npml=10, design=(251, 61), gap=(3, 3), real=real,
                      material=material, filter_radius=filt, filter_fwhm=5.0, snapshot_every=snapshot_every,
                      src_offset=5)
    w.update(I.pulse(800e-9, 200e12))
    return w


def l2rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def solver(w):
    from paper_2203_01462_gb300.binding import Solver
    return Solver(w)


def check_coverage(w, s):
    total, vec = vector_block_count(w)
    inf = s.info()
    assert (inf.step_blocks, inf.vector_blocks) == (total, vec)
    assert vec >= 0.5 * total, (vec, total)
    dl, dh, gl, gh = w["design_lo"], w["design_hi"], w["gap_lo"], w["gap_hi"]
    # design box corners and edges, the gap and the source row all sit in vector tiles
    for i in (dl[0], dh[0] - 1, (dl[0] + dh[0]) // 2):
        for j in (dl[1], dh[1] - 1):
            assert in_vector_tile(w, i, j), (i, j)
    assert dl[0] % 4 and dh[0] % 4 and dl[1] % TILE_Y and dh[1] % TILE_Y
    assert gl[0] // 4 != (gh[0] - 1) // 4
    for i in range(gl[0], gh[0]):
        for j in range(gl[1], gh[1]):
            assert in_vector_tile(w, i, j)
    sy = w["src_lo"][1]
    assert any(in_vector_tile(w, i, sy) for i in range(w["src_lo"][0], w["src_hi"][0]))


def test_geometry_covers_the_vector_path():
    w = wide_case("f64")
    total, vec = vector_block_count(w)
    assert vec / total > 0.54
    check_coverage(w, solver(w))


@pytest.mark.parametrize("snap,material", [(0, "gold"), (64, "silver")])
def test_fp64_vector_path_matches_oracle(snap, material):
    """U[0,1] densities through the Gaussian filter; full history (the
    single-state step) and lossless checkpoints every 64 steps (the paired
    recompute + adjoint step)."""
    mat = I.SILVER if material == "silver" else I.GOLD
    w = wide_case("f64", snapshot_every=snap, material=mat)
    rho = I.rho_uniform(w, 31)
    smax, gs = 5e5, 3.0
    ref = O.gradient(w, rho, smax, gs)
    gh_ref = O.forward(w, rho, smax, gs, record_gap=True)["gap_hist"]
    s = solver(w)
    check_coverage(w, s)
    W, g = s.evaluate(rho, smax, gs)
    s.sync()
    assert abs(float(W.item()) - ref["W"]) <= 1e-10 * abs(ref["W"])
    gh = s.gap_history().cpu().numpy()
    assert np.max(np.abs(gh - gh_ref)) <= 1e-10 * np.max(np.abs(gh_ref))
    assert l2rel(g.cpu().numpy(), ref["grad"]) <= 1e-9


@pytest.mark.parametrize("snap", [0, 64])
def test_fp32_vector_path_matches_oracle(snap):
    """0.3 U[0,1] densities (a lossy film that leaves the gap field well
    above FP32 rounding), filtered, with damping."""
    w = wide_case("f32", snapshot_every=snap)
    rho = 0.3 * I.rho_uniform(w, 32)
    ref = O.gradient(w, rho, 5e5, 3.0)
    s = solver(w)
    W, g = s.evaluate(rho, 5e5, 3.0)
    s.sync()
    assert abs(float(W.item()) - ref["W"]) <= 1e-4 * abs(ref["W"])
    assert l2rel(g.cpu().numpy(), ref["grad"]) <= 1e-3


def test_fp32_vector_path_bowtie_silver_unfiltered():
    """A binary bowtie in silver, no filter (rho~ = rho), checkpoints every 32."""
    w = wide_case("f32", filt=0, snapshot_every=32, material=I.SILVER)
    rho = I.rho_bowtie(w)
    ref = O.gradient(w, rho, 0.0, 1.0)
    s = solver(w)
    W, g = s.evaluate(rho, 0.0, 1.0)
    s.sync()
    assert abs(float(W.item()) - ref["W"]) <= 1e-4 * abs(ref["W"])
    assert l2rel(g.cpu().numpy(), ref["grad"]) <= 1e-3


def test_fp64_vector_path_each_sensitivity_term():
    """Each Eq. (25) term alone, accumulated in the vector path, against the
    oracle's term (silver, so that eps_inf differs from the background), and
    the three terms add up to the full gradient."""
    from test_sensitivity_terms import check
    w = wide_case("f64", snapshot_every=64, material=I.SILVER, nsteps=700)
    check(w, I.rho_uniform(w, 33))
