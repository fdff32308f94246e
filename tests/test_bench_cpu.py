"""The benchmark's host-side contract, checked without a GPU: the reference
arm's JSON line (the FP64 oracle on the host cores), the sizing of the
bounded oracle samples, and the algorithmic bytes per step that the
roofline divides by the kernel time."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

import bench
from paper_2203_01462_gb300 import inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_sample_steps_follow_the_node_budget():
    w = I.cfg_3d_256()
    assert bench.sample_nsteps(w, 0, bench.CPU_CELL_STEPS) == 75
    assert bench.sample_nsteps(w, 0, bench.REF_CELL_STEPS) == 30
    # a larger grid gets fewer steps, never fewer than 10 nor more than the run
    w3 = I.cfg_3d_512()
    n3 = bench.sample_nsteps(w3, 0, bench.CPU_CELL_STEPS)
    assert 10 <= n3 < 75
    assert n3 * I.n_cells(w3) <= bench.CPU_CELL_STEPS
    small = I.cfg_2d_160()
    assert bench.sample_nsteps(small, 0, bench.CPU_CELL_STEPS) == min(small["nsteps"], 1000)
    # an explicit request wins but is capped by the workload's own count
    assert bench.sample_nsteps(w, 7, bench.CPU_CELL_STEPS) == 7
    assert bench.sample_nsteps(small, 10 ** 6, bench.CPU_CELL_STEPS) == small["nsteps"]


def test_reference_arm_prints_one_contract_line():
    cmd = [sys.executable, "bench.py", "--impl", "reference", "--workload", "cfg_2d_160",
           "--nsteps", "60", "--steps", "2", "--warmup", "1"]
    out = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=300, check=True)
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference"
    assert d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["steps"] == 2 and d["warmup"] == 1 and d["n_gpus"] == 1
    assert d["higher_is_better"] is True and d["value"] > 0
    assert d["config"]["sample_nsteps"] == 60
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0


def _explicit_bytes(w):
    """Per-node count of the algorithmic bytes of one step (forward, recompute,
    adjoint): every state word read and written once; psi words per CPML slab
    a node lies in (a corner node lies in two or three); J and rho~ on design
    entries; checkpoint copy amortised over the interval."""
    rb = 8 if w["real"] == "f64" else 4
    L = w["npml"]
    dims = [w["nx"], w["ny"]] + ([w["nz"]] if w["ndim"] == 3 else [])
    ncomp = 6 if w["ndim"] == 3 else 3
    psi_per_slab = 4 if w["ndim"] == 3 else 2
    ne = 3 if w["ndim"] == 3 else 1
    md = I.n_design(w)
    grid = pml = psi_words = 0
    for idx in np.ndindex(*dims):
        grid += 2 * ncomp * rb
        slabs = sum(1 for a, p in enumerate(idx) if p < L or p >= dims[a] - L)
        pml += 2 * psi_per_slab * rb * slabs
        psi_words += 2 * psi_per_slab * slabs
    design = (2 * ne + 1) * rb * md
    K = w.get("snapshot_every", 0)
    snap_rb = {"f32": rb, "bf16": 2, "f16": 2}[w.get("snapshot_dtype", "f32")]
    state_words = ncomp * int(np.prod(dims)) + ne * md + psi_words
    fwd = grid + design + pml + ((rb + snap_rb) * state_words / K if K else ne * rb * md)
    rec = grid + design + pml + ne * rb * md
    adj = grid + design + pml + ne * rb * md + 16 * md
    return fwd, rec, adj


@pytest.mark.parametrize("make", [
    lambda: I.small_2d(nx=41, ny=37, npml=6, design=(17, 15), real="f32", snapshot_every=16),
    lambda: I.small_2d(nx=23, ny=29, npml=4, design=(9, 7), real="f64"),
    lambda: I.workload_2d_inplane(31, 27, dx=20e-9, nsteps=10, npml=5, design=(11, 9), gap=(3, 3), real="f32",
                                  snapshot_every=8, snapshot_dtype="f16"),
    lambda: I.workload_3d(21, 19, 17, dx=20e-9, nsteps=10, npml=4, design=(9, 7, 5), gap=(2, 2, 2), real="f32",
                          snapshot_every=32, snapshot_dtype="bf16"),
])
def test_algorithmic_bytes_count_every_node(make):
    w = make()
    ab = bench.algorithmic_bytes(w)
    fwd, rec, adj = _explicit_bytes(w)
    assert ab["forward"] == pytest.approx(fwd, rel=1e-12)
    assert ab["recompute"] == pytest.approx(rec, rel=1e-12)
    assert ab["adjoint"] == pytest.approx(adj, rel=1e-12)


def test_benchmark_step_bytes_agree_with_the_worked_total():
    """2048^2 forward step: 24 B per node for E_z, H_x, H_y, 12 B per design
    node, 16 B per CPML node, plus the checkpoint copy: about 116 MB (the
    roofline's numerator)."""
    ab = bench.algorithmic_bytes(I.cfg_2d_2048())
    assert 115e6 < ab["forward"] < 118e6


@pytest.mark.parametrize("name", sorted(bench.WORKLOADS))
def test_every_bench_workload_is_a_valid_configuration(name):
    """Each workload bench.py can time passes the library's configuration
    checks and fits in the 280 GB of one GB300 (sized through the C ABI,
    no GPU needed)."""
    from paper_2203_01462_gb300 import binding as B
    w = bench.workload(name, None)
    nbytes = B.workspace_bytes(w)
    assert 0 < nbytes < 280e9, (name, nbytes)


def test_3d_benchmark_step_bytes():
    """256^3 forward step (the default workload): 48 B per node for the six
    field components, 28 B more per design node, 32 B per CPML slab crossed,
    plus the BF16 checkpoint copy every 32 steps: about 1.01 GB."""
    ab = bench.algorithmic_bytes(I.cfg_3d_256())
    assert 1.00e9 < ab["forward"] < 1.03e9
