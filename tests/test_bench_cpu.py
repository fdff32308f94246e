"""The benchmark's host-side contract, checked without a GPU: the reference
arm's JSON line (the FP64 oracle on the host cores) and the sizing of the
bounded oracle samples."""
import json
import os
import subprocess
import sys

import bench
from paper_2203_01462_gb300 import inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_sample_steps_follow_the_node_budget():
    w = I.cfg_2d_2048()
    assert bench.sample_nsteps(w, 0, bench.CPU_CELL_STEPS) == 300
    assert bench.sample_nsteps(w, 0, bench.REF_CELL_STEPS) == 200
    # a larger grid gets fewer steps, never fewer than 10 nor more than the run
    w3 = I.cfg_3d_512()
    n3 = bench.sample_nsteps(w3, 0, bench.CPU_CELL_STEPS)
    assert 10 <= n3 < 300
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
