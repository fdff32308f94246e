"""Checkpointed adjoint: lossless FP32 snapshots reproduce the full-history
gradient bit for bit; BF16 / FP16 per-slab-scaled snapshots perturb only the
recomputed fields, so W~ is unchanged and the gradient error against the
FP64 oracle stays within the stated bounds."""

import numpy as np
import pytest

from oracle import oracle as O
from paper_2203_01462_gb300 import inputs as I

pytestmark = pytest.mark.gpu

# Gradient L2-relative error bounds against the FP64 oracle (FP32 fields).
BOUND = {"f32": 1e-3, "f16": 1e-3, "bf16": 3e-3}


def medium_2d(**kw):
    w = I.workload_2d(150, 140, dx=10e-9, nsteps=1200, npml=10, design=(90, 80), gap=(3, 3), real="f32",
                      filter_radius=5, filter_fwhm=5.0, src_offset=5, **kw)
    w.update(I.pulse(800e-9, 200e12))
    return w


def small_3d(**kw):
    w = I.workload_3d(26, 24, 30, dx=20e-9, nsteps=300, npml=6, design=(10, 9, 6), gap=(2, 2, 2), source="sheet",
                      substrate=True, real="f32", **kw)
    w.update(I.pulse(800e-9, 300e12))
    return w


def grad(w, rho, smax=5e5, gs=2.0):
    from paper_2203_01462_gb300.binding import Solver
    s = Solver(w)
    W, g = s.evaluate(rho, smax, gs)
    s.sync()
    return float(W.item()), g.cpu().numpy()


@pytest.mark.parametrize("make", [medium_2d, small_3d])
def test_snapshot_precisions(make, save_report):
    base = make(snapshot_every=0)
    rho = I.rho_uniform(base, 31)
    ref = O.gradient(base, rho, 5e5, 2.0)["grad"]
    W_full, g_full = grad(base, rho)
    report = {}
    for dt in ("f32", "f16", "bf16"):
        W, g = grad(make(snapshot_every=32, snapshot_dtype=dt), rho)
        assert W == W_full
        err = float(np.linalg.norm(g - ref) / np.linalg.norm(ref))
        report[dt] = err
        if dt == "f32":
            np.testing.assert_array_equal(g, g_full)
        assert err <= BOUND[dt], (dt, err)
    report["full_history_fp32"] = float(np.linalg.norm(g_full - ref) / np.linalg.norm(ref))
    save_report("snapshot_errors_%s.json" % make.__name__, report)
