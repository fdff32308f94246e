"""Host-side helpers of the optimisation loops and the monitors, on the CPU:
the damping continuation, the surrogate's input and target maps, and the
field-enhancement reductions."""
import math
import types

import numpy as np
import pytest
import torch

from paper_2203_01462_gb300 import inputs as I
from paper_2203_01462_gb300 import monitors as M
from paper_2203_01462_gb300 import optimize as OP
from paper_2203_01462_gb300 import surrogate_loop as SL


def test_damping_schedule_decays_geometrically_to_one():
    start, n = 10.0, 50
    vals = [OP.damping_schedule(k, start, n) for k in range(n + 5)]
    assert vals[0] == start
    assert all(v == 1.0 for v in vals[n:])
    assert all(a > b for a, b in zip(vals[:n], vals[1:n + 1]))
    # geometric: equal ratios between consecutive iterations
    ratios = np.array(vals[1:n + 1]) / np.array(vals[:n])
    np.testing.assert_allclose(ratios, start ** (-1.0 / n), rtol=1e-12)
    assert OP.damping_schedule(3, start, 0) == 1.0


def test_damping_levels_span_start_to_one():
    lv = OP.damping_levels(10.0, 6)
    assert len(lv) == 6 and lv[0] == 10.0 and lv[-1] == pytest.approx(1.0, abs=1e-15)
    np.testing.assert_allclose(np.array(lv[1:]) / np.array(lv[:-1]), 10.0 ** (-1.0 / 5), rtol=1e-12)
    assert OP.damping_levels(10.0, 1) == [1.0]


def test_normalised_target_has_unit_peak_and_keeps_signs():
    g = torch.tensor([[-4.0, 2.0], [1.0, 0.5]], dtype=torch.float64)
    n = SL.normalised(g)
    assert n.dtype == torch.float32
    assert float(n.abs().max()) == 1.0
    assert torch.equal(torch.sign(n), torch.sign(g).float())
    z = torch.zeros(3, dtype=torch.float64)
    assert torch.equal(SL.normalised(z), z.float())


def test_net_input_stacks_density_and_damping_level():
    rho = torch.rand(5, 7, dtype=torch.float64)
    x = SL.net_input(rho, 10.0 ** 0.6)
    assert x.shape == (2, 1, 5, 7) and x.dtype == torch.float32 and x.is_contiguous()
    assert torch.allclose(x[0, 0], rho.float())
    assert torch.allclose(x[1, 0], torch.full((5, 7), 0.6))


def test_design_map_is_rows_of_y():
    w = I.small_2d(nx=41, ny=37, design=(17, 15))
    s = types.SimpleNamespace(w=w)
    rho = torch.arange(17 * 15, dtype=torch.float64)
    m = SL.design_map(s, rho)
    assert m.shape == (15, 17)
    assert float(m[1, 0]) == 17.0  # x fastest


def test_pairs_collects_in_order():
    p = SL.Pairs()
    for k in range(3):
        p.add(torch.full((2, 1, 2, 2), float(k)), torch.full((1, 1, 2, 2), -float(k)))
    assert len(p) == 3 and float(p.x[2][0, 0, 0, 0]) == 2.0 and float(p.t[1][0, 0, 0, 0]) == -1.0


def test_magnitude_and_enhancement():
    # 2D: one complex value per gap node
    spec = np.array([[3 + 4j, 1j]])
    np.testing.assert_allclose(M.magnitude(spec), [[5.0, 1.0]])
    # 3D: vector magnitude over the components axis
    spec3 = np.zeros((2, 3, 2), dtype=complex)
    spec3[:, 0, :] = 3.0
    spec3[:, 1, :] = 4j
    np.testing.assert_allclose(M.magnitude(spec3), np.full((2, 2), 5.0))
    ref = np.ones((2, 3, 2), dtype=complex)
    np.testing.assert_allclose(M.field_enhancement(spec3, ref), np.full(2, 5.0 / math.sqrt(3.0)))


def test_incident_workload_removes_only_the_structure():
    w = I.cfg_2d_160()
    v = M.incident_workload(w)
    assert v["psi_s_ratio"] < 1e-9 and w["psi_s_ratio"] == 0.01
    assert {k: v[k] for k in v if k != "psi_s_ratio"} == {k: w[k] for k in w if k != "psi_s_ratio"}
