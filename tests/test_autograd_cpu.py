"""The autograd wrapper's bookkeeping, on the CPU with a stand-in solver.

The adjoint needs the forward run of the same design and damping.  These
tests drive ``FdtdObjective`` with a fake solver whose "objective" is a known
function of rho, so they check that backward re-runs the forward when the
solver's state changed after the objective was evaluated, and only then.
"""
import torch

from paper_2203_01462_gb300.autograd import objective


class FakeSolver:
    """W(rho) = sum(c * rho^2) with gradient 2 c rho, computed from the last
    forward's design, like the library's adjoint."""

    def __init__(self, n):
        self.c = torch.arange(1, n + 1, dtype=torch.float64)
        self.generation = 0
        self.calls = []
        self._rho = None
        self._fwd_rho = None
        self._damp = None

    def set_design(self, rho):
        self.generation += 1
        self.calls.append("set_design")
        self._rho = rho.detach().to(torch.float64).reshape(-1).clone()
        self._fwd_rho = None

    def set_damping(self, sigma_max, gamma_scale):
        self.generation += 1
        self.calls.append("set_damping")
        self._damp = (sigma_max, gamma_scale)
        self._fwd_rho = None

    def forward(self):
        self.generation += 1
        self.calls.append("forward")
        self._fwd_rho = self._rho.clone()
        return (self.c * self._fwd_rho ** 2 * self._damp[1]).sum().reshape(1)

    def adjoint(self):
        self.calls.append("adjoint")
        assert self._fwd_rho is not None, "adjoint without a forward (the library returns FDTD_ESTATE)"

    def gradient(self):
        return 2.0 * self.c * self._fwd_rho * self._damp[1]


def test_backward_after_another_objective_uses_its_own_design():
    s = FakeSolver(6)
    r1 = torch.linspace(0.1, 0.6, 6, dtype=torch.float64, requires_grad=True)
    r2 = torch.linspace(0.9, 0.4, 6, dtype=torch.float64, requires_grad=True)
    W1 = objective(r1, s, 0.0, 2.0)
    W2 = objective(r2, s, 0.0, 3.0)
    s.calls.clear()
    W1.backward()
    assert s.calls == ["set_design", "set_damping", "forward", "adjoint"]
    torch.testing.assert_close(r1.grad, 2.0 * s.c * r1.detach() * 2.0)
    s.calls.clear()
    W2.backward()
    assert s.calls[-2:] == ["forward", "adjoint"]
    torch.testing.assert_close(r2.grad, 2.0 * s.c * r2.detach() * 3.0)


def test_backward_right_after_forward_reuses_the_run():
    s = FakeSolver(4)
    r = torch.full((4,), 0.5, dtype=torch.float64, requires_grad=True)
    W = objective(r, s, 0.0, 1.0, scale=10.0)
    s.calls.clear()
    W.backward()
    assert s.calls == ["adjoint"]
    torch.testing.assert_close(r.grad, 10.0 * 2.0 * s.c * 0.5)


def test_design_changed_in_place_after_forward():
    """The wrapper keeps its own copy of rho: an optimizer step applied to
    rho before backward does not change which design the gradient is for."""
    s = FakeSolver(3)
    r = torch.tensor([0.2, 0.4, 0.6], dtype=torch.float64, requires_grad=True)
    W = objective(r, s, 0.0, 1.0)
    s.set_design(torch.zeros(3, dtype=torch.float64))  # someone else uses the solver
    with torch.no_grad():
        r.add_(0.1)
    W.backward()
    torch.testing.assert_close(r.grad, 2.0 * s.c * torch.tensor([0.2, 0.4, 0.6], dtype=torch.float64))
