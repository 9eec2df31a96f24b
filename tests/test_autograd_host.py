"""Host logic of the autograd wrapper (autograd.py) with a stand-in solver on
the CPU: which inputs receive gradients, in which dtype, and that the
parameters reach the solver unchanged.  The stand-in's forward is
u = 2 v + eps and its reverse mode returns the matching adjoints; the GPU
path itself is tested against the oracle in test_gpu_adjoint.py."""
import torch

from paper_2510_00562_gb300.autograd import _Unrolled


class _StandIn:
    def __init__(self):
        self.params = {}
        self.calls = []

    def set_params(self, **kw):
        self.params.update(kw)

    def solve(self, v):
        return 2.0 * v + self.params["eps"], None, None, self.params["max_iter"]

    def load(self, v):
        self.calls.append("load")

    def unrolled_vjp(self, iters, ubar, ckpt_every=0):
        self.calls.append(("vjp", iters, ckpt_every))
        return 2.0 * ubar, {"eps": float(ubar.sum()), "alpha": 0.0, "beta": 0.0, "omega": 0.0}


def test_gradients_reach_tensor_inputs_in_their_dtype():
    sol = _StandIn()
    v = torch.rand(3, 4, 5, requires_grad=True)
    eps = torch.tensor(0.5, dtype=torch.float64, requires_grad=True)
    omega = torch.tensor(0.03, dtype=torch.float32, requires_grad=True)
    u = _Unrolled.apply(v, eps, 2.0, 3.0, omega, sol, 7, 5)
    assert torch.allclose(u, 2.0 * v.detach() + 0.5)
    assert sol.params == {"eps": 0.5, "alpha": 2.0, "beta": 3.0, "omega": omega.item(), "max_iter": 7, "tol": 0.0}
    w = torch.rand_like(u)
    (u * w).sum().backward()
    assert torch.allclose(v.grad, 2.0 * w)
    assert eps.grad.dtype == torch.float64 and float(eps.grad) == float(w.sum())
    assert omega.grad.dtype == torch.float32 and float(omega.grad) == 0.0
    assert ("vjp", 7, 5) in sol.calls and "load" in sol.calls


def test_constant_parameters_get_no_gradient():
    sol = _StandIn()
    v = torch.rand(2, 3, 4)                      # no gradient wanted for v either
    eps = torch.tensor(0.1, requires_grad=True)
    u = _Unrolled.apply(v, eps, 1.0, 1.0, 0.05, sol, 3, 0)
    u.sum().backward()
    assert eps.grad is not None and v.grad is None
