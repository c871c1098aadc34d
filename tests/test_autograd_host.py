"""Host logic of the torch.autograd wrapper (paper_2506_04157_gb300/autograd.py) on the CPU:
a stand-in problem solves a small dense nonsymmetric system K(eta) u = f (p = g) exactly, with
its adjoint K^T lam = du and the gradient -eta_k lam^T (dK/d eta_k) u, so that gradcheck tests
the wrapper's plumbing: which solve runs in backward, the order of the returned gradients, and
the restoration of the forward pass's checkpointed state when another forward pass changed the
viscosity in between."""
import types

import pytest

torch = pytest.importorskip("torch")

from paper_2506_04157_gb300.autograd import stokes_solve

NU, NP, NE = 6, 2, 4


class DenseProblem:
    def __init__(self, seed=0):
        gen = torch.Generator().manual_seed(seed)
        self.A0 = torch.randn(NU, NU, generator=gen, dtype=torch.float64) * 0.1 + 3 * torch.eye(NU, dtype=torch.float64)
        V = torch.randn(NE, NU, generator=gen, dtype=torch.float64)
        self.E = torch.einsum("ki,kj->kij", V, V)          # eta_k's rank-one parts
        self.log_eta = None
        self.setups = 0
        self.restores = 0
        self.mesh = types.SimpleNamespace(l_max=1, info=lambda L: types.SimpleNamespace(n_p1=NP))

    def K(self):
        return self.A0 + torch.einsum("k,kij->ij", torch.exp(self.log_eta), self.E)

    def set_viscosity(self, x, is_log=False):
        assert is_log
        self.log_eta = x.detach().clone()

    def setup_multigrid(self, l_min):
        self.setups += 1

    def mg_checkpoint(self):
        return self.log_eta.clone()

    def mg_restore(self, state):
        self.restores += 1
        self.log_eta = state.clone()

    def solve(self, f, g, u, p, **opts):
        u.copy_(torch.linalg.solve(self.K(), f))
        p.copy_(g)

    def adjoint_solve(self, gu, gp, lam_u, lam_p, **opts):
        lam_u.copy_(torch.linalg.solve(self.K().T, gu))
        lam_p.copy_(gp)

    def grad_log_eta(self, u, lam_u, grad):
        grad.copy_(-torch.exp(self.log_eta) * torch.einsum("i,kij,j->k", lam_u, self.E, u))


def test_gradcheck_through_the_wrapper():
    prob = DenseProblem()
    gen = torch.Generator().manual_seed(1)
    le = (0.3 * torch.randn(NE, generator=gen, dtype=torch.float64)).requires_grad_()
    f = torch.randn(NU, generator=gen, dtype=torch.float64, requires_grad=True)
    g = torch.randn(NP, generator=gen, dtype=torch.float64, requires_grad=True)
    fn = lambda a, b, c: stokes_solve(a, b, c, prob)
    assert torch.autograd.gradcheck(fn, (le, f, g), eps=1e-6, atol=1e-7)


def test_backward_restores_the_viscosity_of_its_forward():
    prob = DenseProblem(2)
    gen = torch.Generator().manual_seed(3)
    le1 = torch.randn(NE, generator=gen, dtype=torch.float64).requires_grad_()
    le2 = torch.randn(NE, generator=gen, dtype=torch.float64)
    f = torch.randn(NU, generator=gen, dtype=torch.float64)
    g = torch.zeros(NP, dtype=torch.float64)
    u1, _ = stokes_solve(le1, f, g, prob)
    stokes_solve(le2, f, g, prob)                           # another viscosity in between
    setups = prob.setups
    (u1 ** 2).sum().backward()
    # the checkpoint of the first forward pass is restored: no second hierarchy setup
    assert prob.setups == setups and prob.restores == 1 and torch.equal(prob.log_eta, le1.detach())
    # against the same derivative with no forward pass in between
    prob2 = DenseProblem(2)
    le1b = le1.detach().clone().requires_grad_()
    u1b, _ = stokes_solve(le1b, f, g, prob2)
    (u1b ** 2).sum().backward()
    assert prob2.setups == 1 and prob2.restores == 0 and torch.allclose(le1.grad, le1b.grad, rtol=1e-12, atol=0)
