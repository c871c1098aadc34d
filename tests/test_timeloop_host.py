"""Host logic of the coupled time step (paper_2506_04157_gb300/timeloop.py; Sec. 3 and Eq.
StokesSub) on CPU tensors with a recording stand-in for the library problem: the order of the
library calls, the buoyancy scale Ra alpha / Pe, the Dirichlet values carried by the initial
guess, and the rotation of the time levels."""
import types

import pytest

torch = pytest.importorskip("torch")

from paper_2506_04157_gb300.timeloop import CoupledStepper

N2, NP = 7, 3


class RecordingProblem:
    """Stand-in with the sizes and entry points the stepper calls; records every call."""

    def __init__(self):
        self.calls = []
        self.mesh = types.SimpleNamespace(l_max=2, ctx=types.SimpleNamespace(device=0))

    def _sizes(self, level):
        return 3 * N2, NP

    def set_temperature(self, T):
        self.calls.append(("set_temperature", T.clone()))

    def setup_multigrid(self, l_min):
        self.calls.append(("setup_multigrid", l_min))

    def rhs_buoyancy(self, Td, f, scale):
        self.calls.append(("rhs_buoyancy", Td.clone(), scale))
        f.copy_(scale * Td.repeat(3))

    def solve(self, f, g, u, p, **opts):
        self.calls.append(("solve", u.clone(), opts))
        u.add_(f)
        p.fill_(1.0)
        return {"status": "MFS_OK"}

    def temperature_step(self, T_n, T_nm1, u_n, u_nm1, tau1, tau0, T_bc, T1, **tp):
        self.calls.append(("temperature_step", tau1, tau0, tp))
        T1.copy_(2 * T_n - T_nm1)
        return {"status": "MFS_OK"}


def test_stokes_orders_calls_and_scales_buoyancy():
    pr = RecordingProblem()
    tp = dict(Ra=10.0, alpha=2.0, Pe=4.0, k=1.0)
    T_ref = torch.full((N2,), 0.25, dtype=torch.float64)
    u_bc = torch.arange(3 * N2, dtype=torch.float64)
    S = CoupledStepper(pr, temp_params=tp, solve_opts=dict(rtol=1e-9), l_min=1, T_ref=T_ref, u_bc=u_bc,
                       device="cpu")
    T = torch.linspace(0, 1, N2, dtype=torch.float64)
    u = torch.zeros(3 * N2, dtype=torch.float64)
    p = torch.zeros(NP, dtype=torch.float64)
    st = S.stokes(T, u, p)
    assert st["status"] == "MFS_OK"
    names = [c[0] for c in pr.calls]
    assert names == ["set_temperature", "setup_multigrid", "rhs_buoyancy", "solve"]
    assert torch.equal(pr.calls[0][1], T) and pr.calls[1][1] == 1
    _, Td, scale = pr.calls[2]
    assert scale == pytest.approx(10.0 * 2.0 / 4.0) and torch.allclose(Td, T - 0.25)
    _, u_guess, opts = pr.calls[3]
    assert torch.equal(u_guess, u_bc) and opts == dict(rtol=1e-9)   # guess carries the Dirichlet values
    assert torch.allclose(u, u_bc + scale * (T - 0.25).repeat(3)) and torch.all(p == 1.0)


def test_step_rotates_time_levels():
    pr = RecordingProblem()
    S = CoupledStepper(pr, temp_params=dict(Ra=1.0, alpha=1.0, Pe=1.0), device="cpu")
    T0 = torch.rand(N2, dtype=torch.float64)
    Tm = torch.rand(N2, dtype=torch.float64)
    u0 = torch.rand(3 * N2, dtype=torch.float64)
    um = torch.rand(3 * N2, dtype=torch.float64)
    state = dict(T_n=T0, T_nm1=Tm, u_n=u0, u_nm1=um, p=torch.zeros(NP, dtype=torch.float64))
    new, stats = S.step(state, 0.1, 0.2, torch.zeros(N2, dtype=torch.float64))
    assert [c[0] for c in pr.calls][0] == "temperature_step" and pr.calls[0][1:3] == (0.1, 0.2)
    assert torch.allclose(new["T_n"], 2 * T0 - Tm)
    assert new["T_nm1"] is T0 and new["u_nm1"] is u0
    assert not torch.equal(new["u_n"], u0) and set(stats) == {"temperature", "stokes"}
    assert torch.equal(pr.calls[1][1], new["T_n"])      # the viscosity follows the new temperature
