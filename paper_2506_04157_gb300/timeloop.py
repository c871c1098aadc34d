"""Coupled time stepping of the mantle-convection model (arxiv 2506.04157, Sec. 3): per step
the temperature splitting step (MMOC + Eq. WeakTemp), the viscosity law at the new temperature
on every level, the buoyancy load of Eq. (StokesSub) and the Stokes solve.

Orchestration only: every step is a call into the library (its kernels); the state lives in
FP64 device tensors.  With g = -x/|x| the momentum right-hand side is the buoyancy load
(Ra alpha / Pe) int rho (T - T_ref) x/|x| . phi; the velocity's Dirichlet values are zero or
a prescribed field (plate velocities on the surface, Sec. 7.2)."""
from __future__ import annotations

import torch


class CoupledStepper:
    """Time stepping on a problem whose viscosity law (set_viscosity_law) and density table
    (set_density) are set.  temp_params: mfs_temp_params fields (k, Pe, Cp, Di, alpha, H, Ra,
    tolerances); solve_opts: mfs_solve_opts fields for the Stokes solves; device: where the
    state lives (default: the problem's CUDA device)."""

    def __init__(self, problem, temp_params=None, solve_opts=None, l_min=1, T_ref=None, u_bc=None, device=None):
        self.prob = problem
        self.tp = dict(temp_params or {})
        self.opts = dict(solve_opts or {})
        self.l_min = l_min
        L = problem.mesh.l_max
        nu, npp = problem._sizes(L)
        dev = torch.device("cuda", problem.mesh.ctx.device) if device is None else torch.device(device)
        self.n2, self.np = nu // 3, npp
        self.T_ref = torch.zeros(self.n2, dtype=torch.float64, device=dev) if T_ref is None else T_ref
        self.f = torch.zeros(nu, dtype=torch.float64, device=dev)
        self.g = torch.zeros(npp, dtype=torch.float64, device=dev)
        self._Td = torch.zeros(self.n2, dtype=torch.float64, device=dev)
        # Dirichlet values of the velocity ([3][n_p2]; read at the Dirichlet nodes only)
        self.u_bc = torch.zeros(nu, dtype=torch.float64, device=dev) if u_bc is None else u_bc

    def stokes(self, T, u, p):
        """(u, p) for the temperature T in place: u starts from the Dirichlet values u_bc (zero
        elsewhere), p from its value on entry; returns the solver statistics."""
        pr = self.prob
        pr.set_temperature(T)
        pr.setup_multigrid(self.l_min)
        torch.sub(T, self.T_ref, out=self._Td)
        scale = self.tp.get("Ra", 1.0) * self.tp.get("alpha", 1.0) / self.tp.get("Pe", 1.0)
        pr.rhs_buoyancy(self._Td, self.f, scale)
        u.copy_(self.u_bc)   # initial guess carrying the Dirichlet values
        return pr.solve(self.f, self.g, u, p, **self.opts)

    def step(self, state, tau_np1, tau_n, T_bc):
        """state: dict of FP64 device tensors T_n, T_nm1, u_n, u_nm1, p; returns the new state
        and the statistics of both solves."""
        T1 = torch.empty_like(state["T_n"])
        st_T = self.prob.temperature_step(state["T_n"], state["T_nm1"], state["u_n"], state["u_nm1"], tau_np1, tau_n,
                                          T_bc, T1, **self.tp)
        u1 = torch.empty_like(state["u_n"])   # stokes() starts it from the Dirichlet values
        p1 = state["p"].clone()               # the pressure starts from the previous one
        st_S = self.stokes(T1, u1, p1)
        new = dict(T_n=T1, T_nm1=state["T_n"], u_n=u1, u_nm1=state["u_n"], p=p1)
        return new, dict(temperature=st_T, stokes=st_S)
