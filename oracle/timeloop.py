"""Oracle of the coupled time step: the temperature step, then the Stokes system with the
viscosity and the buoyancy of the new temperature.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  FP64.

Paper passages followed (arxiv 2506.04157):
  * Sec. 3: per time step, the temperature T^{n+1} from the splitting step (oracle/temperature.py),
    then the Stokes system of Eq. (StokesSub) with eta(x, T^{n+1}) and the right-hand side
    -(Ra/Pe) g rho alpha T_d^{n+1}, g = -x/|x|, and the compressible constraint.
  * Sec. 7.2, Eq. (ViscosityDef): the Frank-Kamenetskii law.

Readings:
  * With g = -x/|x| the momentum right-hand side is the buoyancy load vector
    (Ra alpha / Pe) int rho T_d (x/|x|) . phi (oracle.fem.buoyancy_rhs with that scale).
  * T_d = T - T_ref for a given reference field (the paper's T_d is the deviation from its
    reference temperature; T_ref = 0 by default).
  * The viscosity of every multigrid level is the law at that level's vertices (above l_eta)
    or at the quadrature points (up to l_eta), as in oracle.solver.Hierarchy.
  * The Stokes solve is exact (direct), the end point of the paper's FGMRES.
"""
from __future__ import annotations

import numpy as np

from .mesh import Level
from .fem import buoyancy_rhs
from .solver import Hierarchy, direct_solve
from .temperature import TemperatureOperators, Locator, temperature_step, DEFAULT_PARAMS


class CoupledOracle:
    """Temperature step + Stokes solve on the level-L shell."""

    def __init__(self, mesh, L, law, dlnrho_table=(0.0,), bc=(0, 1), l_eta=-1, T_ref=None):
        self.mesh, self.L, self.law, self.table, self.bc, self.l_eta = mesh, L, law, dlnrho_table, bc, l_eta
        self.level = Level(mesh, L)
        self.ops = TemperatureOperators(self.level, dlnrho_table)
        self.loc = Locator(self.level)
        self.T_ref = np.zeros(self.level.n_p2) if T_ref is None else np.asarray(T_ref, dtype=np.float64)

    def stokes(self, T, params):
        """(u, p) of Eq. (StokesSub) for the temperature T (zero Dirichlet velocity values)."""
        p = dict(DEFAULT_PARAMS, **(params or {}))
        H = Hierarchy(self.mesh, self.L, None, dlnrho_table=self.table, bc=self.bc, law=self.law, T_fine=T,
                      l_eta=self.l_eta, bounds={l: (0.1, 2.0) for l in range(2, self.L + 1)})
        f = buoyancy_rhs(self.level, np.asarray(T) - self.T_ref, self.table, scale=p["Ra"] * p["alpha"] / p["Pe"])
        nu, npp = 3 * self.level.n_p2, self.level.n_p1
        return direct_solve(H, f, np.zeros(npp), np.zeros(nu), np.zeros(npp))

    def step(self, state, tau_np1, tau_n, params, T_bc):
        """state: dict with T_n, T_nm1, u_n, u_nm1; returns the state one step later (with p)."""
        T1, _, _ = temperature_step(self.ops, self.loc, state["T_n"], state["T_nm1"], state["u_n"], state["u_nm1"],
                                    tau_np1, tau_n, params, T_bc, law=self.law)
        u1, p1 = self.stokes(T1, params)
        return dict(T_n=T1, T_nm1=state["T_n"], u_n=u1, u_nm1=state["u_n"], p=p1)
