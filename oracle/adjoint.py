"""Oracle adjoint: transposed projected saddle-point solve and the gradient of an objective
w.r.t. the nodal log-viscosity.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  FP64.

Definitions (the paper has no adjoint; derived from its discrete system, Sec. 5.1):
  K x = b with K = [A B^T; (B+C) 0] on the projected space (Eq. SaddlePointStructureDirichlet),
  A linear in the P1 viscosity: A = sum_k eta_k dA/deta_k with
  (dA/deta_k)_ij = int 2 psi_k eps(phi_j):eps(phi_i) (quadrature as in A).
  For J(x):  K^T lam = dJ/dx,  dJ/d(log eta_k) = -eta_k lam_u^T (dA/deta_k) u.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .fem import Geometry, QUAD_BARY, project_mean_zero


def adjoint_direct(hier, ju, jp):
    """Exact multiplier of the transposed projected system (small levels):
    [P0 A P0, P0 (B+C)^T; B P0, 0] lam = P (ju, jp), mean-zero pressure part."""
    L = hier.l_max
    ops, cons = hier.ops[L], hier.cons[L]
    nu, npp = 3 * hier.levels[L].n_p2, hier.levels[L].n_p1
    P0 = cons.Pv_matrix()
    Ifree = sp.identity(nu) - P0
    A = P0 @ ops.A @ P0 + Ifree
    BbT = P0 @ (ops.B + ops.C).T
    Bp = ops.B @ P0
    one = np.ones((npp, 1))
    K = sp.bmat([[A, BbT, None], [Bp, None, sp.csr_matrix(one)], [None, sp.csr_matrix(one.T), None]]).tocsc()
    r = np.concatenate([cons.P0(ju), project_mean_zero(jp), [0.0]])
    sol = spla.spsolve(K, r)
    return P0 @ sol[:nu], project_mean_zero(sol[nu:nu + npp])


def grad_log_eta(level, eta_p1, u, lam):
    """g_k = -eta_k sum_e sum_q 2 W_q psi_k(q) eps(u)(q):eps(lam)(q), element by element."""
    mesh = level.mesh
    geo = Geometry(mesh, level.tet_x, level.tet_prism)
    n = level.n_p2
    U = np.asarray(u).reshape(3, n)[:, level.tet_p2]        # (3,E,10)
    Lm = np.asarray(lam).reshape(3, n)[:, level.tet_p2]
    gu = np.einsum("cea,eqad->eqcd", U, geo.grad)           # grad u at qps (E,Q,3,3)
    gl = np.einsum("cea,eqad->eqcd", Lm, geo.grad)

    def dev(G):
        S = 0.5 * (G + np.swapaxes(G, -1, -2))
        tr = np.trace(G, axis1=-2, axis2=-1)
        return S - tr[..., None, None] / 3.0 * np.eye(3)
    contr = np.einsum("eqcd,eqcd->eq", dev(gu), dev(gl))    # (E,Q)
    ge = np.einsum("eq,qk->ek", 2.0 * geo.W * contr, QUAD_BARY)
    g = np.zeros(level.n_p1)
    np.add.at(g, level.tet_p1.reshape(-1), ge.reshape(-1))
    return -np.asarray(eta_p1) * g
