"""Oracle of the weighted BFBT Schur approximation: the inverse-square-root-viscosity P1
Laplacian K_{1/sqrt(eta)}, the square-root-viscosity vector mass M_{sqrt(eta)} (consistent or
lumped) and their composition.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  FP64, assembled scipy matrices.

Paper passages followed (arxiv 2506.04157):
  * Sec. 5.2.3, Eq. (schurWBFBT): S_w^-1 = (B M^-1 B^T)^-1 (B M^-1 A M^-1 B^T) (B M^-1 B^T)^-1
    with M = M_{sqrt(eta)}, the vector mass weighted by the square root of the viscosity.
  * Sec. 5.2.3, the form used in practice: (B M_{sqrt(eta)}^-1 B^T)^-1 is replaced by the
    inverse of K_{1/sqrt(eta)}, a Poisson operator with coefficient 1/sqrt(eta) and natural
    (Neumann) boundary conditions, and the viscosity is rescaled near the outer surface:
        S_w^-1 ~ K_{1/sqrt(eta_l)}^-1 (B M_{sqrt(eta_l)}^-1 A M_{sqrt(eta_r)}^-1 B^T) K_{1/sqrt(eta_r)}^-1,
        eta_{l,r} = a_{l,r}^2 eta on D_eta (the elements whose boundary meets the surface),
        eta elsewhere.
  * Table parametertable: tol_wBFBT = 1e-10, a_l = a_r = 1.

Readings:
  * Vector mass M_{sqrt(eta)}: the paper allows a lumped one but solves it by CG to
    tol_VectorMass, i.e. the consistent mass.  Both are built: consistent (P2 scalar mass with
    weight sqrt(eta_a), the degree-5 conical rule since the P2 mass is of degree 4, the same
    matrix for every velocity component, inverted exactly on the constrained velocity space,
    (P0 M P0 + I - P0)^-1 P0: the limit of the CG) is the solver's default; lumped by the diagonal scaling of Hinton, Rock and Zienkiewicz (1976)
    (each element's consistent-mass diagonal scaled to keep the element's total mass; row-sum
    lumping gives P2 vertices negative mass) is the alternative the library implements.
  * The K solves (tolerance 1e-10 in the paper) are exact here: a sparse direct solve on
    the mean-zero subspace, the constant null space of the Neumann problem removed by a
    Lagrange multiplier.
  * eta at a quadrature point is the P1 interpolant of the nodal viscosity (as for A); the
    weights there are 1/sqrt(eta_q) (K) and sqrt(eta_q) (M).
  * D_eta: the micro-tets with at least one vertex on the outer surface r = r_surf.
  * B without C in the middle factor, as in the other BFBT forms; the velocity-side
    inverses act on the constrained velocity space (Dirichlet rows zero, P_v).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .mesh import CLASS_SURFACE
from .fem import Geometry, QUAD_BARY, assemble, velocity_dofs, project_mean_zero
from .temperature import GeometryRule, QUAD5_BARY


def surface_tets(level):
    """D_eta: boolean mask of the micro-tets with a vertex on the outer surface."""
    return (level.p1_class[level.tet_p1] == CLASS_SURFACE).any(axis=1)


def element_stiffness_p1(geo, weight_q):
    """(E,4,4): int w grad psi_j . grad psi_k with quadrature-point weight w (E,Q)."""
    return np.einsum("eq,eqai,eqbi->eab", geo.W * weight_q, geo.grad1, geo.grad1)


def element_lumped_mass_p2(geo, weight_q):
    """(E,10): HRZ-lumped scalar P2 mass of int w phi_a phi_b: the consistent element
    diagonal times (element total) / (element trace)."""
    m = np.einsum("eq,qa,qb->eab", geo.W * weight_q, geo.phi, geo.phi)
    diag = np.diagonal(m, axis1=1, axis2=2)
    return diag * (m.sum(axis=(1, 2)) / diag.sum(axis=1))[:, None]


class WbfbtOperators:
    """K_{1/sqrt(eta_a)} (n_p1 x n_p1), the lumped M_{sqrt(eta_a)} diagonal d (n_p2) and, with
    mass="consistent", the consistent scalar M_{sqrt(eta_a)} (n_p2 x n_p2) on one level,
    eta_a = a^2 eta on D_eta and eta elsewhere (eta: nodal P1 viscosity).  M_inv applies the
    selected mass's inverse."""

    def __init__(self, level, eta_p1, a=1.0, chunk=4096, mass="lumped"):
        mesh = level.mesh
        eta_p1 = np.asarray(eta_p1, dtype=np.float64)
        surf = surface_tets(level)
        E = level.tet_p1.shape[0]
        Ks = []
        d = np.zeros(level.n_p2)
        for s in range(0, E, chunk):
            sl = slice(s, min(E, s + chunk))
            geo = Geometry(mesh, level.tet_x[sl], level.tet_prism[sl])
            etaq = eta_p1[level.tet_p1[sl]] @ QUAD_BARY.T                          # (E,Q)
            etaq = etaq * np.where(surf[sl], a * a, 1.0)[:, None]
            pd = level.tet_p1[sl]
            Ks.append(assemble(pd, pd, element_stiffness_p1(geo, 1.0 / np.sqrt(etaq)), (level.n_p1, level.n_p1)))
            np.add.at(d, level.tet_p2[sl].reshape(-1), element_lumped_mass_p2(geo, np.sqrt(etaq)).reshape(-1))
        self.K = sum(Ks[1:], Ks[0]).tocsr()
        self.d = d
        self.level = level
        self.mass = mass
        if mass == "consistent":
            Ms = []
            for s in range(0, E, chunk):
                sl = slice(s, min(E, s + chunk))
                geo = GeometryRule(mesh, level.tet_x[sl], level.tet_prism[sl])
                etaq = eta_p1[level.tet_p1[sl]] @ QUAD5_BARY.T * np.where(surf[sl], a * a, 1.0)[:, None]
                p2 = level.tet_p2[sl]
                Ms.append(assemble(p2, p2, np.einsum("eq,qa,qb->eab", geo.W * np.sqrt(etaq), geo.phi, geo.phi),
                                   (level.n_p2, level.n_p2)))
            self.Mc = sum(Ms[1:], Ms[0]).tocsr()
            self._mlu = {}
        elif mass != "lumped":
            raise ValueError(mass)
        n = level.n_p1
        one = sp.csr_matrix(np.ones((n, 1)))
        self._lu = spla.splu(sp.bmat([[self.K, one], [one.T, None]]).tocsc())

    def K_solve(self, b):
        """Mean-zero x with K x = P_p b (the exact K_{1/sqrt(eta_a)}^-1 on mean-zero vectors)."""
        rhs = np.concatenate([project_mean_zero(b), [0.0]])
        return project_mean_zero(self._lu.solve(rhs)[:-1])

    def M_inv(self, u, cons):
        """M_{sqrt(eta_a)}^-1 (lumped or consistent) on the constrained velocity space ([3][n_p2])."""
        if self.mass == "consistent":
            key = id(cons)
            if key not in self._mlu:   # (P0 M P0 + I - P0) on the three components
                P0 = cons.Pv_matrix()
                Mv = sp.block_diag([self.Mc] * 3).tocsr()
                I = sp.identity(Mv.shape[0], format="csr")
                self._mlu[key] = spla.splu((P0 @ Mv @ P0 + I - P0).tocsc())
            return cons.P0(self._mlu[key].solve(cons.P0(u)))
        return cons.P0(np.asarray(u) / np.tile(self.d, 3))


def wbfbt_apply(co, cons, A_apply, wl, wr, r):
    """S_w^-1 r = K_l^-1 (B M_l^-1 A M_r^-1 B^T) K_r^-1 r with the constrained blocks of co
    (apply_B, apply_BT) and A_apply; wl, wr: WbfbtOperators for eta_l and eta_r."""
    y = wr.K_solve(r)
    w = wr.M_inv(co.apply_BT(y), cons)
    w = co.apply_B(wl.M_inv(A_apply(w), cons))
    return wl.K_solve(w)


def icosahedron_volume(R):
    """Volume of the regular icosahedron with circumradius R (edge a = R / sin(2 pi / 5))."""
    a = R / np.sin(2.0 * np.pi / 5.0)
    return 5.0 * (3.0 + np.sqrt(5.0)) / 12.0 * a ** 3
