"""Oracle FEM: quadrature, P2/P1 bases, blended element matrices and assembled operators.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  FP64 throughout.

Paper passages followed (arxiv 2506.04157):
  * Sec. 4.1, pulled-back integrals: physical gradients are
    grad_x phi = J_B^{-T} J_F^{-T} grad_ref phi, the measure is |det J_B| |det J_F|.
  * Sec. 2, deviatoric strain rate eps(u) = sym grad u - (div u) I / dim, tau = 2 eta eps.
  * Sec. 5.1, Eq. (SaddlePointStructure): blocks A, B, C of the discrete system,
      B_ij = -int (div phi_j^u) phi_i^p,   C_ij = -int (grad ln rho . phi_j^u) phi_i^p.
  * Sec. 5.2.2: eta is a P1 function on every level, evaluated at quadrature points.
  * Sec. 5.2.3, Eq. (schurMass): the inverse-viscosity weighted P1 mass matrix.

Readings:
  * A_ij = int 2 eta eps(phi_j):eps(phi_i): the printed second term drops eta; the
    stress tau = 2 eta eps of Sec. 2 fixes it.
  * Quadrature: the symmetric 4-point degree-2 rule (weights 1/24).
  * grad ln rho is radial: (d ln rho / dr)(r) x/|x|, with d ln rho/dr a table on a
    uniform radial grid, linearly interpolated at the physical radius.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .mesh import LOCAL_EDGES, CLASS_SURFACE, CLASS_CMB, CLASS_INNER

QA = (5.0 + 3.0 * 5.0 ** 0.5) / 20.0
QB = (5.0 - 5.0 ** 0.5) / 20.0
QUAD_BARY = np.array([[QA, QB, QB, QB], [QB, QA, QB, QB], [QB, QB, QA, QB], [QB, QB, QB, QA]])
QUAD_W = np.full(4, 1.0 / 24.0)

# gradients of the barycentric coordinates w.r.t. reference coordinates zeta
_GRAD_LAMBDA = np.array([[-1.0, -1.0, -1.0], [1.0, 0, 0], [0, 1.0, 0], [0, 0, 1.0]])


def p2_values(bary):
    """The 10 P2 basis values (4 vertices, then edges in LOCAL_EDGES order)."""
    lam = np.asarray(bary)
    v = [lam[..., a] * (2 * lam[..., a] - 1) for a in range(4)]
    v += [4 * lam[..., a] * lam[..., b] for (a, b) in LOCAL_EDGES]
    return np.stack(v, axis=-1)


def p2_ref_grads(bary):
    """(…,10,3) gradients w.r.t. the reference coordinates of the P2 basis."""
    lam = np.asarray(bary)
    g = [(4 * lam[..., a] - 1)[..., None] * _GRAD_LAMBDA[a] for a in range(4)]
    g += [4 * (lam[..., b][..., None] * _GRAD_LAMBDA[a] + lam[..., a][..., None] * _GRAD_LAMBDA[b])
          for (a, b) in LOCAL_EDGES]
    return np.stack(g, axis=-2)


def interp_table(table, r, r_cmb, r_surf):
    """Linear interpolation of a table on a uniform grid over [r_cmb, r_surf]."""
    t = np.asarray(table, dtype=np.float64)
    if t.size == 1:
        return np.full_like(r, t[0])
    s = (r - r_cmb) / (r_surf - r_cmb) * (t.size - 1)
    s = np.clip(s, 0.0, t.size - 1)
    i = np.minimum(np.floor(s).astype(np.int64), t.size - 2)
    f = s - i
    return (1 - f) * t[i] + f * t[i + 1]


class Geometry:
    """Per micro-tet, per quadrature point: physical gradients, weights, positions."""

    def __init__(self, mesh, X, prism):
        # X: (E,4,3) straight vertex positions; prism: (E,) prism ids
        X = np.asarray(X, dtype=np.float64)
        JF = np.stack([X[:, 1] - X[:, 0], X[:, 2] - X[:, 0], X[:, 3] - X[:, 0]], axis=-1)  # (E,3,3)
        xq = np.einsum("qa,eai->eqi", QUAD_BARY, X)                                        # (E,Q,3)
        JB = mesh.blend_jacobian(xq, prism[:, None])                                       # (E,Q,3,3)
        J = JB @ JF[:, None]
        self.detJ = np.abs(np.linalg.det(J))                                               # (E,Q)
        Jinv = np.linalg.inv(J)
        gref = p2_ref_grads(QUAD_BARY)                                                     # (Q,10,3)
        self.grad = np.einsum("qad,eqdi->eqai", gref, Jinv)                                # (E,Q,10,3)
        self.grad1 = np.einsum("ad,eqdi->eqai", _GRAD_LAMBDA, Jinv)                         # (E,Q,4,3) P1
        self.W = QUAD_W[None, :] * self.detJ                                               # (E,Q)
        self.x = mesh.blend(xq, prism[:, None])                                            # physical qp
        self.phi = p2_values(QUAD_BARY)                                                    # (Q,10)
        self.psi = QUAD_BARY                                                               # P1 values


def element_A(geo, eta_vertex):
    """(E,30,30) element matrices of A = int 2 eta eps(phi_j):eps(phi_i); local dof
    index c*10 + a for component c of node a; eta_vertex: (E,4) P1 nodal viscosity."""
    return element_A_q(geo, eta_vertex @ QUAD_BARY.T)


def element_A_q(geo, etaq):
    """element_A with the viscosity given at the quadrature points, etaq: (E,Q)."""
    E = geo.grad.shape[0]
    g = geo.grad                                                                           # (E,Q,10,3)
    # grad(phi_a e_c) has row c equal to g_a: build eps for all 30 vector basis fns
    eps = np.zeros((E, 4, 3, 10, 3, 3))
    for c in range(3):
        eps[:, :, c, :, c, :] += 0.5 * g
        eps[:, :, c, :, :, c] += 0.5 * g
        for d in range(3):
            eps[:, :, c, :, d, d] -= g[..., c] / 3.0
    eps = eps.reshape(E, 4, 30, 9)
    wq = 2.0 * etaq * geo.W
    return np.einsum("eq,eqik,eqjk->eij", wq, eps, eps)


def element_B(geo):
    """(E,4,30): B_ki = -int (div phi_i) psi_k."""
    div = np.transpose(geo.grad, (0, 1, 3, 2)).reshape(geo.grad.shape[0], 4, 30)          # (E,Q,c*10+a)
    return -np.einsum("eq,qk,eqi->eki", geo.W, geo.psi, div)


def element_C(geo, mesh, dlnrho_table):
    """(E,4,30): C_ki = -int (grad ln rho . phi_i) psi_k, grad ln rho radial."""
    r = np.linalg.norm(geo.x, axis=-1)                                                     # (E,Q)
    g = interp_table(dlnrho_table, r, mesh.r_cmb, mesh.r_surf)[..., None] * geo.x / r[..., None]
    val = np.einsum("eqc,qa->eqca", g, geo.phi).reshape(geo.x.shape[0], 4, 30)
    return -np.einsum("eq,qk,eqi->eki", geo.W, geo.psi, val)


def element_B_rho(geo, mesh, dlnrho_table):
    """(E,4,30): the density-weighted constraint -int psi_k div(rho phi_i)
    = -int rho psi_k (div phi_i + grad ln rho . phi_i): the integrand of B + C weighted by
    rho(r) at the quadrature point (rho(r_surf) = 1; the form int q div(rho u) of the
    compressible continuity equation, Sec. 2, with the sign of B)."""
    r = np.linalg.norm(geo.x, axis=-1)                                                     # (E,Q)
    rho = rho_profile(dlnrho_table, r, mesh.r_cmb, mesh.r_surf)
    div = np.transpose(geo.grad, (0, 1, 3, 2)).reshape(geo.grad.shape[0], 4, 30)
    g = interp_table(dlnrho_table, r, mesh.r_cmb, mesh.r_surf)[..., None] * geo.x / r[..., None]
    val = div + np.einsum("eqc,qa->eqca", g, geo.phi).reshape(geo.x.shape[0], 4, 30)
    return -np.einsum("eq,qk,eqi->eki", geo.W * rho, geo.psi, val)


def element_mass_p1(geo, weight_q):
    """(E,4,4): int w psi_j psi_k with quadrature-point weight w (E,Q)."""
    return np.einsum("eq,qk,qj->ekj", geo.W * weight_q, geo.psi, geo.psi)


def velocity_dofs(level, sel=slice(None)):
    """(E,30) global velocity dof ids (component-major [3][n_p2]) of micro-tets."""
    p2 = level.tet_p2[sel]
    return np.concatenate([p2 + c * level.n_p2 for c in range(3)], axis=1)


def assemble(rows, cols, vals, shape):
    E = vals.shape[0]
    R = np.broadcast_to(rows[:, :, None], vals.shape).reshape(-1)
    C = np.broadcast_to(cols[:, None, :], vals.shape).reshape(-1)
    return sp.coo_matrix((vals.reshape(-1), (R, C)), shape=shape).tocsr()


def viscosity_law(x, T, law):
    """Frank-Kamenetskii viscosity (Sec. 7.2, Eq. ViscosityDef):
        eta(x, T) = eta_base(|x|) exp(-E_A T + V_A (r_surf - |x|)),
    law: dict with E_A, V_A, r_cmb, r_surf and log10_base, the base profile's log10 values on
    a uniform radial grid over [r_cmb, r_surf] (linear interpolation; the paper gives the
    profile as a figure)."""
    r = np.linalg.norm(np.asarray(x, dtype=np.float64), axis=-1)
    base = 10.0 ** interp_table(law["log10_base"], r, law["r_cmb"], law["r_surf"])
    return base * np.exp(-law["E_A"] * np.asarray(T, dtype=np.float64) + law["V_A"] * (law["r_surf"] - r))


class Operators:
    """Assembled FP64 blocks on one level (matrix entries are the definition, the
    matrix-vector product is the operator application).  rho_weighted: the constraint is
    -int q div(rho u) (element_B_rho) in place of B + C of Eq. SaddlePointStructure; C then
    holds the difference, so that B + C is always the constraint and B stays the momentum
    equation's (incompressible) block.  With `law` and the level's P2
    temperature T_p2, A takes the viscosity at the quadrature points, eta(x_q, T(x_q)) with
    T(x_q) the P2 interpolant (Sec. 5.2.2, levels up to l_eta); M_{1/eta} keeps eta_p1."""

    def __init__(self, level, eta_p1, dlnrho_table=(0.0,), chunk=4096, law=None, T_p2=None, rho_weighted=False):
        mesh = level.mesh
        nu, npp = 3 * level.n_p2, level.n_p1
        E = level.tet_p2.shape[0]
        As, Bs, Cs, Ms = [], [], [], []
        eta_p1 = np.asarray(eta_p1, dtype=np.float64)
        for s in range(0, E, chunk):
            sl = slice(s, min(E, s + chunk))
            geo = Geometry(mesh, level.tet_x[sl], level.tet_prism[sl])
            ev = eta_p1[level.tet_p1[sl]]
            vd = velocity_dofs(level, sl)
            pd = level.tet_p1[sl]
            if law is not None:
                Tq = np.asarray(T_p2, dtype=np.float64)[level.tet_p2[sl]] @ geo.phi.T          # (E,Q)
                As.append(assemble(vd, vd, element_A_q(geo, viscosity_law(geo.x, Tq, law)), (nu, nu)))
            else:
                As.append(assemble(vd, vd, element_A(geo, ev), (nu, nu)))
            Bs.append(assemble(pd, vd, element_B(geo), (npp, nu)))
            if rho_weighted:   # C holds B_rho - B, so that B + C is the density-weighted constraint
                Cs.append(assemble(pd, vd, element_B_rho(geo, mesh, dlnrho_table) - element_B(geo), (npp, nu)))
            else:
                Cs.append(assemble(pd, vd, element_C(geo, mesh, dlnrho_table), (npp, nu)))
            etaq = ev @ QUAD_BARY.T
            Ms.append(assemble(pd, pd, element_mass_p1(geo, 1.0 / etaq), (npp, npp)))
        self.A = sum(As[1:], As[0]).tocsr()
        self.B = sum(Bs[1:], Bs[0]).tocsr()
        self.C = sum(Cs[1:], Cs[0]).tocsr()
        self.M_inv_eta = sum(Ms[1:], Ms[0]).tocsr()
        self.level = level


# ---------------------------------------------------------------------- boundary handling
BC_DIRICHLET, BC_FREESLIP = 0, 1


class Constraints:
    """Dirichlet elimination and free-slip projection P_v (Sec. 5.1,
    Eqs. SaddlePointStructureDirichlet / InnerSaddlePointSystem)."""

    def __init__(self, level, bc_surface=BC_DIRICHLET, bc_cmb=BC_FREESLIP):
        n = level.n_p2
        cls = level.p2_class
        bc_of = {CLASS_SURFACE: bc_surface, CLASS_CMB: bc_cmb}
        dir_nodes = np.zeros(n, dtype=bool)
        fs_nodes = np.zeros(n, dtype=bool)
        for k, b in bc_of.items():
            if b == BC_DIRICHLET:
                dir_nodes |= cls == k
            else:
                fs_nodes |= cls == k
        self.n = n
        self.dirichlet = dir_nodes
        self.freeslip = fs_nodes
        x = level.p2_x
        self.normal = x / np.linalg.norm(x, axis=1, keepdims=True)

    def P0(self, u):
        """Zero the Dirichlet velocity dofs and project free-slip nodes: u - (u.n) n."""
        n = self.n
        U = np.array(u, dtype=np.float64).reshape(3, n).copy()
        U[:, self.dirichlet] = 0.0
        fs = self.freeslip
        un = np.einsum("cn,nc->n", U[:, fs], self.normal[fs])
        U[:, fs] -= un[None, :] * self.normal[fs].T
        return U.reshape(-1)

    def Pv_matrix(self):
        """Sparse matrix of P0 (useful for assembling constrained operators)."""
        n = self.n
        keep = (~self.dirichlet).astype(np.float64)
        rows, cols, vals = [], [], []
        for c in range(3):
            for d in range(3):
                v = keep * ((1.0 if c == d else 0.0) - np.where(self.freeslip, self.normal[:, c] * self.normal[:, d], 0.0))
                nzr = np.nonzero(v)[0]
                rows.append(c * n + nzr); cols.append(d * n + nzr); vals.append(v[nzr])
        return sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                             shape=(3 * n, 3 * n)).tocsr()

    def identity_rows(self):
        """Diagonal matrix with ones on the Dirichlet velocity dofs."""
        d = np.tile(self.dirichlet.astype(np.float64), 3)
        return sp.diags(d).tocsr()


def project_mean_zero(p):
    """P_p: subtract the arithmetic mean (Sec. 5.1: P_p only enforces mean zero)."""
    p = np.asarray(p, dtype=np.float64)
    return p - p.mean()


class ConstrainedOperators:
    """The projected, Dirichlet-eliminated blocks the solver works with:
         A_c = I_D + P0 A P0,  Bbar_c = P_p (B + C) P0,  BT_c = P0 B^T P_p,
    where I_D is the identity on Dirichlet dofs (block-row modification)."""

    def __init__(self, ops: Operators, cons: Constraints, with_C=True):
        P0 = cons.Pv_matrix()
        self.P0 = P0
        self.cons = cons
        self.A = (cons.identity_rows() + P0 @ ops.A @ P0).tocsr()
        Bbar = ops.B + ops.C if with_C else ops.B
        self.Bbar_raw = (Bbar @ P0).tocsr()      # P_p is applied to the output separately
        self.B_raw = (ops.B @ P0).tocsr()
        self.BT_raw = (P0 @ ops.B.T).tocsr()     # applied to P_p p
        self.BbarT_raw = (P0 @ Bbar.T).tocsr()

    def apply_A(self, u):
        return self.A @ u

    def apply_Bbar(self, u):
        return project_mean_zero(self.Bbar_raw @ u)

    def apply_B(self, u):
        return project_mean_zero(self.B_raw @ u)

    def apply_BT(self, p):
        return self.BT_raw @ project_mean_zero(p)

    def apply_BbarT(self, q):
        return self.BbarT_raw @ project_mean_zero(q)


def stokes_apply_elements(level, eta_p1, dlnrho_table, u, p, sel):
    """Raw fused operator restricted to the micro-tets `sel`:
         yu = sum_e (A_e u_e + B_e^T p_e),   yp = sum_e (B_e + C_e) u_e
    (element matrices are the definition, the sum over all tets is the operator).
    Returns dense yu [3 n_p2], yp [n_p1] holding only those contributions."""
    mesh = level.mesh
    geo = Geometry(mesh, level.tet_x[sel], level.tet_prism[sel])
    Ae = element_A(geo, np.asarray(eta_p1)[level.tet_p1[sel]])
    Be = element_B(geo)
    Ce = element_C(geo, mesh, dlnrho_table)
    vd = velocity_dofs(level, sel)
    pd = level.tet_p1[sel]
    ue = np.asarray(u)[vd]
    pe = np.asarray(p)[pd]
    yu_e = np.einsum("eij,ej->ei", Ae, ue) + np.einsum("eki,ek->ei", Be, pe)
    yp_e = np.einsum("eki,ei->ek", Be + Ce, ue)
    yu = np.zeros(3 * level.n_p2)
    yp = np.zeros(level.n_p1)
    np.add.at(yu, vd.reshape(-1), yu_e.reshape(-1))
    np.add.at(yp, pd.reshape(-1), yp_e.reshape(-1))
    return yu, yp


def tets_touching(level, p2_nodes=None, p1_nodes=None):
    """Indices of the micro-tets that contain any of the given P2 nodes / P1 vertices."""
    mask = np.zeros(level.tet_p2.shape[0], dtype=bool)
    if p2_nodes is not None:
        mask |= np.isin(level.tet_p2, p2_nodes).any(axis=1)
    if p1_nodes is not None:
        mask |= np.isin(level.tet_p1, p1_nodes).any(axis=1)
    return np.nonzero(mask)[0]


def rho_profile(table, r, r_cmb, r_surf):
    """rho(r) = exp(int_{r_surf}^{r} d ln rho/dr) for the piecewise-linear table (rho(r_surf)
    = 1).  The antiderivative of a piecewise-linear function is exact with the trapezoidal
    rule on its breakpoints: G at the table nodes by cumulative trapezoids, inside a cell
    one more trapezoid up to r."""
    table = np.atleast_1d(np.asarray(table, dtype=np.float64))
    r = np.asarray(r, dtype=np.float64)
    if table.size == 1:
        return np.exp(table[0] * (r - r_surf))
    nodes = np.linspace(r_cmb, r_surf, table.size)
    G_nodes = np.concatenate([[0.0], np.cumsum(0.5 * (table[1:] + table[:-1]) * np.diff(nodes))])
    rc = np.clip(r, r_cmb, r_surf)
    k = np.minimum(np.searchsorted(nodes, rc, side="right") - 1, table.size - 2)
    G_r = G_nodes[k] + 0.5 * (table[k] + interp_table(table, rc, r_cmb, r_surf)) * (rc - nodes[k])
    return np.exp(-(G_nodes[-1] - G_r))


def buoyancy_rhs(level, T_p2, dlnrho_table, scale=1.0):
    """f_(a,c) = scale sum_e sum_q W_q rho(r_q) T_q (x_q/|x_q|)_c phi_a(q), element by element."""
    mesh = level.mesh
    geo = Geometry(mesh, level.tet_x, level.tet_prism)
    Tq = np.asarray(T_p2)[level.tet_p2] @ geo.phi.T                       # (E,Q)
    r = np.linalg.norm(geo.x, axis=-1)
    rho = rho_profile(dlnrho_table, r, mesh.r_cmb, mesh.r_surf)
    xh = geo.x / r[..., None]
    c = scale * geo.W * rho * Tq                                          # (E,Q)
    fe = np.einsum("eq,eqd,qa->eda", c, xh, geo.phi)                      # (E,3,10)
    f = np.zeros(3 * level.n_p2)
    idx = np.stack([level.tet_p2 + d * level.n_p2 for d in range(3)], axis=1)   # (E,3,10)
    np.add.at(f, idx.reshape(-1), fe.reshape(-1))
    return f
