"""Oracle solver: multigrid hierarchy, Chebyshev smoother, V-cycle, CG, V-cycle BFBT,
symmetric Uzawa, FGMRES and FP64 iterative refinement.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  FP64, assembled scipy matrices.

Paper passages followed (arxiv 2506.04157):
  * Sec. 5.2.1, Eq. (SymmetricUzawaStep1): the symmetric Uzawa step (u, p, u) with B
    replaced by B + C in the pressure update only.
  * Sec. 5.2.2: A^-1 approximated by CG preconditioned with a GMG V-cycle to tol_A;
    Chebyshev smoother preconditioned by the inverse diagonal of A, m_A pre/post steps of
    degree deg_A; diag(A) computed without the free-slip projection; coarse-grid CG to
    tol_coarse.
  * Sec. 5.2.3, Eq. (schurV): S_V^-1 = X^-1 (B A_C^-1 A A_C^-1 B^T) X^-1 with
    X = B A_C^-1 B^T, A_C a cheap V-cycle (m_V pre/post steps of degree deg_V); X solved by
    CG to tol_VBFBT preconditioned by M_{1/eta} (itself solved by CG to tol_invMass).
  * Sec. 5.2.4: FGMRES outer solver preconditioned by the block preconditioner.
  * Table parametertable: the default parameters.
  * Sec. 5.2.1, Eqs. (InexactUzawaStep1), (AdjointInexactUzawaStep1): the inexact and
    adjoint inexact Uzawa steps (the alternatives to the symmetric step), each from (0, 0).
  * Sec. 5.2.2 and Sec. 7.2, Eq. (ViscosityDef): with a temperature-dependent viscosity law,
    eta at the vertices of the levels above l_eta and at the quadrature points (from the
    P2 temperature) on the levels up to l_eta.
  * Sec. 5.2.3, Eq. (schurMass): S_M^-1 = M_{1/eta}^-1 solved by CG to tol_invMass; the
    diag(A)-BFBT approximation (C = D = diag(A) in the BFBT formula of Sec. 5.2.3), whose
    B diag(A)^-1 B^T solve is structured like the V-cycle BFBT's.
  * Sec. 5.2.3, Eq. (schurWBFBT) in its rescaled form: the weighted BFBT approximation
    (oracle/wbfbt.py), with a_l, a_r of Table parametertable.

Readings:
  * Chebyshev iteration in the form of Saad, Iterative Methods, Alg. 12.1 (with the
    Jacobi preconditioner), "degree k" = k applications of A per smoothing step including
    the initial residual; interval [b/20, b] with b = 1.2 x the largest eigenvalue of
    D^-1 A estimated by 15 power iterations from a seeded vector.
  * Coarsest level l_min = 1; coarse CG preconditioned by the diagonal.
  * Coarse-level viscosity: P1 full weighting of the next finer level's nodal values
    (the paper evaluates eta at coarse vertices or, below l_eta, at quadrature points from
    the temperature; for rough synthetic fields injection makes the V-cycle diverge).
  * P2 prolongation = exact P2 interpolation in the straight (pre-blending) coordinates
    (the spaces are nested there); restriction = its transpose; projections applied to
    the transferred vectors.
  * FGMRES restart 30; stop at relative residual ||r||/||r0|| (x0 = 0) in FP64.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .mesh import MacroMesh, Level, LOCAL_EDGES, kuhn_to_bary, micro_tets_kuhn
from .fem import (Operators, Constraints, ConstrainedOperators, project_mean_zero,
                  p2_values, QUAD_BARY, viscosity_law)

DEFAULTS = dict(sigma=1.0, omega=0.3, tol_A=1e-2, m_A=3, deg_A=2, tol_VBFBT=1e-1,
                tol_invMass=1e-10, m_V=1, deg_V=1, tol_coarse=1e-2,
                uzawa="symmetric", schur="vbfbt", a_l=1.0, a_r=1.0, wbfbt_mass="consistent",
                tol_wBFBT=1e-10, tol_VectorMass=1e-4)   # the last two: the oracle solves exactly


# ------------------------------------------------------------------------- transfers
def prolongation(mesh: MacroMesh, lc: int):
    """Sparse P mapping P2 nodal values of level lc to level lc+1 by evaluating the
    coarse P2 interpolant at every fine node (straight coordinates).  Returns the scalar
    (per component) matrix of shape (n_p2(lc+1), n_p2(lc))."""
    n = 2 ** lc
    kt = micro_tets_kuhn(n)                                    # coarse micro-tets (Kuhn, level lc)
    Nc, Nf = 2 * n, 4 * n                                      # coarse / fine P2 lattices
    # coarse P2 nodes of a micro-tet: vertices 2*K, edges K_a + K_b (lattice Nc)
    cnodes = [2 * kt[:, a] for a in range(4)] + [kt[:, a] + kt[:, b] for (a, b) in LOCAL_EDGES]
    cnodes = np.stack(cnodes, axis=1)                          # (T,10,3)
    # fine points inside a coarse micro-tet: 4*K0 + sum_j m_j (4*(K_j - K_0)), m in {0..4}/4
    sub = [(i0, i1, i2, i3) for i3 in range(5) for i2 in range(5 - i3) for i1 in range(5 - i2 - i3)
           for i0 in [4 - i1 - i2 - i3]]
    sub = np.array(sub)                                        # (35,4) quarter barycentrics
    lam = sub / 4.0
    phi = p2_values(lam)                                       # (35,10)
    fpts = np.einsum("sa,tai->tsi", sub, kt)                   # fine Kuhn coords (lattice Nf)
    rows, cols, vals = [], [], []
    n_f = MacroMesh.counts(Nf)["total"]
    seen = np.zeros(n_f, dtype=bool)
    for m in range(len(mesh.cells)):
        fid = mesh.node_ids(m, kuhn_to_bary(fpts.reshape(-1, 3), Nf), Nf).reshape(kt.shape[0], 35)
        cid = mesh.node_ids(m, kuhn_to_bary(cnodes.reshape(-1, 3), Nc), Nc).reshape(kt.shape[0], 10)
        for s in range(35):
            f = fid[:, s]
            new = ~seen[f]
            # first occurrence of each fine node in this batch
            f_new, first = np.unique(f[new], return_index=True)
            idx = np.nonzero(new)[0][first]
            seen[f_new] = True
            for a in range(10):
                if phi[s, a] != 0.0:
                    rows.append(f_new)
                    cols.append(cid[idx, a])
                    vals.append(np.full(f_new.size, phi[s, a]))
    assert seen.all()
    P = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(n_f, MacroMesh.counts(Nc)["total"])).tocsr()
    return P


def vector_prolongation(P):
    return sp.block_diag([P, P, P]).tocsr()


# ------------------------------------------------------------------------- smoothers
def chebyshev(Aop, Dinv, proj, x, b, steps, degree, lam_lo, lam_hi):
    """`steps` Chebyshev smoothing steps of the given degree on A x = b, Jacobi-
    preconditioned (Saad, Iterative Methods, Alg. 12.1): degree = applications of A per
    step including the initial residual; `proj` keeps vectors in the constrained space."""
    theta = 0.5 * (lam_hi + lam_lo)
    delta = 0.5 * (lam_hi - lam_lo)
    sigma1 = theta / delta
    x = x.copy()
    for _ in range(steps):
        r = b - Aop(x)
        z = proj(Dinv * r)
        rho = 1.0 / sigma1
        d = z / theta
        for k in range(1, degree + 1):
            x = x + d
            if k == degree:
                break
            r = r - Aop(d)
            z = proj(Dinv * r)
            rho_new = 1.0 / (2.0 * sigma1 - rho)
            d = rho_new * rho * d + (2.0 * rho_new / delta) * z
            rho = rho_new
    return x


def power_max_eig(Aop, Dinv, proj, n, iters=15, seed=0):
    """Largest eigenvalue of D^-1 A by power iteration from a seeded vector."""
    v = proj(np.random.default_rng(seed).standard_normal(n))
    lam = 0.0
    for _ in range(iters):
        v = v / np.linalg.norm(v)
        w = proj(Dinv * Aop(v))
        lam = np.linalg.norm(w)
        v = w
    return lam


def cg(Aop, b, x0=None, M=None, rtol=1e-8, maxit=1000, fixed_iters=None):
    """Preconditioned conjugate gradients; stops at ||r|| <= rtol ||r0|| (or after
    exactly `fixed_iters` iterations when given).  Returns (x, iterations)."""
    x = np.zeros_like(b) if x0 is None else x0.copy()
    r = b - Aop(x) if x0 is not None else b.copy()
    r0 = np.linalg.norm(r)
    if r0 == 0.0:
        return x, 0
    z = M(r) if M is not None else r.copy()
    p = z.copy()
    rz = r @ z
    it = 0
    nmax = fixed_iters if fixed_iters is not None else maxit
    while it < nmax:
        if fixed_iters is None and np.linalg.norm(r) <= rtol * r0:
            break
        Ap = Aop(p)
        pAp = p @ Ap
        if pAp == 0.0:
            break
        alpha = rz / pAp
        x = x + alpha * p
        r = r - alpha * Ap
        it += 1
        z = M(r) if M is not None else r.copy()
        rz_new = r @ z
        p = z + (rz_new / rz) * p
        rz = rz_new
    return x, it


# ------------------------------------------------------------------------- hierarchy
class Hierarchy:
    """Per-level constrained operators, diagonals, transfers and Chebyshev bounds."""

    def __init__(self, mesh, l_max, eta_fine, dlnrho_table=(0.0,), bc=(0, 1), l_min=1,
                 bounds=None, with_C=True, law=None, T_fine=None, l_eta=-1, rho_weighted=False):
        self.mesh, self.l_min, self.l_max = mesh, l_min, l_max
        self.levels, self.ops, self.cons, self.co, self.diag = {}, {}, {}, {}, {}
        Lf = Level(mesh, l_max)
        self.levels[l_max] = Lf
        for l in range(l_min, l_max):
            self.levels[l] = Level(mesh, l)
        # coarse-level viscosity by P1 full weighting (reading: injection of a rough,
        # high-contrast field makes the rediscretised coarse operators unrepresentative).
        # With a temperature-dependent law (Sec. 5.2.2): eta(x_V, T(x_V)) at the vertices of
        # every level above l_eta, eta(x_q, T(x_q)) at the quadrature points up to l_eta.
        self.T = {}
        if law is not None:
            self.etas = {}
            for l in range(l_min, l_max + 1):
                T2, T1 = temperature_on_level(Lf, self.levels[l], T_fine)
                self.T[l] = T2
                self.etas[l] = viscosity_law(self.levels[l].p1_x, T1, law)
        else:
            self.etas = viscosity_hierarchy(mesh, self.levels, eta_fine)
        for l in range(l_min, l_max + 1):
            L = self.levels[l]
            eta = self.etas[l]
            if law is not None and l <= l_eta:
                ops = Operators(L, eta, dlnrho_table, law=law, T_p2=self.T[l], rho_weighted=rho_weighted)
            else:
                ops = Operators(L, eta, dlnrho_table, rho_weighted=rho_weighted)
            cons = Constraints(L, *bc)
            self.ops[l], self.cons[l] = ops, cons
            self.co[l] = ConstrainedOperators(ops, cons, with_C=with_C)
            # diag(A) without the free-slip projection, identity on Dirichlet rows
            d = ops.A.diagonal().copy()
            d[np.tile(cons.dirichlet, 3)] = 1.0
            self.diag[l] = d
        self.P = {l: vector_prolongation(prolongation(mesh, l - 1)) for l in range(l_min + 1, l_max + 1)}
        self.bounds = {}
        for l in range(l_min + 1, l_max + 1):
            if bounds is not None and l in bounds:
                self.bounds[l] = bounds[l]
            else:
                lam = power_max_eig(self.co[l].apply_A, 1.0 / self.diag[l], self.cons[l].P0,
                                    3 * self.levels[l].n_p2)
                self.bounds[l] = (1.2 * lam / 20.0, 1.2 * lam)

    def vcycle(self, l, b, steps, degree, coarse_tol=1e-2, coarse_iters=None, x=None, coarse_exact=False):
        """One V-cycle for A_c x = b on level l from x (default 0).  The coarsest level is
        solved by Jacobi-CG to coarse_tol (or exactly coarse_iters iterations), or exactly
        with a sparse direct solve when coarse_exact (a linear V-cycle, for symmetry pins)."""
        cons = self.cons[l]
        Aop = self.co[l].apply_A
        if l == self.l_min:
            if coarse_exact:
                # A_c is singular only in the free-slip normal directions: regularise them
                import scipy.sparse.linalg as spla
                n = self.co[l].A.shape[0]
                N = sp.identity(n) - cons.Pv_matrix() - cons.identity_rows()
                return cons.P0(spla.spsolve((self.co[l].A + N).tocsc(), b))
            Dinv = 1.0 / self.diag[l]
            xc, _ = cg(Aop, b, M=lambda r: cons.P0(Dinv * r), rtol=coarse_tol, maxit=500,
                       fixed_iters=coarse_iters)
            return xc
        if x is None:
            x = np.zeros_like(b)
        lo, hi = self.bounds[l]
        Dinv = 1.0 / self.diag[l]
        x = chebyshev(Aop, Dinv, cons.P0, x, b, steps, degree, lo, hi)
        r = b - Aop(x)
        P = self.P[l]
        rc = self.cons[l - 1].P0(P.T @ r)
        ec = self.vcycle(l - 1, rc, steps, degree, coarse_tol, coarse_iters, coarse_exact=coarse_exact)
        x = x + cons.P0(P @ ec)
        x = chebyshev(Aop, Dinv, cons.P0, x, b, steps, degree, lo, hi)
        return x


def temperature_on_level(Lfine, Lcoarse, T_fine):
    """A P2 field of the finest level on a coarser level: every P2 node and P1 vertex of the
    coarse level is a P2 node of the finest level (nested lattices); matched by position."""
    from scipy.spatial import cKDTree
    tree = cKDTree(Lfine.p2_x)
    d2, i2 = tree.query(Lcoarse.p2_x)
    d1, i1 = tree.query(Lcoarse.p1_x)
    assert d2.max() < 1e-10 and d1.max() < 1e-10
    T_fine = np.asarray(T_fine, dtype=np.float64)
    return T_fine[i2], T_fine[i1]


def restrict_viscosity(Lfine, Lcoarse, eta_fine):
    """Viscosity on the next coarser level by P1 full weighting: the coarse vertex value is
    the average of the fine vertex at the same point (weight 1) and the fine vertices at the
    midpoints of its coarse edges (weight 1/2), normalised by the weights.  The fine P1
    vertices are the coarse level's P2 nodes, so the coarse tets give the stencil."""
    tp1, tp2 = Lcoarse.tet_p1, Lcoarse.tet_p2
    v = [tp1[:, a] for a in range(4)]
    j = [tp2[:, a] for a in range(4)]
    w = [np.ones(tp1.shape[0]) for _ in range(4)]
    for e, (a, b) in enumerate(LOCAL_EDGES):
        for end in (a, b):
            v.append(tp1[:, end]); j.append(tp2[:, 4 + e]); w.append(np.full(tp1.shape[0], 0.5))
    v, j, w = np.concatenate(v), np.concatenate(j), np.concatenate(w)
    key = v.astype(np.int64) * Lfine.n_p1 + j
    _, first = np.unique(key, return_index=True)
    R = sp.coo_matrix((w[first], (v[first], j[first])), shape=(Lcoarse.n_p1, Lfine.n_p1)).tocsr()
    return (R @ np.asarray(eta_fine)) / (R @ np.ones(Lfine.n_p1))


def viscosity_hierarchy(mesh, levels, eta_fine):
    """eta on every level from the finest by repeated full weighting (levels: dict l -> Level)."""
    L = max(levels)
    etas = {L: np.asarray(eta_fine)}
    for l in range(L, min(levels), -1):
        etas[l - 1] = restrict_viscosity(levels[l], levels[l - 1], etas[l])
    return etas


def inject(Lfine, Lcoarse, eta_fine):
    """Injection of a P1 field: the coarse vertex with barycentrics i (sum N_c) is the
    fine vertex i * 2^(l_f - l_c); matched through the straight coordinates."""
    if Lfine is Lcoarse:
        return np.asarray(eta_fine)
    from scipy.spatial import cKDTree
    tree = cKDTree(Lfine.p1_straight)
    d, idx = tree.query(Lcoarse.p1_straight)
    assert d.max() < 1e-12
    return np.asarray(eta_fine)[idx]


# ------------------------------------------------------------------------- Stokes solver
class StokesOracle:
    """FGMRES + a Uzawa-type block preconditioner (symmetric by default; inexact, adjoint
    inexact) with a Schur approximation (V-cycle BFBT by default; mass, diag(A)-BFBT) on
    the projected saddle-point system."""

    def __init__(self, hier: Hierarchy, params=None):
        self.h = hier
        self.p = dict(DEFAULTS, **(params or {}))
        L = hier.l_max
        self.L = L
        self.co = hier.co[L]
        self.cons = hier.cons[L]
        self.nu = 3 * hier.levels[L].n_p2
        self.np = hier.levels[L].n_p1
        ops = hier.ops[L]
        Md = ops.M_inv_eta.diagonal()
        self.M = ops.M_inv_eta
        self.Mdinv = 1.0 / Md
        self.wl = self.wr = None
        if self.p["schur"] == "wbfbt":
            from .wbfbt import WbfbtOperators
            eta = hier.etas[L]
            mass = self.p["wbfbt_mass"]
            self.wr = WbfbtOperators(hier.levels[L], eta, self.p["a_r"], mass=mass)
            self.wl = self.wr if self.p["a_l"] == self.p["a_r"] else WbfbtOperators(hier.levels[L], eta, self.p["a_l"],
                                                                                     mass=mass)

    # blocks of the constrained system
    def K(self, x):
        u, p = x[:self.nu], x[self.nu:]
        return np.concatenate([self.co.apply_A(u) + self.co.apply_BT(p), self.co.apply_Bbar(u)])

    def Ahat_inv(self, r):
        p = self.p
        h = self.h
        x, _ = cg(self.co.apply_A, r, M=lambda v: h.vcycle(self.L, v, p["m_A"], p["deg_A"], p["tol_coarse"]),
                  rtol=p["tol_A"], maxit=200)
        return x

    def Ac_inv(self, r):
        p = self.p
        return self.h.vcycle(self.L, r, p["m_V"], p["deg_V"], p["tol_coarse"])

    def Minv(self, r):
        x, _ = cg(lambda v: project_mean_zero(self.M @ v), project_mean_zero(r),
                  M=lambda v: project_mean_zero(self.Mdinv * v), rtol=self.p["tol_invMass"], maxit=500)
        return project_mean_zero(x)

    def Dinv(self, r):
        """diag(A)^-1 on the constrained velocity space."""
        return self.cons.P0(r / self.h.diag[self.L])

    def bfbt(self, r, Cinv):
        """BFBT with C = D: (B C^-1 B^T)^-1 (B C^-1 A C^-1 B^T) (B C^-1 B^T)^-1 r, the outer
        inverses by CG to tol_VBFBT preconditioned by M_{1/eta}."""
        p = self.p
        X = lambda q: self.co.apply_B(Cinv(self.co.apply_BT(q)))
        y, _ = cg(X, project_mean_zero(r), M=self.Minv, rtol=p["tol_VBFBT"], maxit=200)
        w = Cinv(self.co.apply_BT(y))
        w = self.co.apply_B(Cinv(self.co.apply_A(w)))
        z, _ = cg(X, project_mean_zero(w), M=self.Minv, rtol=p["tol_VBFBT"], maxit=200)
        return project_mean_zero(z)

    def X(self, q):
        return self.co.apply_B(self.Ac_inv(self.co.apply_BT(q)))

    def Shat_inv(self, r):
        """The Schur approximation: V-cycle BFBT X^-1 (B A_C^-1 A A_C^-1 B^T) X^-1 r (Eq.
        schurV), the inverse-viscosity mass M_{1/eta}^-1 r (Eq. schurMass), diag(A)-BFBT, or
        the weighted BFBT (Eq. schurWBFBT, rescaled form)."""
        kind = self.p["schur"]
        if kind == "mass":
            return self.Minv(r)
        if kind == "wbfbt":
            from .wbfbt import wbfbt_apply
            return project_mean_zero(wbfbt_apply(self.co, self.cons, self.co.apply_A, self.wl, self.wr, r))
        if kind == "diagbfbt":
            return self.bfbt(r, self.Dinv)
        return self.bfbt(r, self.Ac_inv)

    def uzawa(self, r):
        """One Uzawa-type step from (0, 0) on the residual r = (r_u, r_p); B + C replaces B
        in the pressure updates (Sec. 5.2.1)."""
        p = self.p
        ru, rp = r[:self.nu], r[self.nu:]
        kind = p["uzawa"]
        if kind == "inexact":        # Eq. (InexactUzawaStep1)
            un = p["sigma"] * self.Ahat_inv(ru)
            pn = -p["omega"] * self.Shat_inv(rp - self.co.apply_Bbar(un))
            return np.concatenate([un, pn])
        if kind == "adjoint":        # Eq. (AdjointInexactUzawaStep1)
            pn = -p["omega"] * self.Shat_inv(rp)
            un = p["sigma"] * self.Ahat_inv(ru - self.co.apply_BT(pn))
            return np.concatenate([un, pn])
        uh = p["sigma"] * self.Ahat_inv(ru)                  # Eq. (SymmetricUzawaStep1)
        pn = -p["omega"] * self.Shat_inv(rp - self.co.apply_Bbar(uh))
        un = uh + p["sigma"] * self.Ahat_inv(ru - self.co.apply_A(uh) - self.co.apply_BT(pn))
        return np.concatenate([un, pn])

    def fgmres(self, b, rtol, restart=30, maxit=300, x0=None):
        """Right-preconditioned flexible GMRES (modified Gram-Schmidt, Givens)."""
        x = np.zeros_like(b) if x0 is None else x0.copy()
        r = b - self.K(x)
        beta0 = np.linalg.norm(b)
        hist = [np.linalg.norm(r)]
        it = 0
        while it < maxit:
            beta = np.linalg.norm(r)
            if beta <= rtol * beta0:
                break
            V = [r / beta]
            Z = []
            H = np.zeros((restart + 1, restart))
            cs, sn = np.zeros(restart), np.zeros(restart)
            g = np.zeros(restart + 1); g[0] = beta
            k = 0
            for k in range(restart):
                z = self.uzawa(V[k])
                Z.append(z)
                w = self.K(z)
                for i in range(k + 1):
                    H[i, k] = w @ V[i]
                    w = w - H[i, k] * V[i]
                H[k + 1, k] = np.linalg.norm(w)
                V.append(w / H[k + 1, k] if H[k + 1, k] > 0 else w)
                for i in range(k):
                    t = cs[i] * H[i, k] + sn[i] * H[i + 1, k]
                    H[i + 1, k] = -sn[i] * H[i, k] + cs[i] * H[i + 1, k]
                    H[i, k] = t
                den = np.hypot(H[k, k], H[k + 1, k])
                cs[k], sn[k] = H[k, k] / den, H[k + 1, k] / den
                H[k, k] = den
                H[k + 1, k] = 0.0
                g[k + 1] = -sn[k] * g[k]
                g[k] = cs[k] * g[k]
                it += 1
                hist.append(abs(g[k + 1]))
                if abs(g[k + 1]) <= rtol * beta0 or it >= maxit:
                    break
            kk = k + 1
            y = np.linalg.solve(np.triu(H[:kk, :kk]), g[:kk])
            x = x + sum(y[i] * Z[i] for i in range(kk))
            r = b - self.K(x)
        return x, it, hist

    def residual(self, f, g, u, p):
        """Projected residual of the full system with Dirichlet values carried by u
        (raw operators, then projections; Dirichlet rows zero)."""
        ops = self.h.ops[self.L]
        ru = f - ops.A @ u - ops.B.T @ project_mean_zero(p)
        ru = self.cons.P0(ru)
        rp = project_mean_zero(g - (ops.B + ops.C) @ u)
        return np.concatenate([ru, rp])

    def solve(self, f, g, u0, p0, rtol=1e-8):
        r = self.residual(f, g, u0, p0)
        x, it, hist = self.fgmres(r, rtol)
        return u0 + x[:self.nu], project_mean_zero(p0 + x[self.nu:]), it, hist


def direct_solve(hier: Hierarchy, f, g, u0, p0):
    """Exact solution of the projected system (small levels): Dirichlet values from u0,
    free-slip by the projection basis, mean-zero pressure by a Lagrange multiplier."""
    L = hier.l_max
    ops, cons = hier.ops[L], hier.cons[L]
    nu, npp = 3 * hier.levels[L].n_p2, hier.levels[L].n_p1
    P0 = cons.Pv_matrix()
    # basis of the constrained velocity space: keep columns of P0 with nonzero norm via SVD-free trick:
    # use P0 itself (symmetric projector) and regularise the projected-out directions with identity.
    Ifree = sp.identity(nu) - P0
    A = P0 @ ops.A @ P0 + Ifree
    Bb = (ops.B + ops.C) @ P0
    BT = P0 @ ops.B.T
    one = np.ones((npp, 1))
    K = sp.bmat([[A, BT, None], [Bb, None, sp.csr_matrix(one)], [None, sp.csr_matrix(one.T), None]]).tocsc()
    r = np.concatenate([cons.P0(f - ops.A @ u0 - ops.B.T @ project_mean_zero(p0)),
                        project_mean_zero(g - (ops.B + ops.C) @ u0), [0.0]])
    import scipy.sparse.linalg as spla
    sol = spla.spsolve(K, r)
    du = P0 @ sol[:nu]
    dp = sol[nu:nu + npp]
    return u0 + du, project_mean_zero(p0 + dp)
