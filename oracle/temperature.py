"""Oracle of the temperature step: variable-step BDF2, linear extrapolation, the particle
modified method of characteristics (MMOC) with classical RK4 back-tracking and point location
in the blended shell, and the P2 advection-diffusion system with its direct solve.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  FP64, assembled scipy matrices.

Paper passages followed (arxiv 2506.04157):
  * Sec. 3, Eq. (timeDerivative) and the definition of D[.]: variable-step BDF2,
      D[T1, T0, Tm] = s1 T1 - s0 T0 + sm Tm,  s1 = (2 t1 + t0)/(t1 + t0),
      s0 = (t1 + t0)/t0,  sm = t1^2 / (t0 (t1 + t0)),  t1 = tau^{n+1}, t0 = tau^n.
  * Sec. 3, Eq. (Extrapolation): u*^{n+1} = u^n + (u^n - u^{n-1}) tau^{n+1}/tau^n, same for T.
  * Sec. 3, MMOC: particles traced backwards over [t^n, t^{n+1}] with the classical
    Runge-Kutta method along the velocity interpolated linearly in time between u^{n+1}_*
    (at t^{n+1}) and u^n (at t^n), T^n evaluated at the departure points;
        T^n_hat = MMOC(T^n, u*^{n+1}, u^n, tau^{n+1}),
        T^{n-1}_hat = MMOC(MMOC(T^{n-1}, u*^{n+1}, u^n, tau^{n+1}), u^n, u^{n-1}, tau^n),
    approximations of T(t^n, X(t^{n+1}, t^n, x)) and T(t^{n-1}, X(t^{n+1}, t^{n-1}, x)).
  * Sec. 6, Eq. (WeakTemp): for all w in the P2 space vanishing on both spheres,
      int s1 T w + tau (k/(Pe Cp) int grad T . grad(w/rho) - Di alpha/Cp int T (u*.g) w)
        = int (s0 T0_hat - sm Tm_hat) w
          + tau (H/Cp int w + Pe Di/(Ra Cp) int (1/rho) 2 eta(x, T*) eps(u*):eps(u*) w),
    with Dirichlet values on the surface and the CMB; g = -x/|x|.

Readings:
  * Eq. (WeakTemp) as printed multiplies the s0/sm terms by tau^{n+1} as well; dividing
    D[.]/tau^{n+1} out of Eq. (DiffSolve) leaves them without it, and only that form is
    consistent (a steady field must be a fixed point, and the BDF2 coefficients sum to 0).
  * Eqs. (DiffSolve) and (WeakTemp) as printed keep an advection term u*.grad T in the solve,
    while Sec. 3 calls that solve the rest of the splitting step, the energy equation without
    the advection: the MMOC values already follow the characteristics, so D[.]/tau is the
    material derivative.  With the term the scheme advects twice and converges to another
    equation (a manufactured rotation test keeps an O(1) error as tau -> 0), contradicting
    the second-order convergence of Sec. 7.1; the solve omits it.
  * Quadrature: the P2 mass is of degree 4, beyond the 4-point rule of the Stokes blocks (with
    it the element mass has rank 4 of 10).  All temperature forms use Stroud's conical
    product rule with 3 Gauss-Jacobi points per direction (27 points, exact to degree 5,
    positive weights) on the reference tet.
  * Particles start at the P2 nodes (the MMOC result is the nodal interpolant); one RK4 step
    of length tau per MMOC; a departure point outside the shell is moved radially onto the
    nearer sphere (blended) or onto the nearer of the inner and outer face planes of the prism
    its direction crosses (polyhedral).
  * The nested MMOC for T^{n-1}_hat continues the particles: traced from the nodes over
    [t^n, t^{n+1}] with u*^{n+1}, u^n (the inner MMOC's arguments), then on from where they
    arrived over [t^{n-1}, t^n] with u^n, u^{n-1} (the outer MMOC's), and T^{n-1} evaluated once
    at the end: the characteristic X(t^{n+1}, t^{n-1}, x) the paper defines.  Composing the two
    MMOC maps as nodal fields in the printed nesting order would apply the two sub-steps to a
    point in reverse order (the field MMOC(f)(x) = f(X(x)) composes its maps inside out):
    that misses the characteristic by O(tau^3) per step for a velocity that changes in time
    (and interpolates twice), against the RK4 error O(tau^5) of the continued particles.
  * eps is the deviatoric strain rate (as in A); eta(x, T*) from the viscosity law at the
    quadrature points with the P2 interpolant of T*.
  * rho(r) = exp(int_{r_surf}^r d ln rho/dr) from the density table (as for C and the buoyancy).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla
from scipy.special import roots_jacobi, roots_legendre

from .mesh import CLASS_SURFACE, CLASS_CMB
from .fem import p2_values, p2_ref_grads, rho_profile, interp_table, viscosity_law, assemble


# ------------------------------------------------------------------------- time stepping
def bdf2_coefficients(tau_np1, tau_n):
    """(s1, s0, sm) of D[T^{n+1}, T^n, T^{n-1}] for steps tau^{n+1}, tau^n."""
    t1, t0 = float(tau_np1), float(tau_n)
    return (2 * t1 + t0) / (t1 + t0), (t1 + t0) / t0, t1 * t1 / (t0 * (t1 + t0))


def extrapolate(x_n, x_nm1, tau_np1, tau_n):
    """Linear extrapolation x^n + (x^n - x^{n-1}) tau^{n+1} / tau^n."""
    x_n = np.asarray(x_n, dtype=np.float64)
    return x_n + (x_n - np.asarray(x_nm1, dtype=np.float64)) * (tau_np1 / tau_n)


# ------------------------------------------------------------------------- quadrature
def conical_rule(npts=3):
    """Stroud's conical product rule on the reference tet {z >= 0, z1 + z2 + z3 <= 1}:
    z1 = a, z2 = (1 - a) b, z3 = (1 - a)(1 - b) c with Gauss-Jacobi points in a (weight
    (1-a)^2) and b (weight 1-b) and Gauss-Legendre points in c; exact to degree 2 npts - 1.
    Returns (barycentrics (Q,4), weights (Q,) summing to 1/6)."""
    xa, wa = roots_jacobi(npts, 2.0, 0.0)
    xb, wb = roots_jacobi(npts, 1.0, 0.0)
    xc, wc = roots_legendre(npts)
    a, b, c = (xa + 1) / 2, (xb + 1) / 2, (xc + 1) / 2
    wa, wb, wc = wa / 8, wb / 4, wc / 2          # [-1,1] -> [0,1] with the weights' powers
    Z, W = [], []
    for i in range(npts):
        for j in range(npts):
            for k in range(npts):
                Z.append([a[i], (1 - a[i]) * b[j], (1 - a[i]) * (1 - b[j]) * c[k]])
                W.append(wa[i] * wb[j] * wc[k])
    Z = np.array(Z)
    return np.column_stack([1 - Z.sum(axis=1), Z]), np.array(W)


QUAD5_BARY, QUAD5_W = conical_rule(3)


class GeometryRule:
    """Per micro-tet and quadrature point of a given rule: P2 values and physical gradients,
    weights w |det J|, physical positions (J = J_B J_F as in Sec. 4.1)."""

    def __init__(self, mesh, X, prism, bary=QUAD5_BARY, w=QUAD5_W):
        X = np.asarray(X, dtype=np.float64)
        JF = np.stack([X[:, 1] - X[:, 0], X[:, 2] - X[:, 0], X[:, 3] - X[:, 0]], axis=-1)
        xq = np.einsum("qa,eai->eqi", bary, X)
        J = mesh.blend_jacobian(xq, prism[:, None]) @ JF[:, None]
        self.W = w[None, :] * np.abs(np.linalg.det(J))
        self.grad = np.einsum("qad,eqdi->eqai", p2_ref_grads(bary), np.linalg.inv(J))
        self.phi = p2_values(bary)
        self.x = mesh.blend(xq, prism[:, None])


# ------------------------------------------------------------------------- operators
DEFAULT_PARAMS = dict(k=1.0, Pe=1.0, Cp=1.0, Di=0.0, alpha=1.0, H=0.0, Ra=1.0)


class TemperatureOperators:
    """Assembled P2 scalar blocks on one level:
        M_ij = int phi_j phi_i,   D_ij = int grad phi_j . grad(phi_i / rho),
        Ds_ij = int grad phi_j . grad phi_i / rho  (the symmetric part of D),
    and, per velocity u ([3][n_p2]), C(u)_ij = int (u.grad phi_j) phi_i and
    R(u)_ij = int (u.g) phi_j phi_i with g = -x/|x|."""

    def __init__(self, level, dlnrho_table=(0.0,), chunk=2048):
        self.level, self.table, self.chunk = level, dlnrho_table, chunk
        mesh = level.mesh
        n = level.n_p2
        E = level.tet_p2.shape[0]
        Ms, Ds, Ss = [], [], []
        for s in range(0, E, chunk):
            sl = slice(s, min(E, s + chunk))
            geo = GeometryRule(mesh, level.tet_x[sl], level.tet_prism[sl])
            r = np.linalg.norm(geo.x, axis=-1)
            rho = rho_profile(dlnrho_table, r, mesh.r_cmb, mesh.r_surf)
            dl = interp_table(dlnrho_table, r, mesh.r_cmb, mesh.r_surf)
            xh = geo.x / r[..., None]
            # grad(phi_i / rho) = grad phi_i / rho - phi_i (d ln rho/dr) xhat / rho
            gtest = geo.grad / rho[..., None, None] - (geo.phi[None, :, :, None] * (dl / rho)[..., None, None]
                                                      * xh[:, :, None, :])
            d = level.tet_p2[sl]
            Ms.append(assemble(d, d, np.einsum("eq,qa,qb->eab", geo.W, geo.phi, geo.phi), (n, n)))
            Ds.append(assemble(d, d, np.einsum("eq,eqad,eqbd->eab", geo.W, gtest, geo.grad), (n, n)))
            Ss.append(assemble(d, d, np.einsum("eq,eqad,eqbd->eab", geo.W / rho, geo.grad, geo.grad), (n, n)))
        self.M = sum(Ms[1:], Ms[0]).tocsr()
        self.D = sum(Ds[1:], Ds[0]).tocsr()
        self.Ds = sum(Ss[1:], Ss[0]).tocsr()
        cls = level.p2_class
        self.boundary = (cls == CLASS_SURFACE) | (cls == CLASS_CMB)

    def _chunks(self):
        mesh, level = self.level.mesh, self.level
        E = level.tet_p2.shape[0]
        for s in range(0, E, self.chunk):
            sl = slice(s, min(E, s + self.chunk))
            yield sl, GeometryRule(mesh, level.tet_x[sl], level.tet_prism[sl])

    def _uq(self, u, sl, geo):
        n = self.level.n_p2
        U = np.asarray(u, dtype=np.float64).reshape(3, n)[:, self.level.tet_p2[sl]]     # (3,E,10)
        return np.einsum("ceq->eqc", np.einsum("cea,qa->ceq", U, geo.phi)), U

    def advection(self, u):
        n = self.level.n_p2
        Cs = []
        for sl, geo in self._chunks():
            uq, _ = self._uq(u, sl, geo)
            d = self.level.tet_p2[sl]
            Cs.append(assemble(d, d, np.einsum("eq,eqc,eqbc,qa->eab", geo.W, uq, geo.grad, geo.phi), (n, n)))
        return sum(Cs[1:], Cs[0]).tocsr()

    def adiabatic(self, u):
        n = self.level.n_p2
        Rs = []
        for sl, geo in self._chunks():
            uq, _ = self._uq(u, sl, geo)
            r = np.linalg.norm(geo.x, axis=-1)
            ug = -np.einsum("eqc,eqc->eq", uq, geo.x) / r
            d = self.level.tet_p2[sl]
            Rs.append(assemble(d, d, np.einsum("eq,qa,qb->eab", geo.W * ug, geo.phi, geo.phi), (n, n)))
        return sum(Rs[1:], Rs[0]).tocsr()

    def shear_heating(self, u, T_star, law):
        """int (1/rho) 2 eta(x, T*) eps(u):eps(u) phi_i (eps deviatoric)."""
        level, mesh = self.level, self.level.mesh
        out = np.zeros(level.n_p2)
        for sl, geo in self._chunks():
            _, U = self._uq(u, sl, geo)
            G = np.einsum("cea,eqad->eqcd", U, geo.grad)                               # grad u
            eps = 0.5 * (G + np.swapaxes(G, -1, -2))
            tr = np.trace(G, axis1=-2, axis2=-1)
            eps = eps - (tr / 3.0)[..., None, None] * np.eye(3)
            Tq = np.asarray(T_star, dtype=np.float64)[level.tet_p2[sl]] @ geo.phi.T
            eta = viscosity_law(geo.x, Tq, law)
            r = np.linalg.norm(geo.x, axis=-1)
            rho = rho_profile(self.table, r, mesh.r_cmb, mesh.r_surf)
            val = geo.W * 2.0 * eta * np.einsum("eqcd,eqcd->eq", eps, eps) / rho
            np.add.at(out, level.tet_p2[sl].reshape(-1), np.einsum("eq,qa->ea", val, geo.phi).reshape(-1))
        return out


def temperature_matrix(ops, u_star, tau_np1, tau_n, params):
    """Left-hand side of Eq. (WeakTemp) without the advection term (reading above):
    s1 M + tau (k/(Pe Cp) D - Di alpha/Cp R(u*))."""
    p = dict(DEFAULT_PARAMS, **(params or {}))
    s1, _, _ = bdf2_coefficients(tau_np1, tau_n)
    tau = float(tau_np1)
    return s1 * ops.M + tau * ((p["k"] / (p["Pe"] * p["Cp"])) * ops.D
                               - (p["Di"] * p["alpha"] / p["Cp"]) * ops.adiabatic(u_star))


def temperature_rhs(ops, T0_hat, Tm_hat, u_star, tau_np1, tau_n, params, T_star=None, law=None, load=None):
    """Right-hand side of Eq. (WeakTemp) (reading: no tau on the s0/sm terms); the shear
    heating enters when Di != 0 and a viscosity law is given; `load` (int f phi_i of an extra
    source f, e.g. of a manufactured solution) is added times tau."""
    p = dict(DEFAULT_PARAMS, **(params or {}))
    _, s0, sm = bdf2_coefficients(tau_np1, tau_n)
    tau = float(tau_np1)
    rhs = ops.M @ (s0 * np.asarray(T0_hat) - sm * np.asarray(Tm_hat))
    rhs = rhs + tau * (p["H"] / p["Cp"]) * (ops.M @ np.ones(ops.level.n_p2))
    if law is not None and p["Di"] != 0.0:
        rhs = rhs + tau * (p["Pe"] * p["Di"] / (p["Ra"] * p["Cp"])) * ops.shear_heating(u_star, T_star, law)
    if load is not None:
        rhs = rhs + tau * np.asarray(load)
    return rhs


def solve_temperature(ops, T0_hat, Tm_hat, u_star, tau_np1, tau_n, params, T_bc, T_star=None, law=None,
                      load=None):
    """T^{n+1} of Eq. (WeakTemp) with Dirichlet values T_bc on both spheres, by a sparse
    direct solve."""
    L = temperature_matrix(ops, u_star, tau_np1, tau_n, params)
    rhs = temperature_rhs(ops, T0_hat, Tm_hat, u_star, tau_np1, tau_n, params, T_star, law, load)
    bnd = ops.boundary
    Tb = np.where(bnd, np.asarray(T_bc, dtype=np.float64), 0.0)
    rhs = rhs - L @ Tb
    keep = sp.diags((~bnd).astype(np.float64))
    A = (keep @ L @ keep + sp.diags(bnd.astype(np.float64))).tocsc()
    rhs = np.where(bnd, 0.0, rhs)
    return spla.spsolve(A, rhs) + Tb


# ------------------------------------------------------------------------- point location
class Locator:
    """Point location and P2 evaluation on one level: a physical point is pulled back by each
    prism's inverse blending (x~ = (R delta / (e.n)) e, R = |x|, e = x/R), the macro-tet with
    the largest smallest straight barycentric wins, then the micro-tet of that macro the same
    way (brute force over its n^3 micro-tets)."""

    def __init__(self, level):
        self.level = level
        mesh = level.mesh
        self.mesh = mesh
        self.n3 = level.n ** 3
        V = mesh.verts[mesh.cells]                                   # (60,4,3) straight
        self.macro_v0 = V[:, 0]
        self.macro_Tinv = np.linalg.inv(np.stack([V[:, 1] - V[:, 0], V[:, 2] - V[:, 0], V[:, 3] - V[:, 0]], axis=-1))
        X = level.tet_x
        self.tet_v0 = X[:, 0]
        self.tet_Tinv = np.linalg.inv(np.stack([X[:, 1] - X[:, 0], X[:, 2] - X[:, 0], X[:, 3] - X[:, 0]], axis=-1))

    def _pullback(self, x, prism):
        mesh = self.mesh
        if not mesh.blending:
            return x
        nh, d = mesh.prism_normal[prism], mesh.prism_delta[prism]
        R = np.linalg.norm(x, axis=-1)
        e = x / R[..., None]
        return ((R * d) / np.einsum("...i,...i->...", e, nh))[..., None] * e

    @staticmethod
    def _bary(T_inv, v0, x):
        z = np.einsum("...ij,...j->...i", T_inv, x - v0)
        return np.concatenate([1 - z.sum(axis=-1, keepdims=True), z], axis=-1)

    def locate(self, X):
        """(tet index (N,), straight barycentrics (N,4) clipped to the tet) of points X (N,3)."""
        mesh = self.mesh
        X = np.asarray(X, dtype=np.float64)
        if mesh.blending:   # radial clamp into the shell
            R = np.linalg.norm(X, axis=1)
            X = X * (np.clip(R, mesh.r_cmb, mesh.r_surf) / R)[:, None]
        else:               # polyhedral shell: radially between the prism's inner and outer faces
            dots = X @ mesh.prism_normal.T                              # (N, 20)
            f = np.argmax(dots, axis=1)                                 # the face the ray crosses
            t = dots[np.arange(X.shape[0]), f]
            d = mesh.prism_delta[f]
            X = X * (np.clip(t, mesh.r_cmb * d, mesh.r_surf * d) / t)[:, None]
        N = X.shape[0]
        score = np.full((N, 60), -np.inf)
        xt_all = np.zeros((N, 60, 3))
        for m in range(60):
            f = mesh.cell_prism[m]
            ok = X @ mesh.prism_normal[f] > 0.5 * np.linalg.norm(X, axis=1)   # directions near the prism
            xt = self._pullback(np.where(ok[:, None], X, mesh.prism_normal[f]), f)
            lam = self._bary(self.macro_Tinv[m], self.macro_v0[m], xt)
            score[:, m] = np.where(ok, lam.min(axis=1), -np.inf)
            xt_all[:, m] = xt
        mac = np.argmax(score, axis=1)
        xt = xt_all[np.arange(N), mac]
        tet = np.zeros(N, dtype=np.int64)
        lam = np.zeros((N, 4))
        for m in np.unique(mac):
            sel = np.nonzero(mac == m)[0]
            t0 = m * self.n3
            L = self._bary(self.tet_Tinv[None, t0:t0 + self.n3], self.tet_v0[None, t0:t0 + self.n3],
                           xt[sel][:, None, :])                          # (k, n3, 4)
            best = np.argmax(L.min(axis=2), axis=1)
            tet[sel] = t0 + best
            lam[sel] = L[np.arange(sel.size), best]
        lam = np.clip(lam, 0.0, None)
        lam /= lam.sum(axis=1, keepdims=True)
        return tet, lam

    def eval_p2(self, f, X):
        """Values at the points X of the P2 field(s) f ([n_p2] or [c][n_p2])."""
        tet, lam = self.locate(X)
        ph = p2_values(lam)                                              # (N,10)
        F = np.asarray(f, dtype=np.float64).reshape(-1, self.level.n_p2)
        return np.einsum("cna,na->cn", F[:, self.level.tet_p2[tet]], ph).squeeze(0) if F.shape[0] == 1 else \
            np.einsum("cna,na->cn", F[:, self.level.tet_p2[tet]], ph)


def mmoc_departure(loc, u_new, u_old, tau, X=None):
    """Departure points of the particles at X (default: the P2 nodes) after one classical RK4
    step backwards over a step tau, u linear in time from u_old (start) to u_new (end)."""
    x = loc.level.p2_x if X is None else np.asarray(X, dtype=np.float64)
    u_mid = 0.5 * (np.asarray(u_new) + np.asarray(u_old))
    k1 = loc.eval_p2(u_new, x).T
    k2 = loc.eval_p2(u_mid, x - 0.5 * tau * k1).T
    k3 = loc.eval_p2(u_mid, x - 0.5 * tau * k2).T
    k4 = loc.eval_p2(u_old, x - tau * k3).T
    return x - (tau / 6.0) * (k1 + 2 * k2 + 2 * k3 + k4)


def mmoc(loc, T, u_new, u_old, tau):
    """MMOC(T, u_new, u_old, tau): T at the departure points of the P2 nodes."""
    return loc.eval_p2(T, mmoc_departure(loc, u_new, u_old, tau))


def mmoc_history(loc, T_n, T_nm1, u_star, u_n, u_nm1, tau_np1, tau_n):
    """The two history values of the BDF2 step (Sec. 3): T^n and T^{n-1} at the feet of the
    characteristics through the P2 nodes at t^{n+1}.  The particles leave the nodes at
    t^{n+1}, reach Y at t^n (one RK4 step with u between u*^{n+1} and u^n) and are traced on
    from Y to t^{n-1} (one step with u between u^n and u^{n-1}): T^{n-1} is evaluated once,
    at the end of the same particle paths, T(t^{n-1}, X(t^{n+1}, t^{n-1}, x)) as defined with
    Eq. (timeDerivative)."""
    Y = mmoc_departure(loc, u_star, u_n, tau_np1)
    Z = mmoc_departure(loc, u_n, u_nm1, tau_n, X=Y)
    return loc.eval_p2(T_n, Y), loc.eval_p2(T_nm1, Z)


def temperature_step(ops, loc, T_n, T_nm1, u_n, u_nm1, tau_np1, tau_n, params, T_bc, law=None, load=None):
    """One temperature step of Sec. 3 and Sec. 6: extrapolations, the two MMOC evaluations,
    and the solve of Eq. (WeakTemp).  Returns (T^{n+1}, u*^{n+1}, T*^{n+1})."""
    u_star = extrapolate(u_n, u_nm1, tau_np1, tau_n)
    T_star = extrapolate(T_n, T_nm1, tau_np1, tau_n)
    T0_hat, Tm_hat = mmoc_history(loc, T_n, T_nm1, u_star, u_n, u_nm1, tau_np1, tau_n)
    T_np1 = solve_temperature(ops, T0_hat, Tm_hat, u_star, tau_np1, tau_n, params, T_bc, T_star, law, load)
    return T_np1, u_star, T_star
