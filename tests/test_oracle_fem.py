"""Pins of the oracle's element matrices and assembled blocks (no GPU)."""
from fractions import Fraction
from itertools import product
from math import factorial

import numpy as np
import pytest

from oracle.mesh import MacroMesh, Level, CLASS_INNER
import workloads as W
from oracle.fem import (Geometry, Operators, element_A, element_B, Constraints,
                        ConstrainedOperators, project_mean_zero)

EDGES = [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)]


# ----------------------------------------------------------------- exact rational route
def _inv3(M):
    a, b, c = M[0]; d, e, f = M[1]; g, h, i = M[2]
    det = a * (e * i - f * h) - b * (d * i - f * g) + c * (d * h - e * g)
    adj = [[e * i - f * h, c * h - b * i, b * f - c * e],
           [f * g - d * i, a * i - c * g, c * d - a * f],
           [d * h - e * g, b * g - a * h, a * e - b * d]]
    return [[adj[r][s] / det for s in range(3)] for r in range(3)], det


def _grad_lambda(X):
    """Gradients of the barycentric coordinates of a tet with rational vertices."""
    JF = [[X[k + 1][r] - X[0][r] for k in range(3)] for r in range(3)]
    Jinv, det = _inv3(JF)
    g = [[Jinv[k][r] for r in range(3)] for k in range(3)]           # grad lambda_{k+1}
    g0 = [-(g[0][r] + g[1][r] + g[2][r]) for r in range(3)]
    return [g0] + g, abs(det) / 6


def _p2_grad_poly(a, gl):
    """Gradient of P2 basis fn a as {monomial exponent tuple: vector} in barycentrics."""
    poly = {}

    def add(mono, coef, vec):
        key = tuple(mono)
        cur = poly.get(key, [Fraction(0)] * 3)
        poly[key] = [cur[r] + coef * vec[r] for r in range(3)]
    if a < 4:
        e = [0, 0, 0, 0]; e[a] = 1
        add(e, Fraction(4), gl[a]); add([0, 0, 0, 0], Fraction(-1), gl[a])
    else:
        i, j = EDGES[a - 4]
        ei = [0, 0, 0, 0]; ei[j] = 1
        add(ei, Fraction(4), gl[i])
        ej = [0, 0, 0, 0]; ej[i] = 1
        add(ej, Fraction(4), gl[j])
    return poly


def _int_mono(alpha, vol):
    """int_T prod lambda_k^alpha_k = alpha! 3! |T| / (|alpha| + 3)!"""
    num = 1
    for x in alpha:
        num *= factorial(x)
    return Fraction(num * factorial(3), factorial(sum(alpha) + 3)) * vol


def _exact_A_const_eta(X, eta):
    gl, vol = _grad_lambda(X)
    polys = [_p2_grad_poly(a, gl) for a in range(10)]

    def integ(pa, pb, fn):
        s = Fraction(0)
        for ma, va in pa.items():
            for mb, vb in pb.items():
                s += fn(va, vb) * _int_mono([x + y for x, y in zip(ma, mb)], vol)
        return s
    A = [[Fraction(0)] * 30 for _ in range(30)]
    for a, c, b, d in product(range(10), range(3), range(10), range(3)):
        # eps(phi_a e_c):eps(phi_b e_d) = 1/2(delta_cd ga.gb + ga_d gb_c) - 1/3 ga_c gb_d
        def fn(va, vb, c=c, d=d):
            t = Fraction(0)
            if c == d:
                t += sum(va[r] * vb[r] for r in range(3)) / 2
            t += va[d] * vb[c] / 2
            t -= va[c] * vb[d] / 3
            return t
        A[c * 10 + a][d * 10 + b] = 2 * eta * integ(polys[a], polys[b], fn)
    return A


def _exact_B(X):
    gl, vol = _grad_lambda(X)
    polys = [_p2_grad_poly(a, gl) for a in range(10)]
    B = [[Fraction(0)] * 30 for _ in range(4)]
    for k, a, c in product(range(4), range(10), range(3)):
        s = Fraction(0)
        for ma, va in polys[a].items():
            mono = list(ma); mono[k] += 1
            s += va[c] * _int_mono(mono, vol)
        B[k][c * 10 + a] = -s
    return B


@pytest.fixture(scope="module")
def flat():
    return MacroMesh(blending=False)


def test_element_A_exact_integration(flat):
    """Constant eta, affine element: the degree-2 rule integrates the P1xP1 integrand
    exactly, so the oracle's element matrix equals the rational closed form."""
    X = [[Fraction(1, 3), Fraction(0), Fraction(1, 7)], [Fraction(2), Fraction(1, 5), Fraction(0)],
         [Fraction(1, 2), Fraction(3, 2), Fraction(1, 4)], [Fraction(1, 9), Fraction(2, 5), Fraction(5, 3)]]
    eta = Fraction(3, 2)
    exact = np.array([[float(v) for v in row] for row in _exact_A_const_eta(X, eta)])
    Xf = np.array([[float(v) for v in r] for r in X])[None]
    geo = Geometry(flat, Xf, np.array([0]))
    Ae = element_A(geo, np.full((1, 4), float(eta)))[0]
    assert np.abs(Ae - exact).max() <= 1e-13 * np.abs(exact).max()
    Be = __import__("oracle.fem", fromlist=["x"]).element_B(geo)[0]
    exactB = np.array([[float(v) for v in row] for row in _exact_B(X)])
    assert np.abs(Be - exactB).max() <= 1e-14 * np.abs(exactB).max()


@pytest.fixture(scope="module")
def level2():
    mesh = MacroMesh()
    L = Level(mesh, 2)
    r = np.linalg.norm(L.p1_x, axis=1)
    eta = 10 ** (2 * (1 - r) / 0.5)
    return L, eta, Operators(L, eta, dlnrho_table=(-1.0,))


def test_A_symmetric_constant_kernel(level2):
    L, eta, ops = level2
    A = ops.A
    assert abs(A - A.T).max() <= 1e-15 * abs(A).max()
    n = L.n_p2
    for c in range(3):
        u = np.zeros(3 * n); u[c * n:(c + 1) * n] = 1.0
        assert np.abs(A @ u).max() <= 1e-12 * abs(A).max()
    # positive semidefinite on random vectors
    rng = np.random.default_rng(0)
    for _ in range(3):
        u = rng.standard_normal(3 * n)
        assert u @ (A @ u) > 0


def test_A_scaling_and_B_eta_independent(level2):
    L, eta, ops = level2
    ops2 = Operators(L, 3.0 * eta, dlnrho_table=(-1.0,))
    assert abs(ops2.A - 3.0 * ops.A).max() <= 1e-13 * abs(ops.A).max()
    assert abs(ops2.B - ops.B).max() == 0.0
    assert abs(ops2.M_inv_eta - ops.M_inv_eta / 3.0).max() <= 1e-14 * abs(ops.M_inv_eta).max()


def test_affine_kernel_without_blending(flat):
    """Polyhedral shell: rigid rotations and the uniform dilatation u = x have zero
    deviatoric strain rate, so they lie in the kernel of A; B u = -int div u psi."""
    L = Level(flat, 2)
    ops = Operators(L, np.ones(L.n_p1))
    x = L.p2_x
    for u in (np.concatenate([-x[:, 1], x[:, 0], 0 * x[:, 2]]),
              np.concatenate([0 * x[:, 0], -x[:, 2], x[:, 1]]),
              np.concatenate([x[:, 0], x[:, 1], x[:, 2]])):
        assert np.abs(ops.A @ u).max() <= 1e-13
    # div x = 3: B u = -3 int psi_k, and sum_k int psi_k = volume
    u = np.concatenate([x[:, 0], x[:, 1], x[:, 2]])
    X = L.tet_x
    vol = np.abs(np.linalg.det(np.stack([X[:, k] - X[:, 0] for k in (1, 2, 3)], axis=-1))).sum() / 6
    assert np.isclose((ops.B @ u).sum(), -3 * vol, rtol=1e-13)


def test_constant_pressure_kernel(flat):
    """B^T 1 = -int div phi_i vanishes on inner rows exactly without blending; with
    blending it is a quadrature error that decays under refinement."""
    L = Level(flat, 2)
    ops = Operators(L, np.ones(L.n_p1))
    bt = ops.B.T @ np.ones(L.n_p1)
    inner = np.tile(L.p2_class == CLASS_INNER, 3)
    assert np.abs(bt[inner]).max() <= 1e-15 * np.abs(bt).max() * 1e2
    mesh = MacroMesh()
    errs = []
    for l in (1, 2, 3):
        Lb = Level(mesh, l)
        opsb = Operators(Lb, np.ones(Lb.n_p1))
        btb = opsb.B.T @ np.ones(Lb.n_p1)
        inner = np.tile(Lb.p2_class == CLASS_INNER, 3)
        # relative to the size of a single row entry scale h^2
        errs.append(np.abs(btb[inner]).sum())
    assert errs[2] < errs[1] < errs[0]


def test_constrained_operators(level2):
    L, eta, ops = level2
    cons = Constraints(L)
    co = ConstrainedOperators(ops, cons)
    rng = np.random.default_rng(1)
    n = L.n_p2
    u = rng.standard_normal(3 * n)
    v = rng.standard_normal(3 * n)
    p = rng.standard_normal(L.n_p1)
    # Dirichlet rows are identity, free-slip rows are tangential
    y = co.apply_A(u)
    D = np.tile(cons.dirichlet, 3)
    assert np.array_equal(y[D], u[D])
    Y = y.reshape(3, n)
    fs = cons.freeslip
    assert np.abs(np.einsum("cn,nc->n", Y[:, fs], cons.normal[fs])).max() < 1e-13 * np.abs(Y).max()
    # adjointness of the projected blocks on the constrained space
    u0, v0 = cons.P0(u), cons.P0(v)
    assert np.isclose(v0 @ co.apply_A(u0), u0 @ co.apply_A(v0), rtol=1e-13)
    assert np.isclose(project_mean_zero(p) @ co.apply_B(u0), u0 @ co.apply_BT(p), rtol=1e-12)
    assert abs(co.apply_Bbar(u).mean()) < 1e-15 * np.abs(co.apply_Bbar(u)).max() * 1e3


def test_rho_profile_closed_form():
    """rho(r) = exp(-int_r^R g) for a linear g(r) = g0 + (g1-g0)(r-r0)/(R-r0) in closed form."""
    from oracle.fem import rho_profile
    g0, g1, r0, R = -1.2, 0.4, 0.5, 1.0
    r = np.array([0.5, 0.61, 0.83, 1.0])
    s = (g1 - g0) / (R - r0)
    G = lambda x: g0 * x + 0.5 * s * (x - r0) ** 2          # antiderivative of g
    exact = np.exp(-(G(R) - G(r)))
    assert np.allclose(rho_profile(np.array([g0, g1]), r, r0, R), exact, rtol=1e-12, atol=0)


@pytest.mark.parametrize("g", [0.0, -0.3781])
def test_buoyancy_rhs_against_radial_integral(g):
    """With T = 1, f . I(x) -> int rho(r) (x/|x|) . x dx = 4 pi int_{r0}^{R} rho(r) r^3 dr,
    rho = exp(g (r - R)); measured: 2.5e-3 at level 1, 1.6e-4 at level 2 (fourth order)."""
    from oracle.fem import buoyancy_rhs
    mesh = MacroMesh()
    r0, R = mesh.r_cmb, mesh.r_surf
    rr = np.linspace(r0, R, 20001)
    val = np.exp(g * (rr - R)) * rr ** 3
    exact = 4 * np.pi * (rr[1] - rr[0]) / 3 * (val[0] + val[-1] + 4 * val[1:-1:2].sum() + 2 * val[2:-1:2].sum())
    errs = []
    for lvl in (1, 2):
        L = Level(mesh, lvl)
        f = buoyancy_rhs(L, np.ones(L.n_p2), np.array([g, g]))
        errs.append(abs(f @ L.p2_x.T.reshape(-1) - exact) / exact)
    assert errs[1] < 5e-4 and errs[1] < errs[0] / 8


def test_rho_profile_piecewise_against_adaptive_quadrature():
    """A table with kinks: adaptive quadrature split at the breakpoints is independent."""
    from scipy.integrate import quad
    from oracle.fem import rho_profile, interp_table
    tab, r0, R = np.array([-1.0, -0.2, 0.5, -0.7]), 0.5, 1.0
    nodes = np.linspace(r0, R, tab.size)
    for r in (0.5, 0.61, 0.74, 0.9, 1.0):
        val, _ = quad(lambda s: float(interp_table(tab, np.array([s]), r0, R)[0]), r, R,
                      points=[x for x in nodes if r < x < R], epsabs=1e-14, epsrel=1e-14)
        assert abs(rho_profile(tab, np.array([r]), r0, R)[0] - np.exp(-val)) <= 1e-13


def _law(E_A=4.61, V_A=2.996, table=(1.0, 0.0, -1.0, 2.0)):
    return dict(E_A=E_A, V_A=V_A, r_cmb=0.5, r_surf=1.0, log10_base=np.array(table, dtype=float))


def test_quadrature_viscosity_temperature_scaling():
    """A is linear in eta: with a uniform temperature tau, A(T = tau) = exp(-E_A tau) A(T = 0)."""
    from oracle.fem import Operators
    L = Level(MacroMesh(), 1)
    law = _law()
    eta1 = np.ones(L.n_p1)
    A0 = Operators(L, eta1, law=law, T_p2=np.zeros(L.n_p2)).A
    A1 = Operators(L, eta1, law=law, T_p2=np.full(L.n_p2, 0.37)).A
    assert abs(A1 - np.exp(-4.61 * 0.37) * A0).max() <= 1e-12 * abs(A1).max()


def test_quadrature_viscosity_activation_volume():
    """exp(V_A (r_surf - r)) equals a base profile whose log10 is linear in r (a two-entry
    table represents it exactly): both laws give the same A."""
    from oracle.fem import Operators
    L = Level(MacroMesh(), 1)
    T = W.temperature_blobs(L.p2_x, 5)
    v = 2.996
    with_va = _law(E_A=1.3, V_A=v, table=(0.2, 0.2))
    folded = _law(E_A=1.3, V_A=0.0, table=(0.2 + v * 0.5 / np.log(10.0), 0.2))
    A1 = Operators(L, np.ones(L.n_p1), law=with_va, T_p2=T).A
    A2 = Operators(L, np.ones(L.n_p1), law=folded, T_p2=T).A
    assert abs(A1 - A2).max() <= 1e-12 * abs(A1).max()


def test_temperature_injection_exact_for_linear_fields():
    from oracle.solver import temperature_on_level
    mesh = MacroMesh()
    Lf, Lc = Level(mesh, 3), Level(mesh, 1)
    a = np.array([0.3, -1.2, 0.7])
    T2, T1 = temperature_on_level(Lf, Lc, Lf.p2_x @ a)
    assert np.allclose(T2, Lc.p2_x @ a, rtol=0, atol=1e-13)
    assert np.allclose(T1, Lc.p1_x @ a, rtol=0, atol=1e-13)


def test_density_weighted_constraint_pins():
    """element_B_rho (the constraint -int q div(rho u)): reduces to B for a constant density
    (d ln rho/dr = 0), and its quadrature-point integrand equals div(rho u_h) taken by central
    differences of the vector field rho(x) u_h(x) in physical space (product rule, sign and
    radial direction of grad rho) for a random P2 field u_h on a blended micro-tet."""
    from oracle.mesh import MacroMesh, Level
    from oracle.fem import Geometry, element_B, element_B_rho, rho_profile, QUAD_BARY
    mesh = MacroMesh()
    L = Level(mesh, 1)
    sel = np.arange(0, L.tet_p2.shape[0], 37)
    geo = Geometry(mesh, L.tet_x[sel], L.tet_prism[sel])
    assert np.array_equal(element_B_rho(geo, mesh, [0.0]), element_B(geo))
    table = [-0.8, -0.2, 0.4]
    Br = element_B_rho(geo, mesh, table)
    rng = np.random.default_rng(3)
    e = 5
    ue = rng.standard_normal(30)
    X = L.tet_x[sel][e]
    prism = L.tet_prism[sel][e]
    # the P2 field on this element as a function of the physical point: invert the blended map
    # by Newton on the straight barycentric coordinates
    from oracle.mesh import LOCAL_EDGES

    def phys(lam):
        return mesh.blend((lam @ X)[None], np.array([prism]))[0]

    def lam_of(x):
        lam = np.full(4, 0.25)
        for _ in range(30):
            F = phys(lam) - x
            Jc = np.stack([(phys(lam + h * (np.eye(4)[k] - np.eye(4)[0])) - phys(lam - h * (np.eye(4)[k] - np.eye(4)[0])))
                           / (2 * h) for k in (1, 2, 3) for h in [1e-6]], axis=1)
            d = np.linalg.solve(Jc, -F)
            lam = lam + np.concatenate([[-d.sum()], d])
        return lam

    def p2_vals(lam):
        v = [l * (2 * l - 1) for l in lam] + [4 * lam[a] * lam[b] for (a, b) in LOCAL_EDGES]
        return np.array(v)

    def field(x):
        r = np.linalg.norm(x)
        phi = p2_vals(lam_of(x))
        u = np.array([ue[c * 10:(c + 1) * 10] @ phi for c in range(3)])
        return rho_profile(table, np.array([r]), mesh.r_cmb, mesh.r_surf)[0] * u

    W, psi = geo.W[e], geo.psi
    for q in range(QUAD_BARY.shape[0]):
        xq = geo.x[e, q]
        h = 1e-5
        div = sum((field(xq + h * np.eye(3)[c])[c] - field(xq - h * np.eye(3)[c])[c]) / (2 * h) for c in range(3))
        # integrand of row k at this point: -W_q psi_k(q) div(rho u_h)(x_q); compare with the
        # element matrix restricted to this quadrature point (the rule is a sum over points)
        g1 = Geometry(mesh, L.tet_x[sel][e:e + 1], L.tet_prism[sel][e:e + 1])
        Wq = np.zeros_like(g1.W)
        Wq[0, q] = g1.W[0, q]
        g1.W = Wq
        row = element_B_rho(g1, mesh, table)[0] @ ue
        assert np.allclose(row, -W[q] * psi[q] * div, rtol=1e-6, atol=1e-9 * np.abs(row).max())
