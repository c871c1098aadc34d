"""Manufactured-solution convergence of the oracle's discretisation (no GPU): a smooth
velocity vanishing on both spheres and a smooth pressure, the right-hand sides derived
symbolically from -div(2 eta eps(u)) + grad p and -div u - (d ln rho/dr) x/|x| . u, loads
integrated with the degree-5 conical rule, errors in the L2 / H1 norms with the same rule.

Taylor-Hood P2-P1 rates: velocity L2 3, velocity H1 2, pressure L2 2 — reached with a
constant viscosity (incompressible or compressible), with no-slip on both spheres and with
the paper's free-slip CMB (a rotation-type velocity).  With the config-1 viscosity
eta = 10^(4(1 - r)) entering A as its P1 interpolant (Sec. 5.2.2), the O(h^2) coefficient
error caps the velocity at second order in L2 too; the same viscosity evaluated exactly at the
quadrature points restores the third order.  Levels 1 -> 2 (measured rates to level 3 in the
same setting: 3.10 / 2.00 / 2.07, and 1.92 for the P1 viscosity)."""
import numpy as np
import pytest

sy = pytest.importorskip("sympy")

from oracle.mesh import MacroMesh, Level
from oracle.fem import Geometry, element_A_q, assemble, velocity_dofs, ConstrainedOperators
from oracle.solver import Hierarchy, StokesOracle
from oracle.temperature import GeometryRule, QUAD5_BARY


def _problem(variable_eta, dlnrho):
    X = sy.symbols("x0 x1 x2", real=True)
    x, y, z = X
    r = sy.sqrt(x ** 2 + y ** 2 + z ** 2)
    bubble = (r - sy.Rational(1, 2)) * (1 - r)
    u = [bubble * (-y + z * x), bubble * (x + y * z), bubble * (x * y)]
    p = x * y * z + x ** 2 - y
    eta = 10 ** (4 * (1 - r)) if variable_eta else sy.Integer(1)
    G = sy.Matrix([[sy.diff(u[i], X[j]) for j in range(3)] for i in range(3)])
    div = sum(G[i, i] for i in range(3))
    tau = 2 * eta * ((G + G.T) / 2 - div / 3 * sy.eye(3))
    f = [-sum(sy.diff(tau[i, j], X[j]) for j in range(3)) + sy.diff(p, X[i]) for i in range(3)]
    g = -div - dlnrho * sum(X[i] / r * u[i] for i in range(3))
    lam = lambda e: sy.lambdify(X, e, "numpy")
    return dict(f=lam(f), g=lam(g), u=lam(u), G=lam(G.tolist()), p=lam(p), eta=lam(eta))


def _problem_rotation(dlnrho):
    """The paper's boundary conditions (Dirichlet surface, free-slip CMB): u = s(r) w x x with
    s = 4 r (1 - r), so u = 0 on the surface, u tangential and of full size on the CMB, and
    s'(r_cmb) = 0 makes the CMB shear traction vanish (the natural condition of free slip);
    div u = 0 and x.u = 0, so g = 0 in the compressible constraint too."""
    X = sy.symbols("x0 x1 x2", real=True)
    x, y, z = X
    r = sy.sqrt(x ** 2 + y ** 2 + z ** 2)
    s = 4 * r * (1 - r)
    w = (sy.Rational(1, 3), sy.Rational(-1, 2), 1)
    u = [s * (w[1] * z - w[2] * y), s * (w[2] * x - w[0] * z), s * (w[0] * y - w[1] * x)]
    p = x * y * z + x ** 2 - y
    G = sy.Matrix([[sy.diff(u[i], X[j]) for j in range(3)] for i in range(3)])
    tau = 2 * ((G + G.T) / 2)
    f = [-sum(sy.diff(tau[i, j], X[j]) for j in range(3)) + sy.diff(p, X[i]) for i in range(3)]
    g = -sum(G[i, i] for i in range(3)) - dlnrho * sum(X[i] / r * u[i] for i in range(3))
    lam = lambda e: sy.lambdify(X, e, "numpy")
    return dict(f=lam(f), g=lam(g), u=lam(u), G=lam(G.tolist()), p=lam(p), eta=lam(sy.Integer(1)))


def _at(fun, xq):
    v = fun(xq[..., 0], xq[..., 1], xq[..., 2])
    return np.asarray(np.broadcast_arrays(*v, xq[..., 0])[:-1]) if isinstance(v, list) else \
        np.broadcast_to(v, xq.shape[:-1])


def _errors(mesh, L, prob, dlnrho, exact_eta, bc=(0, 0)):
    Lv = Level(mesh, L)
    eta_v = np.broadcast_to(prob["eta"](*Lv.p1_x.T), (Lv.n_p1,)).astype(np.float64)
    H = Hierarchy(mesh, L, eta_v, dlnrho_table=(dlnrho,), bc=bc)
    n2, n1, E = Lv.n_p2, Lv.n_p1, Lv.tet_p2.shape[0]
    if exact_eta:   # A with eta evaluated at the quadrature points instead of its P1 interpolant
        As = []
        for s in range(0, E, 4096):
            sl = slice(s, min(E, s + 4096))
            geo = Geometry(mesh, Lv.tet_x[sl], Lv.tet_prism[sl])
            vd = velocity_dofs(Lv, sl)
            As.append(assemble(vd, vd, element_A_q(geo, _at(prob["eta"], geo.x)), (3 * n2, 3 * n2)))
        H.ops[L].A = sum(As[1:], As[0]).tocsr()
        H.co[L] = ConstrainedOperators(H.ops[L], H.cons[L])
    fh, gh = np.zeros(3 * n2), np.zeros(n1)
    chunks = [slice(s, min(E, s + 4096)) for s in range(0, E, 4096)]
    for sl in chunks:
        geo = GeometryRule(mesh, Lv.tet_x[sl], Lv.tet_prism[sl])
        fq = _at(prob["f"], geo.x)                                               # (3,E,Q)
        for c in range(3):
            np.add.at(fh, (Lv.tet_p2[sl] + c * n2).reshape(-1), np.einsum("eq,eq,qa->ea", geo.W, fq[c], geo.phi).reshape(-1))
        np.add.at(gh, Lv.tet_p1[sl].reshape(-1),
                  np.einsum("eq,eq,qa->ea", geo.W, _at(prob["g"], geo.x), QUAD5_BARY).reshape(-1))
    uh, ph, it, hist = StokesOracle(H).solve(fh, gh, np.zeros(3 * n2), np.zeros(n1), rtol=1e-11)
    eu = eh = ep = epm = vol = 0.0
    for sl in chunks:
        geo = GeometryRule(mesh, Lv.tet_x[sl], Lv.tet_prism[sl])
        U = np.stack([uh[Lv.tet_p2[sl] + c * n2] for c in range(3)])               # (3,E,10)
        uq = np.einsum("cea,qa->ceq", U, geo.phi)
        Gq = np.einsum("cea,eqad->cdeq", U, geo.grad)
        eu += (geo.W * ((uq - _at(prob["u"], geo.x)) ** 2).sum(0)).sum()
        Ge = np.array([[np.broadcast_to(v, geo.W.shape) for v in row]
                       for row in prob["G"](geo.x[..., 0], geo.x[..., 1], geo.x[..., 2])])
        eh += (geo.W * ((Gq - Ge) ** 2).sum((0, 1))).sum()
        d = np.einsum("ea,qa->eq", ph[Lv.tet_p1[sl]], QUAD5_BARY) - _at(prob["p"], geo.x)
        ep += (geo.W * d * d).sum()
        epm += (geo.W * d).sum()
        vol += geo.W.sum()
    return np.sqrt(eu), np.sqrt(eh), np.sqrt(ep - epm ** 2 / vol)


@pytest.mark.parametrize("case", ["constant_eta", "p1_eta", "exact_eta"])
def test_manufactured_solution_rates(case):
    dlnrho = -1.0
    prob = _problem(case != "constant_eta", dlnrho)
    mesh = MacroMesh()
    e1 = _errors(mesh, 1, prob, dlnrho, case == "exact_eta")
    e2 = _errors(mesh, 2, prob, dlnrho, case == "exact_eta")
    ru, rh, rp = (np.log2(a / b) for a, b in zip(e1, e2))
    assert rh > 1.7 and rp > 1.8, (case, ru, rh, rp)
    if case == "p1_eta":
        assert 1.4 < ru < 2.3, ru           # second order: the P1 viscosity's O(h^2) error
    else:
        assert ru > 2.7, ru                 # optimal third order


def test_manufactured_rotation_free_slip_cmb():
    """With the paper's boundary conditions (free-slip CMB by the nodal projection P_v,
    Sec. 5.1) the rates stay those of Taylor-Hood (levels 1 -> 2: velocity L2 2.83, H1 1.88,
    pressure 2.15); a CMB treated as no-slip could not converge (u there is of size one)."""
    dlnrho = -1.0
    prob = _problem_rotation(dlnrho)
    mesh = MacroMesh()
    e1 = _errors(mesh, 1, prob, dlnrho, False, bc=(0, 1))
    e2 = _errors(mesh, 2, prob, dlnrho, False, bc=(0, 1))
    ru, rh, rp = (np.log2(a / b) for a, b in zip(e1, e2))
    assert ru > 2.6 and rh > 1.7 and rp > 1.8, (ru, rh, rp)
