"""Pins of the oracle's multigrid and Stokes solver (no GPU)."""
import json
import os

import numpy as np
import pytest

import workloads as W
from oracle.mesh import MacroMesh, Level
from oracle.fem import p2_values
from oracle.solver import (DEFAULTS, Hierarchy, StokesOracle, chebyshev, cg, direct_solve,
                           prolongation)

HERE = os.path.dirname(os.path.abspath(__file__))


def test_default_parameters_match_paper_table():
    gold = json.load(open(os.path.join(HERE, "golden", "solver_parameters.json")))
    for k, v in gold.items():
        if k != "_source":
            assert DEFAULTS[k] == v, k
    assert DEFAULTS["uzawa"] == "symmetric" and DEFAULTS["schur"] == "vbfbt"   # Sec. 5.2.4


def test_chebyshev_error_reduction_closed_form():
    """On A = diag(lambda), D = I, b = 0 the error after one step of degree k is
    T_k((theta - lambda)/delta) / T_k(theta/delta) (Chebyshev polynomial optimality)."""
    lo, hi = 0.1, 2.0
    lam = np.linspace(0.05, 2.2, 41)
    theta, delta = (hi + lo) / 2, (hi - lo) / 2

    def T(k, x):
        x = np.asarray(x, dtype=float)
        out = np.empty_like(x)
        m = np.abs(x) <= 1
        out[m] = np.cos(k * np.arccos(x[m]))
        out[~m] = np.cosh(k * np.arccosh(np.abs(x[~m]))) * np.sign(x[~m]) ** k
        return out
    for k in (1, 2, 3, 5):
        x = chebyshev(lambda v: lam * v, np.ones_like(lam), lambda v: v, np.ones_like(lam),
                      np.zeros_like(lam), 1, k, lo, hi)
        ref = T(k, (theta - lam) / delta) / T(k, np.array([theta / delta]))[0]
        assert np.allclose(x, ref, rtol=1e-12, atol=1e-14)


def test_cg_solves_spd():
    rng = np.random.default_rng(3)
    Q = rng.standard_normal((30, 30))
    A = Q @ Q.T + 30 * np.eye(30)
    b = rng.standard_normal(30)
    x, it = cg(lambda v: A @ v, b, rtol=1e-12, maxit=200)
    assert np.allclose(A @ x, b, rtol=0, atol=1e-9 * np.linalg.norm(b))


@pytest.mark.parametrize("lc", [0, 1, 2])
def test_prolongation_exact_for_quadratics(lc):
    """P2 spaces are nested in straight coordinates: prolongating the coarse interpolant
    of a quadratic reproduces the fine interpolant exactly."""
    mesh = MacroMesh()
    Lc, Lf = Level(mesh, lc), Level(mesh, lc + 1)
    P = prolongation(mesh, lc)
    rng = np.random.default_rng(lc)
    c = rng.standard_normal(10)

    def q(x):
        x0, x1, x2 = x[:, 0], x[:, 1], x[:, 2]
        return (c[0] + c[1] * x0 + c[2] * x1 + c[3] * x2 + c[4] * x0 * x0 + c[5] * x1 * x1
                + c[6] * x2 * x2 + c[7] * x0 * x1 + c[8] * x0 * x2 + c[9] * x1 * x2)
    assert np.abs(P @ q(Lc.p2_straight) - q(Lf.p2_straight)).max() < 1e-12
    # rows sum to one (partition of unity)
    assert np.allclose(np.asarray(P.sum(axis=1)).ravel(), 1.0)


@pytest.fixture(scope="module")
def hier2():
    mesh = MacroMesh()
    L = Level(mesh, 2)
    eta = W.viscosity_radial(L.p1_x)
    return Hierarchy(mesh, 2, eta, dlnrho_table=W.dlnrho_table_config1())


def test_vcycle_symmetric_with_exact_coarse(hier2):
    H = hier2
    rng = np.random.default_rng(0)
    n = 3 * H.levels[2].n_p2
    u = H.cons[2].P0(rng.standard_normal(n))
    v = H.cons[2].P0(rng.standard_normal(n))
    Mu = H.vcycle(2, u, 3, 2, coarse_exact=True)
    Mv = H.vcycle(2, v, 3, 2, coarse_exact=True)
    assert abs(v @ Mu - u @ Mv) <= 1e-12 * abs(v @ Mu)
    assert u @ Mu > 0 and v @ Mv > 0


def test_vcycle_contracts(hier2):
    H = hier2
    rng = np.random.default_rng(1)
    n = 3 * H.levels[2].n_p2
    b = H.cons[2].P0(rng.standard_normal(n))
    A = H.co[2].apply_A
    x = np.zeros(n)
    res = []
    for _ in range(4):
        x = x + H.vcycle(2, b - A(x), 3, 2)
        res.append(np.linalg.norm(b - A(x)) / np.linalg.norm(b))
    assert res[-1] < 2e-3 and all(r2 < 0.5 * r1 for r1, r2 in zip(res, res[1:]))


@pytest.mark.slow
def test_stokes_fgmres_matches_direct(hier2):
    H = hier2
    S = StokesOracle(H)
    rng = np.random.default_rng(2)
    n, npp = 3 * H.levels[2].n_p2, H.levels[2].n_p1
    f = rng.standard_normal(n)
    g = np.zeros(npp)
    u, p, it, hist = S.solve(f, g, np.zeros(n), np.zeros(npp), rtol=1e-8)
    assert hist[-1] <= 1e-8 * hist[0]
    assert it < 40
    ud, pd = direct_solve(H, f, g, np.zeros(n), np.zeros(npp))
    assert np.linalg.norm(u - ud) / np.linalg.norm(ud) < 1e-5
    assert np.linalg.norm(p - pd) / np.linalg.norm(pd) < 1e-5
    # the direct solution has (near) zero projected residual
    r = S.residual(f, g, ud, pd)
    assert np.linalg.norm(r) <= 1e-10 * np.linalg.norm(S.residual(f, g, 0 * ud, 0 * pd))


@pytest.mark.slow
@pytest.mark.parametrize("uzawa,schur", [("inexact", "vbfbt"), ("adjoint", "vbfbt"), ("symmetric", "mass"),
                                         ("symmetric", "diagbfbt")])
def test_stokes_preconditioner_variants_match_direct(hier2, uzawa, schur):
    """Every block preconditioner / Schur approximation of Sec. 5.2 leaves the solution
    unchanged: FGMRES with it reaches the direct solution (tol_A = 1e-4 for the one-sided
    Uzawa steps, as in the paper's comparison)."""
    H = hier2
    params = dict(uzawa=uzawa, schur=schur)
    if uzawa != "symmetric":
        params["tol_A"] = 1e-4
    S = StokesOracle(H, params)
    rng = np.random.default_rng(2)
    n, npp = 3 * H.levels[2].n_p2, H.levels[2].n_p1
    f = rng.standard_normal(n)
    g = np.zeros(npp)
    u, p, it, hist = S.solve(f, g, np.zeros(n), np.zeros(npp), rtol=1e-8)
    assert hist[-1] <= 1e-8 * hist[0]
    ud, pd = direct_solve(H, f, g, np.zeros(n), np.zeros(npp))
    assert np.linalg.norm(u - ud) / np.linalg.norm(ud) < 1e-5
    assert np.linalg.norm(p - pd) / np.linalg.norm(pd) < 1e-5


@pytest.fixture(scope="module")
def exact_blocks_level1():
    """Level 1 (blended, free-slip CMB, compressible, variable viscosity) with the exact
    inverses of the constrained A and of the Schur complement S = Bbar A^-1 B^T on mean-free
    pressures, for the pins of the Uzawa steps below."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla
    mesh = MacroMesh()
    Lv = Level(mesh, 1)
    eta = W.viscosity_plumes(Lv.p1_x, seed=3, contrast=1e3)
    H = Hierarchy(mesh, 1, eta, dlnrho_table=W.dlnrho_table_compressible(), bounds={})
    co, cons = H.co[1], H.cons[1]
    P0 = cons.Pv_matrix()
    I = sp.identity(P0.shape[0], format="csc")
    lu = spla.splu((P0 @ H.ops[1].A @ P0 + I - P0).tocsc())
    Ainv = lambda r: cons.P0(lu.solve(cons.P0(r)))
    n = Lv.n_p1
    Qp = np.linalg.qr(np.eye(n) - 1.0 / n)[0][:, :n - 1]                  # mean-free basis
    S = np.column_stack([co.apply_Bbar(Ainv(co.apply_BT(q))) for q in Qp.T])
    Sr = Qp.T @ S
    Sinv = lambda r: Qp @ np.linalg.solve(Sr, Qp.T @ r)
    return H, Ainv, Sinv


def _exact_oracle(H, Ainv, Sinv, kind):
    S = StokesOracle(H, dict(uzawa=kind, sigma=1.0, omega=1.0))
    S.Ahat_inv = Ainv
    S.Shat_inv = Sinv
    return S


def _constrained_residual(S, seed):
    rng = np.random.default_rng(seed)
    r = rng.standard_normal(S.nu + S.np)
    return np.concatenate([S.cons.P0(r[:S.nu]), r[S.nu:] - r[S.nu:].mean()])


def test_symmetric_uzawa_with_exact_blocks_is_the_inverse(exact_blocks_level1):
    """Eq. (SymmetricUzawaStep1) with exact A^-1, the exact Schur complement and sigma =
    omega = 1 is the block LDU inverse of the constrained saddle-point operator: K z = r."""
    S = _exact_oracle(*exact_blocks_level1, "symmetric")
    r = _constrained_residual(S, 4)
    z = S.uzawa(r)
    assert np.linalg.norm(S.K(z) - r) <= 1e-9 * np.linalg.norm(r)


@pytest.mark.parametrize("kind", ["inexact", "adjoint"])
def test_one_sided_uzawa_with_exact_blocks_is_nilpotent_of_order_two(exact_blocks_level1, kind):
    """Eqs. (InexactUzawaStep1), (AdjointInexactUzawaStep1) with exact blocks are the block
    lower / upper triangular preconditioners: (K P^-1 - I)^2 = 0, while K P^-1 - I itself is
    not zero (right-preconditioned GMRES converges in two steps)."""
    S = _exact_oracle(*exact_blocks_level1, kind)
    r = _constrained_residual(S, 5)
    E = lambda v: S.K(S.uzawa(v)) - v
    e1 = E(r)
    assert np.linalg.norm(e1) > 1e-3 * np.linalg.norm(r)
    assert np.linalg.norm(E(e1)) <= 1e-9 * np.linalg.norm(r)


def test_bfbt_with_exact_inner_inverse_is_the_exact_schur_inverse(exact_blocks_level1):
    """Eq. (schurV) with the exact A^-1 in place of the cheap V-cycle A_C^-1 collapses to
    X^-1 (B A^-1 A A^-1 B^T) X^-1 = X^-1, X = B A^-1 B^T: the composition's order and the
    middle factor are pinned by agreement with a dense inverse of X on mean-free pressures."""
    H, Ainv, _ = exact_blocks_level1
    S = StokesOracle(H, dict(tol_VBFBT=1e-13))
    n = H.levels[1].n_p1
    Qp = np.linalg.qr(np.eye(n) - 1.0 / n)[0][:, :n - 1]
    X = Qp.T @ np.column_stack([S.co.apply_B(Ainv(S.co.apply_BT(q))) for q in Qp.T])
    r = np.random.default_rng(6).standard_normal(n)
    r -= r.mean()
    ref = Qp @ np.linalg.solve(X, Qp.T @ r)
    got = S.bfbt(r, Ainv)
    assert np.linalg.norm(got - ref) <= 1e-8 * np.linalg.norm(ref)
    # with the cheap V-cycle it is only an approximation
    cheap = S.bfbt(r, S.Ac_inv)
    assert np.linalg.norm(cheap - ref) > 1e-3 * np.linalg.norm(ref)


def test_viscosity_full_weighting_constants_and_linear_fields():
    """The coarse-level viscosity (P1 full weighting, normalised): constants are kept on
    every vertex, and a field linear in the straight coordinates is kept on the vertices
    inside a macro-tet, where the Freudenthal stencil of coarse edges is centrally symmetric
    (the last 60 (N-1)(N-2)(N-3)/6 vertices of the numbering)."""
    from oracle.solver import restrict_viscosity
    mesh = MacroMesh()
    Lf, Lc = Level(mesh, 3), Level(mesh, 2)
    assert np.abs(restrict_viscosity(Lf, Lc, np.full(Lf.n_p1, 7.5)) - 7.5).max() <= 1e-14
    a = np.array([0.3, -1.2, 0.7])
    f = lambda X: 2.0 + X @ a
    got = restrict_viscosity(Lf, Lc, f(Lf.p1_straight))
    N = 4
    n_ci = 60 * (N - 1) * (N - 2) * (N - 3) // 6
    inner = slice(Lc.n_p1 - n_ci, Lc.n_p1)
    assert np.abs(got[inner] - f(Lc.p1_straight)[inner]).max() <= 1e-13
    # on the macro boundaries the stencil is not symmetric: there the weighting smooths
    assert np.abs(got - f(Lc.p1_straight)).max() > 1e-6


def test_power_iteration_estimate_of_the_chebyshev_interval():
    """The Chebyshev upper bound's estimate (15 power iterations on D^-1 A from the seeded
    vector): on D^-1 A = diag(lambda) with a known spectrum the estimate approaches the largest
    eigenvalue from below, within the power method's (lambda_2/lambda_1)^k rate, and the
    projection keeps the projected-out directions out of it."""
    from oracle.solver import power_max_eig
    lam = np.concatenate([np.linspace(0.01, 1.6, 60), [1.8, 2.0]])
    est = power_max_eig(lambda v: lam * v, np.ones(lam.size), lambda v: v, lam.size)
    assert 1.8 < est <= 2.0 + 1e-12
    assert 2.0 - est < 2.0 * (1.8 / 2.0) ** 14
    # a projection that removes the top eigenvector leaves the next one as the estimate
    proj = lambda v: np.concatenate([v[:-1], [0.0]])
    est2 = power_max_eig(lambda v: lam * v, np.ones(lam.size), proj, lam.size)
    assert 1.6 < est2 <= 1.8 + 1e-12
