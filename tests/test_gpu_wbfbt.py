"""GPU parity of the weighted BFBT Schur approximation (Sec. 5.2.3, Eq. schurWBFBT, rescaled
form) against the oracle: the K_{1/sqrt(eta)} apply on every multigrid level, the lumped
M_{sqrt(eta)}, one application of S_w^-1 (exact K solves in the oracle, CG with the GPU's own
K V-cycle to a tight tolerance on the GPU), and Stokes solves with it."""
import functools

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2506_04157_gb300 as mfs
import workloads as W
from oracle.mesh import MacroMesh, Level
from oracle.fem import project_mean_zero
from oracle.solver import Hierarchy, direct_solve, StokesOracle
from oracle.wbfbt import WbfbtOperators, wbfbt_apply

TOL = {torch.float64: 1e-12, torch.float32: 1e-5}


@functools.lru_cache(maxsize=None)
def setup(L):
    mesh = MacroMesh()
    Lf = Level(mesh, L)
    eta = W.viscosity_plumes(Lf.p1_x, seed=7, contrast=1e4)
    # Chebyshev intervals are not compared here: dummy ones spare the oracle's power iterations
    H = Hierarchy(mesh, L, eta, dlnrho_table=W.dlnrho_table_compressible(),
                  bounds={l: (0.1, 2.0) for l in range(2, L + 1)})
    ctx = mfs.Context(0)
    gm = mfs.Mesh(ctx, L)
    prob = mfs.Problem(gm, "dirichlet", "freeslip")
    prob.set_viscosity(torch.tensor(eta, device="cuda"))
    prob.set_density(W.dlnrho_table_compressible())
    prob.setup_multigrid(1)
    return H, ctx, gm, prob


@functools.lru_cache(maxsize=None)
def oracle_ops(L, l, a):
    H = setup(L)[0]
    return WbfbtOperators(H.levels[l], H.etas[l], a)


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("dt", [torch.float64, torch.float32])
@pytest.mark.parametrize("a", [1.0, 3.0])
def test_poisson_apply_every_level(a, dt):
    H, ctx, gm, prob = setup(3)
    for l in range(1, 4):
        n = H.levels[l].n_p1
        p = W.random_field(n, 10 + l)
        if dt == torch.float32:
            p = p.astype(np.float32).astype(np.float64)
        y = torch.empty(n, dtype=dt, device="cuda")
        prob.apply_poisson(l, a, torch.tensor(p, dtype=dt, device="cuda"), y)
        ref = oracle_ops(3, l, a).K @ p
        assert rel(y.double().cpu().numpy(), ref) <= TOL[dt], (l, a)


def test_poisson_constants_in_kernel():
    """The stored off-diagonal form makes K 1 = 0 up to the atomics' rounding."""
    H, ctx, gm, prob = setup(3)
    n = H.levels[3].n_p1
    for dt, tol in [(torch.float64, 1e-13), (torch.float32, 1e-5)]:
        y = torch.empty(n, dtype=dt, device="cuda")
        prob.apply_poisson(3, 1.0, torch.ones(n, dtype=dt, device="cuda"), y)
        p = torch.tensor(W.random_field(n, 5), dtype=dt, device="cuda")
        yp = torch.empty(n, dtype=dt, device="cuda")
        prob.apply_poisson(3, 1.0, p, yp)
        assert y.abs().max().item() <= tol * yp.abs().max().item()


@pytest.mark.parametrize("L", [2, 3])
@pytest.mark.parametrize("a", [1.0, 2.0])
def test_lumped_mass(L, a):
    H, ctx, gm, prob = setup(L)
    d = torch.empty(H.levels[L].n_p2, dtype=torch.float64, device="cuda")
    prob.lumped_vmass(a, d)
    assert rel(d.cpu().numpy(), oracle_ops(L, L, a).d) <= 1e-12


@pytest.mark.parametrize("L", [2, 3])
@pytest.mark.parametrize("al,ar", [(1.0, 1.0), (1.0, 10.0)])
def test_wbfbt_apply_fp64(L, al, ar):
    """S_w^-1 r with the K solves converged far below the oracle's exact solves."""
    H, ctx, gm, prob = setup(L)
    n = H.levels[L].n_p1
    r = project_mean_zero(W.random_field(n, 21))
    z = torch.empty(n, dtype=torch.float64, device="cuda")
    st = prob.apply_schur(torch.tensor(r, device="cuda"), z, schur=3, a_l=al, a_r=ar, tol_wBFBT=1e-13,
                          max_cg=400, vmass=0)
    wl, wr = oracle_ops(L, L, al), oracle_ops(L, L, ar)
    ref = project_mean_zero(wbfbt_apply(H.co[L], H.cons[L], H.co[L].apply_A, wl, wr, r))
    assert rel(z.cpu().numpy(), ref) <= 1e-8, st
    assert st["cg_X_calls"] == 2 and st["cg_X_max"] < 400


def test_wbfbt_apply_fp32():
    """FP32: each K solve stops at relative residual 1e-5 (the FP32 floor of tol_wBFBT)."""
    H, ctx, gm, prob = setup(3)
    n = H.levels[3].n_p1
    r = project_mean_zero(W.random_field(n, 22)).astype(np.float32)
    z = torch.empty(n, dtype=torch.float32, device="cuda")
    prob.apply_schur(torch.tensor(r, device="cuda"), z, schur=3, vmass=0)
    wl = oracle_ops(3, 3, 1.0)
    ref = project_mean_zero(wbfbt_apply(H.co[3], H.cons[3], H.co[3].apply_A, wl, wl, r.astype(np.float64)))
    assert rel(z.double().cpu().numpy(), ref) <= 1e-2


def test_schur_apply_mass_matches_oracle():
    """The same entry point for the mass approximation (Eq. schurMass): M_{1/eta}^-1 r."""
    H, ctx, gm, prob = setup(2)
    n = H.levels[2].n_p1
    r = project_mean_zero(W.random_field(n, 23))
    z = torch.empty(n, dtype=torch.float64, device="cuda")
    prob.apply_schur(torch.tensor(r, device="cuda"), z, schur=1, tol_invMass=1e-13, max_cg=500)
    # the mean-free x with P_p M x = r (the library's CG works on P_p M P_p): lifting the
    # constants, (P_p M P_p + 1 1^T / n) x = r
    M = H.ops[2].M_inv_eta.toarray()
    Pm = np.eye(n) - 1.0 / n
    ref = project_mean_zero(np.linalg.solve(Pm @ M @ Pm + np.ones((n, n)) / n, r))
    assert rel(z.cpu().numpy(), ref) <= 1e-8


def test_schur_refusals():
    H, ctx, gm, prob = setup(2)
    n = H.levels[2].n_p1
    r = torch.zeros(n, dtype=torch.float64, device="cuda")
    z = torch.empty(n, dtype=torch.float64, device="cuda")
    for bad in [dict(schur=4), dict(schur=3, a_l=0.0), dict(schur=3, a_r=-1.0), dict(schur=3, tol_wBFBT=0.0)]:
        with pytest.raises(mfs.MfsError):
            prob.apply_schur(r, z, **bad)
    n0 = gm.info(0).n_p1   # level 0 lies below the multigrid range (l_min = 1)
    with pytest.raises(mfs.MfsError):
        prob.apply_poisson(0, 1.0, torch.zeros(n0, dtype=torch.float64, device="cuda"),
                           torch.zeros(n0, dtype=torch.float64, device="cuda"))


@pytest.mark.parametrize("mixed", [2, 0])
@pytest.mark.parametrize("al", [1.0, 3.0])
def test_solve_with_wbfbt(mixed, al):
    """FGMRES with the symmetric Uzawa step and the weighted BFBT on the lumped vector mass
    (symmetric and asymmetric surface scaling) reaches the oracle's direct solution (omega =
    0.03: the lumped approximation's spectrum reaches ~20-80 here).  Solved to 1e-10: with the contrast-1e4 plumes and a
    rough forcing, a 1e-8 residual leaves a pressure error of ~5e-5."""
    H, ctx, gm, prob = setup(2)
    S = StokesOracle(H)
    L = H.levels[2]
    rng = np.random.default_rng(31)
    f = rng.standard_normal(3 * L.n_p2) * 1e-3
    g = np.zeros(L.n_p1)
    u = torch.zeros(3 * L.n_p2, dtype=torch.float64, device="cuda")
    p = torch.zeros(L.n_p1, dtype=torch.float64, device="cuda")
    st = prob.solve(torch.tensor(f, device="cuda"), torch.tensor(g, device="cuda"), u, p, mixed=mixed, schur=3,
                    a_l=al, omega=0.03, restart=50, max_iters=1500, rtol=1e-10, vmass=0)
    assert st["status"] == "MFS_OK" and st["rel_residual"] <= 1e-10, st
    un, pn = u.cpu().numpy(), p.cpu().numpy()
    r0 = np.linalg.norm(S.residual(f, g, 0 * un, 0 * pn))
    assert np.linalg.norm(S.residual(f, g, un, pn)) <= 1.5e-10 * r0
    ud, pd = direct_solve(H, f, g, 0 * un, 0 * pn)
    assert np.linalg.norm(un - ud) / np.linalg.norm(ud) < 1e-5
    assert np.linalg.norm(pn - pd) / np.linalg.norm(pd) < 1e-5


# ---- the consistent vector mass (vmass = 1)


@functools.lru_cache(maxsize=None)
def oracle_cmass(L, a):
    H = setup(L)[0]
    return WbfbtOperators(H.levels[L], H.etas[L], a, mass="consistent")


@pytest.mark.parametrize("dt", [torch.float64, torch.float32])
@pytest.mark.parametrize("L,a", [(2, 1.0), (2, 3.0), (3, 2.0)])
def test_consistent_vmass_apply(L, a, dt):
    """y_c = M_{sqrt(eta_a)} x_c on each component against the oracle's assembled matrix."""
    H, ctx, gm, prob = setup(L)
    n2 = H.levels[L].n_p2
    x = W.random_field(3 * n2, 40 + L)
    if dt == torch.float32:
        x = x.astype(np.float32).astype(np.float64)
    y = torch.empty(3 * n2, dtype=dt, device="cuda")
    prob.apply_vmass(a, torch.tensor(x, dtype=dt, device="cuda"), y)
    Mc = oracle_cmass(L, a).Mc
    ref = np.concatenate([Mc @ x[c * n2:(c + 1) * n2] for c in range(3)])
    assert rel(y.double().cpu().numpy(), ref) <= TOL[dt], (L, a)


@pytest.mark.parametrize("al,ar", [(1.0, 1.0), (1.0, 10.0)])
def test_wbfbt_consistent_apply_fp64(al, ar):
    """S_w^-1 r with the consistent mass: the GPU's CGs on K and on M converged far below the
    oracle's exact solves."""
    L = 2
    H, ctx, gm, prob = setup(L)
    n = H.levels[L].n_p1
    r = project_mean_zero(W.random_field(n, 24))
    z = torch.empty(n, dtype=torch.float64, device="cuda")
    st = prob.apply_schur(torch.tensor(r, device="cuda"), z, schur=3, a_l=al, a_r=ar, tol_wBFBT=1e-13,
                          vmass=1, tol_VectorMass=1e-13, max_cg=400)
    wl, wr = oracle_cmass(L, al), oracle_cmass(L, ar)
    ref = project_mean_zero(wbfbt_apply(H.co[L], H.cons[L], H.co[L].apply_A, wl, wr, r))
    assert rel(z.cpu().numpy(), ref) <= 1e-8, st
    assert st["cg_M_calls"] == 2 and 0 < st["cg_M_max"] < 400


def test_solve_with_wbfbt_consistent_mass():
    """FGMRES with the weighted BFBT on the consistent mass (the paper's tol_VectorMass = 1e-4)
    and the default omega = 0.3 (the best scaling with this mass) reaches the oracle's direct
    solution."""
    H, ctx, gm, prob = setup(2)
    L = H.levels[2]
    rng = np.random.default_rng(32)
    f = rng.standard_normal(3 * L.n_p2) * 1e-3
    g = np.zeros(L.n_p1)
    u = torch.zeros(3 * L.n_p2, dtype=torch.float64, device="cuda")
    p = torch.zeros(L.n_p1, dtype=torch.float64, device="cuda")
    st = prob.solve(torch.tensor(f, device="cuda"), torch.tensor(g, device="cuda"), u, p, mixed=2, schur=3,
                    vmass=1, restart=50, max_iters=1500, rtol=1e-10)
    assert st["status"] == "MFS_OK" and st["rel_residual"] <= 1e-10, st
    ud, pd = direct_solve(H, f, g, 0 * f, 0 * g)
    assert np.linalg.norm(u.cpu().numpy() - ud) / np.linalg.norm(ud) < 1e-5
    assert np.linalg.norm(p.cpu().numpy() - pd) / np.linalg.norm(pd) < 1e-5


def test_vmass_refusals():
    H, ctx, gm, prob = setup(2)
    n = H.levels[2].n_p1
    r = torch.zeros(n, dtype=torch.float64, device="cuda")
    z = torch.empty(n, dtype=torch.float64, device="cuda")
    for bad in [dict(schur=3, vmass=2), dict(schur=3, vmass=1, tol_VectorMass=0.0)]:
        with pytest.raises(mfs.MfsError):
            prob.apply_schur(r, z, **bad)
    x = torch.zeros(3 * H.levels[2].n_p2, dtype=torch.float64, device="cuda")
    with pytest.raises(mfs.MfsError):
        prob.apply_vmass(0.0, x, torch.empty_like(x))
    with pytest.raises(mfs.MfsError):
        prob.apply_vmass(1.0, x, x)
