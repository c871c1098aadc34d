"""GPU Stokes solves (mixed FP32 + FP64 refinement, FP64 FGMRES with the FP32 preconditioner,
and plain FP64) against the oracle:
the oracle's own FP64 evaluation of the projected residual of the GPU iterate, and the
oracle's direct solution of the projected system."""
import functools

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2506_04157_gb300 as mfs
import workloads as W
from oracle.mesh import MacroMesh, Level
from oracle.solver import Hierarchy, StokesOracle, direct_solve


@functools.lru_cache(maxsize=None)
def setup(L, bc=("dirichlet", "freeslip"), visc="radial"):
    mesh = MacroMesh()
    Lf = Level(mesh, L)
    eta = W.viscosity_radial(Lf.p1_x) if visc == "radial" else W.viscosity_plumes(Lf.p1_x, 2, 1e4)
    bcm = {"dirichlet": 0, "freeslip": 1}
    H = Hierarchy(mesh, L, eta, dlnrho_table=W.dlnrho_table_config1(), bc=(bcm[bc[0]], bcm[bc[1]]))
    S = StokesOracle(H)
    ctx = mfs.Context(0)
    gm = mfs.Mesh(ctx, L)
    prob = mfs.Problem(gm, *bc)
    prob.set_viscosity(torch.tensor(eta, device="cuda"))
    prob.set_density(W.dlnrho_table_config1())
    prob.setup_multigrid(1)
    return H, S, ctx, gm, prob


def rhs(L, seed=3):
    T = W.temperature_blobs(L.p2_x, seed)
    # a smooth radial body force f = T x/|x| at the nodes (load-vector sized), g = 0
    xh = L.p2_x / np.linalg.norm(L.p2_x, axis=1, keepdims=True)
    f = np.concatenate([T * xh[:, 0], T * xh[:, 1], T * xh[:, 2]]) * 1e-3
    return f, np.zeros(L.n_p1)


@pytest.mark.parametrize("mixed", [1, 2, 0])
@pytest.mark.parametrize("bc", [("dirichlet", "freeslip"), ("freeslip", "dirichlet")])
def test_solve_level2(mixed, bc):
    H, S, ctx, gm, prob = setup(2, bc)
    L = H.levels[2]
    f, g = rhs(L)
    u = torch.zeros(3 * L.n_p2, dtype=torch.float64, device="cuda")
    p = torch.zeros(L.n_p1, dtype=torch.float64, device="cuda")
    st = prob.solve(torch.tensor(f, device="cuda"), torch.tensor(g, device="cuda"), u, p, mixed=mixed)
    assert st["status"] == "MFS_OK" and st["rel_residual"] <= 1e-8
    un, pn = u.cpu().numpy(), p.cpu().numpy()
    r0 = np.linalg.norm(S.residual(f, g, 0 * un, 0 * pn))
    r = np.linalg.norm(S.residual(f, g, un, pn))
    assert r <= 1.5e-8 * r0, (r / r0, st)
    ud, pd = direct_solve(H, f, g, 0 * un, 0 * pn)
    assert np.linalg.norm(un - ud) / np.linalg.norm(ud) < 1e-5
    assert np.linalg.norm(pn - pd) / np.linalg.norm(pd) < 1e-5
    assert abs(pn.mean()) < 1e-12 * np.abs(pn).max()


def test_solve_dirichlet_lifting():
    """Non-zero surface velocities (a rigid rotation, tangential) are kept and lifted."""
    H, S, ctx, gm, prob = setup(2)
    L = H.levels[2]
    f, g = rhs(L, 5)
    x = L.p2_x
    w = np.array([0.3, -0.2, 0.5])
    rot = np.cross(w, x)
    u0 = np.zeros(3 * L.n_p2)
    surf = L.p2_class == 1
    for c in range(3):
        u0[c * L.n_p2:(c + 1) * L.n_p2][surf] = rot[surf, c]
    u = torch.tensor(u0, device="cuda")
    p = torch.zeros(L.n_p1, dtype=torch.float64, device="cuda")
    st = prob.solve(torch.tensor(f, device="cuda"), torch.tensor(g, device="cuda"), u, p)
    un, pn = u.cpu().numpy(), p.cpu().numpy()
    for c in range(3):
        assert np.array_equal(un[c * L.n_p2:(c + 1) * L.n_p2][surf], u0[c * L.n_p2:(c + 1) * L.n_p2][surf])
    ud, pd = direct_solve(H, f, g, u0, np.zeros(L.n_p1))
    assert np.linalg.norm(un - ud) / np.linalg.norm(ud) < 1e-5
    r0 = np.linalg.norm(S.residual(f, g, u0, 0 * pn))
    assert np.linalg.norm(S.residual(f, g, un, pn)) <= 1.5e-8 * r0


def test_solve_level3_plumes_mixed_vs_fp64():
    H, S, ctx, gm, prob = setup(3, visc="plumes")
    L = H.levels[3]
    f, g = rhs(L, 7)
    sols = {}
    for mixed in (1, 2, 0):
        u = torch.zeros(3 * L.n_p2, dtype=torch.float64, device="cuda")
        p = torch.zeros(L.n_p1, dtype=torch.float64, device="cuda")
        st = prob.solve(torch.tensor(f, device="cuda"), torch.tensor(g, device="cuda"), u, p, mixed=mixed)
        assert st["rel_residual"] <= 1e-8
        un, pn = u.cpu().numpy(), p.cpu().numpy()
        r0 = np.linalg.norm(S.residual(f, g, 0 * un, 0 * pn))
        assert np.linalg.norm(S.residual(f, g, un, pn)) <= 1.5e-8 * r0
        sols[mixed] = (un, pn)
    assert np.linalg.norm(sols[1][0] - sols[0][0]) / np.linalg.norm(sols[0][0]) < 1e-5
    assert np.linalg.norm(sols[2][0] - sols[0][0]) / np.linalg.norm(sols[0][0]) < 1e-5


@pytest.mark.parametrize("uzawa,schur", [(1, 0), (2, 0), (0, 1), (0, 2)])
def test_solve_preconditioner_variants(uzawa, schur):
    """The inexact and adjoint inexact Uzawa steps and the mass and diag(A)-BFBT Schur
    approximations (Sec. 5.2.1, 5.2.3) reach the same solution as the oracle's direct solve
    (tol_A = 1e-4 for the one-sided Uzawa steps, as in the paper's comparison)."""
    H, S, ctx, gm, prob = setup(2)
    L = H.levels[2]
    f, g = rhs(L, 9)
    u = torch.zeros(3 * L.n_p2, dtype=torch.float64, device="cuda")
    p = torch.zeros(L.n_p1, dtype=torch.float64, device="cuda")
    opts = dict(uzawa=uzawa, schur=schur)
    if uzawa:
        opts["tol_A"] = 1e-4
    st = prob.solve(torch.tensor(f, device="cuda"), torch.tensor(g, device="cuda"), u, p, **opts)
    assert st["status"] == "MFS_OK" and st["rel_residual"] <= 1e-8
    un, pn = u.cpu().numpy(), p.cpu().numpy()
    r0 = np.linalg.norm(S.residual(f, g, 0 * un, 0 * pn))
    assert np.linalg.norm(S.residual(f, g, un, pn)) <= 1.5e-8 * r0
    ud, pd = direct_solve(H, f, g, 0 * un, 0 * pn)
    assert np.linalg.norm(un - ud) / np.linalg.norm(ud) < 1e-5
    assert np.linalg.norm(pn - pd) / np.linalg.norm(pd) < 1e-5
