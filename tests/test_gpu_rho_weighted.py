"""The density-weighted constraint -int q div(rho u) (mfs_set_constraint_form(prob, 1)) on the
GPU against the oracle (oracle.fem.element_B_rho, Operators(rho_weighted=True)): the raw and
constrained constraint block and its transpose, the fused apply and its transpose, and solves
that reach the oracle's direct solution of the system with this constraint."""
import functools

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2506_04157_gb300 as mfs
import workloads as W
from oracle.mesh import MacroMesh, Level
from oracle.fem import Operators, Constraints, ConstrainedOperators
from oracle.solver import Hierarchy, StokesOracle, direct_solve, viscosity_hierarchy

TOL = {torch.float64: 1e-12, torch.float32: 1e-5}
TABLES = {"compressible": tuple(W.dlnrho_table_compressible()), "graded": (-0.8, -0.2, 0.4)}


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@functools.lru_cache(maxsize=None)
def oracle(l, table):
    mesh = MacroMesh()
    Ls = {k: Level(mesh, k) for k in range(l + 1)}
    etas = viscosity_hierarchy(mesh, Ls, W.viscosity_plumes(Ls[l].p1_x, 7, 1e4))
    ops = Operators(Ls[l], etas[l], dlnrho_table=TABLES[table], rho_weighted=True)
    return Ls[l], ops, ConstrainedOperators(ops, Constraints(Ls[l], 0, 1)), etas[l]


@pytest.mark.parametrize("table", ["compressible", "graded"])
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("l", [1, 2, 3])
def test_density_weighted_blocks(l, dtype, table):
    L, ops, co, eta = oracle(l, table)
    ctx = mfs.Context(0)
    mesh = mfs.Mesh(ctx, l)
    prob = mfs.Problem(mesh, "dirichlet", "freeslip")
    prob.set_viscosity(torch.tensor(eta, device="cuda"))
    prob.set_density(np.array(TABLES[table]))
    prob.set_constraint_form(True)
    u = W.random_field(3 * L.n_p2, 61)
    p = W.random_field(L.n_p1, 62)
    if dtype == torch.float32:
        u = u.astype(np.float32).astype(np.float64)
        p = p.astype(np.float32).astype(np.float64)
    ud = torch.tensor(u, dtype=dtype, device="cuda")
    pd = torch.tensor(p, dtype=dtype, device="cuda")
    yu = torch.empty(3 * L.n_p2, dtype=dtype, device="cuda")
    yp = torch.empty(L.n_p1, dtype=dtype, device="cuda")
    get = lambda t: t.double().cpu().numpy()
    prob.apply_B(l, ud, yp, with_C=True)
    assert rel(get(yp), (ops.B + ops.C) @ u) <= TOL[dtype]
    prob.apply_B(l, ud, yp, with_C=False)          # the plain B is unchanged
    assert rel(get(yp), ops.B @ u) <= TOL[dtype]
    prob.apply_BT(l, pd, yu, with_C=True)
    assert rel(get(yu), (ops.B + ops.C).T @ p) <= TOL[dtype]
    prob.apply_B(l, ud, yp, with_C=True, constrained=True)
    assert rel(get(yp), co.apply_Bbar(u)) <= TOL[dtype]
    prob.apply_stokes(l, ud, pd, yu, yp)
    assert rel(get(yu), co.apply_A(u) + co.apply_BT(p)) <= TOL[dtype]
    assert rel(get(yp), co.apply_Bbar(u)) <= TOL[dtype]
    prob.apply_stokes(l, ud, pd, yu, yp, transpose=True)
    assert rel(get(yu), co.apply_A(u) + co.apply_BbarT(p)) <= TOL[dtype]
    assert rel(get(yp), co.apply_B(u)) <= TOL[dtype]
    # the default form is the paper's B + C again
    prob.set_constraint_form(False)
    prob.apply_B(l, ud, yp, with_C=True)
    ref = Operators(L, eta, dlnrho_table=TABLES[table])
    assert rel(get(yp), (ref.B + ref.C) @ u) <= TOL[dtype]


@pytest.mark.parametrize("mixed", [1, 2, 0])
def test_density_weighted_solve(mixed):
    """FGMRES with the symmetric Uzawa / V-cycle BFBT preconditioner on the system with the
    density-weighted constraint reaches the oracle's direct solution of that system."""
    mesh = MacroMesh()
    Lf = Level(mesh, 2)
    eta = W.viscosity_radial(Lf.p1_x)
    table = np.array([-0.8, -0.2, 0.4])
    H = Hierarchy(mesh, 2, eta, dlnrho_table=table, bc=(0, 1), rho_weighted=True)
    S = StokesOracle(H)
    ctx = mfs.Context(0)
    gm = mfs.Mesh(ctx, 2)
    prob = mfs.Problem(gm, "dirichlet", "freeslip")
    prob.set_viscosity(torch.tensor(eta, device="cuda"))
    prob.set_density(table)
    prob.set_constraint_form(True)
    prob.setup_multigrid(1)
    T = W.temperature_blobs(Lf.p2_x, 3)
    xh = Lf.p2_x / np.linalg.norm(Lf.p2_x, axis=1, keepdims=True)
    f = np.concatenate([T * xh[:, 0], T * xh[:, 1], T * xh[:, 2]]) * 1e-3
    g = np.zeros(Lf.n_p1)
    u = torch.zeros(3 * Lf.n_p2, dtype=torch.float64, device="cuda")
    p = torch.zeros(Lf.n_p1, dtype=torch.float64, device="cuda")
    st = prob.solve(torch.tensor(f, device="cuda"), torch.tensor(g, device="cuda"), u, p, mixed=mixed)
    assert st["status"] == "MFS_OK" and st["rel_residual"] <= 1e-8
    un, pn = u.cpu().numpy(), p.cpu().numpy()
    r0 = np.linalg.norm(S.residual(f, g, 0 * un, 0 * pn))
    assert np.linalg.norm(S.residual(f, g, un, pn)) <= 1.5e-8 * r0
    ud, pdd = direct_solve(H, f, g, 0 * un, 0 * pn)
    assert np.linalg.norm(un - ud) / np.linalg.norm(ud) < 1e-5
    assert np.linalg.norm(pn - pdd) / np.linalg.norm(pdd) < 1e-5


def test_batch_refuses_density_weighted_members():
    ctx = mfs.Context(0)
    gm = mfs.Mesh(ctx, 2)
    prob = mfs.Problem(gm)
    prob.set_viscosity(torch.ones(gm.info(2).n_p1, dtype=torch.float64, device="cuda"))
    prob.set_constraint_form(True)
    with pytest.raises(mfs.MfsError):
        mfs.Batch(ctx, [prob])
