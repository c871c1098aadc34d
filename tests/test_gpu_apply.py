"""GPU parity of the operator applies against the oracle (norm-wise relative error:
FP64 <= 1e-12, FP32 <= 1e-5 against the oracle evaluated on the FP32-rounded inputs)."""
import functools

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2506_04157_gb300 as mfs
import workloads as W
from oracle.mesh import MacroMesh, Level
from oracle.fem import Operators, Constraints, ConstrainedOperators, project_mean_zero
from oracle.solver import viscosity_hierarchy

TOL = {torch.float64: 1e-12, torch.float32: 1e-5}
DLNRHO = W.dlnrho_table_config1()


@functools.lru_cache(maxsize=None)
def levels(blending, l_max=3):
    """Oracle levels 0..l_max and eta on each: the formula on the finest level, P1 full
    weighting below (the library's coarse-level viscosity)."""
    mesh = MacroMesh(blending=blending)
    Ls = {l: Level(mesh, l) for l in range(l_max + 1)}
    return mesh, Ls, viscosity_hierarchy(mesh, Ls, W.viscosity_radial(Ls[l_max].p1_x))


@functools.lru_cache(maxsize=None)
def oracle(l, blending, bc=("dirichlet", "freeslip")):
    mesh, Ls, etas = levels(blending)
    L = Ls[l]
    ops = Operators(L, etas[l], dlnrho_table=DLNRHO)
    bcmap = {"dirichlet": 0, "freeslip": 1}
    cons = Constraints(L, bcmap[bc[0]], bcmap[bc[1]])
    return L, ops, ConstrainedOperators(ops, cons)


@functools.lru_cache(maxsize=None)
def gpu_problem(l_max, blending, bc=("dirichlet", "freeslip")):
    ctx = mfs.Context(0)
    mesh = mfs.Mesh(ctx, l_max, blending=blending)
    prob = mfs.Problem(mesh, *bc)
    x = mesh.coords(l_max, p2=False).T
    prob.set_viscosity(torch.tensor(W.viscosity_radial(x), device="cuda"))
    prob.set_density(DLNRHO)
    return ctx, mesh, prob


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def inputs(L, dtype, seed=1):
    u = W.random_field(3 * L.n_p2, seed)
    p = W.random_field(L.n_p1, seed + 1)
    if dtype == torch.float32:
        u = u.astype(np.float32).astype(np.float64)
        p = p.astype(np.float32).astype(np.float64)
    return u, p


def dev(x, dtype):
    return torch.tensor(x, dtype=dtype, device="cuda")


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("blending", [True, False])
@pytest.mark.parametrize("l", [0, 1, 2, 3])
def test_raw_blocks(l, blending, dtype):
    L, ops, _ = oracle(l, blending)
    _, _, prob = gpu_problem(3, blending)
    u, p = inputs(L, dtype)
    ud, pd = dev(u, dtype), dev(p, dtype)
    yu = torch.empty(3 * L.n_p2, dtype=dtype, device="cuda")
    yp = torch.empty(L.n_p1, dtype=dtype, device="cuda")
    prob.apply_A(l, ud, yu)
    assert rel(yu.cpu().double().numpy(), ops.A @ u) <= TOL[dtype]
    prob.apply_B(l, ud, yp, with_C=False)
    assert rel(yp.cpu().double().numpy(), ops.B @ u) <= TOL[dtype]
    prob.apply_B(l, ud, yp, with_C=True)
    assert rel(yp.cpu().double().numpy(), (ops.B + ops.C) @ u) <= TOL[dtype]
    prob.apply_BT(l, pd, yu, with_C=False)
    assert rel(yu.cpu().double().numpy(), ops.B.T @ p) <= TOL[dtype]
    prob.apply_BT(l, pd, yu, with_C=True)
    assert rel(yu.cpu().double().numpy(), (ops.B + ops.C).T @ p) <= TOL[dtype]


@pytest.mark.parametrize("bc", [("dirichlet", "freeslip"), ("freeslip", "dirichlet")])
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("l", [1, 2, 3])
def test_constrained_and_fused(l, dtype, bc):
    L, ops, co = oracle(l, True, bc)
    _, _, prob = gpu_problem(3, True, bc)
    u, p = inputs(L, dtype, seed=5)
    ud, pd = dev(u, dtype), dev(p, dtype)
    yu = torch.empty(3 * L.n_p2, dtype=dtype, device="cuda")
    yp = torch.empty(L.n_p1, dtype=dtype, device="cuda")
    prob.apply_A(l, ud, yu, constrained=True)
    assert rel(yu.cpu().double().numpy(), co.apply_A(u)) <= TOL[dtype]
    prob.apply_B(l, ud, yp, with_C=True, constrained=True)
    assert rel(yp.cpu().double().numpy(), co.apply_Bbar(u)) <= TOL[dtype]
    prob.apply_BT(l, pd, yu, constrained=True)
    assert rel(yu.cpu().double().numpy(), co.apply_BT(p)) <= TOL[dtype]
    # fused [A B^T; (B+C) 0] and its transpose [A (B+C)^T; B 0]
    prob.apply_stokes(l, ud, pd, yu, yp)
    assert rel(yu.cpu().double().numpy(), co.apply_A(u) + co.apply_BT(p)) <= TOL[dtype]
    assert rel(yp.cpu().double().numpy(), co.apply_Bbar(u)) <= TOL[dtype]
    prob.apply_stokes(l, ud, pd, yu, yp, transpose=True)
    assert rel(yu.cpu().double().numpy(), co.apply_A(u) + co.apply_BbarT(p)) <= TOL[dtype]
    assert rel(yp.cpu().double().numpy(), co.apply_B(u)) <= TOL[dtype]


def test_fused_apply_level5_sampled_rows():
    """The bench's workload and launch at full size: level 5 (1,966,080 micro-tets), plume
    viscosity of contrast 1e6 (seed 2), compressible density, the constrained fused apply in
    FP32 and FP64.  The oracle evaluates sampled rows one by one from every micro-tet that
    touches 256 interior P2 nodes and 128 P1 vertices, on the projected inputs: interior
    velocity rows equal A P0 u + B^T P_p p; pressure rows equal (B+C) P0 u up to the one
    constant that P_p removes from the whole output."""
    from oracle.fem import stokes_apply_elements, tets_touching
    lvl = 5
    L = Level(MacroMesh(), lvl)
    dl = W.dlnrho_table_compressible()
    eta = W.viscosity_plumes(L.p1_x, seed=2, contrast=1e6)
    ctx = mfs.Context(0)
    gm = mfs.Mesh(ctx, lvl)
    prob = mfs.Problem(gm, "dirichlet", "freeslip")
    prob.set_viscosity(torch.tensor(eta, device="cuda"))
    prob.set_density(dl)
    rng = np.random.default_rng(11)
    s2 = np.sort(rng.choice(np.flatnonzero(L.p2_class == 0), 256, replace=False))
    s1 = np.sort(rng.choice(L.n_p1, 128, replace=False))
    sel = tets_touching(L, p2_nodes=s2, p1_nodes=s1)
    cons = Constraints(L, 0, 1)
    rows = np.concatenate([s2, s2 + L.n_p2, s2 + 2 * L.n_p2])
    for dtype in (torch.float32, torch.float64):
        u, p = inputs(L, dtype, seed=21)
        yu_ref, yp_ref = stokes_apply_elements(L, eta, dl, cons.P0(u), p - p.mean(), sel)
        yu = torch.empty(3 * L.n_p2, dtype=dtype, device="cuda")
        yp = torch.empty(L.n_p1, dtype=dtype, device="cuda")
        prob.apply_stokes(lvl, dev(u, dtype), dev(p, dtype), yu, yp)
        yu = yu.cpu().double().numpy()
        yp = yp.cpu().double().numpy()
        assert rel(yu[rows], yu_ref[rows]) <= TOL[dtype]
        d = yp[s1] - yp_ref[s1]
        assert np.linalg.norm(d - d.mean()) <= TOL[dtype] * np.linalg.norm(yp_ref[s1])

