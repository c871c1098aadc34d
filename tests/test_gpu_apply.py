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
DEFAULT_VARIANT = 8   # the library's default sweep variant (include/mfs.h)
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


@pytest.mark.parametrize("variant", [0, 1, 2, 3, 4, 5, 6, 7, 8])
@pytest.mark.parametrize("blending", [True, False])
def test_sweep_variants(variant, blending):
    """Every launch variant of the FP32 hot sweeps (shared-memory or register-resident element
    body, 96-192 threads per CTA) gives the oracle's raw A, constrained A and constrained fused
    [A B^T; (B+C) 0] on levels 1-3 to the FP32 tolerance."""
    dtype = torch.float32
    _, _, prob = gpu_problem(3, blending)
    try:
        for l in (1, 2, 3):
            prob.set_tuning(l, variant)
            L, ops, co = oracle(l, blending)
            u, p = inputs(L, dtype, seed=7)
            ud, pd = dev(u, dtype), dev(p, dtype)
            yu = torch.empty(3 * L.n_p2, dtype=dtype, device="cuda")
            yp = torch.empty(L.n_p1, dtype=dtype, device="cuda")
            prob.apply_A(l, ud, yu)
            assert rel(yu.cpu().double().numpy(), ops.A @ u) <= TOL[dtype], l
            prob.apply_A(l, ud, yu, constrained=True)
            assert rel(yu.cpu().double().numpy(), co.apply_A(u)) <= TOL[dtype], l
            prob.apply_stokes(l, ud, pd, yu, yp)
            assert rel(yu.cpu().double().numpy(), co.apply_A(u) + co.apply_BT(p)) <= TOL[dtype], l
            assert rel(yp.cpu().double().numpy(), co.apply_Bbar(u)) <= TOL[dtype], l
    finally:
        for l in (1, 2, 3):
            prob.set_tuning(l, DEFAULT_VARIANT)


def test_fused_apply_level5_sampled_rows():
    """The bench's workload and launch at full size: level 5 (1,966,080 micro-tets), plume
    viscosity of contrast 1e6 (seed 2), compressible density, the constrained fused apply in
    FP32 (sweep variants 0, 6 and 8) and FP64.  The oracle evaluates sampled rows one by one
    from every micro-tet that touches 256 interior, 64 surface and 64 CMB P2 nodes and 128 P1 vertices (32 of them on the
    spheres), on the projected inputs (Sec. 5.1, Eqs. SaddlePointStructureDirichlet /
    InnerSaddlePointSystem): interior velocity rows equal A P0 u + B^T P_p p; surface rows
    (Dirichlet) are the identity, y = u; CMB rows (free-slip) equal P_v (A P0 u + B^T P_p p)
    with P_v u = u - (u.n)n at the node; pressure rows equal (B+C) P0 u up to the one constant
    that P_p removes from the whole output.  Each node class is checked on its own."""
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
    s_in = np.sort(rng.choice(np.flatnonzero(L.p2_class == 0), 256, replace=False))
    s_top = np.sort(rng.choice(np.flatnonzero(L.p2_class == 1), 64, replace=False))
    s_cmb = np.sort(rng.choice(np.flatnonzero(L.p2_class == 2), 64, replace=False))
    s1 = np.sort(np.concatenate([rng.choice(np.flatnonzero(L.p1_class == 0), 96, replace=False),
                                 rng.choice(np.flatnonzero(L.p1_class != 0), 32, replace=False)]))
    s2 = np.concatenate([s_in, s_cmb])
    sel = tets_touching(L, p2_nodes=s2, p1_nodes=s1)
    cons = Constraints(L, 0, 1)
    n2 = L.n_p2
    rows = lambda s: np.concatenate([s, s + n2, s + 2 * n2])
    nrm = L.p2_x[s_cmb] / np.linalg.norm(L.p2_x[s_cmb], axis=1, keepdims=True)
    refs = {}
    for dtype, variant in ((torch.float32, 0), (torch.float32, 6), (torch.float32, 8), (torch.float64, 0)):
        prob.set_tuning(lvl, variant)
        u, p = inputs(L, dtype, seed=21)
        if dtype not in refs:
            refs[dtype] = stokes_apply_elements(L, eta, dl, cons.P0(u), p - p.mean(), sel)
        yu_ref, yp_ref = refs[dtype]
        yu = torch.empty(3 * n2, dtype=dtype, device="cuda")
        yp = torch.empty(L.n_p1, dtype=dtype, device="cuda")
        prob.apply_stokes(lvl, dev(u, dtype), dev(p, dtype), yu, yp)
        yu = yu.cpu().double().numpy()
        yp = yp.cpu().double().numpy()
        assert rel(yu[rows(s_in)], yu_ref[rows(s_in)]) <= TOL[dtype]
        # surface (Dirichlet): identity rows
        assert rel(yu[rows(s_top)], u[rows(s_top)]) <= TOL[dtype]
        # CMB (free-slip): the raw rows projected onto the tangent plane at the node
        R = yu_ref[rows(s_cmb)].reshape(3, -1).T
        R = R - np.einsum("ij,ij->i", R, nrm)[:, None] * nrm
        G = yu[rows(s_cmb)].reshape(3, -1).T
        assert rel(G, R) <= TOL[dtype]
        assert np.abs(np.einsum("ij,ij->i", G, nrm)).max() <= 10 * TOL[dtype] * np.abs(G).max()
        # pressure rows: the P_p constant is common to all rows, estimated from all samples
        d = yp[s1] - yp_ref[s1]
        d = d - d.mean()
        for mask in (L.p1_class[s1] == 0, L.p1_class[s1] != 0):
            assert np.linalg.norm(d[mask]) <= TOL[dtype] * np.linalg.norm(yp_ref[s1][mask])
