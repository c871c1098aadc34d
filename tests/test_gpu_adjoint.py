"""Adjoint gradient of a surface-velocity misfit w.r.t. the nodal log-viscosity:
against the oracle's gradient, central finite differences and the uniform-scaling
identity sum_k g_k = -lam^T A u."""
import functools

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2506_04157_gb300 as mfs
from paper_2506_04157_gb300.autograd import stokes_solve
import workloads as W
from oracle.mesh import MacroMesh, Level
from oracle.solver import Hierarchy, direct_solve
from oracle.adjoint import adjoint_direct, grad_log_eta

BC = ("freeslip", "dirichlet")   # free-slip surface, no-slip CMB (the misfit must vary)
TIGHT = dict(mixed=0, rtol=1e-11, max_iters=400)   # FP64 residual floor ~2e-12 here


@functools.lru_cache(maxsize=None)
def setup(L=2):
    mesh = MacroMesh()
    Lv = Level(mesh, L)
    ctx = mfs.Context(0)
    gm = mfs.Mesh(ctx, L)
    prob = mfs.Problem(gm, *BC)
    prob.set_density(W.dlnrho_table_config1())
    x2 = Lv.p2_x
    T = W.temperature_blobs(x2, 3)
    xh = x2 / np.linalg.norm(x2, axis=1, keepdims=True)
    f = np.concatenate([T * xh[:, 0], T * xh[:, 1], T * xh[:, 2]]) * 1e-3
    log_eta = np.log(W.viscosity_plumes(Lv.p1_x, 5, 1e4))
    log_ref = np.log(W.viscosity_plumes(Lv.p1_x, 4, 1e4))
    return mesh, Lv, ctx, gm, prob, f, log_eta, log_ref


def misfit_and_grad(Lv, u, u_obs):
    """J = 1/2 sum over surface P2 nodes |u - u_obs|^2 and dJ/du."""
    n = Lv.n_p2
    surf = np.tile(Lv.p2_class == 1, 3)
    d = np.where(surf, u - u_obs, 0.0)
    return 0.5 * d @ d, d


def gpu_forward(prob, log_eta, f, npp):
    prob.set_viscosity(torch.tensor(log_eta, device="cuda"), is_log=True)
    prob.setup_multigrid(1)
    u = torch.zeros(f.size, dtype=torch.float64, device="cuda")
    p = torch.zeros(npp, dtype=torch.float64, device="cuda")
    prob.solve(torch.tensor(f, device="cuda"), torch.zeros(npp, dtype=torch.float64, device="cuda"), u, p, **TIGHT)
    return u, p


def test_gradient_vs_oracle_and_identity():
    mesh, Lv, ctx, gm, prob, f, log_eta, log_ref = setup()
    npp = Lv.n_p1
    u_obs = gpu_forward(prob, log_ref, f, npp)[0].cpu().numpy()
    u, p = gpu_forward(prob, log_eta, f, npp)
    J, dJ = misfit_and_grad(Lv, u.cpu().numpy(), u_obs)
    lam_u = torch.zeros_like(u)
    lam_p = torch.zeros_like(p)
    prob.adjoint_solve(torch.tensor(dJ, device="cuda"), torch.zeros_like(p), lam_u, lam_p, **TIGHT)
    g = torch.empty(npp, dtype=torch.float64, device="cuda")
    prob.grad_log_eta(u, lam_u, g)
    g = g.cpu().numpy()
    # oracle: direct forward and adjoint solves, element-loop gradient
    bcm = {"dirichlet": 0, "freeslip": 1}
    H = Hierarchy(mesh, 2, np.exp(log_eta), dlnrho_table=W.dlnrho_table_config1(), bc=(bcm[BC[0]], bcm[BC[1]]))
    uo, po = direct_solve(H, f, np.zeros(npp), 0 * f, np.zeros(npp))
    Jo, dJo = misfit_and_grad(Lv, uo, u_obs)
    lo, _ = adjoint_direct(H, dJo, np.zeros(npp))
    go = grad_log_eta(Lv, np.exp(log_eta), uo, lo)
    assert np.linalg.norm(g - go) / np.linalg.norm(go) < 1e-6
    # uniform scaling: sum_k g_k = -lam^T A u (A linear in eta)
    Au = torch.empty_like(u)
    prob.apply_A(2, u, Au)
    assert abs(g.sum() + lam_u.cpu().numpy() @ Au.cpu().numpy()) <= 1e-9 * np.abs(g).sum()


def test_gradient_finite_differences():
    mesh, Lv, ctx, gm, prob, f, log_eta, log_ref = setup()
    npp = Lv.n_p1
    u_obs = gpu_forward(prob, log_ref, f, npp)[0].cpu().numpy()
    le = torch.tensor(log_eta, device="cuda", requires_grad=True)
    ft = torch.tensor(f, device="cuda")
    gt = torch.zeros(npp, dtype=torch.float64, device="cuda")
    u, p = stokes_solve(le, ft, gt, prob, TIGHT)
    surf = torch.tensor(np.tile(Lv.p2_class == 1, 3), device="cuda")
    J = 0.5 * ((torch.where(surf, u - torch.tensor(u_obs, device="cuda"), 0.0)) ** 2).sum()
    (g,) = torch.autograd.grad(J, le)
    g = g.cpu().numpy()
    rng = np.random.default_rng(6)
    # central step 1e-4: truncation O(h^2) < 1e-7 relative; with h = 1e-6 the FP64 solve
    # floor (relative residual ~2e-12 here) would give ~3e-3 relative FD noise
    h = 1e-4
    for _ in range(4):
        d = rng.standard_normal(npp)
        Jp = misfit_and_grad(Lv, gpu_forward(prob, log_eta + h * d, f, npp)[0].cpu().numpy(), u_obs)[0]
        Jm = misfit_and_grad(Lv, gpu_forward(prob, log_eta - h * d, f, npp)[0].cpu().numpy(), u_obs)[0]
        fd = (Jp - Jm) / (2 * h)
        assert abs(fd - g @ d) <= 1e-4 * abs(g @ d), (fd, g @ d)


def test_gradient_finite_differences_level4_32_directions():
    """The adjoint-gradient workload at full size: level 4 (1,057,512 dofs), contrast 1e4,
    free-slip surface / no-slip CMB, u_obs from the reference viscosity (seed 4), start
    viscosity seed 5, 32 random directions (seed 6).  Central differences with h = 1e-4
    around mixed-precision solves to a relative residual of 1e-11 (observed: median relative
    error 1e-5, largest 4e-4 over the 32 directions)."""
    import time
    L = 4
    ctx = mfs.Context(0)
    gm = mfs.Mesh(ctx, L)
    prob = mfs.Problem(gm, *BC)
    prob.set_density(W.dlnrho_table_config1())
    x1 = gm.coords(L, p2=False).T
    x2 = gm.coords(L).T
    T = W.temperature_blobs(x2, 3)
    xh = x2 / np.linalg.norm(x2, axis=1, keepdims=True)
    f = np.concatenate([T * xh[:, 0], T * xh[:, 1], T * xh[:, 2]]) * 1e-3
    log_eta = np.log(W.viscosity_plumes(x1, 5, 1e4))
    log_ref = np.log(W.viscosity_plumes(x1, 4, 1e4))
    npp = x1.shape[0]
    surf = np.tile(gm.node_class(L) == 1, 3)
    opts = dict(mixed=1, rtol=1e-11, max_iters=600)
    ft = torch.tensor(f, device="cuda")
    gt = torch.zeros(npp, dtype=torch.float64, device="cuda")

    def forward(le):
        prob.set_viscosity(torch.tensor(le, device="cuda"), is_log=True)
        prob.setup_multigrid(1)
        u = torch.zeros(f.size, dtype=torch.float64, device="cuda")
        p = torch.zeros(npp, dtype=torch.float64, device="cuda")
        st = prob.solve(ft, gt, u, p, **opts)
        assert st["rel_residual"] <= 1e-11
        return u.cpu().numpy()

    def J_of(u):
        d = np.where(surf, u - u_obs, 0.0)
        return 0.5 * d @ d

    t0 = time.time()
    u_obs = forward(log_ref)
    le = torch.tensor(log_eta, device="cuda", requires_grad=True)
    u, p = stokes_solve(le, ft, gt, prob, opts)
    J = 0.5 * ((torch.where(torch.tensor(surf, device="cuda"), u - torch.tensor(u_obs, device="cuda"), 0.0)) ** 2).sum()
    (g,) = torch.autograd.grad(J, le)
    g = g.cpu().numpy()
    rng = np.random.default_rng(6)
    h = 1e-4
    errs = []
    for _ in range(32):
        d = rng.standard_normal(npp)
        fd = (J_of(forward(log_eta + h * d)) - J_of(forward(log_eta - h * d))) / (2 * h)
        errs.append(abs(fd - g @ d) / abs(g @ d))
    print(f"level-4 FD check: max rel err {max(errs):.2e}, median {np.median(errs):.2e}, {time.time() - t0:.0f} s")
    assert max(errs) <= 2e-3
