"""GPU parity of the temperature step (Sec. 3, Sec. 6, Eq. WeakTemp) against the oracle: the
P2 blocks M, D, D_s, C(u), R(u) (plain and constrained), the right-hand side with and without
shear heating, the RK4 MMOC with its departure points, and one full step."""
import functools

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2506_04157_gb300 as mfs
import workloads as W
from oracle.mesh import MacroMesh, Level
from oracle.temperature import (TemperatureOperators, Locator, mmoc, mmoc_departure, temperature_rhs,
                                temperature_step)

TABLE = (-0.3781,)
LAW = dict(E_A=4.610, V_A=2.996, r_cmb=0.5, r_surf=1.0, log10_base=[1.0, 0.3, 0.0, 0.5, 2.0])


@functools.lru_cache(maxsize=None)
def setup(L):
    mesh = MacroMesh()
    Lv = Level(mesh, L)
    ops = TemperatureOperators(Lv, TABLE)
    ctx = mfs.Context(0)
    gm = mfs.Mesh(ctx, L)
    prob = mfs.Problem(gm, "dirichlet", "freeslip")
    prob.set_viscosity(torch.ones(Lv.n_p1, dtype=torch.float64, device="cuda"))
    prob.set_density(TABLE)
    prob.set_viscosity_law(LAW["log10_base"], E_A=LAW["E_A"], V_A=LAW["V_A"], l_eta=-1)
    return Lv, ops, ctx, gm, prob


def fields(Lv, seed):
    x = Lv.p2_x
    rng = np.random.default_rng(seed)
    om = rng.standard_normal(3)
    u = (np.cross(om, x) + 0.1 * np.sin(3 * x)).T.reshape(-1)
    T = W.temperature_blobs(x, seed)
    return u, T


def dev(a, dt=torch.float64):
    return torch.tensor(np.asarray(a), dtype=dt, device="cuda")


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("dt,tol", [(torch.float64, 1e-12), (torch.float32, 1e-5)])
def test_temp_blocks(dt, tol):
    Lv, ops, ctx, gm, prob = setup(2)
    u, T = fields(Lv, 1)
    n = Lv.n_p2
    if dt == torch.float32:
        u = u.astype(np.float32).astype(np.float64)
        T = T.astype(np.float32).astype(np.float64)
    y = torch.empty(n, dtype=dt, device="cuda")
    cases = [(dict(cM=1.0), ops.M), (dict(cM=0.0, cD=1.0), ops.D), (dict(cM=0.0, cD=1.0, sym=True), ops.Ds),
             (dict(cM=0.0, cC=1.0, u=u), ops.advection(u)), (dict(cM=0.0, cR=1.0, u=u), ops.adiabatic(u))]
    for kw, A in cases:
        kw = dict(kw)
        if "u" in kw:
            kw["u"] = dev(kw["u"], dt)
        prob.temp_apply(dev(T, dt), y, **kw)
        assert rel(y.double().cpu().numpy(), A @ T) <= tol, kw.keys()
    # constrained combination: identity on the boundary rows and columns
    L = 1.5 * ops.M + 0.1 * (ops.advection(u) + 0.7 * ops.D - 0.2 * ops.adiabatic(u))
    bnd = ops.boundary
    Tin = np.where(bnd, 0.0, T)
    ref = L @ Tin
    ref[bnd] = T[bnd]
    prob.temp_apply(dev(T, dt), y, cM=1.5, cC=0.1, cD=0.07, cR=-0.02, u=dev(u, dt), constrained=True)
    assert rel(y.double().cpu().numpy(), ref) <= tol


@pytest.mark.parametrize("shear", [False, True])
def test_temp_rhs(shear):
    Lv, ops, ctx, gm, prob = setup(2)
    u, T0 = fields(Lv, 2)
    _, Tm = fields(Lv, 3)
    params = dict(H=0.3, Di=0.5 if shear else 0.0, Pe=2.0, Ra=5.0, Cp=1.2)
    b = torch.empty(Lv.n_p2, dtype=torch.float64, device="cuda")
    prob.temp_rhs(dev(T0), dev(Tm), 0.02, 0.03, b, u_star=dev(u), T_star=dev(T0), **params)
    ref = temperature_rhs(ops, T0, Tm, u, 0.02, 0.03, params, T_star=T0, law=LAW if shear else None)
    assert rel(b.cpu().numpy(), ref) <= 1e-12


def test_mmoc_matches_oracle():
    Lv, ops, ctx, gm, prob = setup(2)
    u_new, T = fields(Lv, 4)
    u_old, _ = fields(Lv, 5)
    loc = Locator(Lv)
    X = torch.empty(3 * Lv.n_p2, dtype=torch.float64, device="cuda")
    Th = torch.empty(Lv.n_p2, dtype=torch.float64, device="cuda")
    prob.mmoc(dev(T), dev(u_new), dev(u_old), 0.03, Th, X)
    Xr = mmoc_departure(loc, u_new, u_old, 0.03)
    assert np.abs(X.cpu().numpy().reshape(3, -1).T - Xr).max() <= 1e-12
    assert np.abs(Th.cpu().numpy() - mmoc(loc, T, u_new, u_old, 0.03)).max() <= 1e-10 * np.abs(T).max()
    # the same particles traced on over a second step from where they arrived
    X2 = torch.empty_like(X)
    prob.mmoc(dev(T), dev(u_old), dev(u_new), 0.02, Th, X2, X_start=X)
    Xr2 = mmoc_departure(loc, u_old, u_new, 0.02, X=Xr)
    assert np.abs(X2.cpu().numpy().reshape(3, -1).T - Xr2).max() <= 1e-12
    assert np.abs(Th.cpu().numpy() - loc.eval_p2(T, Xr2)).max() <= 1e-10 * np.abs(T).max()


def test_mmoc_polyhedral_shell():
    """The MMOC on the polyhedral shell (no blending): departure points outside the shell move
    radially onto the prism's inner or outer face plane on both sides; a step long enough to
    cross micro-tets and leave the shell."""
    Lv = Level(MacroMesh(blending=False), 2)
    gm = mfs.Mesh(mfs.Context(0), 2, blending=False)
    prob = mfs.Problem(gm, "dirichlet", "freeslip")
    prob.set_density(TABLE)
    u_new, T = fields(Lv, 6)
    u_old, _ = fields(Lv, 7)
    loc = Locator(Lv)
    X = torch.empty(3 * Lv.n_p2, dtype=torch.float64, device="cuda")
    Th = torch.empty(Lv.n_p2, dtype=torch.float64, device="cuda")
    prob.mmoc(dev(T), dev(u_new), dev(u_old), 0.3, Th, X)
    Xr = mmoc_departure(loc, u_new, u_old, 0.3)
    assert np.abs(X.cpu().numpy().reshape(3, -1).T - Xr).max() <= 1e-12
    assert np.abs(Th.cpu().numpy() - loc.eval_p2(T, Xr)).max() <= 1e-10 * np.abs(T).max()


def test_temperature_step_matches_oracle():
    Lv, ops, ctx, gm, prob = setup(2)
    u_n, T_n = fields(Lv, 6)
    u_nm1, T_nm1 = fields(Lv, 7)
    r = np.linalg.norm(Lv.p2_x, axis=1)
    T_bc = (1 / r - 1) / (1 / 0.5 - 1)
    params = dict(k=0.05, H=0.3, Di=0.2, Pe=2.0, Ra=5.0)
    ref, _, _ = temperature_step(ops, Locator(Lv), T_n, T_nm1, u_n, u_nm1, 0.02, 0.025, params, T_bc, law=LAW)
    T1 = torch.empty(Lv.n_p2, dtype=torch.float64, device="cuda")
    st = prob.temperature_step(dev(T_n), dev(T_nm1), dev(u_n), dev(u_nm1), 0.02, 0.025, dev(T_bc), T1, tol_T=1e-13,
                               **params)
    assert st["status"] == "MFS_OK"
    assert rel(T1.cpu().numpy(), ref) <= 1e-9, st


def test_coupled_step_matches_oracle():
    """Two coupled steps (temperature step, law viscosity, buoyancy, Stokes solve to 1e-10)
    against the oracle's coupled step with an exact Stokes solve."""
    from oracle.timeloop import CoupledOracle
    from paper_2506_04157_gb300.timeloop import CoupledStepper
    law = dict(E_A=4.610, V_A=2.996, r_cmb=0.5, r_surf=1.0, log10_base=[0.0])
    C = CoupledOracle(MacroMesh(), 2, law, dlnrho_table=TABLE)
    Lv = C.level
    ctx = mfs.Context(0)
    gm = mfs.Mesh(ctx, 2)
    prob = mfs.Problem(gm, "dirichlet", "freeslip")
    prob.set_density(TABLE)
    prob.set_viscosity_law(law["log10_base"], E_A=law["E_A"], V_A=law["V_A"], l_eta=-1)
    T = 0.5 + 0.1 * np.sin(4 * Lv.p2_x[:, 0]) * Lv.p2_x[:, 1]
    r = np.linalg.norm(Lv.p2_x, axis=1)
    T_bc = (1 / r - 1) / (1 / 0.5 - 1)
    params = dict(k=0.1, Ra=10.0)
    zero = np.zeros(3 * Lv.n_p2)
    ref = dict(T_n=T, T_nm1=T, u_n=zero, u_nm1=zero)
    S = CoupledStepper(prob, temp_params=dict(params, tol_T=1e-13), solve_opts=dict(rtol=1e-10, mixed=2))
    st = dict(T_n=dev(T), T_nm1=dev(T), u_n=dev(zero), u_nm1=dev(zero), p=torch.zeros(Lv.n_p1, dtype=torch.float64,
                                                                                        device="cuda"))
    for _ in range(2):
        ref = C.step(ref, 0.01, 0.01, params, T_bc)
        st, stats = S.step(st, 0.01, 0.01, dev(T_bc))
        assert stats["stokes"]["status"] == "MFS_OK"
    assert rel(st["T_n"].cpu().numpy(), ref["T_n"]) <= 1e-7
    assert rel(st["u_n"].cpu().numpy(), ref["u_n"]) <= 1e-5
