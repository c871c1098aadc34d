"""GPU parity of the multigrid layer against the oracle: diag(A), M_{1/eta}, transfers and
one V-cycle (same Chebyshev intervals, exact coarse solve on both sides)."""
import functools

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2506_04157_gb300 as mfs
import workloads as W
from oracle.mesh import MacroMesh, Level
from oracle.solver import Hierarchy

TOL = {torch.float64: 1e-12, torch.float32: 1e-5}


@functools.lru_cache(maxsize=None)
def setup(L, bc=("dirichlet", "freeslip")):
    mesh = MacroMesh()
    Lf = Level(mesh, L)
    eta = W.viscosity_plumes(Lf.p1_x, seed=7, contrast=1e4)
    bcm = {"dirichlet": 0, "freeslip": 1}
    H = Hierarchy(mesh, L, eta, dlnrho_table=W.dlnrho_table_compressible(), bc=(bcm[bc[0]], bcm[bc[1]]))
    ctx = mfs.Context(0)
    gm = mfs.Mesh(ctx, L)
    prob = mfs.Problem(gm, *bc)
    x1 = gm.coords(L, p2=False).T
    assert np.abs(x1 - Lf.p1_x).max() < 1e-14
    prob.set_viscosity(torch.tensor(eta, device="cuda"))
    prob.set_density(W.dlnrho_table_compressible())
    prob.setup_multigrid(1)
    for l in range(2, L + 1):
        prob.set_cheb_bounds(l, *H.bounds[l])
    return H, ctx, gm, prob


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def dev(x, dt):
    return torch.tensor(x, dtype=dt, device="cuda")


@pytest.mark.parametrize("dt", [torch.float64, torch.float32])
@pytest.mark.parametrize("L", [2, 3])
def test_diag_and_mass(L, dt):
    H, ctx, gm, prob = setup(L)
    for l in range(1, L + 1):
        y = torch.empty(3 * H.levels[l].n_p2, dtype=dt, device="cuda")
        prob.diag_A(l, y)
        assert rel(y.double().cpu().numpy(), H.diag[l]) <= TOL[dt]
    p = W.random_field(H.levels[L].n_p1, 3)
    if dt == torch.float32:
        p = p.astype(np.float32).astype(np.float64)
    y = torch.empty(H.levels[L].n_p1, dtype=dt, device="cuda")
    prob.apply_mass(L, dev(p, dt), y)
    assert rel(y.double().cpu().numpy(), H.ops[L].M_inv_eta @ p) <= TOL[dt]


@pytest.mark.parametrize("dt", [torch.float64, torch.float32])
@pytest.mark.parametrize("L", [2, 3])
def test_transfers(L, dt):
    H, ctx, gm, prob = setup(L)
    for l in range(2, L + 1):
        nc, nf = 3 * H.levels[l - 1].n_p2, 3 * H.levels[l].n_p2
        xc = H.cons[l - 1].P0(W.random_field(nc, 4))
        rf = W.random_field(nf, 5)
        if dt == torch.float32:
            xc = xc.astype(np.float32).astype(np.float64)
            rf = rf.astype(np.float32).astype(np.float64)
        xf = torch.empty(nf, dtype=dt, device="cuda")
        prob.prolongate(l, dev(xc, dt), xf)
        assert rel(xf.double().cpu().numpy(), H.cons[l].P0(H.P[l] @ xc)) <= TOL[dt]
        rc = torch.empty(nc, dtype=dt, device="cuda")
        prob.restrict(l, dev(rf, dt), rc)
        assert rel(rc.double().cpu().numpy(), H.cons[l - 1].P0(H.P[l].T @ rf)) <= TOL[dt]


@pytest.mark.parametrize("dt", [torch.float64, torch.float32])
@pytest.mark.parametrize("L", [2, 3])
def test_vcycle(L, dt):
    H, ctx, gm, prob = setup(L)
    n = 3 * H.levels[L].n_p2
    f = H.cons[L].P0(W.random_field(n, 6))
    if dt == torch.float32:
        f = f.astype(np.float32).astype(np.float64)
    for steps, deg in ((3, 2), (1, 1)):
        u = torch.empty(n, dtype=dt, device="cuda")
        prob.vcycle(L, dev(f, dt), u, steps=steps, degree=deg)
        ref = H.vcycle(L, f, steps, deg, coarse_exact=True)
        tol = 1e-10 if dt == torch.float64 else 2e-5
        assert rel(u.double().cpu().numpy(), ref) <= tol


@pytest.mark.parametrize("L,bc", [(2, ("dirichlet", "freeslip")), (3, ("dirichlet", "freeslip")),
                                  (2, ("freeslip", "dirichlet"))])
def test_power_iteration_estimate(L, bc):
    """The library's power iteration for the Chebyshev interval (15 FP64 steps on D^-1 A_c,
    Sec. 5.2 reading [b/20, b], b = 1.2 lambda) started from the oracle's seeded vector (numpy
    PCG64, seed 0) gives the oracle's estimate to 1e-10: the same D, A_c, projections and
    iteration count on both sides."""
    from oracle.solver import power_max_eig
    H, ctx, gm, prob = setup(L, bc)
    prob2 = mfs.Problem(gm, *bc)
    prob2.set_viscosity(torch.tensor(H.etas[L], device="cuda"))
    prob2.set_density(W.dlnrho_table_compressible())
    prob2.setup_multigrid(1)
    for l in range(2, L + 1):
        n3 = 3 * H.levels[l].n_p2
        x0 = np.random.default_rng(0).standard_normal(n3)
        lam_ref = power_max_eig(H.co[l].apply_A, 1.0 / H.diag[l], H.cons[l].P0, n3)
        lam = prob.estimate_cheb_bounds(l, torch.tensor(x0, device="cuda"))
        assert abs(lam - lam_ref) <= 1e-10 * lam_ref, (l, lam, lam_ref)
        lo, hi = prob.cheb_bounds(l)
        assert abs(hi - 1.2 * lam_ref) <= 1e-10 * hi and abs(lo - hi / 20) <= 1e-14 * hi
        # the setup's own estimate (its seeded splitmix64 vector) lands near it
        assert abs(prob2.cheb_bounds(l)[1] - 1.2 * lam_ref) <= 0.05 * 1.2 * lam_ref
        prob.set_cheb_bounds(l, *H.bounds[l])   # the shared fixture keeps the oracle's interval


@pytest.mark.parametrize("table", [(-0.3781, -0.3781), (-1.0, -0.2, 0.5, -0.7)])
def test_buoyancy_rhs(table):
    from oracle.fem import buoyancy_rhs
    mesh = MacroMesh()
    L = Level(mesh, 2)
    ctx = mfs.Context(0)
    gm = mfs.Mesh(ctx, 2)
    prob = mfs.Problem(gm)
    prob.set_viscosity(torch.tensor(W.viscosity_radial(L.p1_x), device="cuda"))
    prob.set_density(np.array(table))
    T = W.temperature_blobs(L.p2_x, 9)
    f = torch.empty(3 * L.n_p2, dtype=torch.float64, device="cuda")
    prob.rhs_buoyancy(torch.tensor(T, device="cuda"), f, scale=2.5)
    ref = buoyancy_rhs(L, T, np.array(table), scale=2.5)
    assert rel(f.cpu().numpy(), ref) <= 1e-10


def test_checkpoint_restores_the_hierarchy():
    """mfs_mg_checkpoint / mfs_mg_restore: after another viscosity and a new setup, restoring
    the checkpoint brings back every level's viscosity, inverse diagonal, Chebyshev interval,
    coarse inverse and mass weights: A applies, diagonals, bounds, V-cycles and solves equal
    those before (FP64)."""
    H, ctx, gm, _ = setup(3)
    prob = mfs.Problem(gm)
    L = H.levels[3]
    prob.set_viscosity(torch.tensor(W.viscosity_plumes(L.p1_x, seed=11, contrast=1e4), device="cuda"))
    prob.set_density(W.dlnrho_table_compressible())
    prob.setup_multigrid(1)
    state = prob.mg_checkpoint()
    u = torch.tensor(W.random_field(3 * L.n_p2, 12), device="cuda")
    f = torch.tensor(H.cons[3].P0(W.random_field(3 * L.n_p2, 13)), device="cuda")

    def snapshot():
        out = {}
        for l in (2, 3):
            n3 = 3 * H.levels[l].n_p2
            y = torch.empty(n3, dtype=torch.float64, device="cuda")
            prob.apply_A(l, u[:n3].contiguous(), y, constrained=True)
            d = torch.empty_like(y)
            prob.diag_A(l, d)
            out[l] = (y, d, prob.cheb_bounds(l))
        x = torch.zeros_like(f)
        prob.vcycle(3, f, x, 3, 2)
        out["v"] = x
        g = torch.zeros(L.n_p1, dtype=torch.float64, device="cuda")
        uu, pp = torch.zeros_like(f), torch.zeros_like(g)
        st = prob.solve(f, g, uu, pp, mixed=0)
        out["solve"] = (uu, st["fgmres_iters"])
        return out

    a = snapshot()
    prob.set_viscosity(torch.tensor(W.viscosity_radial(L.p1_x), device="cuda"))
    prob.setup_multigrid(1)
    b = snapshot()
    assert rel(b[3][0].cpu().numpy(), a[3][0].cpu().numpy()) > 1e-3     # the state did change
    prob.mg_restore(state)
    c = snapshot()
    for l in (2, 3):
        assert rel(c[l][0].cpu().numpy(), a[l][0].cpu().numpy()) <= 1e-13
        assert rel(c[l][1].cpu().numpy(), a[l][1].cpu().numpy()) <= 1e-13 and c[l][2] == a[l][2]
    assert rel(c["v"].cpu().numpy(), a["v"].cpu().numpy()) <= 1e-12
    assert rel(c["solve"][0].cpu().numpy(), a["solve"][0].cpu().numpy()) <= 1e-8
    other = mfs.Problem(gm)
    other.set_viscosity(torch.tensor(W.viscosity_radial(L.p1_x), device="cuda"))
    other.setup_multigrid(1)
    with pytest.raises(mfs.MfsError):
        other.mg_restore(state)
