"""Concurrent solves of independent problems on several CUDA streams (mfs_solve_concurrent):
every member's returned iterate is checked by the oracle — the full FP64 projected residual
(Sec. 5.1 system) where the oracle can assemble the level, sampled constrained rows of the
same residual where it cannot — for the 64-member ensemble of levels 3 to 5."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2506_04157_gb300 as mfs
import workloads as W
from oracle.mesh import MacroMesh, Level
from oracle.fem import Constraints
from oracle.sampled import MacroRows, sample_points
from oracle.solver import Hierarchy, StokesOracle

BCS = {"dirichlet": 0, "freeslip": 1}


def forcing(x2, seed):
    """Buoyancy-type nodal forcing T x/|x| from a seeded smooth temperature field; g = 0."""
    T = W.temperature_blobs(x2, seed)
    xh = x2 / np.linalg.norm(x2, axis=1, keepdims=True)
    return np.concatenate([T * xh[:, 0], T * xh[:, 1], T * xh[:, 2]])


def sampled_residual_check(mesh, L, eta, f, u, p, r0, rng, k=24, bc=(0, 1)):
    """Sampled rows of the projected residual r = (P0 (f - A u - B^T P_p p), P_p (g - (B+C) u))
    (g = 0): at P2 nodes and P1 vertices strictly inside random macros the oracle's constrained
    rows give r_i exactly, so |r_i| <= ||r||; the pressure rows carry the common constant of
    P_p, so their spread max - min <= 2 ||r||.  Both against the 1e-8 target (x 1.5)."""
    rows = MacroRows(mesh, L)
    dl = W.dlnrho_table_compressible()
    pm = p - p.mean()
    n2 = rows.n_p2
    worst_u, vals_p = 0.0, []
    for m in rng.choice(60, size=6, replace=False):
        for pt in sample_points(2 * rows.n, k // 6, rng):
            got = rows.constrained_velocity_row(int(m), pt, eta, dl, u, pm, bc)
            if got is None:
                continue
            gid, row, _ = got
            fr = np.array([f[gid + c * n2] for c in range(3)])
            worst_u = max(worst_u, float(np.abs(fr - row).max()))
        for pt in sample_points(rows.n, k // 6, rng):
            got = rows.constrained_pressure_row(int(m), pt, eta, dl, u, pm, bc)
            if got is not None:
                vals_p.append(-got[1])
    assert len(vals_p) >= 4
    assert worst_u <= 1.5e-8 * r0, (worst_u, r0)
    assert max(vals_p) - min(vals_p) <= 3e-8 * r0, (max(vals_p) - min(vals_p), r0)


def test_concurrent_solve_two_streams_vs_oracle_residual():
    """Four members (levels 2 and 3, both boundary-condition pairs) on two streams, solved
    concurrently (FP32 applies in FP64 refinement): the oracle's FP64 projected residual of each
    iterate <= 1.5e-8 of the initial residual, and the members of one stream ran in turn."""
    members = [(3, 120, 1e4, ("dirichlet", "freeslip")), (2, 121, 1e6, ("freeslip", "dirichlet")),
               (2, 122, 1e5, ("dirichlet", "freeslip")), (3, 123, 1e6, ("freeslip", "dirichlet"))]
    streams = [torch.cuda.Stream() for _ in range(2)]
    ctxs = [mfs.Context(0, s.cuda_stream) for s in streams]
    mesh = MacroMesh()
    probs, hiers, host = [], [], []
    for i, (l, seed, c, bc) in enumerate(members):
        Lf = Level(mesh, l)
        eta = W.viscosity_plumes(Lf.p1_x, seed, c)
        hiers.append(Hierarchy(mesh, l, eta, dlnrho_table=W.dlnrho_table_compressible(),
                               bc=(BCS[bc[0]], BCS[bc[1]])))
        P = mfs.Problem(mfs.Mesh(ctxs[i % 2], l), *bc)
        P.set_viscosity(torch.tensor(eta, device="cuda"))
        P.set_density(W.dlnrho_table_compressible())
        P.setup_multigrid(1)
        probs.append(P)
        host.append(forcing(Lf.p2_x, 80 + i))
    fs = [torch.tensor(f, device="cuda") for f in host]
    gs = [torch.zeros(H.levels[H.l_max].n_p1, dtype=torch.float64, device="cuda") for H in hiers]
    us = [torch.zeros_like(f) for f in fs]
    ps = [torch.zeros_like(g) for g in gs]
    stats = mfs.solve_concurrent(probs, fs, gs, us, ps, mixed=1)
    for H, f, u, p, st in zip(hiers, host, us, ps, stats):
        assert st["rel_residual"] <= 1e-8, st
        S = StokesOracle(H)
        un, pn = u.cpu().numpy(), p.cpu().numpy()
        g = np.zeros(H.levels[H.l_max].n_p1)
        r0 = np.linalg.norm(S.residual(f, g, 0 * un, 0 * pn))
        assert np.linalg.norm(S.residual(f, g, un, pn)) <= 1.5e-8 * r0


def test_ensemble_64_members_concurrent_solve():
    """The ensemble workload: 64 shells, refinement levels drawn from {3, 4, 5}, log-uniform
    viscosity contrast in [1e4, 1e6] (seeds 100 + i), buoyancy-type forcing, spread over 8
    streams and solved concurrently with FP32 applies in FP64 refinement (up to 1000 FGMRES
    iterations: the members of contrast near 1e6 take several hundred).  Every member reaches
    the 1e-8 relative residual measured in FP64 by the library; the oracle checks sampled rows
    of each member's projected residual, and the full residual of two level-3 members."""
    rng = np.random.default_rng(3)
    levels = rng.integers(3, 6, size=64)
    contrasts = 10.0 ** rng.uniform(4.0, 6.0, size=64)
    ens = mfs.Ensemble(levels, n_streams=8)
    assert len(set(ens.stream_of)) == 8
    mesh = MacroMesh()
    lv = {int(l): Level(mesh, int(l)) for l in sorted(set(levels.tolist()))}
    etas, host = [], []
    for i, (l, c) in enumerate(zip(levels, contrasts)):
        L = lv[int(l)]
        eta = W.viscosity_plumes(L.p1_x, 100 + i, float(c))
        P = ens.problems[i]
        P.set_viscosity(torch.tensor(eta, device="cuda"))
        P.set_density(W.dlnrho_table_compressible())
        P.setup_multigrid(1)
        etas.append(eta)
        host.append(forcing(L.p2_x, 500 + i))
    torch.cuda.synchronize()
    fs = [torch.tensor(f, device="cuda") for f in host]
    gs = [torch.zeros(lv[int(l)].n_p1, dtype=torch.float64, device="cuda") for l in levels]
    us = [torch.zeros_like(f) for f in fs]
    ps = [torch.zeros_like(g) for g in gs]
    stats = ens.solve(fs, gs, us, ps, mixed=1, max_iters=1000)
    assert all(st["rel_residual"] <= 1e-8 for st in stats), stats
    check = np.random.default_rng(11)
    full_done = 0
    for i, l in enumerate(levels):
        l = int(l)
        u, p = us[i].cpu().numpy(), ps[i].cpu().numpy()
        cons = Constraints(lv[l], 0, 1)
        r0 = float(np.linalg.norm(cons.P0(host[i])))
        sampled_residual_check(mesh, l, etas[i], host[i], u, p, r0, check)
        if l == 3 and full_done < 2:
            H = Hierarchy(mesh, l, etas[i], dlnrho_table=W.dlnrho_table_compressible(), bc=(0, 1))
            S = StokesOracle(H)
            g = np.zeros(lv[l].n_p1)
            assert np.linalg.norm(S.residual(host[i], g, u, p)) <= 1.5e-8 * r0
            full_done += 1
    assert full_done == 2
