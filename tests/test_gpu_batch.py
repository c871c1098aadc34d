"""Ensembles in one sweep launch, and the sweep autotuner: results equal the per-problem
applies / solves."""
import json
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2506_04157_gb300 as mfs
import workloads as W


def make_problem(ctx, level, seed, contrast, bc=("dirichlet", "freeslip")):
    mesh = mfs.Mesh(ctx, level)
    prob = mfs.Problem(mesh, *bc)
    x1 = mesh.coords(level, p2=False).T
    prob.set_viscosity(torch.tensor(W.viscosity_plumes(x1, seed, contrast), device="cuda"))
    prob.set_density(W.dlnrho_table_compressible())
    return prob


@pytest.fixture(scope="module")
def ensemble():
    ctx = mfs.Context(0)
    probs = [make_problem(ctx, 3, 100, 1e4), make_problem(ctx, 2, 101, 1e6, ("freeslip", "dirichlet")),
             make_problem(ctx, 4, 102, 1e5), make_problem(ctx, 3, 103, 1e6)]
    return ctx, probs, mfs.Batch(ctx, probs)


@pytest.mark.parametrize("transpose", [False, True])
@pytest.mark.parametrize("dt", [torch.float64, torch.float32])
def test_batch_apply_matches_individual(ensemble, dt, transpose):
    ctx, probs, batch = ensemble
    us, ps, yus, yps = [], [], [], []
    for i, P in enumerate(probs):
        nu, npp = P._sizes(P.mesh.l_max)
        us.append(torch.tensor(W.random_field(nu, 10 + i), dtype=dt, device="cuda"))
        ps.append(torch.tensor(W.random_field(npp, 20 + i), dtype=dt, device="cuda"))
        yus.append(torch.empty(nu, dtype=dt, device="cuda"))
        yps.append(torch.empty(npp, dtype=dt, device="cuda"))
    batch.apply_stokes(us, ps, yus, yps, transpose=transpose)
    tol = 1e-12 if dt == torch.float64 else 1e-5
    for P, u, p, yu, yp in zip(probs, us, ps, yus, yps):
        ru, rp = torch.empty_like(yu), torch.empty_like(yp)
        P.apply_stokes(P.mesh.l_max, u, p, ru, rp, transpose=transpose)
        assert (torch.linalg.norm(yu - ru) / torch.linalg.norm(ru)).item() <= tol
        assert (torch.linalg.norm(yp - rp) / torch.linalg.norm(rp)).item() <= tol


def test_batch_solve_matches_individual(ensemble):
    ctx, probs, batch = ensemble
    small = [make_problem(ctx, 3, 110, 1e4), make_problem(ctx, 2, 111, 1e3, ("freeslip", "dirichlet"))]
    b2 = mfs.Batch(ctx, small)
    fs, gs = [], []
    for i, P in enumerate(small):
        P.setup_multigrid(1)
        x2 = P.mesh.coords(P.mesh.l_max).T
        T = W.temperature_blobs(x2, 30 + i)
        xh = x2 / np.linalg.norm(x2, axis=1, keepdims=True)
        fs.append(torch.tensor(np.concatenate([T * xh[:, 0], T * xh[:, 1], T * xh[:, 2]]), device="cuda"))
        gs.append(torch.zeros(P._sizes(P.mesh.l_max)[1], dtype=torch.float64, device="cuda"))
    us = [torch.zeros_like(f) for f in fs]
    ps = [torch.zeros_like(g) for g in gs]
    stats = b2.solve(fs, gs, us, ps, mixed=0)
    for P, f, g, u, p, st in zip(small, fs, gs, us, ps, stats):
        assert st["rel_residual"] <= 1e-8
        u1, p1 = torch.zeros_like(u), torch.zeros_like(p)
        st1 = P.solve(f, g, u1, p1, mixed=0)
        assert st1["rel_residual"] <= 1e-8
        # Both iterates stop at a relative residual of 1e-8; atomic accumulation order makes
        # their Krylov paths differ by rounding, so they agree only to about kappa(K) * 1e-8.
        assert (torch.linalg.norm(u - u1) / torch.linalg.norm(u1)).item() < 1e-5


def test_autotune_keeps_results(ensemble, tmp_path):
    ctx, probs, batch = ensemble
    P = probs[2]
    L = P.mesh.l_max
    nu, npp = P._sizes(L)
    u = torch.tensor(W.random_field(nu, 5), dtype=torch.float32, device="cuda")
    p = torch.tensor(W.random_field(npp, 6), dtype=torch.float32, device="cuda")
    y0u, y0p = torch.empty_like(u), torch.empty_like(p)
    P.apply_stokes(L, u, p, y0u, y0p)
    cache = str(tmp_path / "tune.json")
    choice = P.autotune(cache)
    assert all(v in (0, 1) for v in choice) and len(choice) == L + 1
    rows = json.load(open(cache))
    assert [r["variant"] for r in rows] == choice
    assert P.autotune(cache) == choice          # read back from the cache
    y1u, y1p = torch.empty_like(u), torch.empty_like(p)
    P.apply_stokes(L, u, p, y1u, y1p)
    assert (torch.linalg.norm(y1u - y0u) / torch.linalg.norm(y0u)).item() <= 1e-5


def test_ensemble_64_members_uneven_levels():
    """The ensemble workload at full size: 64 shells, refinement levels drawn from {3, 4, 5},
    log-uniform viscosity contrast in [1e4, 1e6], seeds 100 + i.  The one-launch (persistent)
    batched apply equals the per-member applies; repeating the call replays the captured
    graph, a new set of vectors goes back to eager launches."""
    ctx = mfs.Context(0)
    rng = np.random.default_rng(3)
    levels = rng.integers(3, 6, size=64)
    contrasts = 10.0 ** rng.uniform(4.0, 6.0, size=64)
    meshes = {int(l): mfs.Mesh(ctx, int(l)) for l in sorted(set(levels.tolist()))}
    probs = []
    for i, (l, c) in enumerate(zip(levels, contrasts)):
        P = mfs.Problem(meshes[int(l)])
        x1 = meshes[int(l)].coords(int(l), p2=False).T
        P.set_viscosity(torch.tensor(W.viscosity_plumes(x1, 100 + i, float(c)), device="cuda"))
        P.set_density(W.dlnrho_table_compressible())
        probs.append(P)
    batch = mfs.Batch(ctx, probs)
    dt = torch.float32
    us, ps, yus, yps = [], [], [], []
    for i, P in enumerate(probs):
        nu, npp = P._sizes(P.mesh.l_max)
        us.append(torch.tensor(W.random_field(nu, 300 + i), dtype=dt, device="cuda"))
        ps.append(torch.tensor(W.random_field(npp, 400 + i), dtype=dt, device="cuda"))
        yus.append(torch.empty(nu, dtype=dt, device="cuda"))
        yps.append(torch.empty(npp, dtype=dt, device="cuda"))
    refs = []
    for P, u, p in zip(probs, us, ps):
        ru, rp = torch.empty_like(u), torch.empty_like(p)
        P.apply_stokes(P.mesh.l_max, u, p, ru, rp)
        refs.append((ru, rp))
    for rep in range(3):   # eager, captured, replayed
        for y in yus + yps:
            y.fill_(float("nan"))
        batch.apply_stokes(us, ps, yus, yps)
        for (ru, rp), yu, yp in zip(refs, yus, yps):
            assert (torch.linalg.norm(yu - ru) / torch.linalg.norm(ru)).item() <= 1e-5
            assert (torch.linalg.norm(yp - rp) / torch.linalg.norm(rp)).item() <= 1e-5
    # other output vectors: eager again, same results
    yus2 = [torch.empty_like(y) for y in yus]
    yps2 = [torch.empty_like(y) for y in yps]
    batch.apply_stokes(us, ps, yus2, yps2)
    for (ru, rp), yu, yp in zip(refs, yus2, yps2):
        assert (torch.linalg.norm(yu - ru) / torch.linalg.norm(ru)).item() <= 1e-5
