"""The macro-tet sharding path on the GPU (one process standing in for the ranks): the library's
partial applies over the ranks' macro ranges, summed on the shared nodes, reproduce the full
constrained apply, and the sharded V-cycle built from library calls (shard.library_level)
reproduces the library's own V-cycle."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2506_04157_gb300 as mfs
from paper_2506_04157_gb300 import shard
import workloads as W

TOL = {torch.float64: 1e-12, torch.float32: 1e-5}


def make(level, bc=("dirichlet", "freeslip")):
    ctx = mfs.Context(0)
    mesh = mfs.Mesh(ctx, level)
    prob = mfs.Problem(mesh, *bc)
    x1 = mesh.coords(level, p2=False).T
    prob.set_viscosity(torch.tensor(W.viscosity_plumes(x1, 7, 1e4), device="cuda"))
    prob.set_density(W.dlnrho_table_compressible())
    return ctx, mesh, prob


def dirichlet_mask(mesh, level, bc):
    cls = mesh.node_class(level)
    d = np.zeros(cls.shape, bool)
    if bc[0] == "dirichlet":
        d |= cls == 1
    if bc[1] == "dirichlet":
        d |= cls == 2
    return d


@pytest.mark.parametrize("n_ranks", [2, 3])
@pytest.mark.parametrize("bc", [("dirichlet", "freeslip"), ("freeslip", "dirichlet")])
@pytest.mark.parametrize("dt", [torch.float64, torch.float32])
@pytest.mark.parametrize("level", [3, 5])
def test_partial_applies_sum_to_full(level, dt, bc, n_ranks):
    ctx, mesh, prob = make(level, bc)
    topo = mesh.macro_topology()
    ranges = shard.macro_ranges(n_ranks)
    inf = mesh.info(level)
    u = torch.tensor(W.random_field(3 * inf.n_p2, 1), dtype=dt, device="cuda")
    p = torch.tensor(W.random_field(inf.n_p1, 2), dtype=dt, device="cuda")
    pm = p - p.mean()
    dm = torch.tensor(np.tile(dirichlet_mask(mesh, level, bc), 3), device="cuda")
    yu, yp = torch.zeros_like(u), torch.zeros_like(p)
    ya = torch.zeros_like(u)
    for m0, m1 in ranges:
        tu, tp, ta = torch.empty_like(u), torch.empty_like(p), torch.empty_like(u)
        prob.apply_part(level, m0, m1, u, tu, pm, tp)
        prob.apply_part(level, m0, m1, u, ta)
        # every range's identity rows hold u at the Dirichlet nodes it touches
        part = shard.Partition(topo, 2 ** (level + 1), ranges, ranges.index((m0, m1)))
        t = torch.tensor(np.tile(part.touched, 3), device="cuda")
        assert torch.equal(tu[dm & t], u[dm & t]) and torch.equal(ta[dm & t], u[dm & t])
        assert (tu[~t] == 0).all() and (ta[~t] == 0).all()
        yu += tu
        yp += tp
        ya += ta
    yu[dm] = u[dm]
    ya[dm] = u[dm]
    yp -= yp.mean()
    ru, rp, ra = torch.empty_like(u), torch.empty_like(p), torch.empty_like(u)
    prob.apply_stokes(level, u, p, ru, rp)
    prob.apply_A(level, u, ra, constrained=True)
    rel = lambda a, b: (torch.linalg.norm((a - b).double()) / torch.linalg.norm(b.double())).item()
    assert rel(yu, ru) <= TOL[dt] and rel(yp, rp) <= TOL[dt] and rel(ya, ra) <= TOL[dt]


def test_partial_apply_refusals():
    ctx, mesh, prob = make(2)
    n = 3 * mesh.info(2).n_p2
    u = torch.zeros(n, dtype=torch.float64, device="cuda")
    for m0, m1 in ((-1, 30), (0, 61), (30, 30)):
        with pytest.raises(mfs.MfsError):
            prob.apply_part(2, m0, m1, u, torch.empty_like(u))


def test_sharded_vcycle_matches_library_vcycle():
    """Two ranks emulated in one process with the library's kernels: the partial applies of both
    ranges summed (shared nodes added, identity rows kept), restriction per owned rows, the
    coarsest level by the library's exact coarse solve.  One V-cycle (3, 2) on level 4 equals
    mfs_vcycle to 1e-10 (FP64)."""
    level, bc = 4, ("dirichlet", "freeslip")
    ctx, mesh, prob = make(level, bc)
    prob.setup_multigrid(1)
    topo = mesh.macro_topology()
    ranges = shard.macro_ranges(2)
    levels = {}
    for l in range(1, level + 1):
        parts = [shard.Partition(topo, 2 ** (l + 1), ranges, r) for r in range(2)]
        per = [shard.library_level(prob, l, *ranges[r], parts[r], device="cuda",
                                   exclude_dirichlet=dirichlet_mask(mesh, l, bc)) for r in range(2)]
        dm = torch.tensor(np.tile(dirichlet_mask(mesh, l, bc), 3), device="cuda")

        def partial(x, y, per=per, dm=dm):
            acc = torch.zeros_like(x)
            for lv in per:
                t = torch.empty_like(x)
                lv.partial_A(x, t)
                acc += t
            acc[dm] = x[dm]
            y.copy_(acc)
        owned = [lv.owned for lv in per]
        R = per[0].restrict
        restrict = (lambda r, R=R, owned=owned: sum(R(r * o) for o in owned)) if R else None
        one = shard.Partition(topo, 2 ** (l + 1), [(0, 60)], 0)
        levels[l] = shard.ShardedLevel(partial, per[0].dinv, per[0].project, shard.Exchange(one, 3, device="cuda"),
                                       prob.cheb_bounds(l) if l > 1 else (1.0, 2.0), restrict, per[0].prolong,
                                       torch.ones(3 * one.n, dtype=torch.float64, device="cuda"))

    def coarse(bc_full):
        x = torch.zeros_like(bc_full)
        prob.vcycle(1, bc_full, x, 3, 2)
        return x
    V = shard.ShardedVCycle(levels, 1, coarse)
    inf = mesh.info(level)
    b = torch.tensor(W.random_field(3 * inf.n_p2, 9), device="cuda")
    prob.project(level, b)
    x = V(level, b, 3, 2)
    ref = torch.zeros_like(b)
    prob.vcycle(level, b, ref, 3, 2)
    assert (torch.linalg.norm(x - ref) / torch.linalg.norm(ref)).item() <= 1e-10
