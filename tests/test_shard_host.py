"""Macro-tet sharding (paper_2506_04157_gb300/shard.py) on CPU with two gloo ranks.

Each rank owns half of the macro-tets (prism-aligned ranges); its partial operator is the
oracle's element sum over the micro-tets of its macros with the constrained arithmetic of
Sec. 5.1 (P0 on the inputs, P_v on the free-slip outputs, identity rows at the Dirichlet
nodes it touches), standing in for mfs_apply_part.  The two-rank results of the fused apply,
the dot products, the mean removal, one V-cycle and a preconditioned CG on the A block are
checked
  * bit for bit against a one-process evaluation that groups the same partial sums the same
    way (rank 0's part + rank 1's part on shared nodes, owned fine rows restricted per rank),
  * and against the unsharded oracle (ConstrainedOperators, Hierarchy.vcycle) to 1e-12.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

LEVEL = 3
STEPS, DEGREE = 2, 2
CG_ITERS = 10


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _setup():
    import workloads as W
    import paper_2506_04157_gb300 as mfs
    from oracle.mesh import MacroMesh, Level
    from oracle.solver import Hierarchy
    mesh = MacroMesh()
    Lf = Level(mesh, LEVEL)
    eta = W.viscosity_plumes(Lf.p1_x, seed=7, contrast=1e4)
    dl = W.dlnrho_table_compressible()
    H = Hierarchy(mesh, LEVEL, eta, dlnrho_table=dl, bc=(0, 1))
    topo = mfs.Mesh(None, LEVEL).macro_topology()
    assert np.array_equal(np.sort(topo[0], axis=1), np.sort(mesh.cells, axis=1))
    return H, dl, topo


def _partial_A(H, dl, l, m0, m1, touched):
    """Contributions of the micro-tets of macros [m0, m1) to A_c x (constrained arithmetic)."""
    from oracle.fem import stokes_apply_elements
    L, cons = H.levels[l], H.cons[l]
    sel = np.flatnonzero((L.tet_macro >= m0) & (L.tet_macro < m1))
    dmask = np.tile(cons.dirichlet & touched, 3)

    def f(x, y):
        xn = x.numpy()
        yu, _ = stokes_apply_elements(L, H.etas[l], dl, cons.P0(xn), np.zeros(L.n_p1), sel)
        yu = cons.P0(yu)
        yu[dmask] = xn[dmask]
        y.copy_(torch.from_numpy(yu))
    return f


def _partial_fused(H, dl, m0, m1, touched):
    """Contributions of macros [m0, m1) to [A_c u + P0 B^T p; (B + C) P0 u] (p as given)."""
    from oracle.fem import stokes_apply_elements
    l = H.l_max
    L, cons = H.levels[l], H.cons[l]
    sel = np.flatnonzero((L.tet_macro >= m0) & (L.tet_macro < m1))
    dmask = np.tile(cons.dirichlet & touched, 3)

    def f(u, p, yu, yp):
        un = u.numpy()
        a, b = stokes_apply_elements(L, H.etas[l], dl, cons.P0(un), p.numpy(), sel)
        a = cons.P0(a)
        a[dmask] = un[dmask]
        yu.copy_(torch.from_numpy(a))
        yp.copy_(torch.from_numpy(b))
    return f


def _levels(H, dl, topo, ranges, rank, emulate):
    """ShardedLevel per multigrid level for `rank` of `ranges`; emulate: one process holding
    both ranks' partial sums grouped as the two-rank run groups them."""
    from paper_2506_04157_gb300 import shard
    levels = {}
    for l in range(H.l_min, H.l_max + 1):
        N = 2 ** (l + 1)
        parts = [shard.Partition(topo, N, ranges, r) for r in range(len(ranges))]
        cons = H.cons[l]
        dinv = torch.from_numpy(1.0 / H.diag[l])
        proj = lambda x, c=cons: torch.from_numpy(c.P0(x.numpy()))
        P = H.P.get(l)
        restrict = (lambda r, P=P, c=H.cons[l - 1]: torch.from_numpy(c.P0(P.T @ r.numpy()))) if P is not None else None
        prolong = (lambda xc, P=P, c=cons: torch.from_numpy(c.P0(P @ xc.numpy()))) if P is not None else None
        if emulate:
            fs = [_partial_A(H, dl, l, *ranges[r], parts[r].touched) for r in range(len(ranges))]
            dm = np.tile(cons.dirichlet, 3)

            def partial(x, y, fs=fs, dm=dm):
                acc = None
                for f in fs:
                    t = torch.empty_like(x)
                    f(x, t)
                    acc = t if acc is None else acc + t
                acc[dm] = x[dm]
                y.copy_(acc)
            owned = [torch.from_numpy(np.tile(p.owned, 3).astype(np.float64)) for p in parts]
            if restrict is not None:
                restrict = (lambda r, R=restrict, owned=owned: sum(R(r * o) for o in owned))
            ex = shard.Exchange(shard.Partition(topo, N, [(0, 60)], 0), comps=3)
            lv = shard.ShardedLevel(partial, dinv, proj, ex, H.bounds.get(l, (1.0, 2.0)),
                                    (lambda r, R=restrict: R(r)) if restrict else None, prolong,
                                    torch.ones(3 * parts[0].n, dtype=torch.float64))
        else:
            part = parts[rank]
            ex = shard.Exchange(part, comps=3, exclude=cons.dirichlet)
            lv = shard.ShardedLevel(_partial_A(H, dl, l, *ranges[rank], part.touched), dinv, proj, ex,
                                    H.bounds.get(l, (1.0, 2.0)), restrict, prolong,
                                    torch.from_numpy(np.tile(part.owned, 3).astype(np.float64)))
        levels[l] = lv
    return levels


class _GroupedReducer:
    """One-process stand-in for shard.Reducer over several ranks: the owned-entry sums of each
    rank computed apart and added in rank order, as the two-rank all-reduce adds them."""

    def __init__(self, parts, comps=1):
        self.masks = [torch.from_numpy(np.tile(p.owned, comps).astype(np.float64)) for p in parts]
        self.n = parts[0].n * comps

    def total(self, x):
        out = 0.0
        for m in self.masks:
            out = out + (x.double() * m).sum().reshape(1)
        return float(out.item())

    def dot(self, x, y):
        out = 0.0
        for m in self.masks:
            out = out + (x.double() * y.double() * m).sum().reshape(1)
        return float(out.item())

    def remove_mean(self, x):
        x -= self.total(x) / self.n
        return x


def _compute(rank, ranges, emulate, full=True):
    import workloads as W
    from paper_2506_04157_gb300 import shard
    H, dl, topo = _setup()
    L = H.levels[H.l_max]
    n2, n1 = L.n_p2, L.n_p1
    u = torch.from_numpy(W.random_field(3 * n2, 3))
    p = torch.from_numpy(W.random_field(n1, 4))
    b = torch.from_numpy(H.cons[H.l_max].P0(W.random_field(3 * n2, 5)))
    part2 = shard.Partition(topo, 2 ** (H.l_max + 1), ranges, rank)
    part1 = shard.Partition(topo, 2 ** H.l_max, ranges, rank)
    if emulate:
        one2 = shard.Partition(topo, 2 ** (H.l_max + 1), [(0, 60)], 0)
        one1 = shard.Partition(topo, 2 ** H.l_max, [(0, 60)], 0)
        t2 = [shard.Partition(topo, 2 ** (H.l_max + 1), ranges, r).touched for r in range(len(ranges))]
        fs = [_partial_fused(H, dl, *ranges[r], t2[r]) for r in range(len(ranges))]
        dm = np.tile(H.cons[H.l_max].dirichlet, 3)

        def fused(u_, p_, yu, yp):
            a, c = None, None
            for f in fs:
                ta, tc = torch.empty_like(u_), torch.empty_like(p_)
                f(u_, p_, ta, tc)
                a = ta if a is None else a + ta
                c = tc if c is None else c + tc
            a[dm] = u_[dm]
            yu.copy_(a)
            yp.copy_(c)
        all1 = [shard.Partition(topo, 2 ** H.l_max, ranges, r) for r in range(len(ranges))]
        all2 = [shard.Partition(topo, 2 ** (H.l_max + 1), ranges, r) for r in range(len(ranges))]
        op = shard.ShardedStokes(fused, shard.Exchange(one2, 3), shard.Exchange(one1, 1), _GroupedReducer(all1))
        red_u = _GroupedReducer(all2, comps=3)
    else:
        op = shard.ShardedStokes(_partial_fused(H, dl, *ranges[rank], part2.touched),
                                 shard.Exchange(part2, 3, exclude=H.cons[H.l_max].dirichlet), shard.Exchange(part1, 1),
                                 shard.Reducer(part1))
        red_u = shard.Reducer(part2, comps=3)
    yu, yp = torch.empty_like(u), torch.empty_like(p)
    op.apply(u, p, yu, yp)
    dots = (red_u.dot(u, yu), red_u.dot(b, b))
    if not full:
        return dict(yu=yu.numpy(), yp=yp.numpy(), dots=dots, touched2=np.tile(part2.touched, 3),
                    touched1=part1.touched)
    levels = _levels(H, dl, topo, ranges, rank, emulate)
    coarse = lambda bc: torch.from_numpy(H.vcycle(H.l_min, bc.numpy(), STEPS, DEGREE, coarse_exact=True))
    V = shard.ShardedVCycle(levels, H.l_min, coarse)
    x = V(H.l_max, b, STEPS, DEGREE)
    lv = levels[H.l_max]
    jacobi = lambda r: lv.project(lv.dinv * r)
    xc, its, hist = shard.ShardedPCG(V, H.l_max, red_u, precond=jacobi).solve(b, fixed_iters=CG_ITERS)
    return dict(yu=yu.numpy(), yp=yp.numpy(), x=x.numpy(), dots=dots, cg=(xc.numpy(), its, hist),
                touched2=np.tile(part2.touched, 3), touched1=part1.touched)


def _worker(rank, world, port, q, full=True):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_2506_04157_gb300 import shard
        out = _compute(rank, shard.macro_ranges(world), emulate=False, full=full)
        q.put((rank, out))
    finally:
        dist.destroy_process_group()


def _run_ranks(world, full):
    from paper_2506_04157_gb300 import shard
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q, full)) for r in range(world)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=600) for _ in procs)
    for p in procs:
        p.join(timeout=60)
    emu = _compute(0, shard.macro_ranges(world), emulate=True, full=full)
    H, dl, topo = _setup()
    return got, emu, H, dl


@pytest.fixture(scope="module")
def results():
    return _run_ranks(2, full=True)


def test_partition_covers_every_node_once():
    from paper_2506_04157_gb300 import shard
    H, dl, topo = _setup()
    for R in (2, 3, 4):
        ranges = shard.macro_ranges(R)
        assert ranges[0][0] == 0 and ranges[-1][1] == 60
        for N in (4, 8, 16):
            parts = [shard.Partition(topo, N, ranges, r) for r in range(R)]
            owned = np.sum([p.owned for p in parts], axis=0)
            assert (owned == 1).all()                       # one owner per node
            touched = np.sum([p.touched for p in parts], axis=0)
            assert (touched >= 1).all()
            shared = touched >= 2
            assert np.array_equal(np.flatnonzero(shared), parts[0].interface)
            for p in parts:
                assert (p.touched[p.owned]).all()


def test_fused_apply_two_ranks(results):
    got, emu, H, dl = results
    co = H.co[H.l_max]
    import workloads as W
    L = H.levels[H.l_max]
    u = W.random_field(3 * L.n_p2, 3)
    p = W.random_field(L.n_p1, 4)
    ref_u = co.apply_A(u) + co.apply_BT(p)
    ref_p = co.apply_Bbar(u)
    for r in (0, 1):
        t2, t1 = got[r]["touched2"], got[r]["touched1"]
        # bit for bit against the same grouping of partial sums in one process
        assert np.array_equal(got[r]["yu"][t2], emu["yu"][t2])
        assert np.array_equal(got[r]["yp"][t1], emu["yp"][t1])
        # and against the unsharded oracle
        assert np.linalg.norm(got[r]["yu"][t2] - ref_u[t2]) <= 1e-12 * np.linalg.norm(ref_u[t2])
        assert np.linalg.norm(got[r]["yp"][t1] - ref_p[t1]) <= 1e-12 * np.linalg.norm(ref_p[t1])
    # every node is touched by some rank, so the ranks together hold the whole vector
    assert (got[0]["touched2"] | got[1]["touched2"]).all()


def test_dot_products_two_ranks(results):
    got, emu, H, dl = results
    for k in (0, 1):
        assert got[0]["dots"][k] == got[1]["dots"][k] == emu["dots"][k]


def test_vcycle_two_ranks(results):
    """One V-cycle (Chebyshev (2, 2), P2 transfers, exact coarse solve) of the sharded A block:
    bit for bit against the same grouping in one process, and equal to the oracle's unsharded
    V-cycle to 1e-12."""
    got, emu, H, dl = results
    import workloads as W
    L = H.levels[H.l_max]
    b = H.cons[H.l_max].P0(W.random_field(3 * L.n_p2, 5))
    ref = H.vcycle(H.l_max, b, STEPS, DEGREE, coarse_exact=True)
    for r in (0, 1):
        t2 = got[r]["touched2"]
        assert np.array_equal(got[r]["x"][t2], emu["x"][t2])
        assert np.linalg.norm(got[r]["x"][t2] - ref[t2]) <= 1e-12 * np.linalg.norm(ref[t2])


def test_pcg_two_ranks(results):
    """Preconditioned CG on the constrained A block (Jacobi preconditioner, P0-projected; the
    V-cycle preconditioner is checked on its own above), 10 iterations: the two ranks take the
    same steps (residual histories equal, bit for bit against the same grouping in one process)
    and their iterate equals the oracle's own PCG (Sec. 5.2) to 1e-9."""
    got, emu, H, dl = results
    import workloads as W
    from oracle.solver import cg
    L = H.levels[H.l_max]
    cons = H.cons[H.l_max]
    b = cons.P0(W.random_field(3 * L.n_p2, 5))
    M = lambda r: cons.P0(r / H.diag[H.l_max])
    ref, ref_it = cg(H.co[H.l_max].apply_A, b, M=M, fixed_iters=CG_ITERS)
    assert ref_it == CG_ITERS
    for r in (0, 1):
        xc, its, hist = got[r]["cg"]
        t2 = got[r]["touched2"]
        assert its == CG_ITERS and hist == emu["cg"][2]
        assert np.array_equal(xc[t2], emu["cg"][0][t2])
        assert np.linalg.norm(xc[t2] - ref[t2]) <= 1e-9 * np.linalg.norm(ref[t2])
        assert hist[-1] < hist[0]
    assert got[0]["cg"][2] == got[1]["cg"][2]


def test_fused_apply_and_dots_three_ranks():
    """Three gloo ranks (prism-aligned ranges of 21, 18 and 21 macros): an uneven split and
    interface points shared by all three ranges.  With three ranks the all-reduce adds the
    partial sums in an association of its own, so the comparison with the one-process grouping
    is to rounding (1e-14) rather than bit for bit; every rank holds the same interface sums
    and the same dot products (bit for bit), and the fused apply equals the unsharded oracle to
    1e-12 on every rank's touched nodes."""
    got, emu, H, dl = _run_ranks(3, full=False)
    import workloads as W
    co = H.co[H.l_max]
    L = H.levels[H.l_max]
    u = W.random_field(3 * L.n_p2, 3)
    p = W.random_field(L.n_p1, 4)
    ref_u = co.apply_A(u) + co.apply_BT(p)
    ref_p = co.apply_Bbar(u)
    for r in range(3):
        t2, t1 = got[r]["touched2"], got[r]["touched1"]
        assert np.linalg.norm(got[r]["yu"][t2] - emu["yu"][t2]) <= 1e-14 * np.linalg.norm(emu["yu"][t2])
        assert np.linalg.norm(got[r]["yp"][t1] - emu["yp"][t1]) <= 1e-14 * np.linalg.norm(emu["yp"][t1])
        assert np.linalg.norm(got[r]["yu"][t2] - ref_u[t2]) <= 1e-12 * np.linalg.norm(ref_u[t2])
        assert np.linalg.norm(got[r]["yp"][t1] - ref_p[t1]) <= 1e-12 * np.linalg.norm(ref_p[t1])
        for k in (0, 1):
            assert got[r]["dots"][k] == got[0]["dots"][k]
            assert abs(got[r]["dots"][k] - emu["dots"][k]) <= 1e-14 * abs(emu["dots"][k])
        for q in range(3):          # the ranks agree on the points both touch
            both2 = got[r]["touched2"] & got[q]["touched2"]
            both1 = got[r]["touched1"] & got[q]["touched1"]
            assert np.array_equal(got[r]["yu"][both2], got[q]["yu"][both2])
            assert np.array_equal(got[r]["yp"][both1], got[q]["yp"][both1])
    assert (got[0]["touched2"] | got[1]["touched2"] | got[2]["touched2"]).all()
