"""Sharding of the matrix-free hot path by macro-tets (one rank per GPU).

The hybrid hierarchical grid of arxiv 2506.04157 (Sec. 4.1) refines every macro-tet on its
own: each micro-tet, and so each element contribution, belongs to exactly one macro, and
the only nodes two macros share are those on a common macro vertex, edge or face.  A rank
therefore owns a range of macros and

  * applies the operator to the micro-tets of its macros only (mfs_apply_part, or any
    callable with the same meaning),
  * sums the partial results on the shared nodes over the ranks (one all-reduce of the packed
    interface entries per operator application),
  * evaluates dot products over the nodes it owns (each node has one owner: the lowest rank
    touching it) and sums the scalars over the ranks,
  * replicates the coarsest multigrid level (2,430 velocity dofs on level 1).

Every rank holds the whole mesh and full-length vectors in the global numbering; an entry is
meaningful on a rank where the rank's macros touch the node ("consistent on the touched
nodes").  Identity rows of Dirichlet nodes need no exchange: every rank touching such a node
writes the same value.

The module holds the partition, the exchange, the distributed reductions and the distributed
operator / Chebyshev / V-cycle / preconditioned CG orchestration; the arithmetic of every step comes from the
callables it is given (the library's kernels on the GPU).  torch.distributed provides the
all-reduce (NCCL between GPUs, gloo between CPU processes).
"""
from __future__ import annotations

import numpy as np

N_MACROS, N_PRISMS = 60, 20
N_VERTS, N_EDGES, N_FACES = 24, 102, 140


def macro_ranges(n_ranks):
    """Contiguous macro ranges [m0, m1) per rank.  The macros are numbered three per prism, so
    the ranges follow prism boundaries: the 20 prisms are split as evenly as possible."""
    if not 1 <= n_ranks <= N_PRISMS:
        raise ValueError(f"1 <= n_ranks <= {N_PRISMS}")
    bounds = [round(k * N_PRISMS / n_ranks) for k in range(n_ranks + 1)]
    return [(3 * bounds[k], 3 * bounds[k + 1]) for k in range(n_ranks)]


def numbering(N):
    """Offsets of the global lattice numbering with N intervals per macro edge (vertices,
    then edge, face and cell interiors; the layout documented in include/mfs.h)."""
    nE1 = max(N - 1, 0)
    nF1 = (N - 1) * (N - 2) // 2 if N > 2 else 0
    nC1 = (N - 1) * (N - 2) * (N - 3) // 6 if N > 3 else 0
    offE = N_VERTS
    offF = offE + N_EDGES * nE1
    offC = offF + N_FACES * nF1
    return dict(N=N, nE1=nE1, nF1=nF1, nC1=nC1, offE=offE, offF=offF, offC=offC,
                total=offC + N_MACROS * nC1)


class Partition:
    """Which lattice points of one level each rank touches, owns and shares.

    topology: (cells [60,4], edges [60,6], faces [60,4]) from Mesh.macro_topology();
    N: intervals per macro edge of the lattice (2^(l+1) for the P2 nodes of level l, 2^l for
    its P1 vertices); ranges: per-rank macro ranges; rank: this process's rank."""

    def __init__(self, topology, N, ranges, rank):
        cells, edges, faces = (np.asarray(a) for a in topology)
        self.nb = nb = numbering(N)
        self.n = nb["total"]
        self.ranges, self.rank = ranges, rank
        R = len(ranges)
        # which ranks touch each entity
        touch_v = np.zeros((R, N_VERTS), bool)
        touch_e = np.zeros((R, N_EDGES), bool)
        touch_f = np.zeros((R, N_FACES), bool)
        for r, (m0, m1) in enumerate(ranges):
            touch_v[r, cells[m0:m1].ravel()] = True
            touch_e[r, edges[m0:m1].ravel()] = True
            touch_f[r, faces[m0:m1].ravel()] = True
        owner_v = np.argmax(touch_v, axis=0)
        owner_e = np.argmax(touch_e, axis=0)
        owner_f = np.argmax(touch_f, axis=0)
        node_owner = np.full(self.n, -1, np.int64)
        touched = np.zeros(self.n, bool)
        iface = np.zeros(self.n, bool)

        def span(ids, off, cnt):
            ids = np.asarray(ids, np.int64)
            return (off + ids[:, None] * cnt + np.arange(cnt)[None, :]).ravel()

        groups = [(np.arange(N_VERTS), lambda i: np.asarray(i, np.int64), touch_v, owner_v)]
        if nb["nE1"]:
            groups.append((np.arange(N_EDGES), lambda i: span(i, nb["offE"], nb["nE1"]), touch_e, owner_e))
        if nb["nF1"]:
            groups.append((np.arange(N_FACES), lambda i: span(i, nb["offF"], nb["nF1"]), touch_f, owner_f))
        for ids, nodes_of, touch, owner in groups:
            used = touch.any(axis=0)
            ids = ids[used]
            nodes = nodes_of(ids)
            per = len(nodes) // max(len(ids), 1)
            node_owner[nodes] = np.repeat(owner[ids], per)
            touched[nodes] = np.repeat(touch[rank, ids], per)
            iface[nodes] = np.repeat(touch[:, ids].sum(axis=0) >= 2, per)
        if nb["nC1"]:
            for r, (m0, m1) in enumerate(ranges):
                nodes = span(np.arange(m0, m1), nb["offC"], nb["nC1"])
                node_owner[nodes] = r
                if r == rank:
                    touched[nodes] = True
        assert (node_owner >= 0).all()
        self.owner = node_owner
        self.touched = touched
        self.owned = node_owner == rank
        self.interface = np.flatnonzero(iface)          # the same list on every rank

    def macro_range(self):
        return self.ranges[self.rank]


class Exchange:
    """Sum over the ranks of the interface entries of a vector with `comps` component blocks
    ([comps][n], component-major): gather into one buffer, all-reduce, scatter back.
    exclude: node mask (length n) of entries left out (e.g. Dirichlet nodes, whose identity
    rows every rank already holds)."""

    def __init__(self, part, comps=1, exclude=None, group=None, device=None):
        import torch
        idx = part.interface
        if exclude is not None:
            idx = idx[~np.asarray(exclude)[idx]]
        full = np.concatenate([idx + c * part.n for c in range(comps)])
        self.idx = torch.as_tensor(full, dtype=torch.int64, device=device)
        self.group = group
        self.size = full.size

    def sum_interface(self, x):
        import torch.distributed as dist
        if self.size == 0 or not dist.is_initialized() or dist.get_world_size(self.group) == 1:
            return x
        buf = x.index_select(0, self.idx)
        dist.all_reduce(buf, op=dist.ReduceOp.SUM, group=self.group)
        x.index_copy_(0, self.idx, buf)
        return x


class Reducer:
    """Global reductions over owned entries (each node counted once over the ranks)."""

    def __init__(self, part, comps=1, group=None, device=None):
        import torch
        m = np.tile(part.owned, comps).astype(np.float64)
        self.mask64 = torch.as_tensor(m, device=device)
        self.n = part.n * comps
        self.group = group

    def _allreduce(self, v):
        import torch.distributed as dist
        if dist.is_initialized() and dist.get_world_size(self.group) > 1:
            dist.all_reduce(v, op=dist.ReduceOp.SUM, group=self.group)
        return v

    def dot(self, x, y):
        """sum_i x_i y_i over all nodes (FP64 accumulation)."""
        v = (x.double() * y.double() * self.mask64).sum().reshape(1)
        return float(self._allreduce(v).item())

    def total(self, x):
        v = (x.double() * self.mask64).sum().reshape(1)
        return float(self._allreduce(v).item())

    def remove_mean(self, x):
        """x <- x - mean(x) over the global vector (P_p of Sec. 5.1)."""
        x -= self.total(x) / self.n
        return x


class ShardedStokes:
    """The constrained fused operator [A_c, B^T_c; Bbar_c, 0] of one level on the macro range
    of this rank.  partial(u, p, yu, yp): the range's contributions with p used as given and
    no mean removal (mfs_apply_part's meaning); inputs consistent on the touched nodes,
    outputs consistent on the touched nodes after the call."""

    def __init__(self, partial, ex_u, ex_p, red_p):
        self.partial, self.ex_u, self.ex_p, self.red_p = partial, ex_u, ex_p, red_p

    def apply(self, u, p, yu, yp):
        pm = self.red_p.remove_mean(p.clone())
        self.partial(u, pm, yu, yp)
        self.ex_u.sum_interface(yu)
        self.ex_p.sum_interface(yp)
        self.red_p.remove_mean(yp)
        return yu, yp


class ShardedLevel:
    """One multigrid level of A_c on this rank: partial_A(x, y) (the range's contributions to
    A_c x, mfs_apply_part with fused = 0), dinv (inverse diagonal, consistent), project(x)
    (P0 in place, pointwise), the exchange of the level's velocity vectors, the Chebyshev
    interval, and for l > l_min restrict(r) -> P0_c P^T r and prolong(xc) -> P0 P xc (full-
    vector transfers of the level pair)."""

    def __init__(self, partial_A, dinv, project, exchange, bounds, restrict=None, prolong=None, owned=None):
        self.partial_A, self.dinv, self.project, self.ex = partial_A, dinv, project, exchange
        self.bounds, self.restrict, self.prolong = bounds, restrict, prolong
        self.owned = owned          # velocity-entry mask of the nodes this rank owns

    def A(self, x):
        import torch
        y = torch.empty_like(x)
        self.partial_A(x, y)
        return self.ex.sum_interface(y)


class ShardedVCycle:
    """The multigrid V-cycle of the A block (Sec. 5.2: Jacobi-preconditioned Chebyshev smoothing,
    P2 transfers, coarsest level solved exactly) over macro-sharded levels.  levels: dict
    l -> ShardedLevel for l_min..l_max; coarse_solve(b_full) -> x_full on the coarsest level,
    replicated: the coarse right-hand side is completed by an all-reduce of the owned entries
    first.  Restriction sums owned fine rows only (partial P^T) and then the coarse interface,
    so every fine contribution enters once; prolongation is local (a fine node's stencil lies in
    its macro)."""

    def __init__(self, levels, l_min, coarse_solve, group=None):
        self.levels, self.l_min, self.coarse_solve, self.group = levels, l_min, coarse_solve, group

    def chebyshev(self, lv, x, b, steps, degree):
        lo, hi = lv.bounds
        theta, delta = 0.5 * (hi + lo), 0.5 * (hi - lo)
        sigma1 = theta / delta
        x = x.clone()
        for _ in range(steps):
            r = b - lv.A(x)
            z = lv.project(lv.dinv * r)
            rho = 1.0 / sigma1
            d = z / theta
            for k in range(1, degree + 1):
                x = x + d
                if k == degree:
                    break
                r = r - lv.A(d)
                z = lv.project(lv.dinv * r)
                rho_new = 1.0 / (2.0 * sigma1 - rho)
                d = rho_new * rho * d + (2.0 * rho_new / delta) * z
                rho = rho_new
        return x

    def _complete(self, lv, x):
        """The full vector from the owned entries of every rank (all-reduce)."""
        import torch.distributed as dist
        y = x * lv.owned
        if dist.is_initialized() and dist.get_world_size(self.group) > 1:
            dist.all_reduce(y, op=dist.ReduceOp.SUM, group=self.group)
        return y

    def __call__(self, l, b, steps=3, degree=2, x=None):
        import torch
        lv = self.levels[l]
        if l == self.l_min:
            return self.coarse_solve(self._complete(lv, b))
        if x is None:
            x = torch.zeros_like(b)
        x = self.chebyshev(lv, x, b, steps, degree)
        r = b - lv.A(x)
        rc = lv.restrict(r * lv.owned)
        self.levels[l - 1].ex.sum_interface(rc)
        ec = self(l - 1, rc, steps, degree)
        x = x + lv.prolong(ec)
        return self.chebyshev(lv, x, b, steps, degree)


class ShardedPCG:
    """Preconditioned conjugate gradients on the constrained A block of one level (the A-block
    solve of the Uzawa preconditioner, Sec. 5.2, with the multigrid V-cycle as preconditioner)
    over macro-sharded levels: A x by the sharded operator (partial sums and the interface
    exchange), the preconditioner a callable on consistent vectors (by default the sharded
    V-cycle of the level), and every inner product over the owned entries summed over the
    ranks (reducer.dot), so that all ranks take the same step lengths and stop at the same
    iteration.  b and the returned x are full-length and consistent on the touched nodes."""

    def __init__(self, vcycle, level, reducer, steps=3, degree=2, precond=None):
        self.level_op = vcycle.levels[level]
        self.red = reducer
        self.precond = precond if precond is not None else (lambda r: vcycle(level, r, steps, degree))

    def solve(self, b, x=None, rtol=1e-8, max_iters=200, fixed_iters=None):
        """(x, iterations, residual norms per iteration); stops at ||r|| <= rtol ||r0||, or
        after exactly fixed_iters iterations when given."""
        import math
        import torch
        A = self.level_op.A
        x = torch.zeros_like(b) if x is None else x.clone()
        r = b - A(x)
        r0 = math.sqrt(self.red.dot(r, r))
        hist = [r0]
        if r0 == 0.0:
            return x, 0, hist
        z = self.precond(r)
        p = z.clone()
        rz = self.red.dot(r, z)
        n = fixed_iters if fixed_iters is not None else max_iters
        for it in range(1, n + 1):
            q = A(p)
            alpha = rz / self.red.dot(p, q)
            x = x + alpha * p
            r = r - alpha * q
            hist.append(math.sqrt(self.red.dot(r, r)))
            if fixed_iters is None and hist[-1] <= rtol * r0:
                return x, it, hist
            z = self.precond(r)
            rz_new = self.red.dot(r, z)
            p = z + (rz_new / rz) * p
            rz = rz_new
        return x, n, hist


def library_level(prob, level, m0, m1, part, group=None, device=None, bounds=None, exclude_dirichlet=None):
    """A ShardedLevel backed by the library's kernels on this rank's GPU: mfs_apply_part for the
    partial A, mfs_diag_A, mfs_project, mfs_restrict / mfs_prolongate (multigrid set up on the
    problem).  exclude_dirichlet: node mask of the level's Dirichlet nodes."""
    import torch
    info = prob.mesh.info(level)
    n3 = 3 * info.n_p2
    dinv = torch.empty(n3, dtype=torch.float64, device=device)
    prob.diag_A(level, dinv)
    dinv = 1.0 / dinv

    def partial_A(x, y):
        prob.apply_part(level, m0, m1, x, y)

    def project(x):
        prob.project(level, x)
        return x

    restrict = prolong = None
    if level > 0:
        def restrict(r):
            rc = torch.empty(3 * prob.mesh.info(level - 1).n_p2, dtype=r.dtype, device=r.device)
            prob.restrict(level, r, rc)
            return rc

        def prolong(xc):
            xf = torch.empty(n3, dtype=xc.dtype, device=xc.device)
            prob.prolongate(level, xc, xf)
            return xf

    if bounds is None:
        from . import MfsError
        try:
            bounds = prob.cheb_bounds(level)
        except MfsError:            # the coarsest level has no smoother
            bounds = None
    ex = Exchange(part, comps=3, exclude=exclude_dirichlet, group=group, device=device)
    owned = torch.as_tensor(np.tile(part.owned, 3).astype(np.float64), device=device)
    return ShardedLevel(partial_A, dinv, project, ex, bounds, restrict, prolong, owned)
