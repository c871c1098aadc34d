"""Sampled rows of the fused constrained Stokes apply on levels too large to assemble: the row
of a P2 node or P1 vertex strictly inside a macro-tet collects the element contributions of
the micro-tets of that macro which contain it (an interior point belongs to no other macro).
The same holds for a point strictly inside a macro face that lies on one of the two spheres
(the face bounds the shell, so no other macro touches it): the constrained rows there apply
the boundary conditions of Sec. 5.1 (Eqs. SaddlePointStructureDirichlet /
InnerSaddlePointSystem) locally — P0 on the inputs of every micro-tet, and at the row's own
node the identity (Dirichlet) or the tangential projection P_v (free-slip).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  FP64.  Element matrices, quadrature and
geometry are those of oracle/fem.py (Sec. 4.1, Sec. 5.1, Eq. SaddlePointStructure); the rows
are sums of element contributions, the definition of the assembled operator.
"""
from __future__ import annotations

import numpy as np

from .mesh import micro_tets_kuhn, kuhn_to_bary, LOCAL_EDGES, CLASS_INNER, CLASS_SURFACE, CLASS_CMB
from .fem import Geometry, element_A, element_B, element_C, BC_DIRICHLET


class MacroRows:
    """Rows of [A B^T; (B+C) 0] at interior points of the macros of a level with 2^L micro
    intervals per macro edge (the same Kuhn subdivision for every macro)."""

    def __init__(self, mesh, L):
        self.mesh, self.L = mesh, L
        n = 2 ** L
        self.n = n
        kt = micro_tets_kuhn(n)                                              # (n^3,4,3)
        self.kt = kt
        F = [2 * kt[:, a] for a in range(4)] + [kt[:, a] + kt[:, b] for (a, b) in LOCAL_EDGES]
        self.F = np.stack(F, axis=1)                                          # (n^3,10,3) fine Kuhn coords
        counts = mesh.counts
        self.n_p2 = counts(2 * n)["total"]
        self.n_p1 = counts(n)["total"]

    def tets_at(self, fine=None, coarse=None):
        """Indices (within a macro) of the micro-tets with a P2 node at fine Kuhn coordinates
        `fine`, or a vertex at Kuhn coordinates `coarse`."""
        if fine is not None:
            return np.nonzero((self.F == np.asarray(fine)).all(axis=-1).any(axis=-1))[0]
        return np.nonzero((self.kt == np.asarray(coarse)).all(axis=-1).any(axis=-1))[0]

    def interior(self, m, sel):
        """True when no P2 node of the micro-tets sel lies on the surface or CMB sphere (so the
        constrained operator acts on them as the raw one): a lattice point is on a sphere when
        all macro vertices with a nonzero barycentric weight lie on it."""
        b = kuhn_to_bary(self.F[sel].reshape(-1, 3), 2 * self.n)
        lay = self.mesh.layer[self.mesh.cells[m]]
        nz = b > 0
        top = np.all(~nz | (lay[None, :] == 1), axis=1)
        bot = np.all(~nz | (lay[None, :] == 0), axis=1)
        return not bool((top | bot).any())

    def contributions(self, m, sel, eta_p1, dlnrho_table, u, p):
        """Element contributions of the micro-tets sel of macro m: (p2 ids (k,10), yu_e (k,30),
        p1 ids (k,4), yp_e (k,4)) for velocity u [3][n_p2] and pressure p [n_p1]."""
        mesh, n = self.mesh, self.n
        kt = self.kt[sel]
        p2 = mesh.node_ids(m, kuhn_to_bary(self.F[sel].reshape(-1, 3), 2 * n), 2 * n).reshape(-1, 10)
        b1 = kuhn_to_bary(kt.reshape(-1, 3), n)
        p1 = mesh.node_ids(m, b1, n).reshape(-1, 4)
        X = mesh.straight(m, b1, n).reshape(-1, 4, 3)
        geo = Geometry(mesh, X, np.full(len(sel), mesh.cell_prism[m]))
        Ae = element_A(geo, np.asarray(eta_p1)[p1])
        Be = element_B(geo)
        Ce = element_C(geo, mesh, dlnrho_table)
        vd = np.concatenate([p2 + c * self.n_p2 for c in range(3)], axis=1)
        ue = np.asarray(u)[vd]
        pe = np.asarray(p)[p1]
        yu = np.einsum("eij,ej->ei", Ae, ue) + np.einsum("eki,ek->ei", Be, pe)
        yp = np.einsum("eki,ei->ek", Be + Ce, ue)
        return p2, yu, p1, yp

    def velocity_row(self, m, fine, eta_p1, dlnrho_table, u, p):
        """(global P2 id, the 3 velocity rows) at the fine point of macro m (strictly inside the
        macro), or None when a micro-tet around it touches a sphere."""
        sel = self.tets_at(fine=fine)
        if len(sel) == 0 or not self.interior(m, sel):
            return None
        p2, yu, _, _ = self.contributions(m, sel, eta_p1, dlnrho_table, u, p)
        loc = (self.F[sel] == np.asarray(fine)).all(axis=-1)                 # (k,10)
        gid = int(p2[loc][0])
        rows = np.zeros(3)
        for c in range(3):
            rows[c] = yu[:, c * 10:(c + 1) * 10][loc].sum()
        return gid, rows

    def pressure_row(self, m, vertex, eta_p1, dlnrho_table, u, p):
        """(global P1 id, the (B + C) u row) at the vertex of macro m (strictly inside the
        macro), or None when a micro-tet around it touches a sphere."""
        sel = self.tets_at(coarse=vertex)
        if len(sel) == 0 or not self.interior(m, sel):
            return None
        _, _, p1, yp = self.contributions(m, sel, eta_p1, dlnrho_table, u, p)
        loc = (self.kt[sel] == np.asarray(vertex)).all(axis=-1)              # (k,4)
        return int(p1[loc][0]), float(yp[loc].sum())

    # ------------------------------------------------------------------ constrained rows
    def _point_owned(self, m, bary):
        """True when the lattice point (barycentrics w.r.t. macro m's vertices) belongs to
        macro m alone: strictly inside it, or strictly inside a face of it on a sphere."""
        if (np.asarray(bary) < 0).any():
            return False
        nz = np.asarray(bary) > 0
        if nz.all():
            return True
        if nz.sum() != 3:
            return False
        lay = self.mesh.layer[self.mesh.cells[m]]
        return bool(np.all(lay[nz] == lay[nz][0]))

    def _node_classes(self, m, sel):
        """Class (inner / surface / CMB) and outward unit normal x/|x| at the blended position of
        every P2 node of the micro-tets sel of macro m: (k,10), (k,10,3)."""
        b = kuhn_to_bary(self.F[sel].reshape(-1, 3), 2 * self.n)
        lay = self.mesh.layer[self.mesh.cells[m]]
        nz = b > 0
        top = np.all(~nz | (lay[None, :] == 1), axis=1)
        bot = np.all(~nz | (lay[None, :] == 0), axis=1)
        cls = np.where(top, CLASS_SURFACE, np.where(bot, CLASS_CMB, CLASS_INNER))
        x = self.mesh.blend(self.mesh.straight(m, b, 2 * self.n), self.mesh.cell_prism[m])
        nrm = x / np.linalg.norm(x, axis=1, keepdims=True)
        return cls.reshape(-1, 10), nrm.reshape(-1, 10, 3)

    def _project_inputs(self, m, sel, ue, bc):
        """P0 on the element velocity vectors ue (k,30), component-major within an element:
        Dirichlet nodes zeroed, free-slip nodes u - (u.n)n."""
        cls, nrm = self._node_classes(m, sel)
        U = ue.reshape(-1, 3, 10).transpose(0, 2, 1).copy()                   # (k,10,3)
        for c, kind in ((CLASS_SURFACE, bc[0]), (CLASS_CMB, bc[1])):
            on = cls == c
            if kind == BC_DIRICHLET:
                U[on] = 0.0
            else:
                un = np.einsum("ij,ij->i", U[on], nrm[on])
                U[on] -= un[:, None] * nrm[on]
        return U.transpose(0, 2, 1).reshape(-1, 30)

    def _constrained_contributions(self, m, sel, eta_p1, dlnrho_table, u, p, bc):
        mesh, n = self.mesh, self.n
        kt = self.kt[sel]
        p2 = mesh.node_ids(m, kuhn_to_bary(self.F[sel].reshape(-1, 3), 2 * n), 2 * n).reshape(-1, 10)
        b1 = kuhn_to_bary(kt.reshape(-1, 3), n)
        p1 = mesh.node_ids(m, b1, n).reshape(-1, 4)
        X = mesh.straight(m, b1, n).reshape(-1, 4, 3)
        geo = Geometry(mesh, X, np.full(len(sel), mesh.cell_prism[m]))
        Ae = element_A(geo, np.asarray(eta_p1)[p1])
        Be = element_B(geo)
        Ce = element_C(geo, mesh, dlnrho_table)
        vd = np.concatenate([p2 + c * self.n_p2 for c in range(3)], axis=1)
        ue = self._project_inputs(m, sel, np.asarray(u)[vd], bc)
        pe = np.asarray(p)[p1]
        yu = np.einsum("eij,ej->ei", Ae, ue) + np.einsum("eki,ek->ei", Be, pe)
        yp = np.einsum("eki,ei->ek", Be + Ce, ue)
        return p2, yu, p1, yp

    def constrained_velocity_row(self, m, fine, eta_p1, dlnrho_table, u, p, bc=(BC_DIRICHLET, 1)):
        """(global P2 id, its 3 rows of the constrained fused apply A_c u + P0 B^T p) at a fine
        point of macro m that belongs to no other macro (see _point_owned), or None.  p is used
        as given (pass it mean-free for the P_p p of the constrained operator); bc = (surface,
        CMB) boundary conditions."""
        b = kuhn_to_bary(np.asarray(fine)[None], 2 * self.n)[0]
        if not self._point_owned(m, b):
            return None
        sel = self.tets_at(fine=fine)
        p2, yu, _, _ = self._constrained_contributions(m, sel, eta_p1, dlnrho_table, u, p, bc)
        loc = (self.F[sel] == np.asarray(fine)).all(axis=-1)                 # (k,10)
        gid = int(p2[loc][0])
        cls, nrm = self._node_classes(m, sel)
        cl, nr = cls[loc][0], nrm[loc][0]
        rows = np.array([yu[:, c * 10:(c + 1) * 10][loc].sum() for c in range(3)])
        kind = {CLASS_SURFACE: bc[0], CLASS_CMB: bc[1]}.get(int(cl))
        if kind == BC_DIRICHLET:
            rows = np.array([u[gid + c * self.n_p2] for c in range(3)], dtype=np.float64)
        elif kind is not None:
            rows = rows - (rows @ nr) * nr
        return gid, rows, int(cl)

    def constrained_pressure_row(self, m, vertex, eta_p1, dlnrho_table, u, p, bc=(BC_DIRICHLET, 1)):
        """(global P1 id, the (B + C) P0 u row) at a vertex of macro m that belongs to no other
        macro, or None (the constrained operator subtracts the output's mean from all rows)."""
        b = kuhn_to_bary(np.asarray(vertex)[None], self.n)[0]
        if not self._point_owned(m, b):
            return None
        sel = self.tets_at(coarse=vertex)
        _, _, p1, yp = self._constrained_contributions(m, sel, eta_p1, dlnrho_table, u, p, bc)
        loc = (self.kt[sel] == np.asarray(vertex)).all(axis=-1)
        return int(p1[loc][0]), float(yp[loc].sum())

    def sphere_faces(self, m):
        """Local faces z (opposite local vertex z) of macro m on a sphere: [(z, layer)],
        layer 1 = surface, 0 = CMB."""
        lay = self.mesh.layer[self.mesh.cells[m]]
        out = []
        for z in range(4):
            rest = np.delete(lay, z)
            if np.all(rest == rest[0]):
                out.append((z, int(rest[0])))
        return out


def face_points(n, z, k, rng):
    """k random Kuhn lattice points (A, B, C) of the lattice with n intervals strictly inside
    the face z of the Kuhn simplex (barycentric z zero, the other three positive)."""
    out = []
    while len(out) < k:
        i = np.sort(rng.integers(1, n, 2))[::-1]
        if i[0] == i[1]:
            continue
        hi, lo = int(i[0]), int(i[1])
        # barycentrics (n - A, A - B, B - C, C); three positive numbers summing to n, z zero
        if z == 0:
            pt = (n, hi, lo)
        elif z == 1:
            pt = (hi, hi, lo)
        elif z == 2:
            pt = (hi, lo, lo)
        else:
            pt = (hi, lo, 0)
        out.append(pt)
    return out


def sample_points(n, k, rng, margin=1):
    """k random Kuhn lattice points (A > B > C) of the lattice with n intervals, at least
    `margin` steps from every face of the Kuhn simplex."""
    out = []
    while len(out) < k:
        A, B, C = np.sort(rng.integers(0, n + 1, 3))[::-1]
        if n - A >= margin and A - B >= margin and B - C >= margin and C >= margin:
            out.append((int(A), int(B), int(C)))
    return out
