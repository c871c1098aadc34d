"""Sampled rows of the fused constrained Stokes apply on levels too large to assemble: the row
of a P2 node or P1 vertex strictly inside a macro-tet collects the element contributions of
the micro-tets of that macro which contain it (an interior point belongs to no other macro).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  FP64.  Element matrices, quadrature and
geometry are those of oracle/fem.py (Sec. 4.1, Sec. 5.1, Eq. SaddlePointStructure); the rows
are sums of element contributions, the definition of the assembled operator.
"""
from __future__ import annotations

import numpy as np

from .mesh import micro_tets_kuhn, kuhn_to_bary, LOCAL_EDGES
from .fem import Geometry, element_A, element_B, element_C


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


def sample_points(n, k, rng, margin=1):
    """k random Kuhn lattice points (A > B > C) of the lattice with n intervals, at least
    `margin` steps from every face of the Kuhn simplex."""
    out = []
    while len(out) < k:
        A, B, C = np.sort(rng.integers(0, n + 1, 3))[::-1]
        if n - A >= margin and A - B >= margin and B - C >= margin and C >= margin:
            out.append((int(A), int(B), int(C)))
    return out
