"""Oracle mesh: icosahedral shell macro mesh, uniform refinement, node numbering, blending.

TEST INFRASTRUCTURE ONLY.  This package is the plain FP64 CPU oracle that the CUDA
library is checked against.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it.  It shares
no code with ``paper_2506_04157_gb300``.

Paper passages followed (arxiv 2506.04157):
  * Sec. 4.1 (Mesh and Blending): icosahedral shell built from truncated pyramids
    (one radial layer here), each cut into tetrahedra, then uniformly refined
    [Bey95]; a blending map B from the straight macro mesh onto the shell,
    C^0 globally and C^1 on each macro-element (Fig. BlendedDomain).
  * Sec. 4.2 / Eq. (Lagrange): P2 nodes are the vertex and edge-midpoint Lagrange
    points, split into inner, surface and CMB sets.

Readings where the paper is silent:
  * Prism split: each quad face of a prism is cut along the diagonal through its
    lowest-numbered vertex; with bottom vertices a<b<c and tops a'<b'<c' this gives
    the tets (a,b,c,c'), (a,b,c',b'), (a,b',c',a').
  * Refinement: every macro-tet, with its vertices in increasing global order, is
    identified with the Kuhn simplex {n >= x1 >= x2 >= x3 >= 0} and cut by
    Freudenthal's rule into n^3 = 8^L congruent micro-tets.  The restriction to any
    face is the uniform "red" triangle refinement, so neighbours conform.
  * Blending: with unit prism normal nh and plane offset delta = V.nh of the
    icosahedral face, B(x) = (x.nh / delta) * x / |x|: radial projection that maps
    the plane x.nh = r*delta onto the sphere of radius r.
  * Numbering (the library's vector layout, documented in include/mfs.h): P1
    vertices of level l (N = 2^l intervals per macro edge) are numbered macro
    vertices first, then macro-edge interiors, macro-face interiors, macro-cell
    interiors; P2 nodes of level l are the P1 vertices of level l+1.
"""
from __future__ import annotations

import numpy as np

PHI = (1.0 + 5.0 ** 0.5) / 2.0
N_MACRO_VERTS = 24
N_MACRO_EDGES = 102
N_MACRO_FACES = 140
N_MACRO_CELLS = 60

# local edge order of a tetrahedron (pairs of local vertex ids)
LOCAL_EDGES = [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)]

CLASS_INNER, CLASS_SURFACE, CLASS_CMB = 0, 1, 2


def _mask_tables():
    edge = np.full(16, -1, dtype=np.int64)
    hi = np.full(16, -1, dtype=np.int64)
    mid = np.full(16, -1, dtype=np.int64)
    zz = np.full(16, -1, dtype=np.int64)
    for mk in range(16):
        pos = [q for q in range(4) if mk >> q & 1]
        if pos:
            hi[mk] = pos[-1]
        if len(pos) == 2:
            edge[mk] = LOCAL_EDGES.index(tuple(pos))
        if len(pos) == 3:
            mid[mk] = pos[1]
            zz[mk] = [q for q in range(4) if q not in pos][0]
    return edge, hi, mid, zz


_EDGE_OF_MASK, _HI_OF_MASK, _MID_OF_MASK, _Z_OF_MASK = _mask_tables()


def icosahedron():
    """12 unit vertices (cyclic permutations of (0, +-1, +-phi), normalised) and the
    20 faces as increasing vertex triples, in lexicographic order."""
    V = []
    for p in range(3):
        for q in range(4):
            s1 = 1.0 if (q >> 1) else -1.0
            s2 = 1.0 if (q & 1) else -1.0
            base = (0.0, s1, s2 * PHI)
            V.append((base[(0 - p) % 3], base[(1 - p) % 3], base[(2 - p) % 3]))
    V = np.array(V, dtype=np.float64)
    V /= np.linalg.norm(V, axis=1, keepdims=True)
    edge_len = 2.0 / np.sqrt(1.0 + PHI ** 2)
    F = []
    for i in range(12):
        for j in range(i + 1, 12):
            if abs(np.linalg.norm(V[i] - V[j]) - edge_len) > 1e-9:
                continue
            for k in range(j + 1, 12):
                if abs(np.linalg.norm(V[i] - V[k]) - edge_len) < 1e-9 and \
                   abs(np.linalg.norm(V[j] - V[k]) - edge_len) < 1e-9:
                    F.append((i, j, k))
    return V, np.array(F, dtype=np.int64)


def tet_number(m):
    """m(m+1)(m+2)/6, with the value 0 for m <= 0."""
    m = np.asarray(m, dtype=np.int64)
    return np.where(m > 0, m * (m + 1) * (m + 2) // 6, 0)


class MacroMesh:
    """The 60-tet macro mesh of the shell r_cmb <= |x| <= r_surf (one radial layer)."""

    def __init__(self, r_cmb=0.5, r_surf=1.0, blending=True):
        self.r_cmb, self.r_surf, self.blending = float(r_cmb), float(r_surf), bool(blending)
        U, F = icosahedron()
        self.ico_faces = F
        self.unit = np.vstack([U, U])                               # direction of each macro vertex
        self.layer = np.array([0] * 12 + [1] * 12)                  # 0 = CMB sphere, 1 = surface
        self.verts = np.vstack([self.r_cmb * U, self.r_surf * U])   # straight positions
        cells, prism = [], []
        for f, (a, b, c) in enumerate(F):
            A, Bp, C = a + 12, b + 12, c + 12
            for t in ((a, b, c, C), (a, b, C, Bp), (a, Bp, C, A)):
                cells.append(sorted(t))
                prism.append(f)
        self.cells = np.array(cells, dtype=np.int64)
        self.cell_prism = np.array(prism, dtype=np.int64)
        # prism normals and plane offsets
        nh = np.cross(U[F[:, 1]] - U[F[:, 0]], U[F[:, 2]] - U[F[:, 0]])
        nh /= np.linalg.norm(nh, axis=1, keepdims=True)
        sgn = np.sign(np.einsum("ij,ij->i", nh, U[F[:, 0]]))
        nh *= sgn[:, None]
        self.prism_normal = nh
        self.prism_delta = np.einsum("ij,ij->i", nh, U[F[:, 0]])
        # macro edges and faces: unique increasing tuples, lexicographic
        E = sorted({(int(c[i]), int(c[j])) for c in self.cells for (i, j) in LOCAL_EDGES})
        Fc = sorted({tuple(int(v) for v in np.delete(c, z)) for c in self.cells for z in range(4)})
        self.edges = np.array(E, dtype=np.int64)
        self.faces = np.array(Fc, dtype=np.int64)
        eidx = {e: i for i, e in enumerate(E)}
        fidx = {f: i for i, f in enumerate(Fc)}
        self.cell_edges = np.array([[eidx[(int(c[i]), int(c[j]))] for (i, j) in LOCAL_EDGES]
                                    for c in self.cells], dtype=np.int64)
        self.cell_faces = np.array([[fidx[tuple(int(v) for v in np.delete(c, z))] for z in range(4)]
                                    for c in self.cells], dtype=np.int64)
        assert len(self.edges) == N_MACRO_EDGES and len(self.faces) == N_MACRO_FACES
        assert len(self.cells) == N_MACRO_CELLS

    # ------------------------------------------------------------------ numbering
    @staticmethod
    def counts(N):
        """Sizes of the four primitive blocks of the level with N intervals per edge."""
        nE1 = max(N - 1, 0)
        nF1 = max((N - 1) * (N - 2) // 2, 0)
        nC1 = int(tet_number(N - 3))
        return dict(nE1=nE1, nF1=nF1, nC1=nC1,
                    offE=N_MACRO_VERTS,
                    offF=N_MACRO_VERTS + N_MACRO_EDGES * nE1,
                    offC=N_MACRO_VERTS + N_MACRO_EDGES * nE1 + N_MACRO_FACES * nF1,
                    total=N_MACRO_VERTS + N_MACRO_EDGES * nE1 + N_MACRO_FACES * nF1
                    + N_MACRO_CELLS * nC1)

    @staticmethod
    def face_interior_index(i1, i2, N):
        """Index of the face-interior point with barycentric (N-i1-i2, i1, i2)."""
        return (i2 - 1) * (N - 1) - (i2 - 1) * i2 // 2 + (i1 - 1)

    @staticmethod
    def cell_interior_index(i1, i2, i3, N):
        """Index of the cell-interior point with barycentric (N-i1-i2-i3, i1, i2, i3):
        layers of constant i3, rows of constant i2, i1 fastest."""
        K = N - 2
        before = tet_number(K - 1) - tet_number(K - i3)
        M = N - 1 - i3
        return before + (i2 - 1) * M - (i2 - 1) * i2 // 2 + (i1 - 1)

    def node_ids(self, m, I, N):
        """Global ids of lattice points of macro cell m.  I: (k,4) integer barycentric
        coordinates w.r.t. the cell's increasing vertex order, summing to N."""
        I = np.asarray(I, dtype=np.int64)
        k = I.shape[0]
        cnt = self.counts(N)
        out = np.full(k, -1, dtype=np.int64)
        nz = I > 0
        nnz = nz.sum(1)
        cell = self.cells[m]
        # macro vertex
        sel = nnz == 1
        if sel.any():
            out[sel] = cell[np.argmax(I[sel], axis=1)]
        mask = nz[:, 0] * 1 + nz[:, 1] * 2 + nz[:, 2] * 4 + nz[:, 3] * 8
        rows = np.arange(k)
        # macro edge: interior position t = weight of the higher local vertex
        sel = nnz == 2
        if sel.any():
            e = self.cell_edges[m][_EDGE_OF_MASK[mask[sel]]]
            t = I[rows[sel], _HI_OF_MASK[mask[sel]]]
            out[sel] = cnt["offE"] + e * cnt["nE1"] + (t - 1)
        # macro face: (i1, i2) = weights of the middle and highest of its 3 vertices
        sel = nnz == 3
        if sel.any():
            f = self.cell_faces[m][_Z_OF_MASK[mask[sel]]]
            i1 = I[rows[sel], _MID_OF_MASK[mask[sel]]]
            i2 = I[rows[sel], _HI_OF_MASK[mask[sel]]]
            out[sel] = cnt["offF"] + f * cnt["nF1"] + self.face_interior_index(i1, i2, N)
        # macro cell interior
        sel = nnz == 4
        if sel.any():
            out[sel] = cnt["offC"] + m * cnt["nC1"] + self.cell_interior_index(
                I[sel, 1], I[sel, 2], I[sel, 3], N)
        return out

    # ------------------------------------------------------------------ geometry
    def straight(self, m, I, N):
        """Straight (pre-blending) position of lattice points of cell m."""
        X = self.verts[self.cells[m]]
        return (np.asarray(I, dtype=np.float64) / N) @ X

    def blend(self, x, prism):
        """Blending map B(x) = (x.nh/delta) x/|x| for points x in the given prism(s)."""
        if not self.blending:
            return np.array(x, dtype=np.float64, copy=True)
        nh = self.prism_normal[prism]
        d = self.prism_delta[prism]
        h = np.einsum("...i,...i->...", x, nh)
        rho = np.linalg.norm(x, axis=-1)
        return ((h / d) / rho)[..., None] * x

    def blend_jacobian(self, x, prism):
        """J_B(x) = (R/rho)(I - e e^T) + (1/delta) e nh^T with R = x.nh/delta, rho = |x|,
        e = x/rho (derivative of the blending map)."""
        x = np.asarray(x, dtype=np.float64)
        eye = np.broadcast_to(np.eye(3), x.shape[:-1] + (3, 3))
        if not self.blending:
            return eye.copy()
        nh = np.broadcast_to(self.prism_normal[prism], x.shape)
        d = np.broadcast_to(self.prism_delta[prism], x.shape[:-1])
        rho = np.linalg.norm(x, axis=-1)
        e = x / rho[..., None]
        R = np.einsum("...i,...i->...", x, nh) / d
        s = (R / rho)[..., None, None]
        return s * (eye - e[..., :, None] * e[..., None, :]) + (1.0 / d)[..., None, None] * (
            e[..., :, None] * nh[..., None, :])


def cell_lattice(N):
    """All integer barycentric 4-tuples summing to N (every lattice point of a cell)."""
    pts = [(N - i1 - i2 - i3, i1, i2, i3)
           for i3 in range(N + 1) for i2 in range(N + 1 - i3) for i1 in range(N + 1 - i2 - i3)]
    return np.array(pts, dtype=np.int64)


def kuhn_to_bary(K, n):
    """Kuhn-simplex coordinates (A,B,C), n >= A >= B >= C >= 0, to barycentric integers."""
    K = np.asarray(K, dtype=np.int64)
    A, B, C = K[..., 0], K[..., 1], K[..., 2]
    return np.stack([n - A, A - B, B - C, C], axis=-1)


PERMS = [(0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)]


def micro_tets_kuhn(n):
    """Freudenthal subdivision of the Kuhn simplex scaled by n, by brute force: every
    unit cube [q, q+1] of [0,n)^3 and every permutation pi gives the simplex
    q, q+e_pi0, q+e_pi0+e_pi1, q+(1,1,1); keep those inside n>=x1>=x2>=x3>=0.
    Cubes in lexicographic (a, b, c) order, permutations in PERMS order within a cube.
    Returns (n^3, 4, 3) integer vertex coordinates."""
    q = np.stack(np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij"), axis=-1).reshape(-1, 3)
    eye = np.eye(3, dtype=np.int64)
    cand = []
    for p in PERMS:
        v1 = q + eye[p[0]]
        v2 = v1 + eye[p[1]]
        cand.append(np.stack([q, v1, v2, q + 1], axis=1))                   # (n^3, 4, 3)
    V = np.stack(cand, axis=1).reshape(-1, 4, 3)                             # cube-major, then perm
    ok = (np.all(V[:, :, 0] <= n, axis=1) & np.all(V[:, :, 0] >= V[:, :, 1], axis=1)
          & np.all(V[:, :, 1] >= V[:, :, 2], axis=1) & np.all(V[:, :, 2] >= 0, axis=1))
    T = V[ok].astype(np.int64)
    assert T.shape[0] == n ** 3
    return T


class Level:
    """Everything the oracle needs at refinement level l: micro-tets with their 10 P2
    node ids and 4 P1 vertex ids, node coordinates and node classes."""

    def __init__(self, mesh: MacroMesh, l: int):
        self.mesh, self.l = mesh, l
        n = 2 ** l
        self.n = n
        self.n_p1 = MacroMesh.counts(n)["total"]
        self.n_p2 = MacroMesh.counts(2 * n)["total"]
        kt = micro_tets_kuhn(n)                                   # (n^3,4,3)
        # P2 nodes of a micro-tet in fine Kuhn coordinates: 2*vertices, then edge sums
        fine = [2 * kt[:, a] for a in range(4)] + [kt[:, a] + kt[:, b] for (a, b) in LOCAL_EDGES]
        fine = np.stack(fine, axis=1)                             # (n^3,10,3)
        bary2 = kuhn_to_bary(fine, 2 * n)
        bary1 = kuhn_to_bary(kt, n)
        p2, p1, xs, mac = [], [], [], []
        for m in range(N_MACRO_CELLS):
            p2.append(mesh.node_ids(m, bary2.reshape(-1, 4), 2 * n).reshape(-1, 10))
            p1.append(mesh.node_ids(m, bary1.reshape(-1, 4), n).reshape(-1, 4))
            xs.append(mesh.straight(m, bary1.reshape(-1, 4), n).reshape(-1, 4, 3))
            mac.append(np.full(n ** 3, m))
        self.tet_p2 = np.concatenate(p2)
        self.tet_p1 = np.concatenate(p1)
        self.tet_x = np.concatenate(xs)
        self.tet_macro = np.concatenate(mac)
        self.tet_prism = mesh.cell_prism[self.tet_macro]
        self.p2_straight, self.p2_class, self.p2_prism = self._nodes(2 * n)
        self.p1_straight, self.p1_class, self.p1_prism = self._nodes(n)
        self.p2_x = mesh.blend(self.p2_straight, self.p2_prism)
        self.p1_x = mesh.blend(self.p1_straight, self.p1_prism)

    def _nodes(self, N):
        return lattice_nodes(self.mesh, N)


def lattice_nodes(mesh, N):
    """Straight positions, classes and prisms of all lattice points of the level with N
    intervals per macro edge, by global id."""
    tot = MacroMesh.counts(N)["total"]
    X = np.full((tot, 3), np.nan)
    cls = np.full(tot, -1, dtype=np.int64)
    prism = np.full(tot, -1, dtype=np.int64)
    lat = cell_lattice(N)
    for m in range(N_MACRO_CELLS):
        ids = mesh.node_ids(m, lat, N)
        x = mesh.straight(m, lat, N)
        lay = mesh.layer[mesh.cells[m]]
        nz = lat > 0
        top = np.all(~nz | (lay[None, :] == 1), axis=1)
        bot = np.all(~nz | (lay[None, :] == 0), axis=1)
        c = np.where(top, CLASS_SURFACE, np.where(bot, CLASS_CMB, CLASS_INNER))
        seen = ~np.isnan(X[ids, 0])
        if seen.any():
            assert np.allclose(X[ids[seen]], x[seen], atol=1e-14, rtol=0)
            assert np.all(cls[ids[seen]] == c[seen])
        X[ids] = x
        cls[ids] = c
        prism[ids] = mesh.cell_prism[m]
    assert not np.isnan(X).any()
    return X, cls, prism
