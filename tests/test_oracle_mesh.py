"""Pins of the oracle mesh against closed forms and invariants (no GPU)."""
import numpy as np
import pytest

from oracle.mesh import MacroMesh, Level, micro_tets_kuhn, cell_lattice, CLASS_SURFACE, CLASS_CMB


def recursion_counts(l):
    """Vertices/edges/faces/tets of uniform refinement from (24,102,140,60):
    V'=V+E, E'=2E+3F+T, F'=4F+8T, T'=8T (each edge splits, each face gives 3 inner
    edges and 4 faces, each tet gives 1 inner edge, 8 inner faces, 8 tets)."""
    V, E, F, T = 24, 102, 140, 60
    for _ in range(l):
        V, E, F, T = V + E, 2 * E + 3 * F + T, 4 * F + 8 * T, 8 * T
    return V, E, F, T


@pytest.fixture(scope="module")
def mesh():
    return MacroMesh()


def test_macro_mesh_euler(mesh):
    V, E, F, T = 24, len(mesh.edges), len(mesh.faces), len(mesh.cells)
    assert (E, F, T) == (102, 140, 60)
    assert V - E + F - T == 2          # solid shell ~ S^2


@pytest.mark.parametrize("l", [0, 1, 2, 3])
def test_level_counts(mesh, l):
    L = Level(mesh, l)
    V, E, F, T = recursion_counts(l)
    V2 = recursion_counts(l + 1)[0]
    assert L.tet_p2.shape[0] == T
    assert L.n_p1 == V and L.n_p2 == V2
    assert (L.p2_class == CLASS_SURFACE).sum() == 10 * 4 ** (l + 1) + 2
    assert (L.p2_class == CLASS_CMB).sum() == 10 * 4 ** (l + 1) + 2
    # every id used, P2 ids of vertices coincide with the coarse P1 positions
    assert np.unique(L.tet_p2).size == L.n_p2
    assert np.unique(L.tet_p1).size == L.n_p1


@pytest.mark.parametrize("l", [1, 2])
def test_refined_complex(mesh, l):
    """Euler characteristic 2 of the refined complex, every interior micro-face in
    exactly two micro-tets, boundary micro-faces only on the two spheres."""
    L = Level(mesh, l)
    tets = L.tet_p1
    edges = {tuple(sorted((t[i], t[j]))) for t in tets for i in range(4) for j in range(i + 1, 4)}
    faces = {}
    for t in tets:
        for z in range(4):
            f = tuple(sorted(np.delete(t, z)))
            faces[f] = faces.get(f, 0) + 1
    V, E, F, T = recursion_counts(l)
    assert (len(edges), len(faces), len(tets)) == (E, F, T)
    assert L.n_p1 - len(edges) + len(faces) - len(tets) == 2
    assert set(faces.values()) <= {1, 2}
    bnd = [f for f, c in faces.items() if c == 1]
    for f in bnd:
        cls = L.p1_class[list(f)]
        assert np.all(cls == cls[0]) and cls[0] in (CLASS_SURFACE, CLASS_CMB)
    assert len(bnd) == 2 * 20 * 4 ** l


def test_micro_tets_volume_and_orientation_free():
    """Freudenthal pieces tile the Kuhn simplex: total volume n^3/6 with n^3 pieces of
    volume 1/6 each, and all lattice points are covered."""
    for n in (1, 2, 3, 4):
        T = micro_tets_kuhn(n)
        vol = np.abs(np.linalg.det(np.stack([T[:, k] - T[:, 0] for k in (1, 2, 3)], axis=-1))) / 6
        assert np.allclose(vol, 1 / 6)
        assert np.isclose(vol.sum(), n ** 3 / 6)
        pts = {tuple(p) for p in T.reshape(-1, 3)}
        assert len(pts) == (n + 1) * (n + 2) * (n + 3) // 6


def test_polyhedral_volume(mesh):
    L = Level(mesh, 2)
    X = L.tet_x
    vol = np.abs(np.linalg.det(np.stack([X[:, k] - X[:, 0] for k in (1, 2, 3)], axis=-1))).sum() / 6
    Xm = mesh.verts[mesh.cells]
    vm = np.abs(np.linalg.det(np.stack([Xm[:, k] - Xm[:, 0] for k in (1, 2, 3)], axis=-1))).sum() / 6
    assert np.isclose(vol, vm, rtol=1e-13)


def test_blending_jacobian_fd(mesh):
    rng = np.random.default_rng(7)
    for m in range(0, 60, 7):
        lam = rng.dirichlet(np.ones(4), size=5)
        x = lam @ mesh.verts[mesh.cells[m]]
        pr = mesh.cell_prism[m]
        J = mesh.blend_jacobian(x, pr)
        h = 1e-6
        for k in range(3):
            e = np.zeros(3); e[k] = h
            fd = (mesh.blend(x + e, pr) - mesh.blend(x - e, pr)) / (2 * h)
            assert np.allclose(J[:, :, k], fd, rtol=0, atol=1e-8)
        # closed-form determinant (R/rho)^2 kappa (nh.e)
        nh, d = mesh.prism_normal[pr], mesh.prism_delta[pr]
        rho = np.linalg.norm(x, axis=1)
        R = x @ nh / d
        det = (R / rho) ** 2 / d * (x @ nh) / rho
        assert np.allclose(np.linalg.det(J), det, rtol=1e-12)


def test_blended_boundary_radii(mesh):
    L = Level(mesh, 2)
    r = np.linalg.norm(L.p2_x, axis=1)
    assert np.allclose(r[L.p2_class == CLASS_SURFACE], 1.0, atol=1e-14)
    assert np.allclose(r[L.p2_class == CLASS_CMB], 0.5, atol=1e-14)
    assert np.all((r > 0.5 - 1e-14) & (r < 1 + 1e-14))


def test_blended_volume_converges():
    """Sum of w|det J| over all qps -> (4 pi / 3)(1 - 1/8) at O(h^2) (degree-2 rule
    and piecewise-polynomial pull-back of a smooth map)."""
    from oracle.fem import Geometry
    mesh = MacroMesh()
    exact = 4 * np.pi / 3 * (1 - 0.125)
    errs = []
    for l in (0, 1, 2, 3):
        L = Level(mesh, l)
        errs.append(abs(Geometry(mesh, L.tet_x, L.tet_prism).W.sum() - exact))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert errs[-1] < 1e-3
    assert np.all(rates[1:] > 1.8), rates
