"""Pins of the sampled-row oracle (no GPU): rows built from one macro's micro-tets around an
interior point equal the rows of the full level's element sums."""
import numpy as np
import pytest

import workloads as W
from oracle.mesh import MacroMesh, Level, lattice_nodes
from oracle.fem import stokes_apply_elements, tets_touching
from oracle.sampled import MacroRows, sample_points, face_points
from oracle.fem import Operators, Constraints, ConstrainedOperators


@pytest.mark.parametrize("L", [2, 3])
def test_sampled_rows_match_full_level(L):
    mesh = MacroMesh()
    Lv = Level(mesh, L)
    eta = W.viscosity_plumes(Lv.p1_x, seed=2, contrast=1e6)
    dl = W.dlnrho_table_compressible()
    u = W.random_field(3 * Lv.n_p2, 21)
    p = W.random_field(Lv.n_p1, 22)
    R = MacroRows(mesh, L)
    assert (R.n_p2, R.n_p1) == (Lv.n_p2, Lv.n_p1)
    rng = np.random.default_rng(5)
    nv = npr = 0
    for _ in range(40):
        m = int(rng.integers(0, 60))
        r = R.velocity_row(m, sample_points(2 * R.n, 1, rng)[0], eta, dl, u, p)
        if r is not None:
            gid, rows = r
            yu, _ = stokes_apply_elements(Lv, eta, dl, u, p, tets_touching(Lv, p2_nodes=[gid]))
            ref = yu[[gid, gid + Lv.n_p2, gid + 2 * Lv.n_p2]]
            assert np.abs(rows - ref).max() <= 1e-13 * np.abs(ref).max()
            assert Lv.p2_class[gid] == 0
            nv += 1
        r1 = R.pressure_row(m, sample_points(R.n, 1, rng)[0], eta, dl, u, p)
        if r1 is not None:
            vid, val = r1
            _, yp = stokes_apply_elements(Lv, eta, dl, u, p, tets_touching(Lv, p1_nodes=[vid]))
            assert abs(val - yp[vid]) <= 1e-13 * abs(yp[vid])
            npr += 1
    assert nv >= 10 and npr >= 5


def test_lattice_nodes_match_level():
    mesh = MacroMesh()
    Lv = Level(mesh, 2)
    X, cls, prism = lattice_nodes(mesh, 4)
    assert np.array_equal(mesh.blend(X, prism), Lv.p1_x) and np.array_equal(cls, Lv.p1_class)


@pytest.mark.parametrize("L,bc", [(2, (0, 1)), (2, (1, 0)), (3, (0, 1))])
def test_constrained_rows_match_full_level(L, bc):
    """Constrained rows at points owned by one macro (strictly inside it, or strictly inside a
    macro face on a sphere) equal the rows of the assembled constrained operators
    A_c u + P0 B^T p and (B + C) P0 u (Sec. 5.1): surface and CMB rows under both boundary
    conditions, and interior rows whose micro-tets touch the spheres."""
    mesh = MacroMesh()
    Lv = Level(mesh, L)
    eta = W.viscosity_plumes(Lv.p1_x, seed=2, contrast=1e6)
    dl = W.dlnrho_table_compressible()
    co = ConstrainedOperators(Operators(Lv, eta, dlnrho_table=dl), Constraints(Lv, *bc))
    u = W.random_field(3 * Lv.n_p2, 23)
    p = W.random_field(Lv.n_p1, 24)
    p = p - p.mean()
    yu = co.A @ u + co.BT_raw @ p
    yp = co.Bbar_raw @ u
    R = MacroRows(mesh, L)
    rng = np.random.default_rng(6)
    seen = {0: 0, 1: 0, 2: 0}
    npr = 0
    for m in range(60):
        for z, lay in R.sphere_faces(m):
            for pt in face_points(2 * R.n, z, 2, rng):
                gid, rows, cl = R.constrained_velocity_row(m, pt, eta, dl, u, p, bc)
                assert cl == (1 if lay == 1 else 2) and Lv.p2_class[gid] == cl
                ref = yu[[gid, gid + Lv.n_p2, gid + 2 * Lv.n_p2]]
                assert np.abs(rows - ref).max() <= 1e-13 * max(np.abs(ref).max(), 1e-300)
                seen[cl] += 1
            if R.n > 2:
                for pt in face_points(R.n, z, 1, rng):
                    vid, val = R.constrained_pressure_row(m, pt, eta, dl, u, p, bc)
                    assert abs(val - yp[vid]) <= 1e-13 * abs(yp[vid])
                    npr += 1
        # an interior point next to a sphere: its micro-tets carry sphere nodes
        if not R.sphere_faces(m):
            continue
        z, lay = R.sphere_faces(m)[0]
        pt = np.array(face_points(2 * R.n, z, 1, rng)[0])
        inward = {0: (-1, 0, 0), 1: (1, 0, 0), 2: (0, 1, 0), 3: (0, 0, 1)}[z]
        q = tuple(int(v) for v in pt + np.array(inward))
        r = R.constrained_velocity_row(m, q, eta, dl, u, p, bc)
        if r is not None:
            gid, rows, cl = r
            ref = yu[[gid, gid + Lv.n_p2, gid + 2 * Lv.n_p2]]
            assert cl == 0 and np.abs(rows - ref).max() <= 1e-13 * np.abs(ref).max()
            seen[0] += 1
    assert seen[1] >= 20 and seen[2] >= 20 and seen[0] >= 10
    assert npr >= 20 or R.n <= 2
