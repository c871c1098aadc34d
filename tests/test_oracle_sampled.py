"""Pins of the sampled-row oracle (no GPU): rows built from one macro's micro-tets around an
interior point equal the rows of the full level's element sums."""
import numpy as np
import pytest

import workloads as W
from oracle.mesh import MacroMesh, Level, lattice_nodes
from oracle.fem import stokes_apply_elements, tets_touching
from oracle.sampled import MacroRows, sample_points


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
