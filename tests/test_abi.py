"""C-ABI library: loads, exports every declared symbol, and its host-side mesh (numbering,
coordinates, node classes) agrees with the independently written oracle (no GPU)."""
import os
import re

import numpy as np
import pytest

import paper_2506_04157_gb300 as mfs
from oracle.mesh import MacroMesh, Level

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    syms = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            syms |= set(re.findall(r"\b(mfs_[A-Za-z0-9_]+)\s*\(", src))
    return syms


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(mfs.LIB_PATH):
        import paper_2506_04157_gb300.build as b
        b.build()
    return mfs.lib()


def test_exports_every_declared_symbol(lib):
    syms = declared_symbols()
    assert len(syms) >= 18
    for s in sorted(syms):
        assert hasattr(lib, s), s
    assert set(mfs._SIGS) <= syms | {"mfs_last_error", "mfs_version"}


def test_errors_without_gpu_or_bad_args(lib):
    with pytest.raises(mfs.MfsError):
        mfs.Mesh(None, 8)
    with pytest.raises(mfs.MfsError):
        mfs.Mesh(None, 2, r_cmb=1.0, r_surf=0.5)
    m = mfs.Mesh(None, 2)
    with pytest.raises(mfs.MfsError) as e:
        mfs.Problem(m)
    assert "host-only" in str(e.value)
    # null handles are refused with MFS_EINVAL (1) and a message, before any device work
    import ctypes
    L = mfs.lib()
    null = ctypes.c_void_p()
    for name, args in [("mfs_apply_vmass", (null, 0, 1.0, null, null)),
                       ("mfs_lumped_vmass", (null, 1.0, null)),
                       ("mfs_apply_poisson", (null, 1, 0, 1.0, null, null)),
                       ("mfs_apply_schur", (null, None, 0, null, null, None)),
                       ("mfs_set_temperature", (null, null)),
                       ("mfs_mesh_law_maps", (null, 0, null, null, null)),
                       ("mfs_mmoc_host", (null, 0, null, null, null, null, 0.1, null, null)),
                       ("mfs_temperature_step", (null, None, null, null, null, null, 0.1, 0.1, null, null, None))]:
        assert getattr(L, name)(*args) == 1, name
        assert L.mfs_last_error(), name
    # the concurrent solve: an empty ensemble is a no-op; a negative count, a negative thread
    # count or null arrays are refused before any device work
    opts = mfs.SolveOpts()
    L.mfs_solve_opts_default(ctypes.byref(opts))
    assert L.mfs_solve_concurrent(0, null, ctypes.byref(opts), null, null, null, null, null, 0) == 0
    assert L.mfs_solve_concurrent(-1, null, ctypes.byref(opts), null, null, null, null, null, 0) == 1
    assert L.mfs_solve_concurrent(0, null, ctypes.byref(opts), null, null, null, null, null, -2) == 1
    assert L.mfs_solve_concurrent(2, null, ctypes.byref(opts), null, null, null, null, null, 0) == 1
    assert b"non-null" in L.mfs_last_error()
    two = (ctypes.c_void_p * 2)(None, None)
    assert L.mfs_solve_concurrent(2, two, ctypes.byref(opts), two, two, two, two, null, 0) == 1
    assert b"member 0" in L.mfs_last_error()


@pytest.mark.parametrize("blending", [True, False])
@pytest.mark.parametrize("l", [0, 1, 2, 3])
def test_numbering_coords_classes_match_oracle(lib, l, blending):
    M = mfs.Mesh(None, l, blending=blending)
    L = Level(MacroMesh(blending=blending), l)
    inf = M.info(l)
    assert (inf.n_p2, inf.n_p1, inf.n_tets) == (L.n_p2, L.n_p1, L.tet_p2.shape[0])
    for p2 in (True, False):
        xs = M.coords(l, p2=p2, blended=False).T
        xb = M.coords(l, p2=p2, blended=True).T
        ref_s = L.p2_straight if p2 else L.p1_straight
        ref_b = L.p2_x if p2 else L.p1_x
        assert np.abs(xs - ref_s).max() < 1e-14
        assert np.abs(xb - ref_b).max() < 1e-14
        cls = M.node_class(l, p2=p2)
        ref_c = L.p2_class if p2 else L.p1_class
        assert np.array_equal(cls, ref_c)


def test_library_default_options_match_paper_table(lib):
    """mfs_solve_opts_default carries the paper's Table parametertable (tests/golden; the
    coarse-grid tolerance has no field: the coarse solve is an exact inverse), the temperature
    defaults its tol_T; the ctypes mirrors have the sizes of the C structs of include/mfs.h
    (136 and 96 bytes under the LP64 ABI of x86_64 and aarch64)."""
    import ctypes
    import json
    import os
    gold = json.load(open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                                       "solver_parameters.json")))
    o = mfs.Problem.default_opts()
    for k, v in gold.items():
        if k not in ("_source", "tol_coarse"):
            assert getattr(o, k) == v, k
    # the weighted BFBT's vector mass is the consistent one, solved by CG (Sec. 5.2.3)
    assert (o.uzawa, o.schur, o.mixed, o.tol_wBFBT, o.vmass) == (0, 0, 1, 1e-10, 1)
    t = mfs.Problem.temp_params()
    assert t.tol_T == 1e-10 and t.restart == 30
    assert ctypes.sizeof(mfs.SolveOpts) == 152 and ctypes.sizeof(mfs.TempParams) == 96


def test_library_quadrature_rule_matches_oracle(lib):
    """The library's own Gauss-Jacobi construction of the 27-point conical rule (host code of
    the temperature kernels) against the oracle's, built from scipy's Gauss-Jacobi roots."""
    from oracle.temperature import QUAD5_BARY, QUAD5_W
    lam, w = mfs.temp_rule()
    assert np.abs(lam - QUAD5_BARY).max() <= 1e-15 and np.abs(w - QUAD5_W).max() <= 1e-16


@pytest.mark.parametrize("l", [1, 2, 3])
def test_library_prolongation_matches_oracle(lib, l):
    """The library's host-built P2 prolongation (the CSR its transfer kernels use) equals the
    oracle's, built independently from the same definition (coarse P2 interpolant at the fine
    nodes), entry for entry."""
    import scipy.sparse as sp
    from oracle.mesh import MacroMesh
    from oracle.solver import prolongation
    m = mfs.Mesh(None, l)
    rp, ci, w = m.prolongation(l)
    nf, nc = m.info(l).n_p2, m.info(l - 1).n_p2
    P = sp.csr_matrix((w, ci, rp), shape=(nf, nc))
    R = prolongation(MacroMesh(), l - 1)
    assert R.shape == P.shape
    assert abs(P - R).max() == 0.0


@pytest.mark.parametrize("l", [1, 2, 3])
def test_library_p1_interpolation_and_viscosity_weighting_match_oracle(lib, l):
    """The library's host-built P1 interpolation reproduces linear fields exactly (on the
    straight vertices), and its row-normalised transpose, the coarse-viscosity full
    weighting, equals the oracle's restriction of a random field."""
    import scipy.sparse as sp
    from oracle.mesh import MacroMesh, Level
    from oracle.solver import restrict_viscosity
    m = mfs.Mesh(None, l)
    cv, fv, w = m.p1_interpolation(l)
    nf, nc = m.info(l).n_p1, m.info(l - 1).n_p1
    T = sp.csr_matrix((w, (fv, cv)), shape=(nf, nc))
    assert np.abs(np.asarray(T.sum(axis=1)).ravel() - 1.0).max() == 0.0
    mesh = MacroMesh()
    Lf, Lc = Level(mesh, l), Level(mesh, l - 1)
    a = np.array([0.3, -0.7, 1.1])
    assert np.abs(T @ (Lc.p1_straight @ a) - Lf.p1_straight @ a).max() <= 1e-14
    eta = np.random.default_rng(l).uniform(1.0, 10.0, nf)
    R = T.T.tocsr()
    got = (R @ eta) / (R @ np.ones(nf))
    assert np.abs(got - restrict_viscosity(Lf, Lc, eta)).max() <= 1e-14 * eta.max()


@pytest.mark.parametrize("blending", [True, False])
def test_library_law_maps_match_oracle(lib, blending):
    """The maps through which the device viscosity law reads the temperature (finest P2 node
    at each vertex and, for the quadrature-point levels, at each P2 node; the vertex radius)
    equal the oracle's matching by position (k-d tree over the finest level's P2 nodes) on
    every level of a level-3 hierarchy, so that eta(x_V, T(x_V)) of Eq. ViscosityDef takes
    the same temperature and radius on both sides."""
    from oracle.solver import temperature_on_level
    mesh = MacroMesh(blending=blending)
    M = mfs.Mesh(None, 3, blending=blending)
    Lf = Level(mesh, 3)
    ids = np.arange(Lf.n_p2, dtype=np.float64)
    for l in range(4):
        L = Level(mesh, l)
        vfine, vrad, p2fine = M.law_maps(l)
        i2, i1 = temperature_on_level(Lf, L, ids)
        assert np.array_equal(vfine, i1.astype(np.int32)), l
        assert np.array_equal(p2fine, i2.astype(np.int32)), l
        assert np.abs(vrad - np.linalg.norm(L.p1_x, axis=1)).max() <= 1e-15, l
    with pytest.raises(mfs.MfsError):
        M.law_maps(4)


@pytest.mark.parametrize("tau", [0.03, 0.3])
@pytest.mark.parametrize("blending", [True, False])
def test_library_mmoc_particle_step_matches_oracle(lib, blending, tau):
    """The library's MMOC particle step (the code the mmoc kernel runs per particle: RK4 back
    along u linear in time, point location, P2 evaluation; Sec. 3), run on the host, against
    the oracle's k-d-tree-free locator and RK4: departure points to 1e-12 and T there, on a
    rotation plus a non-affine field large enough to carry particles across macro faces and
    out of the shell (moved back radially), and particle paths continued over a second step."""
    from oracle.temperature import Locator, mmoc_departure
    import workloads as W
    mesh = MacroMesh(blending=blending)
    Lv = Level(mesh, 2)
    M = mfs.Mesh(None, 2, blending=blending)
    x = Lv.p2_x
    rng = np.random.default_rng(7)
    u_new = (np.cross(rng.standard_normal(3), x) + 0.1 * np.sin(3 * x)).T.reshape(-1)
    u_old = (np.cross(rng.standard_normal(3), x) + 0.3 * x).T.reshape(-1)
    T = W.temperature_blobs(x, 4)
    loc = Locator(Lv)
    Th, X = M.mmoc_host(x, T, u_new, u_old, tau)
    Xr = mmoc_departure(loc, u_new, u_old, tau)
    assert np.abs(X - Xr).max() <= 1e-12
    assert np.abs(Th - loc.eval_p2(T, Xr)).max() <= 1e-10 * np.abs(T).max()
    if tau == 0.3:   # longer than a level-2 micro-tet edge (0.125 radially); some leave the shell
        r = np.linalg.norm(X, axis=1)
        assert np.linalg.norm(X - x, axis=1).max() > 0.125
        assert (r > mesh.r_surf).any() or (r < mesh.r_cmb).any()
    Th2, X2 = M.mmoc_host(X, T, u_old, u_new, 0.02)
    Xr2 = mmoc_departure(loc, u_old, u_new, 0.02, X=Xr)
    assert np.abs(X2 - Xr2).max() <= 1e-12
    assert np.abs(Th2 - loc.eval_p2(T, Xr2)).max() <= 1e-10 * np.abs(T).max()


def test_mmoc_host_refusals(lib):
    """mfs_mmoc_host refuses a negative particle count, missing fields for a non-empty batch and
    a non-finite step with MFS_EINVAL and a message; an empty batch is a no-op."""
    import ctypes
    M = mfs.Mesh(None, 1)
    L = lib
    null = None
    buf = (ctypes.c_double * 8)()
    for args in [(M.handle, -1, null, null, null, null, 0.1, null, null),
                 (M.handle, 1, buf, null, buf, buf, 0.1, buf, null),
                 (M.handle, 1, buf, buf, buf, buf, float("nan"), buf, null)]:
        assert L.mfs_mmoc_host(*args) == 1
        assert L.mfs_last_error()
    assert L.mfs_mmoc_host(M.handle, 0, null, null, null, null, 0.1, null, null) == 0
