"""Pins of the weighted-BFBT oracle (no GPU): the inverse-square-root-viscosity P1 Laplacian
K_{1/sqrt(eta)}, the HRZ-lumped vector mass M_{sqrt(eta)}, the surface layer D_eta and the
composed approximation of Sec. 5.2.3 (Eq. schurWBFBT, rescaled form)."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import workloads as W
from oracle.mesh import MacroMesh, Level, CLASS_SURFACE
from oracle.fem import project_mean_zero
from oracle.solver import Hierarchy, StokesOracle, direct_solve
from oracle.wbfbt import WbfbtOperators, wbfbt_apply, surface_tets, icosahedron_volume

# straight (polyhedral) shell between the icosahedra of circumradius 0.5 and 1
POLY_VOLUME = icosahedron_volume(1.0) - icosahedron_volume(0.5)


def test_icosahedron_volume_closed_form():
    # unit edge length: 5 (3 + sqrt 5) / 12
    assert abs(icosahedron_volume(np.sin(2 * np.pi / 5)) - 2.1816949906249126) < 1e-13


@pytest.mark.parametrize("L", [0, 1, 2])
def test_poisson_energy_of_linear_functions_polyhedral(L):
    """On straight tets P1 holds the coordinate functions: x_i^T K x_j = int w delta_ij,
    the shell's volume times the constant weight 1/sqrt(eta)."""
    Lv = Level(MacroMesh(blending=False), L)
    x = Lv.p1_x
    for eta, wt in [(1.0, 1.0), (16.0, 0.25)]:
        K = WbfbtOperators(Lv, np.full(Lv.n_p1, eta)).K
        G = x.T @ (K @ x)
        assert np.abs(G - wt * POLY_VOLUME * np.eye(3)).max() <= 1e-12 * POLY_VOLUME


def test_poisson_null_space_symmetry_and_definiteness():
    Lv = Level(MacroMesh(), 2)
    eta = W.viscosity_plumes(Lv.p1_x, seed=7, contrast=1e4)
    K = WbfbtOperators(Lv, eta, a=3.0).K
    nrm = abs(K).max()
    assert np.abs(K @ np.ones(Lv.n_p1)).max() <= 1e-12 * nrm        # Neumann: constants
    assert abs(K - K.T).max() <= 1e-14 * nrm
    rng = np.random.default_rng(0)
    for _ in range(5):
        v = project_mean_zero(rng.standard_normal(Lv.n_p1))
        assert v @ (K @ v) > 0


@pytest.mark.parametrize("L", [0, 1, 2])
def test_lumped_mass_total_polyhedral(L):
    """HRZ lumping keeps each element's total mass: sum_i d_i = int sqrt(eta)."""
    Lv = Level(MacroMesh(blending=False), L)
    for eta, wt in [(1.0, 1.0), (9.0, 3.0)]:
        d = WbfbtOperators(Lv, np.full(Lv.n_p1, eta)).d
        assert abs(d.sum() - wt * POLY_VOLUME) <= 1e-12 * POLY_VOLUME
        assert d.min() > 0


def test_lumped_mass_total_blended_converges_to_sphere_shell():
    shell = 4.0 * np.pi / 3.0 * (1.0 - 0.5 ** 3)
    errs = []
    for L in [1, 2, 3]:
        Lv = Level(MacroMesh(), L)
        errs.append(abs(WbfbtOperators(Lv, np.ones(Lv.n_p1)).d.sum() / shell - 1))
    assert errs[-1] < 1e-5 and errs[1] < errs[0] / 8 and errs[2] < errs[1] / 8


def test_lumped_mass_hrz_values_closed_form():
    """With the symmetric 4-point rule every P2 vertex function is +-1/10 at the points and
    the edge functions (1 + sqrt 5)/10 or (3 - sqrt 5)/10, so per straight tet of volume V
    the HRZ masses are V / (64 - 12 sqrt 5) (vertices) and V (10 - 2 sqrt 5)/(64 - 12 sqrt 5)
    (edge midpoints)."""
    Lv = Level(MacroMesh(blending=False), 1)
    X = Lv.tet_x
    V = np.abs(np.linalg.det(np.stack([X[:, 1] - X[:, 0], X[:, 2] - X[:, 0], X[:, 3] - X[:, 0]], axis=-1))) / 6
    den = 64.0 - 12.0 * np.sqrt(5.0)
    fac = np.array([1.0] * 4 + [10.0 - 2.0 * np.sqrt(5.0)] * 6) / den
    expect = np.zeros(Lv.n_p2)
    np.add.at(expect, Lv.tet_p2.reshape(-1), (V[:, None] * fac[None, :]).reshape(-1))
    d = WbfbtOperators(Lv, np.ones(Lv.n_p1)).d
    assert np.abs(d - expect).max() <= 1e-14 * expect.max()


@pytest.mark.parametrize("L", [0, 1, 2])
def test_surface_layer(L):
    """D_eta holds every micro-tet with a face on the surface (20 4^L of them), every
    macro-tet at level 0 (each has a surface vertex), and only tets touching the surface."""
    Lv = Level(MacroMesh(), L)
    mask = surface_tets(Lv)
    on = Lv.p1_class[Lv.tet_p1] == CLASS_SURFACE
    face = on.sum(axis=1) == 3
    assert face.sum() == 20 * 4 ** L
    assert np.all(mask[face])
    assert np.array_equal(mask, on.any(axis=1))
    if L == 0:
        assert mask.all()
    r = np.linalg.norm(Lv.p1_x[Lv.tet_p1], axis=-1).max(axis=1)
    assert np.all(np.abs(r[mask] - 1.0) < 1e-14)


def test_surface_scaling_is_elementwise():
    """eta_a = a^2 eta on D_eta: K(a) = K_rest + K_D / a and d(a) = d_rest + a d_D."""
    Lv = Level(MacroMesh(), 1)
    eta = W.viscosity_radial(Lv.p1_x)
    K1, d1 = WbfbtOperators(Lv, eta, 1.0).K, WbfbtOperators(Lv, eta, 1.0).d
    O2, O4 = WbfbtOperators(Lv, eta, 2.0), WbfbtOperators(Lv, eta, 4.0)
    assert abs(3 * (O2.K - K1) - 2 * (O4.K - K1)).max() <= 1e-13 * abs(K1).max()
    assert np.abs(3 * (O2.d - d1) - (O4.d - d1)).max() <= 1e-13 * d1.max()
    # vertices outside the surface layer keep their rows
    touched = np.unique(Lv.tet_p1[surface_tets(Lv)])
    free = np.setdiff1d(np.arange(Lv.n_p1), touched)
    assert abs((O2.K - K1)[free]).max() == 0.0


@pytest.fixture(scope="module")
def level1_isoviscous():
    mesh = MacroMesh()
    Lv = Level(mesh, 1)
    H = Hierarchy(mesh, 1, np.ones(Lv.n_p1))
    co, cons = H.co[1], H.cons[1]
    n = Lv.n_p1
    reg = sp.identity(co.A.shape[0]) - cons.Pv_matrix() - cons.identity_rows()
    lu = spla.splu((co.A + reg).tocsc())
    S = np.column_stack([co.apply_B(cons.P0(lu.solve(co.apply_BT(e)))) for e in np.eye(n)])
    U, _, _ = np.linalg.svd(np.eye(n) - 1.0 / n)
    return Lv, co, cons, S, U[:, :n - 1]


def _sw(Lv, co, cons, eta, a_l, a_r, a_scale=1.0):
    """Dense S_w^-1 with the viscosity eta in K and M and a_scale times the level's A."""
    wl, wr = WbfbtOperators(Lv, eta, a_l), WbfbtOperators(Lv, eta, a_r)
    A = lambda u: a_scale * co.apply_A(u)
    return np.column_stack([project_mean_zero(wbfbt_apply(co, cons, A, wl, wr, e)) for e in np.eye(Lv.n_p1)])


def test_wbfbt_consistent_mass_spectrum_is_bounded(level1_isoviscous):
    """With the consistent vector mass (the CG solve of Sec. 5.2.3) S_w^-1 S keeps an order-one
    spectrum: measured [0.345, 4.31] on level 1 and [0.333, 4.99] on level 2 (condition 13,
    15), against [0.116, 20.6] and [0.123, 78.5] with the HRZ-lumped mass (condition 177,
    635: the O(1/h) growth is the lumping's)."""
    Lv, co, cons, S, Bm = level1_isoviscous
    wc = WbfbtOperators(Lv, np.ones(Lv.n_p1), 1.0, mass="consistent")
    Sw = np.column_stack([project_mean_zero(wbfbt_apply(co, cons, co.apply_A, wc, wc, e))
                          for e in np.eye(Lv.n_p1)])
    ev = np.linalg.eigvals(Bm.T @ Sw @ S @ Bm)
    assert np.abs(ev.imag).max() < 1e-8 * np.abs(ev.real).max()
    assert 0.3 < ev.real.min() and ev.real.max() < 5.0


def test_wbfbt_spectrum_isoviscous(level1_isoviscous):
    """S_w^-1 S on the mean-zero space (S = B A^-1 B^T, level 1, eta = 1): symmetric S_w^-1
    for a_l = a_r, real positive spectrum of order one (the P1-Laplacian replacement of
    B M^-1 B^T enters twice; measured [0.116, 20.6]); unchanged when eta is scaled by a
    constant, since K^-1 ~ eta^(1/2), M^-1 ~ eta^(-1/2), A ~ eta and S ~ 1/eta."""
    Lv, co, cons, S, Bm = level1_isoviscous
    Sw = _sw(Lv, co, cons, np.ones(Lv.n_p1), 1.0, 1.0)
    assert abs(Sw - Sw.T).max() <= 1e-10 * abs(Sw).max()
    ev = np.linalg.eigvals(Bm.T @ Sw @ S @ Bm)
    assert np.abs(ev.imag).max() < 1e-8 * np.abs(ev.real).max()
    assert 0.1 < ev.real.min() and ev.real.max() < 25.0
    Sw100 = _sw(Lv, co, cons, np.full(Lv.n_p1, 100.0), 1.0, 1.0, a_scale=100.0)
    assert abs(Sw100 - 100.0 * Sw).max() <= 1e-10 * abs(100.0 * Sw).max()


def test_wbfbt_asymmetric_transpose_identity(level1_isoviscous):
    """(K_l^-1 B M_l^-1 A M_r^-1 B^T K_r^-1)^T swaps the roles of a_l and a_r."""
    Lv, co, cons, S, Bm = level1_isoviscous
    eta = W.viscosity_radial(Lv.p1_x)
    A = _sw(Lv, co, cons, eta, 1.0, 10.0)
    Bt = _sw(Lv, co, cons, eta, 10.0, 1.0)
    assert abs(A.T - Bt).max() <= 1e-10 * abs(A).max()
    assert abs(A - A.T).max() > 1e-3 * abs(A).max()


@pytest.mark.slow
@pytest.mark.parametrize("a_l", [1.0, 3.0])
def test_stokes_wbfbt_matches_direct(a_l):
    """FGMRES with the symmetric Uzawa step and the weighted BFBT (symmetric and asymmetric
    surface scaling) reaches the direct solution (level 1)."""
    mesh = MacroMesh()
    Lv = Level(mesh, 1)
    H = Hierarchy(mesh, 1, W.viscosity_radial(Lv.p1_x), dlnrho_table=W.dlnrho_table_config1())
    S = StokesOracle(H, dict(schur="wbfbt", a_l=a_l, omega=0.03))
    rng = np.random.default_rng(2)
    n, npp = 3 * Lv.n_p2, Lv.n_p1
    f = rng.standard_normal(n)
    g = np.zeros(npp)
    u, p, it, hist = S.solve(f, g, np.zeros(n), np.zeros(npp), rtol=1e-8)
    assert hist[-1] <= 1e-8 * hist[0]
    ud, pd = direct_solve(H, f, g, np.zeros(n), np.zeros(npp))
    assert np.linalg.norm(u - ud) / np.linalg.norm(ud) < 1e-5
    assert np.linalg.norm(p - pd) / np.linalg.norm(pd) < 1e-5


def test_poisson_spectrally_equivalent_to_B_Minv_BT(level1_isoviscous):
    """K_{1/sqrt(eta)} stands for B M_{sqrt(eta)}^-1 B^T (two operators built independently:
    a P1 stiffness matrix, and the divergence blocks around the lumped vector mass): the
    generalised eigenvalues of the pair on the mean-zero space are bounded above and below
    by order-one constants, for a constant and a rough viscosity alike (measured at level 1:
    [0.315, 1.708] with eta = 1, [0.139, 1.383] with the contrast-1e4 plumes); a wrong
    weight exponent would stretch the range by up to the square root of the contrast."""
    Lv, co, cons, S, Bm = level1_isoviscous
    for eta in (np.ones(Lv.n_p1), W.viscosity_plumes(Lv.p1_x, seed=7, contrast=1e4)):
        Wo = WbfbtOperators(Lv, eta)
        n = Lv.n_p1
        X = np.column_stack([co.apply_B(Wo.M_inv(co.apply_BT(e), cons)) for e in np.eye(n)])
        ev = np.linalg.eigvals(np.linalg.solve(Bm.T @ Wo.K.toarray() @ Bm, Bm.T @ X @ Bm)).real
        assert 0.1 < ev.min() and ev.max() < 3.0, (ev.min(), ev.max())


def test_consistent_vector_mass():
    """The consistent M_{sqrt(eta)} (degree-5 rule): f^T M g = sqrt(c) int f g for quadratics
    f, g and eta = c on the polyhedral shell (against cone-by-cone integration of the two
    icosahedra); symmetric positive definite; its constrained inverse inverts P0 M P0 on
    constrained vectors."""
    from oracle.temperature import conical_rule
    from oracle.mesh import icosahedron
    from oracle.fem import Constraints
    Lv = Level(MacroMesh(blending=False), 1)
    x = Lv.p2_x
    f = lambda y: 1 + y[:, 0] - 2 * y[:, 1] * y[:, 2] + 0.5 * y[:, 0] ** 2
    g = lambda y: y[:, 1] ** 2 - y[:, 2] + 0.3 * y[:, 0] * y[:, 1]
    U, F = icosahedron()
    bary, w = conical_rule(4)
    ref = 0.0
    for R, sgn in [(1.0, 1.0), (0.5, -1.0)]:
        for (a, b, c) in F:
            V = np.array([[0, 0, 0], R * U[a], R * U[b], R * U[c]])
            y = bary @ V
            ref += sgn * abs(np.linalg.det(np.stack([V[1] - V[0], V[2] - V[0], V[3] - V[0]], -1))) * (w * f(y) * g(y)).sum()
    O = WbfbtOperators(Lv, np.full(Lv.n_p1, 4.0), mass="consistent")
    assert abs(f(x) @ (O.Mc @ g(x)) - 2.0 * ref) <= 1e-12 * abs(ref)
    assert abs(O.Mc - O.Mc.T).max() <= 1e-15 * abs(O.Mc).max()
    cons = Constraints(Lv)
    v = cons.P0(np.random.default_rng(3).standard_normal(3 * Lv.n_p2))
    Mv = np.concatenate([O.Mc @ v.reshape(3, -1)[c] for c in range(3)])
    assert np.abs(O.M_inv(cons.P0(Mv), cons) - v).max() <= 1e-10 * np.abs(v).max()


def test_consistent_vector_mass_variable_viscosity_and_surface_scaling():
    """Variable viscosity: on the polyhedral shell, where P2 reproduces quadratics f and g,
    f^T M_{sqrt(eta_a)} g is the integral of sqrt(eta_a) f g with eta the P1 interpolant of the
    nodal viscosity; a 512-point conical rule (degree 15) integrates it to far below the
    degree-5 rule's error (sqrt(eta) is not a polynomial: 6e-6 relative here), while a
    dropped square root moves the form by tens of percents.  The scaling a multiplies exactly
    the surface micro-tets' share by a."""
    from oracle.temperature import conical_rule
    Lv = Level(MacroMesh(blending=False), 1)
    eta = 10 ** np.random.default_rng(5).uniform(0.0, 1.0, Lv.n_p1)
    f = lambda y: 1 + y[..., 0] - 2 * y[..., 1] * y[..., 2] + 0.5 * y[..., 0] ** 2
    g = lambda y: y[..., 1] ** 2 - y[..., 2] + 0.3 * y[..., 0] * y[..., 1]
    bary, w = conical_rule(8)
    X = Lv.tet_x                                                       # (E,4,3)
    y = np.einsum("qa,eai->eqi", bary, X)
    det = np.abs(np.linalg.det(np.stack([X[:, 1] - X[:, 0], X[:, 2] - X[:, 0], X[:, 3] - X[:, 0]], -1)))
    etaq = eta[Lv.tet_p1] @ bary.T                                     # (E,Q)
    per_tet = det * ((w * np.sqrt(etaq) * f(y) * g(y)).sum(axis=1))
    surf = surface_tets(Lv)
    x = Lv.p2_x
    M1 = WbfbtOperators(Lv, eta, 1.0, mass="consistent").Mc
    M3 = WbfbtOperators(Lv, eta, 3.0, mass="consistent").Mc
    got1 = f(x) @ (M1 @ g(x))
    assert abs(got1 - per_tet.sum()) <= 1e-4 * abs(per_tet).sum(), (got1, per_tet.sum())
    got3 = f(x) @ (M3 @ g(x))
    assert abs((got3 - got1) - 2.0 * per_tet[surf].sum()) <= 1e-4 * abs(per_tet[surf]).sum()
    # the weight eta instead of sqrt(eta) moves the form well outside that band
    alt = (det * ((w * etaq * f(y) * g(y)).sum(axis=1))).sum()
    assert abs(alt - per_tet.sum()) > 1e-1 * abs(per_tet).sum()
