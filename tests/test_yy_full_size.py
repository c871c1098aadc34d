"""Full-size parity at level 6 (the largest configured workload), collected after the other
GPU parity modules: constrained fused apply against the oracle's sampled rows
(oracle/sampled.py)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2506_04157_gb300 as mfs
import workloads as W
from oracle.mesh import MacroMesh

TOL = {torch.float64: 1e-12, torch.float32: 1e-5}


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_fused_apply_level6_sampled_rows():
    """The level-6 workload at full size (15,728,640 micro-tets, 66,069,384 dofs; plume
    viscosity of contrast 1e6, seed 2; compressible density), constrained fused apply in FP32
    and FP64.  The oracle evaluates 192 velocity rows and 64 pressure rows at points strictly
    inside macro-tets from the micro-tets of that macro around them (oracle/sampled.py; no
    sphere node among them, so P0 acts as the identity there): velocity rows equal
    A u + B^T P_p p; pressure rows equal (B+C) u up to the one constant P_p removes.  Then 64
    surface and 64 CMB rows at points strictly inside the macro faces on the spheres (owned by
    one macro, Sec. 5.1): the identity at the Dirichlet surface, P_v (A P0 u + B^T P_p p) at the
    free-slip CMB, and 32 pressure rows (B+C) P0 u at sphere vertices, each class checked on
    its own."""
    from oracle.mesh import lattice_nodes
    from oracle.sampled import MacroRows, sample_points, face_points
    lvl = 6
    mesh = MacroMesh()
    R = MacroRows(mesh, lvl)
    X1, _, pr1 = lattice_nodes(mesh, 2 ** lvl)
    eta = W.viscosity_plumes(mesh.blend(X1, pr1), seed=2, contrast=1e6)
    dl = W.dlnrho_table_compressible()
    ctx = mfs.Context(0)
    gm = mfs.Mesh(ctx, lvl)
    prob = mfs.Problem(gm, "dirichlet", "freeslip")
    prob.set_viscosity(torch.tensor(eta, device="cuda"))
    prob.set_density(dl)
    rng = np.random.default_rng(13)
    vel, pre = [], []
    while len(vel) < 192:
        m = int(rng.integers(0, 60))
        vel.append((m, sample_points(2 * R.n, 1, rng)[0]))
    while len(pre) < 64:
        m = int(rng.integers(0, 60))
        pre.append((m, sample_points(R.n, 1, rng)[0]))
    faces = [(m, z, lay) for m in range(60) for z, lay in R.sphere_faces(m)]
    bvel = {1: [], 0: []}   # layer 1 = surface, 0 = CMB
    bpre = []
    while min(len(bvel[1]), len(bvel[0])) < 64:
        m, z, lay = faces[int(rng.integers(0, len(faces)))]
        if len(bvel[lay]) < 64:
            bvel[lay].append((m, face_points(2 * R.n, z, 1, rng)[0]))
    while len(bpre) < 32:
        m, z, lay = faces[int(rng.integers(0, len(faces)))]
        bpre.append((m, face_points(R.n, z, 1, rng)[0]))
    for dtype in (torch.float32, torch.float64):
        u = W.random_field(3 * R.n_p2, 31)
        p = W.random_field(R.n_p1, 32)
        if dtype == torch.float32:
            u = u.astype(np.float32).astype(np.float64)
            p = p.astype(np.float32).astype(np.float64)
        yu = torch.empty(3 * R.n_p2, dtype=dtype, device="cuda")
        yp = torch.empty(R.n_p1, dtype=dtype, device="cuda")
        prob.apply_stokes(lvl, torch.tensor(u, dtype=dtype, device="cuda"),
                          torch.tensor(p, dtype=dtype, device="cuda"), yu, yp)
        yu = yu.cpu().double().numpy()
        yp = yp.cpu().double().numpy()
        pm = p - p.mean()
        got, ref = [], []
        for m, f in vel:
            r = R.velocity_row(m, f, eta, dl, u, pm)
            if r is None:
                continue
            gid, rows = r
            got.append(yu[[gid, gid + R.n_p2, gid + 2 * R.n_p2]])
            ref.append(rows)
        assert len(ref) >= 100
        assert rel(np.concatenate(got), np.concatenate(ref)) <= TOL[dtype]
        d, refp = [], []
        for m, v in pre:
            r = R.pressure_row(m, v, eta, dl, u, pm)
            if r is None:
                continue
            vid, val = r
            d.append(yp[vid] - val)
            refp.append(val)
        d, refp = np.array(d), np.array(refp)
        assert len(refp) >= 30
        c = d.mean()
        assert np.linalg.norm(d - c) <= TOL[dtype] * np.linalg.norm(refp)
        # boundary rows of the constrained operator
        for lay, cls in ((1, 1), (0, 2)):
            got, ref = [], []
            for m, f in bvel[lay]:
                gid, rows, cl = R.constrained_velocity_row(m, f, eta, dl, u, pm)
                assert cl == cls
                got.append(yu[[gid, gid + R.n_p2, gid + 2 * R.n_p2]])
                ref.append(rows)
            assert rel(np.concatenate(got), np.concatenate(ref)) <= TOL[dtype], cls
        d, refp = [], []
        for m, v in bpre:
            vid, val = R.constrained_pressure_row(m, v, eta, dl, u, pm)
            d.append(yp[vid] - val)
            refp.append(val)
        d, refp = np.array(d), np.array(refp)
        assert np.linalg.norm(d - c) <= 2 * TOL[dtype] * np.linalg.norm(refp)
