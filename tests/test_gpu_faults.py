"""Failure handling with host-side injection only (no GPU fault, trap or hang): NaN data,
an iteration cap, calls out of order and bad arguments return status codes."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2506_04157_gb300 as mfs
import workloads as W


@pytest.fixture(scope="module")
def prob():
    ctx = mfs.Context(0)
    mesh = mfs.Mesh(ctx, 2)
    P = mfs.Problem(mesh)
    P.set_viscosity(torch.tensor(W.viscosity_radial(mesh.coords(2, p2=False).T), device="cuda"))
    return ctx, mesh, P


def test_out_of_order_and_bad_arguments(prob):
    ctx, mesh, P = prob
    nu, npp = P._sizes(2)
    f = torch.zeros(nu, dtype=torch.float64, device="cuda")
    with pytest.raises(mfs.MfsError) as e:
        P.vcycle(2, f, torch.empty_like(f))          # multigrid not set up yet
    assert e.value.status == mfs.EINVAL
    lib = mfs.lib()
    y = torch.empty_like(f)
    rc = lib.mfs_apply_A(P.handle, 5, mfs.F64, 0, ctypes.c_void_p(f.data_ptr()), ctypes.c_void_p(y.data_ptr()))
    assert rc == mfs.EINVAL and b"level" in lib.mfs_last_error()
    rc = lib.mfs_apply_A(P.handle, 2, 7, 0, ctypes.c_void_p(f.data_ptr()), ctypes.c_void_p(y.data_ptr()))
    assert rc == mfs.EINVAL
    rc = lib.mfs_apply_A(P.handle, 2, mfs.F64, 0, None, ctypes.c_void_p(y.data_ptr()))
    assert rc == mfs.EINVAL


def test_nan_rhs_and_iteration_cap(prob):
    ctx, mesh, P = prob
    P.setup_multigrid(1)
    nu, npp = P._sizes(2)
    x2 = mesh.coords(2).T
    f = torch.tensor(np.concatenate([W.temperature_blobs(x2, 1)] * 3), device="cuda")
    g = torch.zeros(npp, dtype=torch.float64, device="cuda")
    fbad = f.clone()
    # an interior node: Dirichlet rows of the constrained system ignore f by design
    interior = int(np.flatnonzero(mesh.node_class(2) == 0)[5])
    fbad[interior] = float("nan")
    u = torch.zeros_like(f)
    p = torch.zeros_like(g)
    st = P.solve(fbad, g, u, p, raise_on_error=False)
    assert st["status"] == "MFS_ENAN"
    st = P.solve(f, g, u, p, raise_on_error=False, mixed=3)   # no such precision mode
    assert st["status"] == "MFS_EINVAL"
    st = P.solve(f, g, u, p, raise_on_error=False, uzawa=5)   # no such block preconditioner
    assert st["status"] == "MFS_EINVAL"
    u.zero_()
    p.zero_()
    st = P.solve(f, g, u, p, raise_on_error=False, max_iters=1, max_outer=1)
    assert st["status"] == "MFS_ENOTCONV"
    assert st["fgmres_iters"] == 1 and 0 < st["rel_residual"] < 1
    assert torch.isfinite(u).all() and torch.isfinite(p).all()     # best iterate returned
