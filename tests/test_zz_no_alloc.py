"""The allocation-free B apply (mfs_apply_B_noalloc) against mfs_apply_B.

Callers that cannot call cudaMalloc at apply time (code under an external memory manager
that owns all device allocations, or a real-time loop where an allocation would
synchronise the device) use mfs_apply_B_noalloc, whose mean-removal scratch is a fixed
static device array.  This file is named so that pytest collects it last."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2506_04157_gb300 as mfs
import workloads as W

TOL = {torch.float64: 1e-12, torch.float32: 1e-5}


@pytest.fixture(scope="module")
def problem():
    ctx = mfs.Context(0)
    mesh = mfs.Mesh(ctx, 4)
    prob = mfs.Problem(mesh)
    x = mesh.coords(4, p2=False).T
    prob.set_viscosity(torch.tensor(W.viscosity_plumes(x, seed=2, contrast=1e4), device="cuda"))
    prob.set_density(W.dlnrho_table_compressible())
    return ctx, mesh, prob


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("level", [2, 4])
def test_noalloc_matches_apply_B_twice(problem, level, dtype):
    ctx, mesh, prob = problem
    inf = mesh.info(level)
    for call in range(2):   # two calls in a row share the static scratch
        u = torch.tensor(W.random_field(3 * inf.n_p2, 40 + call), dtype=dtype, device="cuda")
        q_ref = torch.empty(inf.n_p1, dtype=dtype, device="cuda")
        q_na = torch.full((inf.n_p1,), float("nan"), dtype=dtype, device="cuda")
        prob.apply_B(level, u, q_ref, with_C=True, constrained=True)
        prob.apply_B_noalloc(level, u, q_na, with_C=True, constrained=True)
        torch.cuda.synchronize()
        a, b = q_na.double().cpu().numpy(), q_ref.double().cpu().numpy()
        assert np.isfinite(a).all()
        assert np.linalg.norm(a - b) / np.linalg.norm(b) <= TOL[dtype]
        assert abs(a.mean()) <= 1e3 * np.finfo(np.float32 if dtype == torch.float32 else np.float64).eps * np.abs(a).max()


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_noalloc_raw_mode_matches_apply_B(problem, dtype):
    """MFS_RAW (no mean removal, so no scratch use): the same as mfs_apply_B's raw block."""
    ctx, mesh, prob = problem
    inf = mesh.info(3)
    u = torch.tensor(W.random_field(3 * inf.n_p2, 44), dtype=dtype, device="cuda")
    q_ref = torch.empty(inf.n_p1, dtype=dtype, device="cuda")
    q_na = torch.empty_like(q_ref)
    prob.apply_B(3, u, q_ref, with_C=True, constrained=False)
    prob.apply_B_noalloc(3, u, q_na, with_C=True, constrained=False)
    a, b = q_na.double().cpu().numpy(), q_ref.double().cpu().numpy()
    assert np.linalg.norm(a - b) / np.linalg.norm(b) <= TOL[dtype]
