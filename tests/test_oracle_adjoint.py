"""Pin of the oracle's adjoint gradient against central finite differences of the
objective computed with exact (direct) solves (no GPU)."""
import numpy as np

import workloads as W
from oracle.mesh import MacroMesh, Level
from oracle.solver import Hierarchy, direct_solve
from oracle.adjoint import adjoint_direct, grad_log_eta


def test_oracle_gradient_central_differences():
    M = MacroMesh()
    L = Level(M, 1)
    le = np.log(W.viscosity_plumes(L.p1_x, 5, 1e2))
    npp = L.n_p1
    T = W.temperature_blobs(L.p2_x, 3)
    xh = L.p2_x / np.linalg.norm(L.p2_x, axis=1, keepdims=True)
    f = np.concatenate([T * xh[:, 0], T * xh[:, 1], T * xh[:, 2]])
    surf = np.tile(L.p2_class == 1, 3)

    def J(le):
        H = Hierarchy(M, 1, np.exp(le), bc=(1, 0), l_min=1)
        u, p = direct_solve(H, f, np.zeros(npp), 0 * f, np.zeros(npp))
        d = np.where(surf, u, 0.0)
        return 0.5 * d @ d, u, d, H

    J0, u, d, H = J(le)
    lam, _ = adjoint_direct(H, d, np.zeros(npp))
    g = grad_log_eta(L, np.exp(le), u, lam)
    rng = np.random.default_rng(0)
    h = 1e-6
    for _ in range(3):
        v = rng.standard_normal(npp)
        fd = (J(le + h * v)[0] - J(le - h * v)[0]) / (2 * h)
        assert abs(fd - g @ v) <= 1e-5 * abs(g @ v)
