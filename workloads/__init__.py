"""Seeded synthetic inputs for the shell Stokes workloads.

This module holds no arithmetic of the discretisation or of the solver: it only turns
node coordinates (from either side) and seeds into input fields, so that the oracle
and the CUDA library are fed identical data.  The geometry and viscosity structure
follow the paper's mantle model (Sec. 7.2: radially layered viscosity modulated
laterally, density rho = rho_top exp(Di/Gamma0 (r_surf - |x|))); the paper's plate
reconstructions and temperature checkpoints are not available, so these synthetic
fields stand in for them.
"""
from __future__ import annotations

import numpy as np

R_CMB, R_SURF = 0.5, 1.0
GAMMA_COMPRESSIBLE = 0.3781      # Di / Gamma_0 of the paper's nondimensional model


def radius(x):
    return np.linalg.norm(np.asarray(x, dtype=np.float64), axis=-1)


def viscosity_radial(x):
    """eta(x) = 10^(2 (1 - |x|) / 0.5): contrast 1e2 across the shell."""
    return 10.0 ** (2.0 * (1.0 - radius(x)) / 0.5)


def _unit_vectors(rng, k):
    v = rng.standard_normal((k, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def viscosity_plumes(x, seed, contrast=1e6, noise_sigma=0.5, n_plumes=4, plume_width=0.15):
    """Radial step at r = 0.75 (factor 1e3) times a lateral plume factor
    1 - 0.99 max_k exp(-theta_k^2 / (2 w^2)) (theta_k = angle to plume axis k, axes
    uniform on the sphere) times log-normal noise exp(sigma xi), xi ~ N(0,1) per node;
    then log eta is affinely rescaled so that max/min = contrast exactly and min = 1.
    x: (n,3) node positions (the nodes carrying eta)."""
    rng = np.random.default_rng(seed)
    x = np.asarray(x, dtype=np.float64)
    r = radius(x)
    xh = x / r[:, None]
    axes = _unit_vectors(rng, n_plumes)
    cosang = np.clip(xh @ axes.T, -1.0, 1.0)
    theta = np.arccos(cosang)
    plume = 1.0 - 0.99 * np.exp(-theta ** 2 / (2 * plume_width ** 2)).max(axis=1)
    xi = rng.standard_normal(x.shape[0])
    log10_eta = 3.0 * (r > 0.75) + np.log10(plume) + (noise_sigma / np.log(10.0)) * xi
    lo, hi = log10_eta.min(), log10_eta.max()
    log10_eta = (log10_eta - lo) / (hi - lo) * np.log10(contrast)
    return 10.0 ** log10_eta


def temperature_blobs(x, seed, n_blobs=8, width=0.1):
    """T = sum_k a_k exp(-|x - c_k|^2 / (2 w^2)), c_k uniform in the shell volume,
    a_k ~ U(-1, 1)."""
    rng = np.random.default_rng(seed)
    centers = []
    while len(centers) < n_blobs:
        c = rng.uniform(-R_SURF, R_SURF, size=3)
        if R_CMB <= np.linalg.norm(c) <= R_SURF:
            centers.append(c)
    centers = np.array(centers)
    amp = rng.uniform(-1.0, 1.0, size=n_blobs)
    x = np.asarray(x, dtype=np.float64)
    d2 = ((x[:, None, :] - centers[None, :, :]) ** 2).sum(-1)
    return (amp[None, :] * np.exp(-d2 / (2 * width ** 2))).sum(1)


def dlnrho_table_config1():
    """rho = exp(-(r - 0.5)): d ln rho / dr = -1 everywhere (2-entry table)."""
    return np.array([-1.0, -1.0])


def dlnrho_table_compressible():
    """rho proportional to exp(0.3781 (1 - r)): d ln rho / dr = -0.3781."""
    return np.array([-GAMMA_COMPRESSIBLE, -GAMMA_COMPRESSIBLE])


def random_field(n, seed, dtype=np.float64):
    """i.i.d. standard normal entries (test vectors for operator parity)."""
    return np.random.default_rng(seed).standard_normal(n).astype(dtype)


WORKLOADS = {
    "shell-L2-contrast1e2": dict(level=2, viscosity="radial", dlnrho="config1"),
    "shell-L5-contrast1e6": dict(level=5, viscosity="plumes", contrast=1e6, eta_seed=2,
                                 T_seed=3, dlnrho="compressible"),
    "shell-L4-contrast1e4-adjoint": dict(level=4, viscosity="plumes", contrast=1e4, eta_seed=5,
                                         T_seed=3, dlnrho="compressible"),
    "shell-L6-contrast1e6": dict(level=6, viscosity="plumes", contrast=1e6, eta_seed=2,
                                 T_seed=3, dlnrho="compressible"),
}


# nondimensional numbers of the paper's mantle model (Table dimtable)
MODEL_RA, MODEL_DI, MODEL_PE = 1.692e7, 0.4538, 2.822e4
T_ADIABATIC_ND = 1600.0 / 3900.0     # T_adiabatic / Delta T


def temperature_adiabat(x, seed, di=MODEL_DI, t_adiabatic=T_ADIABATIC_ND, noise=0.03):
    """Initial temperature of the paper's model (Sec. 7.2): the reference adiabat
    T^s = T_adiabatic exp(Di (r_surf - |x|)) times (1 + noise U(-1, 1)) per node (seeded)."""
    rng = np.random.default_rng(seed)
    ts = t_adiabatic * np.exp(di * (R_SURF - radius(x)))
    return ts * (1.0 + noise * rng.uniform(-1.0, 1.0, ts.shape))

