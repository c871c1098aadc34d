"""Python binding of libmfs: matrix-free blended P2-P1 Stokes on one GB300.

A thin ctypes layer over the C ABI in include/mfs.h: it marshals handles, torch device
pointers and the current CUDA stream; every computation runs in the library's CUDA
kernels.  There is no fallback: if libmfs.so is missing, every call raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libmfs.so")

OK, EINVAL, ENOMEM, ECUDA, ENOTCONV, EBREAKDOWN, ENAN, ETIMEOUT = range(8)
F64, F32 = 0, 1
BC = {"dirichlet": 0, "freeslip": 1}
RAW, CONSTRAINED = 0, 1

_STATUS = {0: "MFS_OK", 1: "MFS_EINVAL", 2: "MFS_ENOMEM", 3: "MFS_ECUDA", 4: "MFS_ENOTCONV",
           5: "MFS_EBREAKDOWN", 6: "MFS_ENAN", 7: "MFS_ETIMEOUT"}


class MfsError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


class LevelInfo(ctypes.Structure):
    _fields_ = [("level", ctypes.c_int), ("n_tets", ctypes.c_int64), ("n_p2", ctypes.c_int64),
                ("n_p1", ctypes.c_int64), ("n_surface", ctypes.c_int64), ("n_cmb", ctypes.c_int64)]


class SolveOpts(ctypes.Structure):
    _fields_ = [("mixed", ctypes.c_int), ("rtol", ctypes.c_double), ("restart", ctypes.c_int),
                ("max_iters", ctypes.c_int), ("max_outer", ctypes.c_int), ("inner_rtol", ctypes.c_double),
                ("sigma", ctypes.c_double), ("omega", ctypes.c_double), ("tol_A", ctypes.c_double),
                ("m_A", ctypes.c_int), ("deg_A", ctypes.c_int), ("tol_VBFBT", ctypes.c_double),
                ("tol_invMass", ctypes.c_double), ("m_V", ctypes.c_int), ("deg_V", ctypes.c_int),
                ("max_cg", ctypes.c_int), ("with_C", ctypes.c_int), ("uzawa", ctypes.c_int),
                ("schur", ctypes.c_int), ("a_l", ctypes.c_double), ("a_r", ctypes.c_double),
                ("tol_wBFBT", ctypes.c_double), ("vmass", ctypes.c_int), ("tol_VectorMass", ctypes.c_double)]


class SolveStats(ctypes.Structure):
    _fields_ = [("outer_iters", ctypes.c_int), ("fgmres_iters", ctypes.c_int), ("cg_A_iters", ctypes.c_int),
                ("cg_X_iters", ctypes.c_int), ("cg_M_iters", ctypes.c_int), ("cg_A_calls", ctypes.c_int),
                ("cg_X_calls", ctypes.c_int), ("cg_M_calls", ctypes.c_int), ("cg_A_max", ctypes.c_int),
                ("cg_X_max", ctypes.c_int), ("cg_M_max", ctypes.c_int), ("vcycles", ctypes.c_int),
                ("applies", ctypes.c_int), ("r0_norm", ctypes.c_double), ("r_norm", ctypes.c_double),
                ("rel_residual", ctypes.c_double), ("time_ms", ctypes.c_double),
                ("time_Ahat_ms", ctypes.c_double), ("time_Sinv_ms", ctypes.c_double),
                ("time_Minv_ms", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class TempParams(ctypes.Structure):
    _fields_ = [("k", ctypes.c_double), ("Pe", ctypes.c_double), ("Cp", ctypes.c_double), ("Di", ctypes.c_double),
                ("alpha", ctypes.c_double), ("H", ctypes.c_double), ("Ra", ctypes.c_double),
                ("tol_T", ctypes.c_double), ("rtol", ctypes.c_double), ("restart", ctypes.c_int),
                ("max_iters", ctypes.c_int), ("max_cg", ctypes.c_int), ("cg_rtol", ctypes.c_double)]


class TempStats(ctypes.Structure):
    _fields_ = [("fgmres_iters", ctypes.c_int), ("cg_iters", ctypes.c_int), ("r0_norm", ctypes.c_double),
                ("r_norm", ctypes.c_double), ("time_ms", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_vp = ctypes.c_void_p
_i = ctypes.c_int
_d = ctypes.c_double
_SIGS = {
    "mfs_last_error": ([], ctypes.c_char_p),
    "mfs_version": ([], ctypes.c_char_p),
    "mfs_ctx_create": ([_i, _vp, ctypes.POINTER(_vp)], _i),
    "mfs_ctx_set_stream": ([_vp, _vp], _i),
    "mfs_ctx_destroy": ([_vp], _i),
    "mfs_ctx_timing": ([_vp, _i], _i),
    "mfs_ctx_kernel_time": ([_vp, ctypes.POINTER(_d), ctypes.POINTER(ctypes.c_int64)], _i),
    "mfs_mesh_shell": ([_vp, _d, _d, _i, _i, ctypes.POINTER(_vp)], _i),
    "mfs_mesh_destroy": ([_vp], _i),
    "mfs_mesh_info": ([_vp, _i, ctypes.POINTER(LevelInfo)], _i),
    "mfs_mesh_coords": ([_vp, _i, _i, _i, _vp], _i),
    "mfs_mesh_node_class": ([_vp, _i, _i, _vp], _i),
    "mfs_problem_create": ([_vp, _i, _i, ctypes.POINTER(_vp)], _i),
    "mfs_problem_destroy": ([_vp], _i),
    "mfs_set_viscosity": ([_vp, _vp, _i], _i),
    "mfs_set_density": ([_vp, _i, _vp], _i),
    "mfs_set_constraint_form": ([_vp, _i], _i),
    "mfs_apply_A": ([_vp, _i, _i, _i, _vp, _vp], _i),
    "mfs_apply_B": ([_vp, _i, _i, _i, _i, _vp, _vp], _i),
    "mfs_apply_BT": ([_vp, _i, _i, _i, _i, _vp, _vp], _i),
    "mfs_apply_stokes": ([_vp, _i, _i, _i, _vp, _vp, _vp, _vp], _i),
    "mfs_apply_B_noalloc": ([_vp, _i, _i, _i, _i, _vp, _vp], _i),
    "mfs_fma_peak": ([_vp, _i, _i, _i, ctypes.POINTER(_d), ctypes.POINTER(_d)], _i),
    "mfs_apply_part": ([_vp, _i, _i, _i, _i, _i, _vp, _vp, _vp, _vp], _i),
    "mfs_mesh_macro_topology": ([_vp, _vp, _vp, _vp], _i),
    "mfs_setup_multigrid": ([_vp, _i], _i),
    "mfs_set_cheb_bounds": ([_vp, _i, _d, _d], _i),
    "mfs_get_cheb_bounds": ([_vp, _i, ctypes.POINTER(_d), ctypes.POINTER(_d)], _i),
    "mfs_estimate_cheb_bounds": ([_vp, _i, _vp, ctypes.POINTER(_d)], _i),
    "mfs_diag_A": ([_vp, _i, _i, _vp], _i),
    "mfs_apply_mass": ([_vp, _i, _i, _vp, _vp], _i),
    "mfs_prolongate": ([_vp, _i, _i, _vp, _vp], _i),
    "mfs_restrict": ([_vp, _i, _i, _vp, _vp], _i),
    "mfs_project": ([_vp, _i, _i, _vp], _i),
    "mfs_mg_checkpoint": ([_vp, ctypes.POINTER(_vp)], _i),
    "mfs_mg_restore": ([_vp, _vp], _i),
    "mfs_mg_state_destroy": ([_vp], _i),
    "mfs_vcycle": ([_vp, _i, _i, _i, _i, _vp, _vp], _i),
    "mfs_solve_opts_default": ([ctypes.POINTER(SolveOpts)], None),
    "mfs_adjoint_solve": ([_vp, ctypes.POINTER(SolveOpts), _vp, _vp, _vp, _vp, ctypes.POINTER(SolveStats)], _i),
    "mfs_grad_log_eta": ([_vp, _vp, _vp, _vp], _i),
    "mfs_autotune": ([_vp, ctypes.c_char_p], _i),
    "mfs_set_viscosity_law": ([_vp, _d, _d, _i, _vp, _i], _i),
    "mfs_set_temperature": ([_vp, _vp], _i),
    "mfs_rhs_buoyancy": ([_vp, _vp, _d, _vp], _i),
    "mfs_get_tuning": ([_vp, _i, ctypes.POINTER(_i)], _i),
    "mfs_set_tuning": ([_vp, _i, _i], _i),
    "mfs_batch_create": ([_vp, _i, _vp, ctypes.POINTER(_vp)], _i),
    "mfs_batch_destroy": ([_vp], _i),
    "mfs_batch_apply_stokes": ([_vp, _i, _i, _vp, _vp, _vp, _vp], _i),
    "mfs_batch_solve": ([_vp, ctypes.POINTER(SolveOpts), _vp, _vp, _vp, _vp, _vp], _i),
    "mfs_solve_concurrent": ([_i, _vp, ctypes.POINTER(SolveOpts), _vp, _vp, _vp, _vp, _vp, _i], _i),
    "mfs_stokes_solve": ([_vp, ctypes.POINTER(SolveOpts), _vp, _vp, _vp, _vp, ctypes.POINTER(SolveStats)], _i),
    "mfs_apply_schur": ([_vp, ctypes.POINTER(SolveOpts), _i, _vp, _vp, ctypes.POINTER(SolveStats)], _i),
    "mfs_apply_poisson": ([_vp, _i, _i, _d, _vp, _vp], _i),
    "mfs_lumped_vmass": ([_vp, _d, _vp], _i),
    "mfs_apply_vmass": ([_vp, _i, _d, _vp, _vp], _i),
    "mfs_temp_rule": ([_vp, _vp], _i),
    "mfs_mesh_prolongation": ([_vp, _i, _vp, _vp, _vp, _vp], _i),
    "mfs_mesh_p1_interpolation": ([_vp, _i, _vp, _vp, _vp, _vp], _i),
    "mfs_mesh_law_maps": ([_vp, _i, _vp, _vp, _vp], _i),
    "mfs_mmoc_host": ([_vp, _i, _vp, _vp, _vp, _vp, _d, _vp, _vp], _i),
    "mfs_temp_params_default": ([ctypes.POINTER(TempParams)], None),
    "mfs_temp_apply": ([_vp, _i, _d, _d, _d, _d, _i, _i, _vp, _vp, _vp], _i),
    "mfs_temp_rhs": ([_vp, ctypes.POINTER(TempParams), _vp, _vp, _vp, _vp, _d, _d, _vp], _i),
    "mfs_mmoc": ([_vp, _vp, _vp, _vp, _d, _vp, _vp, _vp], _i),
    "mfs_temperature_step": ([_vp, ctypes.POINTER(TempParams), _vp, _vp, _vp, _vp, _d, _d, _vp, _vp,
                              ctypes.POINTER(TempStats)], _i),
}

_lib = None


def lib():
    """The loaded libmfs.so (raises MfsError if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise MfsError(EINVAL, f"{LIB_PATH} not built (python -m paper_2506_04157_gb300.build)")
        L = ctypes.CDLL(LIB_PATH)
        for name, (args, res) in _SIGS.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


def _check(status):
    if status != OK:
        raise MfsError(status, lib().mfs_last_error().decode())


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def _prec_of(t):
    import torch
    if t.dtype == torch.float64:
        return F64
    if t.dtype == torch.float32:
        return F32
    raise MfsError(EINVAL, f"unsupported dtype {t.dtype}")


def _need(t, n, dtype=None, name="tensor"):
    if not t.is_cuda or not t.is_contiguous():
        raise MfsError(EINVAL, f"{name} must be a contiguous CUDA tensor")
    if t.numel() != n:
        raise MfsError(EINVAL, f"{name} has {t.numel()} entries, expected {n}")
    if dtype is not None and t.dtype != dtype:
        raise MfsError(EINVAL, f"{name} has dtype {t.dtype}, expected {dtype}")


class Context:
    """Device + stream; the stream defaults to torch's current stream."""

    def __init__(self, device=0, stream=None):
        if stream is None:
            import torch
            stream = torch.cuda.current_stream(device).cuda_stream
        h = ctypes.c_void_p()
        _check(lib().mfs_ctx_create(device, ctypes.c_void_p(stream), ctypes.byref(h)))
        self.handle, self.device = h, device

    def set_stream(self, stream):
        _check(lib().mfs_ctx_set_stream(self.handle, ctypes.c_void_p(stream)))

    def enable_timing(self, on=True):
        _check(lib().mfs_ctx_timing(self.handle, int(on)))

    def fma_peak(self, kind, launches=10, iters=20000):
        """(TFLOP/s, ms) of the FMA-chain throughput kernel: kind "f32", "f32x2" or "f64"."""
        k = {"f32": 0, "f32x2": 1, "f64": 2}[kind]
        tf, ms = ctypes.c_double(), ctypes.c_double()
        _check(lib().mfs_fma_peak(self.handle, k, launches, iters, ctypes.byref(tf), ctypes.byref(ms)))
        return tf.value, ms.value

    def kernel_time(self):
        """(total ms, launches) of the timed element-sweep kernels since the last call."""
        ms, n = ctypes.c_double(), ctypes.c_int64()
        _check(lib().mfs_ctx_kernel_time(self.handle, ctypes.byref(ms), ctypes.byref(n)))
        return ms.value, n.value

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.mfs_ctx_destroy(self.handle)
            self.handle = None


class Mesh:
    """Blended icosahedral shell mesh with levels 0..l_max (ctx=None: host-only)."""

    def __init__(self, ctx, l_max, r_cmb=0.5, r_surf=1.0, blending=True):
        h = ctypes.c_void_p()
        _check(lib().mfs_mesh_shell(ctx.handle if ctx is not None else None, r_cmb, r_surf, l_max,
                                    1 if blending else 0, ctypes.byref(h)))
        self.handle, self.ctx, self.l_max = h, ctx, l_max
        self.r_cmb, self.r_surf = r_cmb, r_surf

    def info(self, level):
        out = LevelInfo()
        _check(lib().mfs_mesh_info(self.handle, level, ctypes.byref(out)))
        return out

    def coords(self, level, p2=True, blended=True):
        n = self.info(level).n_p2 if p2 else self.info(level).n_p1
        buf = np.empty((3, n), dtype=np.float64)
        _check(lib().mfs_mesh_coords(self.handle, level, int(p2), int(blended),
                                     buf.ctypes.data_as(ctypes.c_void_p)))
        return buf

    def prolongation(self, level):
        """(rp, ci, w): CSR of the scalar P2 prolongation from level-1 to level (host)."""
        nnz = ctypes.c_int()
        _check(lib().mfs_mesh_prolongation(self.handle, level, ctypes.byref(nnz), None, None, None))
        rp = np.empty(self.info(level).n_p2 + 1, dtype=np.int32)
        ci = np.empty(nnz.value, dtype=np.int32)
        w = np.empty(nnz.value, dtype=np.float64)
        vp = lambda a: a.ctypes.data_as(ctypes.c_void_p)
        _check(lib().mfs_mesh_prolongation(self.handle, level, ctypes.byref(nnz), vp(rp), vp(ci), vp(w)))
        return rp, ci, w

    def p1_interpolation(self, level):
        """(coarse, fine, w): triplets of the P1 interpolation from level-1 to level (host)."""
        nnz = ctypes.c_int()
        _check(lib().mfs_mesh_p1_interpolation(self.handle, level, ctypes.byref(nnz), None, None, None))
        cv = np.empty(nnz.value, dtype=np.int32)
        fv = np.empty(nnz.value, dtype=np.int32)
        w = np.empty(nnz.value, dtype=np.float64)
        vp = lambda a: a.ctypes.data_as(ctypes.c_void_p)
        _check(lib().mfs_mesh_p1_interpolation(self.handle, level, ctypes.byref(nnz), vp(cv), vp(fv), vp(w)))
        return cv, fv, w

    def law_maps(self, level):
        """(vfine, vrad, p2fine): the viscosity law's finest-node maps of a level (host)."""
        inf = self.info(level)
        vfine = np.empty(inf.n_p1, dtype=np.int32)
        vrad = np.empty(inf.n_p1, dtype=np.float64)
        p2fine = np.empty(inf.n_p2, dtype=np.int32)
        vp = lambda a: a.ctypes.data_as(ctypes.c_void_p)
        _check(lib().mfs_mesh_law_maps(self.handle, level, vp(vfine), vp(vrad), vp(p2fine)))
        return vfine, vrad, p2fine

    def mmoc_host(self, X_start, T, u_new, u_old, tau):
        """(T_hat, X_dep): the MMOC particle step on the host for particles at X_start (n, 3);
        T [n_p2], u_new, u_old [3 n_p2] on the finest level (numpy float64)."""
        X = np.ascontiguousarray(np.asarray(X_start, dtype=np.float64).T)
        n = X.shape[1]
        n2 = self.info(self.l_max).n_p2
        T = np.ascontiguousarray(T, dtype=np.float64)
        un = np.ascontiguousarray(u_new, dtype=np.float64)
        uo = np.ascontiguousarray(u_old, dtype=np.float64)
        if T.size != n2 or un.size != 3 * n2 or uo.size != 3 * n2:
            raise ValueError("T needs n_p2 and u_new, u_old 3 n_p2 entries of the finest level")
        Th = np.empty(n)
        Xo = np.empty((3, n))
        vp = lambda a: a.ctypes.data_as(ctypes.c_void_p)
        _check(lib().mfs_mmoc_host(self.handle, n, vp(X), vp(T), vp(un), vp(uo), tau, vp(Th), vp(Xo)))
        return Th, Xo.T

    def macro_topology(self):
        """(cells [60,4], edges [60,6], faces [60,4]): global vertex, macro-edge and macro-face
        ids of every macro-tet (host, int32)."""
        cells = np.empty((60, 4), dtype=np.int32)
        edges = np.empty((60, 6), dtype=np.int32)
        faces = np.empty((60, 4), dtype=np.int32)
        vp = lambda a: a.ctypes.data_as(ctypes.c_void_p)
        _check(lib().mfs_mesh_macro_topology(self.handle, vp(cells), vp(edges), vp(faces)))
        return cells, edges, faces

    def node_class(self, level, p2=True):
        n = self.info(level).n_p2 if p2 else self.info(level).n_p1
        buf = np.empty(n, dtype=np.int8)
        _check(lib().mfs_mesh_node_class(self.handle, level, int(p2), buf.ctypes.data_as(ctypes.c_void_p)))
        return buf

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.mfs_mesh_destroy(self.handle)
            self.handle = None


class Problem:
    """Mesh + boundary conditions + viscosity/density; operator applies on torch tensors."""

    def __init__(self, mesh, bc_surface="dirichlet", bc_cmb="freeslip"):
        h = ctypes.c_void_p()
        _check(lib().mfs_problem_create(mesh.handle, BC[bc_surface], BC[bc_cmb], ctypes.byref(h)))
        self.handle, self.mesh = h, mesh

    def set_viscosity(self, eta, is_log=False):
        import torch
        _need(eta, self.mesh.info(self.mesh.l_max).n_p1, torch.float64, "eta")
        _check(lib().mfs_set_viscosity(self.handle, _ptr(eta), int(is_log)))

    def set_density(self, dlnrho_dr):
        t = np.ascontiguousarray(np.atleast_1d(dlnrho_dr), dtype=np.float64)
        _check(lib().mfs_set_density(self.handle, t.size, t.ctypes.data_as(ctypes.c_void_p)))

    def set_constraint_form(self, rho_weighted):
        """The constraint row: the paper's B + C (False) or -int q div(rho u) (True)."""
        _check(lib().mfs_set_constraint_form(self.handle, int(bool(rho_weighted))))

    def _sizes(self, level):
        inf = self.mesh.info(level)
        return 3 * inf.n_p2, inf.n_p1

    def apply_A(self, level, u, y, constrained=False):
        nu, _ = self._sizes(level)
        _need(u, nu, None, "u"); _need(y, nu, u.dtype, "y")
        _check(lib().mfs_apply_A(self.handle, level, _prec_of(u), int(constrained), _ptr(u), _ptr(y)))

    def apply_B(self, level, u, q, with_C=True, constrained=False):
        nu, npp = self._sizes(level)
        _need(u, nu, None, "u"); _need(q, npp, u.dtype, "q")
        _check(lib().mfs_apply_B(self.handle, level, _prec_of(u), int(constrained), int(with_C),
                                 _ptr(u), _ptr(q)))

    def apply_part(self, level, m0, m1, u, yu, p=None, yp=None):
        """Partial constrained apply over macros m0 <= m < m1 (mfs_apply_part): A_c alone when p
        is None, else the fused [A_c, P0 B^T; (B+C) P0] with p used as given and yp not made
        mean-free."""
        nu, npp = self._sizes(level)
        _need(u, nu, None, "u"); _need(yu, nu, u.dtype, "yu")
        fused = p is not None
        if fused:
            _need(p, npp, u.dtype, "p"); _need(yp, npp, u.dtype, "yp")
        _check(lib().mfs_apply_part(self.handle, level, _prec_of(u), int(fused), m0, m1, _ptr(u),
                                    _ptr(p) if fused else None, _ptr(yu), _ptr(yp) if fused else None))

    def apply_B_noalloc(self, level, u, q, with_C=True, constrained=False):
        """mfs_apply_B without device allocation: the mean-removal scratch lives in a
        fixed static device array (for callers that cannot call cudaMalloc)."""
        nu, npp = self._sizes(level)
        _need(u, nu, None, "u"); _need(q, npp, u.dtype, "q")
        _check(lib().mfs_apply_B_noalloc(self.handle, level, _prec_of(u), int(constrained), int(with_C),
                                         _ptr(u), _ptr(q)))

    def apply_BT(self, level, p, y, with_C=False, constrained=False):
        nu, npp = self._sizes(level)
        _need(p, npp, None, "p"); _need(y, nu, p.dtype, "y")
        _check(lib().mfs_apply_BT(self.handle, level, _prec_of(p), int(constrained), int(with_C),
                                  _ptr(p), _ptr(y)))

    def apply_stokes(self, level, u, p, yu, yp, transpose=False):
        nu, npp = self._sizes(level)
        _need(u, nu, None, "u"); _need(p, npp, u.dtype, "p")
        _need(yu, nu, u.dtype, "yu"); _need(yp, npp, u.dtype, "yp")
        _check(lib().mfs_apply_stokes(self.handle, level, _prec_of(u), int(transpose), _ptr(u), _ptr(p),
                                      _ptr(yu), _ptr(yp)))

    # ---- multigrid layer
    def setup_multigrid(self, l_min=1):
        _check(lib().mfs_setup_multigrid(self.handle, l_min))

    def set_cheb_bounds(self, level, lo, hi):
        _check(lib().mfs_set_cheb_bounds(self.handle, level, lo, hi))

    def cheb_bounds(self, level):
        lo, hi = ctypes.c_double(), ctypes.c_double()
        _check(lib().mfs_get_cheb_bounds(self.handle, level, ctypes.byref(lo), ctypes.byref(hi)))
        return lo.value, hi.value

    def mg_checkpoint(self):
        """Device copy of the viscosity-dependent multigrid state (MgState; restore with
        mg_restore)."""
        h = ctypes.c_void_p()
        _check(lib().mfs_mg_checkpoint(self.handle, ctypes.byref(h)))
        return MgState(h)

    def mg_restore(self, state):
        _check(lib().mfs_mg_restore(self.handle, state.handle))

    def estimate_cheb_bounds(self, level, x0):
        """Re-run the power iteration of the level's Chebyshev interval from x0 (FP64 CUDA
        tensor [3 n_p2]); returns the eigenvalue estimate."""
        import torch
        nu, _ = self._sizes(level)
        _need(x0, nu, torch.float64, "x0")
        lam = ctypes.c_double()
        _check(lib().mfs_estimate_cheb_bounds(self.handle, level, _ptr(x0), ctypes.byref(lam)))
        return lam.value

    def diag_A(self, level, y):
        nu, _ = self._sizes(level)
        _need(y, nu, None, "y")
        _check(lib().mfs_diag_A(self.handle, level, _prec_of(y), _ptr(y)))

    def apply_mass(self, level, p, y):
        _, npp = self._sizes(level)
        _need(p, npp, None, "p"); _need(y, npp, p.dtype, "y")
        _check(lib().mfs_apply_mass(self.handle, level, _prec_of(p), _ptr(p), _ptr(y)))

    def apply_poisson(self, level, a, p, y):
        """y = K_{1/sqrt(eta_a)} p (weighted-BFBT Poisson operator) on a multigrid level."""
        _, npp = self._sizes(level)
        _need(p, npp, None, "p"); _need(y, npp, p.dtype, "y")
        _check(lib().mfs_apply_poisson(self.handle, level, _prec_of(p), float(a), _ptr(p), _ptr(y)))

    def lumped_vmass(self, a, d):
        """d = lumped M_{sqrt(eta_a)} diagonal (one FP64 entry per P2 node, finest level)."""
        import torch
        nu, _ = self._sizes(self.mesh.l_max)
        _need(d, nu // 3, torch.float64, "d")
        _check(lib().mfs_lumped_vmass(self.handle, float(a), _ptr(d)))

    def apply_vmass(self, a, x, y):
        """y = consistent M_{sqrt(eta_a)} x on the three velocity components ([3][n_p2], finest
        level; FP64 or FP32, no boundary rows removed)."""
        nu, _ = self._sizes(self.mesh.l_max)
        _need(x, nu, None, "x"); _need(y, nu, x.dtype, "y")
        _check(lib().mfs_apply_vmass(self.handle, _prec_of(x), float(a), _ptr(x), _ptr(y)))

    def prolongate(self, level, xc, xf):
        nf, _ = self._sizes(level)
        nc, _ = self._sizes(level - 1)
        _need(xc, nc, None, "xc"); _need(xf, nf, xc.dtype, "xf")
        _check(lib().mfs_prolongate(self.handle, level, _prec_of(xc), _ptr(xc), _ptr(xf)))

    def restrict(self, level, rf, rc):
        nf, _ = self._sizes(level)
        nc, _ = self._sizes(level - 1)
        _need(rf, nf, None, "rf"); _need(rc, nc, rf.dtype, "rc")
        _check(lib().mfs_restrict(self.handle, level, _prec_of(rf), _ptr(rf), _ptr(rc)))

    def project(self, level, x):
        """x <- P0 x in place (Dirichlet entries zeroed, free-slip nodes projected)."""
        nu, _ = self._sizes(level)
        _need(x, nu, None, "x")
        _check(lib().mfs_project(self.handle, level, _prec_of(x), _ptr(x)))

    def vcycle(self, level, f, u, steps=3, degree=2):
        nu, _ = self._sizes(level)
        _need(f, nu, None, "f"); _need(u, nu, f.dtype, "u")
        _check(lib().mfs_vcycle(self.handle, level, _prec_of(f), steps, degree, _ptr(f), _ptr(u)))

    def set_viscosity_law(self, log10_base, E_A=4.610, V_A=2.996, l_eta=-1):
        """Frank-Kamenetskii viscosity law; quadrature-point viscosity on levels <= l_eta."""
        tab = np.ascontiguousarray(np.asarray(log10_base, dtype=np.float64).ravel())
        _check(lib().mfs_set_viscosity_law(self.handle, float(E_A), float(V_A), tab.size,
                                            tab.ctypes.data_as(ctypes.c_void_p), int(l_eta)))

    def set_temperature(self, T_p2):
        """Finest-level P2 temperature (FP64 device tensor): sets the viscosity from the law."""
        import torch
        nu, _ = self._sizes(self.mesh.l_max)
        _need(T_p2, nu // 3, torch.float64, "T_p2")
        _check(lib().mfs_set_temperature(self.handle, _ptr(T_p2)))

    def rhs_buoyancy(self, T_p2, f, scale=1.0):
        """f = scale * int rho T (x/|x|) . phi (FP64 device tensors: T [n_p2], f [3 n_p2])."""
        import torch
        nu, _ = self._sizes(self.mesh.l_max)
        _need(T_p2, nu // 3, torch.float64, "T_p2"); _need(f, nu, torch.float64, "f")
        _check(lib().mfs_rhs_buoyancy(self.handle, _ptr(T_p2), float(scale), _ptr(f)))

    # ---- autotuning
    def set_tuning(self, level, variant):
        """Select the sweep launch variant of a level by hand (0..8, see include/mfs.h)."""
        _check(lib().mfs_set_tuning(self.handle, level, variant))

    def get_tuning(self, level):
        """The sweep launch variant in use on a level."""
        v = ctypes.c_int()
        _check(lib().mfs_get_tuning(self.handle, level, ctypes.byref(v)))
        return v.value

    def autotune(self, cache_path=None):
        """Pick the fastest sweep variant per level (cached in cache_path if given)."""
        _check(lib().mfs_autotune(self.handle, cache_path.encode() if cache_path else None))
        out = []
        for l in range(self.mesh.l_max + 1):
            v = ctypes.c_int()
            _check(lib().mfs_get_tuning(self.handle, l, ctypes.byref(v)))
            out.append(v.value)
        return out

    # ---- Stokes solver
    @staticmethod
    def default_opts(**kw):
        o = SolveOpts()
        lib().mfs_solve_opts_default(ctypes.byref(o))
        for k, v in kw.items():
            if not hasattr(o, k):
                raise MfsError(EINVAL, f"unknown solver option {k}")
            setattr(o, k, v)
        return o

    def solve(self, f, g, u, p, raise_on_error=True, **opts):
        """Solve the projected Stokes system in place (u, p: FP64 device tensors holding
        the initial guess / Dirichlet values).  Returns the statistics as a dict
        (with the status under 'status')."""
        import torch
        L = self.mesh.l_max
        nu, npp = self._sizes(L)
        _need(f, nu, torch.float64, "f"); _need(g, npp, torch.float64, "g")
        _need(u, nu, torch.float64, "u"); _need(p, npp, torch.float64, "p")
        o = self.default_opts(**opts)
        st = SolveStats()
        rc = lib().mfs_stokes_solve(self.handle, ctypes.byref(o), _ptr(f), _ptr(g), _ptr(u), _ptr(p),
                                    ctypes.byref(st))
        d = st.as_dict()
        d["status"] = _STATUS.get(rc, rc)
        if rc != OK and raise_on_error:
            raise MfsError(rc, lib().mfs_last_error().decode())
        return d

    def apply_schur(self, r, z, **opts):
        """z = S^-1 r for the Schur approximation opts['schur'] (finest level, precision of r);
        returns the statistics as a dict."""
        _, npp = self._sizes(self.mesh.l_max)
        _need(r, npp, None, "r"); _need(z, npp, r.dtype, "z")
        o = self.default_opts(**opts)
        st = SolveStats()
        _check(lib().mfs_apply_schur(self.handle, ctypes.byref(o), _prec_of(r), _ptr(r), _ptr(z), ctypes.byref(st)))
        return st.as_dict()

    # ---- temperature step (finest level; FP64 unless stated)
    @staticmethod
    def temp_params(**kw):
        o = TempParams()
        lib().mfs_temp_params_default(ctypes.byref(o))
        for k, v in kw.items():
            if not hasattr(o, k):
                raise MfsError(EINVAL, f"unknown temperature parameter {k}")
            setattr(o, k, v)
        return o

    def temp_apply(self, x, y, cM=1.0, cC=0.0, cD=0.0, cR=0.0, u=None, sym=False, constrained=False):
        """y = (cM M + cC C(u) + cD D + cR R(u)) x (precision of x)."""
        nu, _ = self._sizes(self.mesh.l_max)
        _need(x, nu // 3, None, "x"); _need(y, nu // 3, x.dtype, "y")
        if u is not None:
            _need(u, nu, x.dtype, "u")
        _check(lib().mfs_temp_apply(self.handle, _prec_of(x), cM, cC, cD, cR, int(sym), int(constrained),
                                    _ptr(u) if u is not None else None, _ptr(x), _ptr(y)))

    def temp_rhs(self, T0_hat, Tm_hat, tau_np1, tau_n, b, u_star=None, T_star=None, **params):
        import torch
        nu, _ = self._sizes(self.mesh.l_max)
        for t, nm in [(T0_hat, "T0_hat"), (Tm_hat, "Tm_hat"), (b, "b")]:
            _need(t, nu // 3, torch.float64, nm)
        o = self.temp_params(**params)
        _check(lib().mfs_temp_rhs(self.handle, ctypes.byref(o), _ptr(T0_hat), _ptr(Tm_hat),
                                  _ptr(u_star) if u_star is not None else None,
                                  _ptr(T_star) if T_star is not None else None, tau_np1, tau_n, _ptr(b)))

    def mmoc(self, T, u_new, u_old, tau, T_hat, X_dep=None, X_start=None):
        """T_hat = T at the departure points of particles starting at the P2 nodes (or at
        X_start [3][n_p2]) after one RK4 step back over tau; X_dep receives those points."""
        import torch
        nu, _ = self._sizes(self.mesh.l_max)
        _need(T, nu // 3, torch.float64, "T"); _need(T_hat, nu // 3, torch.float64, "T_hat")
        _need(u_new, nu, torch.float64, "u_new"); _need(u_old, nu, torch.float64, "u_old")
        for t, name in ((X_dep, "X_dep"), (X_start, "X_start")):
            if t is not None:
                _need(t, nu, torch.float64, name)
        _check(lib().mfs_mmoc(self.handle, _ptr(T), _ptr(u_new), _ptr(u_old), tau,
                              _ptr(X_start) if X_start is not None else None, _ptr(T_hat),
                              _ptr(X_dep) if X_dep is not None else None))

    def temperature_step(self, T_n, T_nm1, u_n, u_nm1, tau_np1, tau_n, T_bc, T_np1, raise_on_error=True, **params):
        """One temperature step; returns the statistics as a dict (status under 'status')."""
        import torch
        nu, _ = self._sizes(self.mesh.l_max)
        for t, nm in [(T_n, "T_n"), (T_nm1, "T_nm1"), (T_bc, "T_bc"), (T_np1, "T_np1")]:
            _need(t, nu // 3, torch.float64, nm)
        _need(u_n, nu, torch.float64, "u_n"); _need(u_nm1, nu, torch.float64, "u_nm1")
        o = self.temp_params(**params)
        st = TempStats()
        rc = lib().mfs_temperature_step(self.handle, ctypes.byref(o), _ptr(T_n), _ptr(T_nm1), _ptr(u_n), _ptr(u_nm1),
                                        tau_np1, tau_n, _ptr(T_bc), _ptr(T_np1), ctypes.byref(st))
        d = st.as_dict()
        d["status"] = _STATUS.get(rc, rc)
        if rc != OK and raise_on_error:
            raise MfsError(rc, lib().mfs_last_error().decode())
        return d

    def adjoint_solve(self, ju, jp, lam_u, lam_p, raise_on_error=True, **opts):
        """Solve K^T lam = (ju, jp) in place (FP64 device tensors); returns statistics."""
        import torch
        L = self.mesh.l_max
        nu, npp = self._sizes(L)
        _need(ju, nu, torch.float64, "ju"); _need(jp, npp, torch.float64, "jp")
        _need(lam_u, nu, torch.float64, "lam_u"); _need(lam_p, npp, torch.float64, "lam_p")
        o = self.default_opts(**opts)
        st = SolveStats()
        rc = lib().mfs_adjoint_solve(self.handle, ctypes.byref(o), _ptr(ju), _ptr(jp), _ptr(lam_u), _ptr(lam_p),
                                     ctypes.byref(st))
        d = st.as_dict()
        d["status"] = _STATUS.get(rc, rc)
        if rc != OK and raise_on_error:
            raise MfsError(rc, lib().mfs_last_error().decode())
        return d

    def grad_log_eta(self, u, lam_u, g):
        import torch
        L = self.mesh.l_max
        nu, npp = self._sizes(L)
        _need(u, nu, torch.float64, "u"); _need(lam_u, nu, torch.float64, "lam_u")
        _need(g, npp, torch.float64, "g")
        _check(lib().mfs_grad_log_eta(self.handle, _ptr(u), _ptr(lam_u), _ptr(g)))

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.mfs_problem_destroy(self.handle)
            self.handle = None


def temp_rule():
    """(barycentrics [27, 4], weights [27]) of the library's degree-5 conical rule (host)."""
    lam = np.empty((27, 4), dtype=np.float64)
    w = np.empty(27, dtype=np.float64)
    _check(lib().mfs_temp_rule(lam.ctypes.data_as(ctypes.c_void_p), w.ctypes.data_as(ctypes.c_void_p)))
    return lam, w


def _ptr_array(tensors):
    arr = (ctypes.c_void_p * len(tensors))(*[t.data_ptr() for t in tensors])
    return arr


class MgState:
    """A checkpoint of a problem's viscosity-dependent multigrid state (mfs_mg_checkpoint)."""

    def __init__(self, handle):
        self.handle = handle

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.mfs_mg_state_destroy(self.handle)
            self.handle = None


class Batch:
    """An ensemble of problems on one context: one sweep launch applies all of them."""

    def __init__(self, ctx, problems):
        self.problems = list(problems)
        h = ctypes.c_void_p()
        arr = (ctypes.c_void_p * len(self.problems))(*[p.handle.value for p in self.problems])
        _check(lib().mfs_batch_create(ctx.handle, len(self.problems), arr, ctypes.byref(h)))
        self.handle, self.ctx = h, ctx

    def apply_stokes(self, us, ps, yus, yps, transpose=False):
        for P, u, p, yu, yp in zip(self.problems, us, ps, yus, yps):
            nu, npp = P._sizes(P.mesh.l_max)
            _need(u, nu, None, "u"); _need(p, npp, u.dtype, "p")
            _need(yu, nu, u.dtype, "yu"); _need(yp, npp, u.dtype, "yp")
        prec = _prec_of(us[0])
        _check(lib().mfs_batch_apply_stokes(self.handle, prec, int(transpose), _ptr_array(us), _ptr_array(ps),
                                            _ptr_array(yus), _ptr_array(yps)))

    def solve(self, fs, gs, us, ps, **opts):
        o = Problem.default_opts(**opts)
        stats = (SolveStats * len(self.problems))()
        rc = lib().mfs_batch_solve(self.handle, ctypes.byref(o), _ptr_array(fs), _ptr_array(gs), _ptr_array(us),
                                   _ptr_array(ps), stats)
        if rc != OK:
            raise MfsError(rc, lib().mfs_last_error().decode())
        return [s.as_dict() for s in stats]

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.mfs_batch_destroy(self.handle)
            self.handle = None


def solve_concurrent(problems, fs, gs, us, ps, n_threads=0, raise_on_error=True, **opts):
    """mfs_stokes_solve for every problem, the problems of different contexts (streams) at the
    same time (mfs_solve_concurrent): one host thread per context works through its problems
    in turn.  fs, gs, us, ps: FP64 device tensors per problem (us, ps: initial guesses, solved
    in place).  Returns the statistics per problem (dicts with 'status')."""
    import torch
    probs = list(problems)
    if not (len(probs) == len(fs) == len(gs) == len(us) == len(ps)):
        raise MfsError(EINVAL, "one right-hand side and one solution per problem")
    for P, f, g, u, p in zip(probs, fs, gs, us, ps):
        nu, npp = P._sizes(P.mesh.l_max)
        _need(f, nu, torch.float64, "f"); _need(g, npp, torch.float64, "g")
        _need(u, nu, torch.float64, "u"); _need(p, npp, torch.float64, "p")
    o = Problem.default_opts(**opts)
    stats = (SolveStats * max(len(probs), 1))()
    arr = (ctypes.c_void_p * max(len(probs), 1))(*[P.handle.value for P in probs])
    rc = lib().mfs_solve_concurrent(len(probs), arr, ctypes.byref(o), _ptr_array(fs), _ptr_array(gs),
                                    _ptr_array(us), _ptr_array(ps), stats, int(n_threads))
    if rc not in (OK, ENOTCONV) or (rc != OK and raise_on_error):
        raise MfsError(rc, lib().mfs_last_error().decode())
    out = [stats[i].as_dict() for i in range(len(probs))]
    return out


def place_members(levels, n_streams):
    """Stream of each ensemble member: members taken largest first (work ~ 8^level, the
    micro-tet count), each onto the stream with the least work so far (ties: the lowest
    stream).  Returns (stream index per member, work per stream)."""
    levels = [int(l) for l in levels]
    n_streams = max(1, min(int(n_streams), max(len(levels), 1)))
    load = [0] * n_streams
    stream_of = [0] * len(levels)
    for i in sorted(range(len(levels)), key=lambda i: (-levels[i], i)):
        k = min(range(n_streams), key=lambda k: (load[k], k))
        stream_of[i] = k
        load[k] += 8 ** levels[i]
    return stream_of, load


class Ensemble:
    """Independent Stokes problems (levels may differ) spread over n_streams CUDA streams of one
    device, for mfs_solve_concurrent: one context and one mesh per (stream, level), members
    placed by place_members."""

    def __init__(self, levels, n_streams=8, device=0):
        import torch
        self.levels = [int(l) for l in levels]
        self.stream_of, _ = place_members(self.levels, n_streams)
        n_streams = max(self.stream_of) + 1 if self.levels else 1
        self.streams = [torch.cuda.Stream(device) for _ in range(n_streams)]
        self.ctxs = [Context(device, s.cuda_stream) for s in self.streams]
        self.meshes = {}
        self.problems = []
        for i, l in enumerate(self.levels):
            key = (self.stream_of[i], l)
            if key not in self.meshes:
                self.meshes[key] = Mesh(self.ctxs[key[0]], l)
            self.problems.append(Problem(self.meshes[key]))

    def solve(self, fs, gs, us, ps, n_threads=0, raise_on_error=True, **opts):
        return solve_concurrent(self.problems, fs, gs, us, ps, n_threads=n_threads,
                                raise_on_error=raise_on_error, **opts)
