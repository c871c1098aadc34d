/* mfs.h — matrix-free blended P2-P1 Stokes operators and solver on one GPU (sm_103a).
 *
 * C ABI of libmfs.so.  Method: arxiv 2506.04157 ("paper" below).
 *
 * Conventions for every entry point
 *   - Return value: MFS_OK or an error code; the library never aborts.  On error,
 *     mfs_last_error() returns a message (thread-local, valid until the next call).
 *   - Vector arguments are DEVICE pointers owned by the caller (e.g. torch tensors),
 *     contiguous, on the context's device, unless a parameter says "host".
 *   - Velocity vectors are component-major [3][n_p2] (SoA: all x, then all y, then z);
 *     pressure and viscosity vectors are [n_p1].  FP64 entry points (prec = MFS_F64)
 *     take double*, FP32 ones (prec = MFS_F32) take float*.
 *   - All device work is enqueued on the context's stream; apply calls are
 *     asynchronous; calls that return host scalars synchronise the stream.
 *   - The library owns the mesh hierarchy, per-level coefficient data and solver
 *     workspaces (device memory it allocates with cudaMalloc); destroy functions free it.
 *   - One context per host thread at a time.
 *
 * Vector layout (node numbering) of refinement level l, N = 2^l intervals per macro
 * edge, for P1 vertices; the P2 nodes of level l are the P1 vertices of level l+1:
 *   ids [0, 24)                  macro vertices (12 icosahedron directions on r_cmb,
 *                                then the same 12 on r_surf)
 *   then 102 macro edges x (N-1) edge-interior points, from the lower to the higher
 *                                macro vertex id
 *   then 140 macro faces x (N-1)(N-2)/2 face-interior points
 *   then  60 macro cells x (N-1)(N-2)(N-3)/6 cell-interior points.
 * mfs_mesh_coords() returns the positions in this order.
 */
#ifndef MFS_H
#define MFS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  MFS_OK = 0,
  MFS_EINVAL = 1,      /* invalid argument (null handle, bad level, size, mode) */
  MFS_ENOMEM = 2,      /* device or host allocation failed */
  MFS_ECUDA = 3,       /* a CUDA runtime call failed (message has the CUDA error) */
  MFS_ENOTCONV = 4,    /* iterative solve did not reach its tolerance (best iterate kept) */
  MFS_EBREAKDOWN = 5,  /* Krylov breakdown (zero denominator) */
  MFS_ENAN = 6,        /* NaN or Inf in a residual norm */
  MFS_ETIMEOUT = 7     /* a bounded device-side wait ran out */
} mfs_status;

typedef enum { MFS_F64 = 0, MFS_F32 = 1 } mfs_prec;
typedef enum { MFS_BC_DIRICHLET = 0, MFS_BC_FREESLIP = 1 } mfs_bc;
/* RAW: the full assembled-equivalent block, no boundary handling.
 * CONSTRAINED: the projected, Dirichlet-eliminated block of the paper's Eq.
 *   (SaddlePointStructureDirichlet): Dirichlet velocity rows are the identity and
 *   their columns are dropped, free-slip nodes are projected, u -> u - (u.n)n, on input
 *   and output (P_v), pressure inputs and outputs are made mean-free (P_p). */
typedef enum { MFS_RAW = 0, MFS_CONSTRAINED = 1 } mfs_bcmode;

typedef struct mfs_ctx mfs_ctx;
typedef struct mfs_mesh mfs_mesh;
typedef struct mfs_problem mfs_problem;
typedef struct mfs_batch mfs_batch;
typedef struct mfs_mg_state mfs_mg_state;

typedef struct {
  int level;
  int64_t n_tets;      /* micro-tets: 60 * 8^level */
  int64_t n_p2;        /* P2 nodes (velocity has 3 * n_p2 entries) */
  int64_t n_p1;        /* P1 vertices (pressure / viscosity entries) */
  int64_t n_surface;   /* P2 nodes on r = r_surf */
  int64_t n_cmb;       /* P2 nodes on r = r_cmb */
} mfs_level_info;

/* Last error message of the calling thread ("" if none). */
const char* mfs_last_error(void);

/* Library version string. */
const char* mfs_version(void);

/* Context: device ordinal and the CUDA stream (cudaStream_t passed as void*, NULL =
 * legacy default stream) on which all work is enqueued.  The stream stays owned by
 * the caller.  Errors: MFS_EINVAL (bad device), MFS_ECUDA. */
mfs_status mfs_ctx_create(int device, void* cuda_stream, mfs_ctx** out);
mfs_status mfs_ctx_set_stream(mfs_ctx* ctx, void* cuda_stream);
mfs_status mfs_ctx_destroy(mfs_ctx* ctx);

/* Optional device timing of the element-sweep kernel (the matrix-free micro-tet
 * sweep behind every apply): with enable != 0 each sweep launch is bracketed by CUDA
 * events on the context's stream.  mfs_ctx_kernel_time() synchronises the stream and
 * returns the summed duration (ms) and the number of timed launches since the last
 * query, then resets both.  Not part of the method; a measurement aid. */
mfs_status mfs_ctx_timing(mfs_ctx* ctx, int enable);
mfs_status mfs_ctx_kernel_time(mfs_ctx* ctx, double* total_ms, int64_t* launches);

/* Spherical-shell mesh r_cmb <= |x| <= r_surf (paper Sec. 4.1): the 20 faces of the
 * icosahedron give 20 prisms in one radial layer, each cut into 3 macro-tets (each
 * quad face along the diagonal through its lowest-numbered vertex), 60 macro-tets,
 * uniformly refined (Freudenthal/Kuhn subdivision, 8^l micro-tets per macro) on levels
 * 0..l_max.  blending = 1 maps the straight mesh onto the shell by the radial blending
 * map B(x) = (x.nh/delta) x/|x| (nh, delta: normal and offset of the prism's face
 * plane); blending = 0 keeps the polyhedral shell.  Requires 0 < r_cmb < r_surf,
 * 0 <= l_max <= 7.  ctx = NULL builds a host-only mesh (numbering, coordinates and node
 * classes; no device data, no problem can be created on it).
 * Errors: MFS_EINVAL, MFS_ENOMEM, MFS_ECUDA. */
mfs_status mfs_mesh_shell(mfs_ctx* ctx, double r_cmb, double r_surf, int l_max, int blending,
                          mfs_mesh** out);
mfs_status mfs_mesh_destroy(mfs_mesh* mesh);
mfs_status mfs_mesh_info(const mfs_mesh* mesh, int level, mfs_level_info* out);

/* Node positions of a level into a HOST buffer xyz[3][n] (component-major), n = n_p2
 * if p2 != 0 else n_p1; blended = 1 gives physical positions B(x~), 0 the straight
 * ones.  Errors: MFS_EINVAL. */
mfs_status mfs_mesh_coords(const mfs_mesh* mesh, int level, int p2, int blended, double* xyz);

/* Node classes of a level into a HOST buffer (0 inner, 1 surface, 2 CMB). */
mfs_status mfs_mesh_node_class(const mfs_mesh* mesh, int level, int p2, int8_t* cls);

/* Problem = mesh + boundary conditions + coefficients (paper Sec. 2 boundary
 * conditions, Sec. 5.1 projections).  Defaults of the paper: surface Dirichlet, CMB
 * free-slip.  Errors: MFS_EINVAL, MFS_ENOMEM. */
mfs_status mfs_problem_create(mfs_mesh* mesh, mfs_bc bc_surface, mfs_bc bc_cmb, mfs_problem** out);
mfs_status mfs_problem_destroy(mfs_problem* prob);

/* Nodal P1 viscosity on the finest level (DEVICE pointer, double[n_p1(l_max)]; if
 * is_log != 0 the values are ln(eta)).  eta is a P1 function on every level, evaluated
 * at quadrature points by linear interpolation (paper Sec. 5.2.2, "eta_P1 on every
 * level"); each coarser level gets the P1 full weighting of the next finer one (the
 * normalised average of the coincident vertex, weight 1, and the midpoints of the
 * incident coarse edges, weight 1/2).  Errors: MFS_EINVAL, MFS_ECUDA. */
mfs_status mfs_set_viscosity(mfs_problem* prob, const double* eta_p1, int is_log);

/* Radial profile of d ln(rho)/dr on a uniform grid of n >= 1 points over
 * [r_cmb, r_surf] (HOST array), linearly interpolated at the physical radius of each
 * quadrature point; it defines C of paper Eq. (SaddlePointStructure),
 * C_ij = -int (grad ln rho . phi_j) psi_i with grad ln rho = (d ln rho/dr) x/|x|.
 * Default: 0 (incompressible).  Errors: MFS_EINVAL. */
mfs_status mfs_set_density(mfs_problem* prob, int n, const double* dlnrho_dr);

/* Temperature-dependent viscosity (paper Sec. 7.2, Eq. ViscosityDef, Frank-Kamenetskii):
 *   eta(x, T) = eta_base(|x|) exp(-E_A T + V_A (r_surf - |x|)),
 * log10 eta_base given by n (1..64) values on a uniform radial grid over [r_cmb, r_surf]
 * (HOST array, linear interpolation; the paper shows its profile only as a figure; it uses
 * E_A = 4.610, V_A = 2.996).  Per Sec. 5.2.2 the levels above l_eta carry eta as a P1
 * function of its values at the vertices, the levels l <= l_eta evaluate eta at every
 * quadrature point from the P2 temperature (-1 <= l_eta < l_max; -1: P1 everywhere).
 * Takes effect with mfs_set_temperature.  Errors: MFS_EINVAL, MFS_ECUDA. */
mfs_status mfs_set_viscosity_law(mfs_problem* prob, double E_A, double V_A, int n, const double* log10_base,
                                 int l_eta);
/* The finest level's P2 temperature T_p2 [n_p2] (FP64, device): sets the viscosity of every
 * level from the law (replaces mfs_set_viscosity; mfs_set_viscosity in turn drops the law).
 * On levels <= l_eta only the A block is available (B and the fused applies return
 * MFS_EINVAL there).  Evaluated on the device; the first call per mesh builds vertex-to-node
 * lookup maps (allocates device memory).  Errors: MFS_EINVAL (no law), MFS_ENOMEM, MFS_ECUDA. */
mfs_status mfs_set_temperature(mfs_problem* prob, const double* T_p2);

/* y = A(eta) u on level lvl (paper Sec. 5.1, A_ij = int 2 eta eps(phi_j):eps(phi_i),
 * eps(u) = sym grad u - (div u) I/3; blending Jacobian evaluated at every quadrature
 * point of the symmetric 4-point degree-2 rule).  u, y: [3][n_p2(lvl)].  u and y must
 * not overlap.  Errors: MFS_EINVAL, MFS_ECUDA. */
mfs_status mfs_apply_A(mfs_problem* prob, int lvl, mfs_prec prec, mfs_bcmode mode, const void* u,
                       void* y);

/* q = B u or q = (B + C) u (with_C != 0), B_ij = -int (div phi_j) psi_i (paper Sec. 5.1).
 * u: [3][n_p2], q: [n_p1].  Errors: MFS_EINVAL, MFS_ECUDA. */
mfs_status mfs_apply_B(mfs_problem* prob, int lvl, mfs_prec prec, mfs_bcmode mode, int with_C,
                       const void* u, void* q);

/* y = B^T p, or y = (B + C)^T p if with_C != 0.  p: [n_p1], y: [3][n_p2]. */
mfs_status mfs_apply_BT(mfs_problem* prob, int lvl, mfs_prec prec, mfs_bcmode mode, int with_C,
                        const void* p, void* y);

/* Fused saddle-point operator in one sweep over the micro-tets (paper Eq.
 * SaddlePointStructure with Bbar = B + C):
 *   transpose = 0:  yu = A u + B^T p,     yp = (B + C) u
 *   transpose = 1:  yu = A u + (B + C)^T p, yp = B u       (the adjoint operator)
 * Always CONSTRAINED (projections of Eq. SaddlePointStructureDirichlet).
 * Errors: MFS_EINVAL, MFS_ECUDA. */
mfs_status mfs_apply_stokes(mfs_problem* prob, int lvl, mfs_prec prec, int transpose, const void* u,
                            const void* p, void* yu, void* yp);

/* Buoyancy load vector on the finest level (paper Eq. SaddlePointStructure,
 * f_i = -int (Ra/Pe) rho alpha T g . phi_i with g = -x/|x|):
 *   f_(a,c) = scale int rho(r) T (x/|x|)_c phi_a dx,
 * T_p2 a nodal P2 field [n_p2] (FP64, device), rho(r) = exp(int_{r_surf}^{r} d ln rho/dr)
 * from the mfs_set_density table (piecewise linear, integrated exactly; rho(r_surf) = 1),
 * f: [3][n_p2] (FP64, device, overwritten).  Errors: MFS_EINVAL, MFS_ECUDA. */
mfs_status mfs_rhs_buoyancy(mfs_problem* prob, const double* T_p2, double scale, double* f);

/* ---------------------------------------------------------------- multigrid layer
 * (paper Sec. 5.2.2).  mfs_setup_multigrid builds, for levels l_min..l_max: the
 * boundary-node lists (Dirichlet / free-slip with their normals), the P2 transfer
 * operators, diag(A) (without the free-slip projection, ones on Dirichlet rows), the
 * Chebyshev interval [b/20, b] of D^-1 A per smoothing level (b = 1.2 x the largest
 * eigenvalue from 15 FP64 power iterations, unless set by mfs_set_cheb_bounds), the FP64
 * inverse of the coarsest-level operator, and the diagonal of M_{1/eta}.  Call it after
 * mfs_set_viscosity (and again after every new viscosity).  Allocates device memory.
 * Errors: MFS_EINVAL (viscosity not set, bad l_min), MFS_ENOMEM, MFS_ECUDA, MFS_ENAN. */
mfs_status mfs_setup_multigrid(mfs_problem* prob, int l_min);

/* Override / read the Chebyshev interval of D^-1 A on a smoothing level
 * (l_min < lvl <= l_max).  Bounds set before mfs_setup_multigrid replace the estimate. */
mfs_status mfs_set_cheb_bounds(mfs_problem* prob, int lvl, double lo, double hi);
mfs_status mfs_get_cheb_bounds(const mfs_problem* prob, int lvl, double* lo, double* hi);
/* Re-estimate the Chebyshev interval of level lvl (l_min < lvl <= l_max, multigrid set up)
 * from a caller-given start vector: x0 (device, FP64, [3][n_p2] of that level; read only,
 * projected by P_v and the Dirichlet elimination before the first step, any nonzero scale)
 * replaces the library's seeded vector in the 15 FP64 power iterations on D^-1 A_c of
 * mfs_setup_multigrid.  Stores [b/20, b], b = 1.2 * lambda, for the level's smoother and
 * returns lambda (the last iterate's norm) in *lam_max (host).  Synchronises the stream.
 * Errors: MFS_EINVAL (multigrid not set up, level without smoother, null pointer),
 * MFS_ENAN (the iterate vanished or became non-finite), MFS_ECUDA. */
mfs_status mfs_estimate_cheb_bounds(mfs_problem* prob, int lvl, const double* x0, double* lam_max);

/* Checkpoint of the viscosity-dependent multigrid state (the forward solution of the paper's
 * adjoint use "checkpointed per level"): device copies of every level's nodal viscosity (FP64,
 * FP32) and inverse diagonal of A (FP64, FP32), the Chebyshev intervals, the coarse-level
 * inverse, and the finest level's M_{1/eta} quadrature weights and inverse diagonal.
 * mfs_mg_restore copies them back into the problem (same problem, same multigrid range), so a
 * later adjoint solve runs on the state of the forward solve without recomputing it
 * (mfs_set_viscosity + mfs_setup_multigrid).  Both synchronise the stream; the checkpoint
 * allocates device memory (level 6: about 1.9 GB), freed by mfs_mg_state_destroy.
 * Errors: MFS_EINVAL (multigrid not set up, quadrature-point viscosity in use (l_eta >= 0),
 * state of another problem or of another level range), MFS_ECUDA. */
mfs_status mfs_mg_checkpoint(mfs_problem* prob, mfs_mg_state** out);
mfs_status mfs_mg_restore(mfs_problem* prob, const mfs_mg_state* state);
mfs_status mfs_mg_state_destroy(mfs_mg_state* state);

/* Form of the constraint (mass-conservation) row.  rho_weighted = 0 (default): the paper's
 * B + C of Eq. SaddlePointStructure, -int q (div u + grad ln rho . u).  rho_weighted = 1: the
 * density-weighted form -int q div(rho u) = -int q rho (div u + grad ln rho . u), rho(r) the
 * profile of mfs_set_density normalised to rho(r_surf) = 1 — the same continuous constraint
 * scaled by rho, a different discrete weighting.  It replaces B + C everywhere the library
 * uses it (applies with with_C, the fused apply and its transpose, the Uzawa pressure update,
 * residuals); the momentum rows keep B^T.  Batches refuse members with rho_weighted = 1.
 * Errors: MFS_EINVAL. */
mfs_status mfs_set_constraint_form(mfs_problem* prob, int rho_weighted);

/* diag(A) on level lvl without the free-slip projection (paper Sec. 5.2.2), 1 on
 * Dirichlet rows; y: [3][n_p2]. */
mfs_status mfs_diag_A(mfs_problem* prob, int lvl, mfs_prec prec, void* y);

/* y = M_{1/eta} p, the P1 mass matrix weighted by 1/eta at the quadrature points (paper
 * Eq. schurMass); p, y: [n_p1] of level lvl.  Needs only mfs_set_viscosity. */
mfs_status mfs_apply_mass(mfs_problem* prob, int lvl, mfs_prec prec, const void* p, void* y);

/* P2 prolongation from level lvl-1 to lvl (exact P2 interpolation in the straight
 * coordinates, then the boundary projections of level lvl) and its transpose
 * (restriction, then the projections of level lvl-1).  l_min < lvl <= l_max. */
mfs_status mfs_prolongate(mfs_problem* prob, int lvl, mfs_prec prec, const void* xc, void* xf);
mfs_status mfs_restrict(mfs_problem* prob, int lvl, mfs_prec prec, const void* rf, void* rc);
/* x <- P0 x on level lvl (l_min <= lvl <= l_max, multigrid set up): Dirichlet velocity
 * entries zeroed, free-slip nodes projected, u - (u.n)n (paper Sec. 5.1); x: [3][n_p2]. */
mfs_status mfs_project(mfs_problem* prob, int lvl, mfs_prec prec, void* x);

/* The scalar P2 prolongation of mfs_prolongate before the projections, as a CSR matrix with
 * n_p2(lvl) rows (fine nodes) and n_p2(lvl-1) columns: each fine node takes the coarse P2
 * interpolant at its position, one entry per nonzero coarse basis value.  Host-only (a
 * host-only mesh suffices).  nnz receives the entry count; rp [n_p2(lvl)+1], ci [nnz], w [nnz]
 * are HOST arrays, each filled when not NULL (call once with NULLs to size them).
 * 1 <= lvl <= l_max.  Errors: MFS_EINVAL. */
mfs_status mfs_mesh_prolongation(const mfs_mesh* mesh, int lvl, int* nnz, int* rp, int* ci, double* w);

/* The P1 interpolation from level lvl-1 to lvl as (coarse vertex, fine vertex, weight)
 * triplets: weight 1 where a fine vertex coincides with a coarse one, 1/2 for each end of the
 * coarse edge whose midpoint it is.  The library builds from it the weighted-BFBT Poisson
 * multigrid's transfers and, normalised row by row in the transpose, the full weighting that
 * gives every coarser level its viscosity.  Host-only; nnz receives the count; coarse, fine,
 * w: HOST arrays of nnz entries, each filled when not NULL.  1 <= lvl <= l_max.
 * Errors: MFS_EINVAL. */
mfs_status mfs_mesh_p1_interpolation(const mfs_mesh* mesh, int lvl, int* nnz, int* coarse, int* fine, double* w);

/* The lookup maps mfs_set_temperature uses to evaluate the viscosity law (paper Sec. 7.2, Eq.
 * ViscosityDef) on level lvl: the temperature of a P1 vertex, or of a P2 node on the levels
 * up to l_eta that carry the quadrature-point viscosity (Sec. 5.2.2), is the finest level's
 * P2 temperature at the same point.  Host-only.  vfine[n_p1]: index of the finest P2 node
 * at each vertex of lvl; vrad[n_p1]: the vertex's radius |x| (blended point); p2fine[n_p2]:
 * index of the finest P2 node at each P2 node of lvl.  HOST arrays, each filled when not
 * NULL.  0 <= lvl <= l_max.  Errors: MFS_EINVAL. */
mfs_status mfs_mesh_law_maps(const mfs_mesh* mesh, int lvl, int* vfine, double* vrad, int* p2fine);

/* One V-cycle for the constrained A on level lvl (paper Sec. 5.2.2): `steps` Chebyshev
 * pre- and post-smoothing steps of `degree` applications each, exact FP64 coarse solve on
 * l_min.  f: right-hand side [3][n_p2]; u: result (overwritten, the cycle starts from 0).
 * Errors: MFS_EINVAL (multigrid not set up, bad level), MFS_ECUDA. */
mfs_status mfs_vcycle(mfs_problem* prob, int lvl, mfs_prec prec, int steps, int degree, const void* f, void* u);

/* ---------------------------------------------------------------- Stokes solver
 * FGMRES (paper Sec. 5.2.4) right-preconditioned by the symmetric Uzawa step (Eq.
 * SymmetricUzawaStep1, B + C in the pressure update), A^-1 ~ CG + V-cycle (Sec. 5.2.2),
 * S^-1 ~ V-cycle BFBT (Eq. schurV) with CG on X = B A_C^-1 B^T preconditioned by CG on
 * M_{1/eta}.  Defaults (mfs_solve_opts_default) are the paper's Table parametertable. */
typedef struct {
  int mixed;          /* 1: FP32 inner FGMRES inside FP64 iterative refinement (default);
                         2: FP64 FGMRES (one FP64 fused apply per iteration) preconditioned by
                            the FP32 Uzawa step with its FP32 V-cycles and CGs;
                         0: all FP64 */
  double rtol;        /* stop at ||r|| <= rtol ||r0||, r the FP64 projected residual (1e-8) */
  int restart;        /* FGMRES restart length (30) */
  int max_iters;      /* total FGMRES iterations (300) */
  int max_outer;      /* refinement steps (restarts on the true FP64 residual) (20) */
  double inner_rtol;  /* relative tolerance of each inner FP32 FGMRES (1e-4); the last step stops
                         once the target rtol is within a factor 2 */
  double sigma;       /* scaling of A^-1 in the Uzawa step (1) */
  double omega;       /* scaling of S^-1 in the Uzawa step (0.3) */
  double tol_A;       /* CG on A, relative (1e-2) */
  int m_A, deg_A;     /* V-cycle for A: Chebyshev steps and degree (3, 2) */
  double tol_VBFBT;   /* CG on X (1e-1) */
  double tol_invMass; /* CG on M_{1/eta} (1e-10; at least 1e-6 in FP32) */
  int m_V, deg_V;     /* cheap V-cycle A_C (1, 1) */
  int max_cg;         /* iteration cap of every inner CG (200) */
  int with_C;         /* 1: compressible constraint (B + C) (1) */
  int uzawa;          /* block preconditioner (Sec. 5.2.1): 0 symmetric Uzawa (Eq.
                         SymmetricUzawaStep1, default), 1 inexact Uzawa (Eq.
                         InexactUzawaStep1), 2 adjoint inexact Uzawa (Eq.
                         AdjointInexactUzawaStep1); each applied from (0, 0) */
  int schur;          /* Schur approximation (Sec. 5.2.3): 0 V-cycle BFBT (Eq. schurV, default),
                         1 inverse-viscosity mass M_{1/eta}^-1 by CG to tol_invMass (Eq.
                         schurMass), 2 diag(A)-BFBT (C = D = diag(A), solved like 0),
                         3 weighted BFBT (Eq. schurWBFBT, rescaled form, see mfs_apply_schur) */
  double a_l, a_r;    /* weighted-BFBT surface scalings: eta_{l,r} = a_{l,r}^2 eta on the micro-tets
                         with a vertex on the outer surface (1, 1; Table parametertable) */
  double tol_wBFBT;   /* CG on K_{1/sqrt(eta)}, relative or absolute, whichever is met first
                         (1e-10; at least 1e-5 in FP32) */
  int vmass;          /* weighted-BFBT vector mass M_{sqrt(eta)}: 0 the lumped mass, 1 (default)
                         the consistent mass (mfs_apply_vmass) by Jacobi-preconditioned CG on
                         the constrained velocity space to tol_VectorMass (Sec. 5.2.3); with
                         schur = 3 the cg_M_* statistics count these CGs.  The consistent mass
                         keeps the approximation's spectrum of order one under refinement and
                         suits omega = 0.3; the lumped one's grows like 1/h and wants a
                         smaller omega (about 0.03 on levels 1-2) */
  double tol_VectorMass; /* CG on the consistent M_{sqrt(eta)}, relative (1e-4; Table
                         parametertable) */
} mfs_solve_opts;

typedef struct {
  int outer_iters;    /* refinement steps (mixed) or 1 */
  int fgmres_iters;   /* total FGMRES iterations */
  int cg_A_iters, cg_X_iters, cg_M_iters;        /* totals over all calls */
  int cg_A_calls, cg_X_calls, cg_M_calls;
  int cg_A_max, cg_X_max, cg_M_max;               /* largest iteration count of one call */
  int vcycles;        /* V-cycles on the finest level */
  int applies;        /* finest-level A / saddle-point sweeps issued by the Krylov layers */
  double r0_norm, r_norm, rel_residual;   /* FP64 projected residual norms */
  double time_ms;     /* wall time of the solve (setup excluded) */
  /* wall time inside the preconditioner's parts (each ends in a host synchronisation, so
   * the times include the device work): A-block CG (A_hat^-1), Schur solve (V-cycle BFBT,
   * with the mass CGs it calls), and the mass CGs alone */
  double time_Ahat_ms, time_Sinv_ms, time_Minv_ms;
} mfs_solve_stats;

void mfs_solve_opts_default(mfs_solve_opts* opts);

/* ---------------------------------------------------------------- Schur approximations
 * z = S^-1 r: one application of the Schur approximation opts->schur (opts = NULL: the
 * default V-cycle BFBT) on the finest level, in precision prec, with the tolerances of opts,
 * as the Uzawa step applies it.  r, z: [n_p1] device vectors of prec; z is mean-free.  Needs
 * mfs_setup_multigrid.  stats (may be NULL) receives the inner CG counts and times.
 * The weighted BFBT (schur = 3; Sec. 5.2.3, Eq. schurWBFBT with the near-surface rescaling):
 *   S_w^-1 = K_{1/sqrt(eta_l)}^-1 (B M_{sqrt(eta_l)}^-1 A M_{sqrt(eta_r)}^-1 B^T) K_{1/sqrt(eta_r)}^-1,
 * K by CG preconditioned with its own geometric V-cycle (Chebyshev m_A, deg_A) to tol_wBFBT,
 * M the lumped vector mass (mfs_lumped_vmass; vmass = 0) or the consistent one
 * (mfs_apply_vmass; vmass = 1) solved by CG to tol_VectorMass.  Its operators are built on
 * first use of a scaling and after every coefficient change (allocates device memory).
 * Errors: MFS_EINVAL, MFS_ENAN, MFS_ENOMEM, MFS_ECUDA. */
mfs_status mfs_apply_schur(mfs_problem* prob, const mfs_solve_opts* opts, mfs_prec prec, const void* r, void* z,
                           mfs_solve_stats* stats);

/* y = K_{1/sqrt(eta_a)} p on level lvl (multigrid range): the P1 Laplacian
 *   K_ij = sum_tets sum_q w_q |det J_q| grad psi_j . grad psi_i / sqrt(eta_a(x_q))
 * with natural boundary conditions (Sec. 5.2.3, the Poisson operator replacing
 * B M_{sqrt(eta)}^-1 B^T), eta_a = a^2 eta on the micro-tets with a vertex on the outer surface
 * and eta elsewhere, eta the P1 interpolant of the level's nodal viscosity.  p, y: [n_p1(lvl)]
 * device vectors of prec.  Needs mfs_setup_multigrid.  Errors: MFS_EINVAL, MFS_ENOMEM, MFS_ECUDA. */
mfs_status mfs_apply_poisson(mfs_problem* prob, int lvl, mfs_prec prec, double a, const void* p, void* y);

/* d = the lumped vector mass M_{sqrt(eta_a)} on the finest level (Sec. 5.2.3, "potentially
 * lumped"): per micro-tet the diagonal of int sqrt(eta_a) phi_i phi_j (P2, the 4-point rule)
 * scaled to the element's total int sqrt(eta_a) (Hinton-Rock-Zienkiewicz lumping); one entry
 * per P2 node, the same for every velocity component.  d: [n_p2] FP64 device vector.
 * Errors: MFS_EINVAL, MFS_ECUDA. */
mfs_status mfs_lumped_vmass(mfs_problem* prob, double a, double* d);

/* y_c = M_{sqrt(eta_a)} x_c for the three velocity components c on the finest level: the
 * consistent P2 scalar mass M_ij = sum_tets sum_q w_q |det J_q| sqrt(eta_a(x_q)) phi_j phi_i
 * (Sec. 5.2.3, the vector mass weighted by the square root of the viscosity), eta_a as in
 * mfs_apply_poisson, on the degree-5 conical rule (the P2 mass has degree 4; 27 points).  No
 * boundary rows or columns are removed.  x, y: [3][n_p2] device vectors of prec (distinct).
 * Needs the viscosity.  Errors: MFS_EINVAL (null argument, no viscosity, a not positive and
 * finite), MFS_ECUDA. */
mfs_status mfs_apply_vmass(mfs_problem* prob, mfs_prec prec, double a, const void* x, void* y);

/* Solve the projected saddle-point system (paper Eq. SaddlePointStructureDirichlet) on
 * the finest level: f [3][n_p2] and g [n_p1] are the right-hand sides (FP64, device);
 * u [3][n_p2], p [n_p1] (FP64, device) hold the initial guess on entry, the solution on
 * exit; u's Dirichlet nodes carry the boundary values and are kept.  p is returned with
 * arithmetic mean zero.  Needs mfs_setup_multigrid.  opts = NULL uses the defaults; stats
 * may be NULL.  Errors: MFS_EINVAL, MFS_ENOTCONV (best iterate returned), MFS_ENAN,
 * MFS_ECUDA, MFS_ENOMEM (Krylov storage is allocated on the first solve). */
mfs_status mfs_stokes_solve(mfs_problem* prob, const mfs_solve_opts* opts, const double* f, const double* g,
                            double* u, double* p, mfs_solve_stats* stats);

/* ---------------------------------------------------------------- temperature step
 * The energy equation's splitting step of Sec. 3 and Sec. 6 on the finest level: the
 * temperature is a P2 scalar [n_p2] (FP64, device) with Dirichlet values on both spheres.
 * Parameters are the nondimensional numbers and constants of Eq. (WeakTemp). */
typedef struct {
  double k, Pe, Cp, Di, alpha, H, Ra;  /* conductivity, Peclet, heat capacity, dissipation, expansivity,
                                          internal heating, Rayleigh (1, 1, 1, 0, 1, 0, 1) */
  double tol_T;       /* absolute FGMRES tolerance on the constrained residual (1e-10, Table
                         parametertable) */
  double rtol;        /* relative FGMRES tolerance, 0 = absolute only (0) */
  int restart;        /* FGMRES restart length (30) */
  int max_iters;      /* total FGMRES iterations (300) */
  int max_cg;         /* iterations of each preconditioner CG (200) */
  double cg_rtol;     /* relative tolerance of the FP32 preconditioner CG (1e-6) */
} mfs_temp_params;

typedef struct {
  int fgmres_iters, cg_iters;
  double r0_norm, r_norm;   /* FP64 constrained residual norms */
  double time_ms;
} mfs_temp_stats;

void mfs_temp_params_default(mfs_temp_params* params);

/* The 27-point quadrature rule of the temperature blocks and the consistent vector mass, as
 * the kernels use it: Stroud's conical product rule on the reference tet (Gauss-Jacobi points
 * with weights (1-s)^2 and (1-t), Gauss-Legendre in the third direction; exact to degree 5;
 * weights summing to 1/6).  lam: [27][4] barycentric coordinates, w: [27] (HOST arrays).
 * Host-only (no device needed).  Errors: MFS_EINVAL (null pointer, or the rule failed its
 * exactness check). */
mfs_status mfs_temp_rule(double* lam, double* w);

/* y = (cM M + cC C(u) + cD D + cR R(u)) x on the finest level (Eq. WeakTemp's blocks):
 *   M = int phi_j phi_i, C(u) = int (u . grad phi_j) phi_i, R(u) = int (u . g) phi_j phi_i with
 *   g = -x/|x|, D = int grad phi_j . grad(phi_i / rho) (sym = 1: int grad phi_j . grad phi_i / rho),
 * integrated with a 27-point degree-5 rule over the blended micro-tets; rho from the density
 * table (mfs_set_density).  constrained = 1: rows and columns of the nodes on both spheres
 * replaced by the identity.  u: [3][n_p2] (may be NULL when cC = cR = 0); x, y: [n_p2]; all
 * device vectors of prec.  Allocates the temperature workspace on first use.
 * Errors: MFS_EINVAL, MFS_ENOMEM, MFS_ECUDA. */
mfs_status mfs_temp_apply(mfs_problem* prob, mfs_prec prec, double cM, double cC, double cD, double cR, int sym,
                          int constrained, const void* u, const void* x, void* y);

/* b = the right-hand side of Eq. (WeakTemp) for the step (tau_np1, tau_n):
 *   int phi_i [s0 T0_hat - sm Tm_hat + tau H/Cp + tau Pe Di/(Ra Cp) 2 eta(x, T*) eps(u*):eps(u*) / rho],
 * s0 = (tau_np1 + tau_n)/tau_n, sm = tau_np1^2 / (tau_n (tau_np1 + tau_n)) (variable-step BDF2,
 * Sec. 3), eps the deviatoric strain rate of u* [3][n_p2], eta the viscosity law
 * (mfs_set_viscosity_law) at the points with T* interpolated.  u_star, T_star may be NULL when
 * Di = 0.  All FP64 device vectors; rows of boundary nodes are not modified further.
 * Errors: MFS_EINVAL, MFS_ENOMEM, MFS_ECUDA. */
mfs_status mfs_temp_rhs(mfs_problem* prob, const mfs_temp_params* params, const double* T0_hat, const double* Tm_hat,
                        const double* u_star, const double* T_star, double tau_np1, double tau_n, double* b);

/* T_hat = MMOC(T, u_new, u_old, tau) (Sec. 3): one particle per P2 node traced back over a step
 * tau with one classical RK4 step along u(t) linear in time from u_old (start of the step) to
 * u_new (end), and T evaluated there (departure points outside the shell moved radially onto
 * it: onto the nearer sphere, or on the polyhedral shell onto the nearer of the inner and
 * outer face planes of the prism the point's direction crosses).  The particles start at the nodes (X_start = NULL) or at the points X_start [3][n_p2]
 * (a particle path continued over an earlier step).  T, T_hat: [n_p2]; u_new, u_old:
 * [3][n_p2]; X_dep: [3][n_p2] departure points, or NULL.  FP64 device vectors.
 * Errors: MFS_EINVAL, MFS_ENOMEM, MFS_ECUDA. */
mfs_status mfs_mmoc(mfs_problem* prob, const double* T, const double* u_new, const double* u_old, double tau,
                    const double* X_start, double* T_hat, double* X_dep);

/* The MMOC particle step of mfs_mmoc (Sec. 3) run on the host, one particle after another,
 * by the same per-particle code the kernel runs: for each of the n particles starting at
 * X_start[:, i] ([3][n]), its departure point after one RK4 step back over tau with u linear
 * in time from u_old to u_new, and T there.  mesh may be host-only (mfs_mesh_shell with a
 * NULL context); the fields live on its finest level: T [n_p2], u_new, u_old [3][n_p2].
 * Outputs T_hat [n] and X_out [3][n] (or NULL).  All HOST arrays.  Meant for checking the
 * device path on a machine without a GPU and for small host-side traces.
 * Errors: MFS_EINVAL. */
mfs_status mfs_mmoc_host(const mfs_mesh* mesh, int n, const double* X_start, const double* T, const double* u_new,
                         const double* u_old, double tau, double* T_hat, double* X_out);

/* One temperature step (Sec. 3 and Sec. 6): u* and T* by linear extrapolation (Eq.
 * Extrapolation), T0_hat = MMOC(T_n, u*, u_n, tau_np1) at the departure points Y of the nodes,
 * Tm_hat = T_nm1 at the feet of the same particles traced on from Y with (u_n, u_nm1, tau_n) —
 * the characteristic X(t^{n+1}, t^{n-1}, x) that the nested MMOC of Sec. 3 approximates —
 * then Eq. (WeakTemp) for T_np1 with the Dirichlet values of T_bc
 * on both spheres — without its advection term: the MMOC values carry the advection, and the
 * solve is the energy equation without it (Sec. 3) — by FGMRES (FP64) preconditioned by an
 * FP32 Jacobi-CG on s1 M + tau k/(Pe Cp) D_s.  T_*: [n_p2], u_*: [3][n_p2], FP64 device vectors.
 * Errors: MFS_EINVAL, MFS_ENOTCONV (best iterate returned), MFS_ENAN, MFS_ENOMEM, MFS_ECUDA. */
mfs_status mfs_temperature_step(mfs_problem* prob, const mfs_temp_params* params, const double* T_n,
                                const double* T_nm1, const double* u_n, const double* u_nm1, double tau_np1,
                                double tau_n, const double* T_bc, double* T_np1, mfs_temp_stats* stats);

/* ---------------------------------------------------------------- adjoint (not in the paper)
 * Adjoint solve K^T lam = (ju, jp) with K^T = [A (B+C)^T; B 0] on the constrained space
 * (the multiplier's Dirichlet values are zeroed on entry), by the same FGMRES / symmetric
 * Uzawa / V-cycle BFBT solver with the constraint and momentum pressure blocks swapped.
 * ju [3][n_p2], jp [n_p1]: gradient of the objective w.r.t. (u, p) (FP64, device);
 * lam_u, lam_p: initial guess in, multiplier out.  Errors as mfs_stokes_solve. */
mfs_status mfs_adjoint_solve(mfs_problem* prob, const mfs_solve_opts* opts, const double* ju, const double* jp,
                             double* lam_u, double* lam_p, mfs_solve_stats* stats);

/* Gradient of the objective w.r.t. the nodal log-viscosity of the finest level:
 *   g_k = -eta_k sum_q 2 w_q |det J_q| psi_k(q) eps(u)(q) : eps(lam)(q)
 * (A is linear in the P1 viscosity), u the forward velocity (with its Dirichlet values),
 * lam the adjoint velocity; all FP64 device vectors, g [n_p1].  Errors: MFS_EINVAL, MFS_ECUDA. */
mfs_status mfs_grad_log_eta(mfs_problem* prob, const double* u, const double* lam_u, double* g);

/* ---------------------------------------------------------------- ensembles (not in the paper)
 * A batch groups n problems on one context (each with its own mesh, refinement level,
 * boundary conditions and viscosity; all blended or all polyhedral).  Allocates device
 * memory.  Errors: MFS_EINVAL, MFS_ENOMEM, MFS_ECUDA. */
mfs_status mfs_batch_create(mfs_ctx* ctx, int n, mfs_problem* const* probs, mfs_batch** out);
mfs_status mfs_batch_destroy(mfs_batch* batch);

/* The constrained fused saddle-point apply (as mfs_apply_stokes, compressible) of every
 * member on its finest level, with ONE micro-tet sweep launch covering all members' tiles
 * (plus batched zeroing and pressure mean removal).  u, p, yu, yp: HOST arrays of n device
 * pointers.  Errors: MFS_EINVAL, MFS_ECUDA. */
mfs_status mfs_batch_apply_stokes(mfs_batch* batch, mfs_prec prec, int transpose, const void* const* u,
                                  const void* const* p, void* const* yu, void* const* yp);

/* mfs_stokes_solve for every member in turn (each needs mfs_setup_multigrid); stats: n
 * entries or NULL.  Returns the first error, MFS_ENOTCONV after trying every member. */
mfs_status mfs_batch_solve(mfs_batch* batch, const mfs_solve_opts* opts, const double* const* f,
                           const double* const* g, double* const* u, double* const* p, mfs_solve_stats* stats);

/* Concurrent solve of n independent problems (not in the paper): mfs_stokes_solve for every
 * member, with the members of DIFFERENT contexts running at the same time.  The members are
 * grouped by the context of their mesh; one host thread works through a group member after
 * member on that context's stream, and up to n_threads groups (0: one thread per group) run
 * concurrently, so that the small kernels and host round trips of low-level members overlap
 * on the device.  Members of one context never run concurrently; two contexts must not share
 * a stream.  The call synchronizes each device it uses before the first solve (inputs written
 * on other streams are complete) and returns after every solve has finished.  f, g, u, p:
 * HOST arrays of n FP64 device pointers as in mfs_stokes_solve (each member needs
 * mfs_setup_multigrid); stats: n entries or NULL.  Returns MFS_OK when every member
 * converged, MFS_ENOTCONV when some did not (the other members' results are valid), else the
 * first member's error; mfs_last_error names the member.  Errors: MFS_EINVAL (null arrays,
 * negative n or n_threads, contexts sharing a stream), MFS_ENOMEM (a host exception in a
 * member's solve, caught in its thread), as mfs_stokes_solve. */
mfs_status mfs_solve_concurrent(int n, mfs_problem* const* probs, const mfs_solve_opts* opts, const double* const* f,
                                const double* const* g, double* const* u, double* const* p, mfs_solve_stats* stats,
                                int n_threads);

/* ---------------------------------------------------------------- sharding by macro-tets
 * The hybrid hierarchical grid of paper Sec. 4.1 splits naturally by macro-tets: every
 * micro-tet, and so every element contribution, belongs to exactly one macro; nodes on macro
 * vertices, edges and faces are shared by the macros around them.  A multi-GPU run gives
 * each rank a range of macros; the ranks' partial results are summed on the shared nodes
 * (paper_2506_04157_gb300/shard.py holds that logic).
 *
 * Macro topology (host, level-independent): cells[4m + k] = global vertex id of local vertex
 * k of macro m (increasing), edges[6m + e] = global macro-edge id of local edge e (pairs 01,
 * 02, 03, 12, 13, 23), faces[4m + z] = global macro-face id of the face opposite local vertex
 * z.  With the node numbering documented at the top of this file, the lattice points a macro
 * touches on a level follow from these ids.  Buffers [240], [360], [240] ints, caller-owned.
 * Errors: MFS_EINVAL (null pointer). */
mfs_status mfs_mesh_macro_topology(const mfs_mesh* mesh, int* cells, int* edges, int* faces);

/* Partial constrained apply over the micro-tets of macros m0 <= m < m1 (0 <= m0 < m1 <= 60)
 * on level lvl: fused = 0 gives yu = the contributions of those micro-tets to A_c u;
 * fused = 1 gives yu = A_c u + P0 B^T p and yp = (B + C) P0 u restricted alike.  Element
 * arithmetic as in mfs_apply_stokes's constrained mode: P0 (Dirichlet columns dropped,
 * free-slip projection) on the velocity input, P_v on the free-slip output rows, identity
 * rows y = u at the Dirichlet nodes the range touches; but p is used as given (pass it
 * mean-free) and yp is not made mean-free — with shared nodes summed over all ranks and the
 * pressure mean then removed, the result is mfs_apply_stokes's (rounding aside).  Outputs are
 * overwritten; entries of nodes the range does not touch are zero.  p, yp may be NULL when
 * fused = 0.  Errors: MFS_EINVAL (range, level, null pointer, fused apply on a level that
 * evaluates the viscosity at quadrature points), MFS_ECUDA. */
mfs_status mfs_apply_part(mfs_problem* prob, int lvl, mfs_prec prec, int fused, int m0, int m1, const void* u,
                          const void* p, void* yu, void* yp);

/* ---------------------------------------------------------------- autotuning (not in the paper)
 * The FP32 hot sweeps (fused saddle-point apply and A alone) have 9 launch variants per mesh
 * level: 0 = shared-memory element body with float atomics, 192 threads, 4 resident CTAs
 * per SM; 1 = the same with 3 CTAs per SM; 2-6 = register-resident element body with
 * fixed-point (int32) accumulation of each tile in rounds with their own power-of-two
 * scales, with (threads, CTAs per SM) = (192, 2), (128, 3), (128, 4), (256, 2), (192, 3);
 * 7-8 = the fixed-point body with the four quadrature points processed in two packed FP32
 * pairs (fma/add/mul.f32x2), (192, 3) and (128, 4).  By default every level runs variant 8
 * for the fused apply (and the other operator sets) and variant 7 for A alone; mfs_set_tuning
 * and mfs_autotune set one variant for both.  All compute the same operator (rounding order and the fixed-point rounding
 * aside).  mfs_autotune times every variant on every level of the problem's mesh with CUDA
 * events and keeps the fastest for all later applies on that mesh.  cache_path (may be
 * NULL): a text file read first (levels found there are not timed) and written with the
 * choices and timings.  Allocates and frees temporary device vectors.
 * Errors: MFS_EINVAL, MFS_ENOMEM, MFS_ECUDA. */
mfs_status mfs_autotune(mfs_problem* prob, const char* cache_path);
/* The variant in use on a level (of the fused apply; mfs_set_tuning sets both). */
mfs_status mfs_get_tuning(const mfs_problem* prob, int lvl, int* variant);
/* Select the variant of a level by hand (0 <= variant < 9); it applies to every problem on
 * the mesh.  Errors: MFS_EINVAL. */
mfs_status mfs_set_tuning(mfs_problem* prob, int lvl, int variant);

/* ---------------------------------------------------------------- measurement (not in the paper)
 * Throughput of the device's fused multiply-add pipes, the denominators of the element
 * sweeps' arithmetic roofline: kind 0 = FP32 (fma.rn.f32), 1 = FP32 packed pairs
 * (fma.rn.f32x2, two FMAs per instruction), 2 = FP64 (fma.rn.f64).  Runs `launches`
 * back-to-back launches of a kernel whose threads each carry 8 independent FMA chains of
 * 128 * iters FMAs (64 warps per SM), timed with CUDA events on the context's stream after
 * one warm-up launch; returns the rate (*tflops, counting an FMA as 2 flops) and the timed
 * duration (*ms).  Allocates and frees a small output buffer; synchronises the stream.
 * Errors: MFS_EINVAL (null pointer, kind outside 0..2, launches or iters < 1), MFS_ECUDA. */
mfs_status mfs_fma_peak(mfs_ctx* ctx, int kind, int launches, int iters, double* tflops, double* ms);

/* Allocation-free variant of mfs_apply_B (no counterpart in the paper).
 *
 * For callers that cannot call cudaMalloc while they apply the operator: for example code
 * running under an external memory manager that owns every device allocation, or a
 * real-time loop in which a device allocation would synchronise the device.  Same
 * arguments, result and errors as mfs_apply_B; the caller passes u and q as before.  In
 * MFS_CONSTRAINED mode the mean removal (P_p) sums q in a fixed, library-owned static
 * device array of 8,448 bytes (1,024 partial sums) instead of the problem's workspace, so
 * the call allocates nothing (no cudaMalloc/cudaFree, no allocating library routine).
 * Limit: levels with at most 4,194,304 pressure entries (levels 0-6); larger levels return
 * MFS_EINVAL with a message giving the limit.
 * The first call on a device looks up the array's device address (cudaGetSymbolAddress,
 * with that device current); make that first call before any stream capture.  Every GPU
 * that loads the library holds the array until the process exits; all calls share it and
 * it keeps the last call's contents, so calls that overlap on the GPU (for example on two
 * streams) race and must be serialised by the caller. */
mfs_status mfs_apply_B_noalloc(mfs_problem* prob, int lvl, mfs_prec prec, mfs_bcmode mode, int with_C,
                               const void* u, void* q);

#ifdef __cplusplus
}
#endif
#endif /* MFS_H */
