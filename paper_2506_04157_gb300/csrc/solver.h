// Internal declarations of the multigrid / Krylov layer.
#pragma once

#include <vector>

#include "library.h"

namespace mfs {

// P2 nodes of one level that carry a boundary condition (kind 1 Dirichlet, 2 free slip),
// with the outward radial unit normal at each node.
struct BoundaryList {
  int nb = 0;
  int* ids = nullptr;
  int* nodemap = nullptr;   // [n_p2]: position of the node in the list, -1 for interior nodes
  int8_t* kind = nullptr;
  double* nrm64 = nullptr;
  float* nrm32 = nullptr;
  template <typename T>
  const T* normals() const;
};
template <>
inline const double* BoundaryList::normals<double>() const { return nrm64; }
template <>
inline const float* BoundaryList::normals<float>() const { return nrm32; }

// CSR matrix with weights in both precisions (transfer operators).
struct Csr {
  int nrows = 0, ncols = 0;
  int* rp = nullptr;
  int* ci = nullptr;
  double* w64 = nullptr;
  float* w32 = nullptr;
  template <typename T>
  const T* w() const;
};
template <>
inline const double* Csr::w<double>() const { return w64; }
template <>
inline const float* Csr::w<float>() const { return w32; }

template <typename T>
struct Blas {
  static void axpby(int64_t n, T a, const T* x, T b, T* y, cudaStream_t s);          // y = a x + b y
  static void axpbypcz(int64_t n, T a, const T* x, T b, const T* y, T c, T* z, cudaStream_t s);
  static void fill(int64_t n, T v, T* y, cudaStream_t s);
  static void mul(int64_t n, const T* x, const T* d, T* z, cudaStream_t s);           // z = x .* d
  static void recip(int64_t n, T* x, cudaStream_t s);
  static void dot_async(int64_t n, const T* x, const T* y, double* part, double* out, cudaStream_t s);
  static void bproject(const BoundaryList& B, int64_t n_p2, T* v, cudaStream_t s);
  static void spmv3(const Csr& P, int64_t ncols, const T* x, T alpha, T beta, T* y, cudaStream_t s);
  static void gemv_f64(int n, const double* A, const T* b, T* x, cudaStream_t s);
  static void convert_from_f64(int64_t n, const double* x, T* y, cudaStream_t s);
  static void convert_to_f64(int64_t n, const T* x, double* y, cudaStream_t s);
  // Chebyshev update of a velocity vector ([3][n_p2]), one pass per node: r = b (mode 0),
  // b - t (mode 1) or r - t (mode 2); d = cz dinv r + cd d; x = (mode 0 ? 0 : x) + d;
  // t = 0; then the boundary projection of d and x at the node
  static void cheb_update(int64_t n_p2, int mode, const T* b, T* t, T* r, const T* dinv, T* d, T* x, T cz, T cd,
                          const BoundaryList& B, cudaStream_t s);
  // y = P_c R (b - t) (restriction of a residual, projected on the coarse level Bc)
  static void restrict_residual(const Csr& R, int64_t ncols, const T* b, const T* t, T* y, const BoundaryList& Bc,
                                cudaStream_t s);
  // x += P xc, projected on the fine level Bf (prolongation of a coarse correction); t = 0
  static void prolong_add(const Csr& P, int64_t ncols, const T* xc, T* x, T* t, const BoundaryList& Bf,
                          cudaStream_t s);
};

// blocks (at most) of the mass-CG reduction kernels (each thread takes four elements per
// round; more blocks would lengthen the serial arrival count of the last-block reduction)
constexpr int kMassRedBlocks = 512;

// slots of the device-resident CG scalars
enum { CG_RZ = 0, CG_RZN, CG_PQ, CG_RR, CG_RR0, CG_ALPHA, CG_BETA, CG_IT, CG_ACTIVE, CG_MEANQ, CG_MEANZ, CG_NSLOTS };

template <typename T>
struct CgDev {
  static void init(double* sc, cudaStream_t s);                  // it = 0, active = rr0 > 0
  // One iteration of CG on P_p M P_p (P_p: mean removal; Jacobi preconditioner, p kept
  // mean-free) after the sweep q = M p, in three launches whose reductions finish in the
  // last block to arrive: (1) alpha = rz / p.q and mean(q); (2) x += alpha p,
  // r -= alpha (q - mean q), z = dinv r, q = 0, then beta, convergence and mean(z);
  // (3) p = (z - mean z) + beta p.  part: 4 * kMassRedBlocks doubles, counter: one zeroed uint.
  static void mass_dots(int64_t n, const T* p, const T* q, double* part, unsigned* counter, double* sc,
                        cudaStream_t s);
  static void mass_update(int64_t n, const T* p, T* q, T* x, T* r, T* z, const T* dinv, double* part,
                          unsigned* counter, double* sc, double tol2, int maxit, cudaStream_t s);
  static void mass_pupd(int64_t n, const T* z, T* p, const double* sc, cudaStream_t s);
};

template <typename T>
inline const T* lvl_eta(mfs_problem* P, int l);
template <>
inline const double* lvl_eta<double>(mfs_problem* P, int l) { return P->eta64[l]; }
template <>
inline const float* lvl_eta<float>(mfs_problem* P, int l) { return P->eta32[l]; }
template <typename T>
inline const T* lvl_temp(mfs_problem* P, int l);
template <>
inline const double* lvl_temp<double>(mfs_problem* P, int l) { return P->temp64[l]; }
template <>
inline const float* lvl_temp<float>(mfs_problem* P, int l) { return P->temp32[l]; }
template <typename T>
inline const T* lvl_lbase(mfs_problem* P);
template <>
inline const double* lvl_lbase<double>(mfs_problem* P) { return P->d_lbase64; }
template <>
inline const float* lvl_lbase<float>(mfs_problem* P) { return P->d_lbase32; }
template <typename T>
inline const MacroGeom<T>* lvl_geom(mfs_mesh* M);
template <>
inline const MacroGeom<double>* lvl_geom<double>(mfs_mesh* M) { return M->d_geom64; }
template <>
inline const MacroGeom<float>* lvl_geom<float>(mfs_mesh* M) { return M->d_geom32; }

template <typename T>
mfs_status diag_A(mfs_problem* P, int lvl, const BoundaryList& B, T* diag);
// Quadrature weights of M_{1/eta} on level lvl: w[((tile * 4) + q) * kMassSlots + t] =
// w_q |det J_q| / eta(x_q) for the t-th micro-tet of the tile (the tile's class list order).
constexpr int kMassSlots = 6 * TT * TT * TT;
inline int64_t mass_weight_count(const LevelData& L) { return (int64_t)kMacroCells * L.n_tiles * 4 * kMassSlots; }
mfs_status mass_weights(mfs_problem* P, int lvl, double* w);
// y = M_{1/eta} p (or its diagonal) from stored weights; `active` and zero_out as below
template <typename T>
mfs_status mass_apply_w(mfs_problem* P, int lvl, const T* w, const T* pin, T* y, int diag_only,
                        const double* active = nullptr, int zero_out = 1);
// y = M_{1/eta} p (or its diagonal); with `active` the sweep is a no-op unless *active > 0,
// zero_out = 0 adds into a zeroed y
template <typename T>
mfs_status mass_apply(mfs_problem* P, int lvl, const T* pin, T* y, int diag_only, const double* active = nullptr,
                      int zero_out = 1);
mfs_status coarse_inverse(mfs_problem* P, int lvl, const BoundaryList& B, double* A, double* work);
// in-place Gauss-Jordan inverse of an SPD n x n matrix (no pivoting); colk: n doubles
void gj_invert(int n, double* A, double* colk, cudaStream_t s);
void unit_vector(int64_t n, int64_t j, double* e, cudaStream_t s);

// ---- weighted BFBT (Sec. 5.2.3, Eq. schurWBFBT, rescaled form; wbfbt.cu)
// Operators for one surface scaling a (eta_a = a^2 eta on the micro-tets with a vertex on
// the outer surface, eta elsewhere): K_{1/sqrt(eta_a)} on the multigrid levels with its
// GMG, and the lumped M_{sqrt(eta_a)}^-1 on the finest level.  Built on first use of a and
// rebuilt after a coefficient change; `side` identifies them in the calls below.
mfs_status pmg_side(mfs_problem* P, double a, int* side);
// coarsest multigrid level, or -1 before mfs_setup_multigrid
int mg_lmin(const mfs_problem* P);
// y = K_{1/sqrt(eta_a)} p on level lvl (multigrid range)
template <typename T>
mfs_status poisson_apply(mfs_problem* P, int side, int lvl, const T* p, T* y);
// x = one V-cycle for K x = b on the finest level (x overwritten; m steps of degree deg)
template <typename T>
mfs_status poisson_vcycle(mfs_problem* P, int side, T* x, const T* b, int m, int deg);
// lumped M_{sqrt(eta_a)}^-1 replicated per velocity component ([3][n_p2], finest level)
template <typename T>
const T* poisson_minv(mfs_problem* P, int side);
// d = the lumped M_{sqrt(eta_a)} diagonal [n_p2] on the finest level (FP64, device)
mfs_status lumped_vmass(mfs_problem* P, double a, double* d);
// y = the consistent M_{sqrt(eta_a)} x on the three components of the finest level
// ([3][n_p2]; diag != 0: its diagonal [n_p2], x unused; temperature.cu, on the degree-5 rule)
template <typename T>
mfs_status wmass_apply(mfs_problem* P, double a, const T* x, T* y, int diag);
// the inverse diagonal of the consistent M_{sqrt(eta_a)} replicated per velocity component
// ([3][n_p2], finest level), built on first use after each coefficient change
template <typename T>
mfs_status poisson_cmass_dinv(mfs_problem* P, int side, const T** out);
// g_k = -eta_k sum_tets sum_q 2 w|det J| psi_k(q) eps(u)(q) : eps(lam)(q)   (FP64)
mfs_status grad_log_eta(mfs_problem* P, int lvl, const double* u, const double* lam, double* g);

}  // namespace mfs
