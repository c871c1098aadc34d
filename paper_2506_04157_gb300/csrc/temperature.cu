// Temperature step of the mantle-convection model (arxiv 2506.04157, Sec. 3 and Sec. 6) on the
// finest level of a problem's blended shell:
//  * the P2 scalar operator  y = cM M x + cC C(u) x + cD D x + cR R(u) x  with
//      M = int phi_j phi_i,  C(u) = int (u.grad phi_j) phi_i,  R(u) = int (u.g) phi_j phi_i,
//      D = int grad phi_j . grad(phi_i / rho)  (or its symmetric part int grad phi_j . grad phi_i / rho),
//    g = -x/|x|, as a micro-tet sweep (one CTA per tile, one thread per micro-tet) with a
//    27-point conical product rule of degree 5 (the P2 mass is of degree 4), optionally
//    with the Dirichlet rows and columns of both spheres replaced by the identity;
//  * the right-hand side of Eq. (WeakTemp): BDF2 history, internal heating and shear heating
//    2 eta(x, T*) eps(u*):eps(u*) / rho (deviatoric eps, the viscosity law at the points);
//  * the particle MMOC: one classical RK4 step backwards from every P2 node along the velocity
//    interpolated linearly in time, then the P2 field at the departure point, with point
//    location in the blended shell (face by the largest e.n, inverse blending, macro Kuhn
//    coordinates, Freudenthal cube and type); for T^{n-1} the same particles are traced on
//    over the second step (the characteristic X(t^{n+1}, t^{n-1}, x) of Sec. 3);
//  * the solve: FGMRES in FP64 preconditioned by a Jacobi-CG in FP32 on the symmetric part
//    s1 M + tau k/(Pe Cp) D_s of the left-hand side.  The left-hand side has no advection
//    block: Sec. 3 solves the energy equation without the advection after the MMOC (the
//    printed u*.grad T term would advect twice and break the second-order convergence).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "apply.cuh"
#include "library.h"
#include "qp_geometry.cuh"
#include "solver.h"
#include "sweep_params.cuh"

namespace mfs {

constexpr int kTQ = 27;   // points of the conical product rule
__constant__ double c_tq_lam[kTQ][4];
__constant__ double c_tq_w[kTQ];

namespace {
inline int tblk(int64_t n, int threads = 256, int cap = 8192) {
  int64_t b = (n + threads - 1) / threads;
  if (b < 1) b = 1;
  return (int)(b < cap ? b : cap);
}

// Jacobi polynomial P_k^{(a,b)}(x) by its three-term recurrence
double jacobi_p(int k, double a, double b, double x) {
  if (k == 0) return 1.0;
  double p0 = 1.0, p1 = 0.5 * ((a + b + 2) * x + (a - b));
  for (int j = 2; j <= k; ++j) {
    const double c = 2 * j + a + b;
    const double p2 = ((c - 1) * (c * (c - 2) * x + a * a - b * b) * p1 - 2 * (j + a - 1) * (j + b - 1) * c * p0) /
                      (2 * j * (j + a + b) * (c - 2));
    p0 = p1;
    p1 = p2;
  }
  return p1;
}

// Gauss-Jacobi rule on [-1, 1] with weight (1-x)^a (1+x)^b: the k simple roots of P_k by
// bracketing on a fine grid and bisection, weights from
//   w_i = Gamma(k+a+1) Gamma(k+b+1) 2^(a+b+1) / (Gamma(k+a+b+1) k! (1 - x_i^2) P_k'(x_i)^2),
//   P_k' = (k + a + b + 1)/2 P_{k-1}^{(a+1,b+1)}
bool gauss_jacobi(int k, double a, double b, double* x, double* w) {
  int found = 0;
  const int grid = 4000;
  double xl = -1.0, fl = jacobi_p(k, a, b, xl + 1e-14);
  for (int g = 1; g <= grid && found < k; ++g) {
    const double xr = -1.0 + 2.0 * g / grid;
    const double fr = jacobi_p(k, a, b, g == grid ? xr - 1e-14 : xr);
    if ((fl < 0) != (fr < 0)) {
      double lo = xl, hi = xr, flo = fl;
      for (int it = 0; it < 200; ++it) {
        const double mid = 0.5 * (lo + hi);
        const double fm = jacobi_p(k, a, b, mid);
        if ((fm < 0) == (flo < 0)) {
          lo = mid;
          flo = fm;
        } else {
          hi = mid;
        }
      }
      x[found++] = 0.5 * (lo + hi);
    }
    xl = xr;
    fl = fr;
  }
  if (found != k) return false;
  const double c = std::exp(std::lgamma(k + a + 1) + std::lgamma(k + b + 1) - std::lgamma(k + a + b + 1) -
                            std::lgamma(k + 1.0)) * std::pow(2.0, a + b + 1);
  for (int i = 0; i < k; ++i) {
    const double dp = 0.5 * (k + a + b + 1) * jacobi_p(k - 1, a + 1, b + 1, x[i]);
    w[i] = c / ((1 - x[i] * x[i]) * dp * dp);
  }
  return true;
}

// Stroud's conical product rule on the reference tet (z1 = s, z2 = (1-s) t, z3 = (1-s)(1-t) v;
// Gauss-Jacobi in s (weight (1-s)^2) and t (weight 1-t), Gauss-Legendre in v), checked
// against the exact integrals of the monomials up to degree 5
bool conical_rule27(double lam[kTQ][4], double w[kTQ]) {
  double xs[3], ws[3], xt[3], wt[3], xv[3], wv[3];
  if (!gauss_jacobi(3, 2.0, 0.0, xs, ws) || !gauss_jacobi(3, 1.0, 0.0, xt, wt) || !gauss_jacobi(3, 0.0, 0.0, xv, wv))
    return false;
  int q = 0;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      for (int k = 0; k < 3; ++k, ++q) {
        const double s = 0.5 * (xs[i] + 1), t = 0.5 * (xt[j] + 1), v = 0.5 * (xv[k] + 1);
        const double z1 = s, z2 = (1 - s) * t, z3 = (1 - s) * (1 - t) * v;
        lam[q][0] = 1 - z1 - z2 - z3;
        lam[q][1] = z1;
        lam[q][2] = z2;
        lam[q][3] = z3;
        w[q] = ws[i] / 8 * wt[j] / 4 * wv[k] / 2;
      }
  auto fact = [](int m) {
    double f = 1;
    for (int i = 2; i <= m; ++i) f *= i;
    return f;
  };
  for (int deg = 0; deg <= 5; ++deg)
    for (int a = 0; a <= deg; ++a)
      for (int b = 0; a + b <= deg; ++b) {
        const int c = deg - a - b;
        double sum = 0;
        for (int p = 0; p < kTQ; ++p) sum += w[p] * std::pow(lam[p][1], a) * std::pow(lam[p][2], b) * std::pow(lam[p][3], c);
        if (std::fabs(sum - fact(a) * fact(b) * fact(c) / fact(deg + 3)) > 1e-15) return false;
      }
  return true;
}
}  // namespace

#define TM_STRIDE(i, n) \
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (n); i += (int64_t)gridDim.x * blockDim.x)

// ------------------------------------------------------------------------- sweep arguments
template <typename T>
struct TempArgs {
  const MacroGeom<T>* geom;
  const Tile* tiles;
  const uint16_t* tets;
  const int2* classes;
  const int* ids2;
  int n, n_p2;
  const double* dlnrho;
  int n_dlnrho;
  double r_cmb, r_surf;
  T cM, cC, cD, cR;
  const T* u;        // [3][n_p2] velocity (for cC, cR), or null
  const T* x;
  T* y;
  int constrained;   // 1: boundary columns dropped, boundary rows skipped
};

// lattice-frame gradients of the 10 P2 basis functions at barycentrics lam
template <typename T>
__device__ __forceinline__ void p2_lattice_grads(const T lam[4], T gl[10][3]) {
  const T GL[4][3] = {{-1, 0, 0}, {1, -1, 0}, {0, 1, -1}, {0, 0, 1}};
  for (int a = 0; a < 4; ++a)
    for (int j = 0; j < 3; ++j) gl[a][j] = (T(4) * lam[a] - T(1)) * GL[a][j];
  for (int e = 0; e < 6; ++e) {
    const int i0 = e < 3 ? 0 : (e < 5 ? 1 : 2);
    const int i1 = e < 3 ? e + 1 : (e < 5 ? e - 1 : 3);
    for (int j = 0; j < 3; ++j) gl[4 + e][j] = T(4) * (lam[i1] * GL[i0][j] + lam[i0] * GL[i1][j]);
  }
}
template <typename T>
__host__ __device__ __forceinline__ void p2_values_at(const T lam[4], T phi[10]) {
  for (int a = 0; a < 4; ++a) phi[a] = lam[a] * (T(2) * lam[a] - T(1));
  phi[4] = T(4) * lam[0] * lam[1];
  phi[5] = T(4) * lam[0] * lam[2];
  phi[6] = T(4) * lam[0] * lam[3];
  phi[7] = T(4) * lam[1] * lam[2];
  phi[8] = T(4) * lam[1] * lam[3];
  phi[9] = T(4) * lam[2] * lam[3];
}
// d ln rho / dr from the uniform radial table
__device__ __forceinline__ double dlnrho_tab(const double* tab, int nt, double r, double r0, double r1) {
  if (nt <= 1) return tab[0];
  const double top = nt - 1;
  double s = (r - r0) / (r1 - r0) * top;
  s = s < 0 ? 0 : (s > top ? top : s);
  int i = (int)s;
  i = i > nt - 2 ? nt - 2 : i;
  const double f = s - i;
  return (1 - f) * tab[i] + f * tab[i + 1];
}

// y (+)= (cM M + cC C(u) + cD D + cR R(u)) x  (DIAG: the diagonal of cM M + cD D, x unused)
template <typename T, bool BLEND, bool SYM, bool VEL, bool DIAG>
__global__ void __launch_bounds__(128) k_temp_apply(const TempArgs<T> P) {
  __shared__ T xs[NSLOT2], ys[NSLOT2];
  __shared__ T us[VEL ? 3 * NSLOT2 : 1];
  const int m = blockIdx.y, tidx = blockIdx.x;
  const size_t lin = (size_t)m * gridDim.x + tidx;
  const Tile tile = P.tiles[tidx];
  const MacroGeom<T>& G = P.geom[m];
  const int n = P.n;
  const int* tab2 = P.ids2 + lin * NSLOT2;
  for (int s = threadIdx.x; s < NSLOT2; s += blockDim.x) {
    const int code = tab2[s];
    const bool ok = code >= 0;
    const bool drop = !ok || (P.constrained && slot_class(code) != 0);
    const int64_t id = slot_node(code);
    xs[s] = (!DIAG && !drop) ? P.x[id] : T(0);
    ys[s] = T(0);
    if (VEL)
      for (int c = 0; c < 3; ++c) us[c * NSLOT2 + s] = ok ? P.u[c * (int64_t)P.n_p2 + id] : T(0);
  }
  __syncthreads();
  const T vol = G.absdet / (T(n) * T(n) * T(n));
  const int2 cinfo = P.classes[tile.cls];
  for (int t = threadIdx.x; t < cinfo.y; t += blockDim.x) {
    const int code = P.tets[cinfo.x + t];
    const int ci = code & 15, cj = (code >> 4) & 15, ck = (code >> 8) & 15, pmu = code >> 12;
    const int p0 = perm_at(pmu, 0), p1 = perm_at(pmu, 1), p2 = perm_at(pmu, 2);
    const int base = ci + 5 * cj + 25 * ck;
    int slot[10];
    T xv[10], uv[3][10], acc[10];
    for (int a = 0; a < 10; ++a) {
      slot[a] = base + slot_off(pmu, a);
      xv[a] = xs[slot[a]];
      acc[a] = T(0);
      if (VEL)
        for (int c = 0; c < 3; ++c) uv[c][a] = us[c * NSLOT2 + slot[a]];
    }
    const T qb[3] = {T(tile.ta * TT + ci), T(tile.tb * TT + cj), T(tile.tc * TT + ck)};
#pragma unroll 1
    for (int q = 0; q < kTQ; ++q) {
      T lam[4];
      for (int a = 0; a < 4; ++a) lam[a] = T(c_tq_lam[q][a]);
      T xi[3];
      for (int d = 0; d < 3; ++d)
        xi[d] = qb[d] + lam[3] + (d == p0 ? lam[1] + lam[2] : T(0)) + (d == p1 ? lam[2] : T(0));
      T K[3][3], hr, rinv, x[3];
      lattice_geometry<T, BLEND>(G, n, p0, p1, p2, xi[0], xi[1], xi[2], K, hr, rinv, x);
      const T W = T(c_tq_w[q]) * vol * hr * hr * hr;
      T phi[10], gl[10][3], g[10][3];
      p2_values_at<T>(lam, phi);
      p2_lattice_grads<T>(lam, gl);
      const T ihr = T(1) / hr;
      for (int a = 0; a < 10; ++a)
        for (int d = 0; d < 3; ++d) g[a][d] = (gl[a][0] * K[0][d] + gl[a][1] * K[1][d] + gl[a][2] * K[2][d]) * ihr;
      const T h = x[0] * G.nh[0] + x[1] * G.nh[1] + x[2] * G.nh[2];
      const double rad = BLEND ? double(h / G.delta) : double(T(1) / rinv);
      const T rho = T(rho_of(P.dlnrho, P.n_dlnrho, rad, P.r_cmb, P.r_surf));
      const T e[3] = {x[0] * rinv, x[1] * rinv, x[2] * rinv};
      if (DIAG) {
        for (int a = 0; a < 10; ++a)
          acc[a] += W * (P.cM * phi[a] * phi[a] + P.cD / rho * (g[a][0] * g[a][0] + g[a][1] * g[a][1] + g[a][2] * g[a][2]));
        continue;
      }
      T Tq = T(0), gT[3] = {T(0), T(0), T(0)};
      for (int a = 0; a < 10; ++a) {
        Tq += phi[a] * xv[a];
        for (int d = 0; d < 3; ++d) gT[d] += xv[a] * g[a][d];
      }
      T cphi = P.cM * Tq;
      if (VEL) {
        T uq[3] = {T(0), T(0), T(0)};
        for (int a = 0; a < 10; ++a)
          for (int c = 0; c < 3; ++c) uq[c] += phi[a] * uv[c][a];
        cphi += P.cC * (uq[0] * gT[0] + uq[1] * gT[1] + uq[2] * gT[2]) -
                P.cR * (uq[0] * e[0] + uq[1] * e[1] + uq[2] * e[2]) * Tq;
      }
      if (!SYM) {   // grad(phi_i / rho) = grad phi_i / rho - phi_i (d ln rho/dr) e / rho
        const T dl = T(dlnrho_tab(P.dlnrho, P.n_dlnrho, rad, P.r_cmb, P.r_surf));
        cphi -= P.cD * dl / rho * (gT[0] * e[0] + gT[1] * e[1] + gT[2] * e[2]);
      }
      const T cg[3] = {P.cD / rho * gT[0], P.cD / rho * gT[1], P.cD / rho * gT[2]};
      for (int a = 0; a < 10; ++a) acc[a] += W * (cphi * phi[a] + cg[0] * g[a][0] + cg[1] * g[a][1] + cg[2] * g[a][2]);
    }
    for (int a = 0; a < 10; ++a) atomicAdd(&ys[slot[a]], acc[a]);
  }
  __syncthreads();
  for (int s = threadIdx.x; s < NSLOT2; s += blockDim.x) {
    const int code = tab2[s];
    if (code < 0 || (P.constrained && slot_class(code) != 0)) continue;
    atomicAdd(&P.y[slot_node(code)], ys[s]);
  }
}

// b += int phi_i [s0 T0 - sm Tm + cH + cS 2 eta(x, T*) eps(u*):eps(u*) / rho]
struct RhsArgs {
  const MacroGeom<double>* geom;
  const Tile* tiles;
  const uint16_t* tets;
  const int2* classes;
  const int* ids2;
  int n, n_p2;
  const double* dlnrho;
  int n_dlnrho;
  double r_cmb, r_surf;
  const double *T0, *Tm, *us, *Ts;   // us: [3][n_p2]
  double s0, sm, cH, cS;
  const double* lbase;               // viscosity law (cS != 0)
  int n_lbase;
  double E_A, V_A;
  double* b;
};

template <bool BLEND, bool SHEAR>
__global__ void __launch_bounds__(128) k_temp_rhs(const RhsArgs P) {
  __shared__ double hs[NSLOT2], bs[NSLOT2];
  __shared__ double ts[SHEAR ? NSLOT2 : 1];
  __shared__ double vs[SHEAR ? 3 * NSLOT2 : 1];
  const int m = blockIdx.y, tidx = blockIdx.x;
  const size_t lin = (size_t)m * gridDim.x + tidx;
  const Tile tile = P.tiles[tidx];
  const MacroGeom<double>& G = P.geom[m];
  const int n = P.n;
  const int* tab2 = P.ids2 + lin * NSLOT2;
  for (int s = threadIdx.x; s < NSLOT2; s += blockDim.x) {
    const int code = tab2[s];
    const int64_t id = slot_node(code);
    hs[s] = code >= 0 ? P.s0 * P.T0[id] - P.sm * P.Tm[id] : 0.0;
    bs[s] = 0.0;
    if (SHEAR) {
      ts[s] = code >= 0 ? P.Ts[id] : 0.0;
      for (int c = 0; c < 3; ++c) vs[c * NSLOT2 + s] = code >= 0 ? P.us[c * (int64_t)P.n_p2 + id] : 0.0;
    }
  }
  __syncthreads();
  const double vol = G.absdet / ((double)n * n * n);
  const int2 cinfo = P.classes[tile.cls];
  for (int t = threadIdx.x; t < cinfo.y; t += blockDim.x) {
    const int code = P.tets[cinfo.x + t];
    const int ci = code & 15, cj = (code >> 4) & 15, ck = (code >> 8) & 15, pmu = code >> 12;
    const int p0 = perm_at(pmu, 0), p1 = perm_at(pmu, 1), p2 = perm_at(pmu, 2);
    const int base = ci + 5 * cj + 25 * ck;
    int slot[10];
    double hv[10], acc[10];
    for (int a = 0; a < 10; ++a) {
      slot[a] = base + slot_off(pmu, a);
      hv[a] = hs[slot[a]];
      acc[a] = 0.0;
    }
    const double qb[3] = {double(tile.ta * TT + ci), double(tile.tb * TT + cj), double(tile.tc * TT + ck)};
#pragma unroll 1
    for (int q = 0; q < kTQ; ++q) {
      double lam[4];
      for (int a = 0; a < 4; ++a) lam[a] = c_tq_lam[q][a];
      double xi[3];
      for (int d = 0; d < 3; ++d)
        xi[d] = qb[d] + lam[3] + (d == p0 ? lam[1] + lam[2] : 0.0) + (d == p1 ? lam[2] : 0.0);
      double K[3][3], hr, rinv, x[3];
      lattice_geometry<double, BLEND>(G, n, p0, p1, p2, xi[0], xi[1], xi[2], K, hr, rinv, x);
      const double W = c_tq_w[q] * vol * hr * hr * hr;
      double phi[10];
      p2_values_at<double>(lam, phi);
      double val = P.cH;
      for (int a = 0; a < 10; ++a) val += phi[a] * hv[a];
      if (SHEAR) {
        double gl[10][3];
        p2_lattice_grads<double>(lam, gl);
        double Gu[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}}, Tq = 0.0;
        for (int a = 0; a < 10; ++a) {
          double ga[3];
          for (int d = 0; d < 3; ++d) ga[d] = (gl[a][0] * K[0][d] + gl[a][1] * K[1][d] + gl[a][2] * K[2][d]) / hr;
          const int sa = slot[a];
          for (int c = 0; c < 3; ++c)
            for (int d = 0; d < 3; ++d) Gu[c][d] += vs[c * NSLOT2 + sa] * ga[d];
          Tq += phi[a] * ts[sa];
        }
        const double tr = (Gu[0][0] + Gu[1][1] + Gu[2][2]) / 3.0;
        double ee = 0.0;
        for (int c = 0; c < 3; ++c)
          for (int d = 0; d < 3; ++d) {
            const double eps = 0.5 * (Gu[c][d] + Gu[d][c]) - (c == d ? tr : 0.0);
            ee += eps * eps;
          }
        const double h = x[0] * G.nh[0] + x[1] * G.nh[1] + x[2] * G.nh[2];
        const double rad = BLEND ? h / G.delta : 1.0 / rinv;
        const double rho = rho_of(P.dlnrho, P.n_dlnrho, rad, P.r_cmb, P.r_surf);
        const double eta = exp(2.302585092994045684 * radial_table<double>(P.lbase, P.n_lbase, rad, P.r_cmb, P.r_surf) -
                               P.E_A * Tq + P.V_A * (P.r_surf - rad));
        val += P.cS * 2.0 * eta * ee / rho;
      }
      for (int a = 0; a < 10; ++a) acc[a] += W * val * phi[a];
    }
    for (int a = 0; a < 10; ++a) atomicAdd(&bs[slot[a]], acc[a]);
  }
  __syncthreads();
  for (int s = threadIdx.x; s < NSLOT2; s += blockDim.x) {
    const int code = tab2[s];
    if (code < 0) continue;
    atomicAdd(&P.b[slot_node(code)], bs[s]);
  }
}

// ------------------------------------------------------------------------- weighted vector mass
// y_c = M_w x_c (c = 0..2), M_w the consistent P2 scalar mass with weight sqrt(s eta_q): eta_q
// the P1 interpolant of the level's nodal viscosity at the point, s = a^2 on micro-tets with a
// vertex on the outer surface and 1 elsewhere (the M_{sqrt(eta_a)} of the weighted BFBT,
// Sec. 5.2.3), on the degree-5 rule.  DIAG: its diagonal [n_p2] (x unused).  The components
// pass one after the other through the same shared staging (16 KB in FP64).
template <typename T, bool BLEND, bool DIAG>
__global__ void __launch_bounds__(128) k_wmass(const ApplyParams<T> P, T a2, int64_t n_p2, const T* __restrict__ x,
                                               T* __restrict__ y) {
  __shared__ T xs[NSLOT2], ys[NSLOT2];
  __shared__ T eta_s[NSLOT1];
  __shared__ int surf_s[NSLOT1];
  const int m = blockIdx.y, tidx = blockIdx.x;
  const size_t lin = (size_t)m * gridDim.x + tidx;
  const Tile tile = P.tiles[tidx];
  const MacroGeom<T>& G = P.geom[m];
  const int n = P.n;
  const int* tab2 = P.ids2 + lin * NSLOT2;
  for (int s = threadIdx.x; s < NSLOT1; s += blockDim.x) {
    const int id = P.ids1[lin * NSLOT1 + s];
    eta_s[s] = id >= 0 ? P.eta[id] : T(1);
    const int code = tab2[s];   // P2 slot s < NSLOT1 is the vertex slot s of the P1 block
    surf_s[s] = (code >= 0 && slot_class(code) == 1) ? 1 : 0;
  }
  const T vol = G.absdet / (T(n) * T(n) * T(n));
  const int2 cinfo = P.classes[tile.cls];
  for (int c = 0; c < (DIAG ? 1 : 3); ++c) {
    __syncthreads();   // staging of eta done; the previous component flushed
    for (int s = threadIdx.x; s < NSLOT2; s += blockDim.x) {
      const int code = tab2[s];
      xs[s] = (!DIAG && code >= 0) ? x[c * n_p2 + slot_node(code)] : T(0);
      ys[s] = T(0);
    }
    __syncthreads();
    for (int t = threadIdx.x; t < cinfo.y; t += blockDim.x) {
      const int code = P.tets[cinfo.x + t];
      const int ci = code & 15, cj = (code >> 4) & 15, ck = (code >> 8) & 15, pmu = code >> 12;
      const int p0 = perm_at(pmu, 0), p1 = perm_at(pmu, 1), p2 = perm_at(pmu, 2);
      const int base = ci + 5 * cj + 25 * ck;
      int slot[10];
      T xv[10], acc[10];
      for (int a = 0; a < 10; ++a) {
        slot[a] = base + slot_off(pmu, a);
        xv[a] = xs[slot[a]];
        acc[a] = T(0);
      }
      T ev[4];
      int on = 0;
      for (int a = 0; a < 4; ++a) {   // vertex slots lie in parity class 0: P1 slot = P2 slot
        ev[a] = eta_s[slot[a]];
        on |= surf_s[slot[a]];
      }
      const T sc = on ? a2 : T(1);
      const T qb[3] = {T(tile.ta * TT + ci), T(tile.tb * TT + cj), T(tile.tc * TT + ck)};
#pragma unroll 1
      for (int q = 0; q < kTQ; ++q) {
        T lam[4];
        for (int a = 0; a < 4; ++a) lam[a] = T(c_tq_lam[q][a]);
        T xi[3];
        for (int d = 0; d < 3; ++d)
          xi[d] = qb[d] + lam[3] + (d == p0 ? lam[1] + lam[2] : T(0)) + (d == p1 ? lam[2] : T(0));
        T K[3][3], hr, rinv, xq[3];
        lattice_geometry<T, BLEND>(G, n, p0, p1, p2, xi[0], xi[1], xi[2], K, hr, rinv, xq);
        const T etaq = lam[0] * ev[0] + lam[1] * ev[1] + lam[2] * ev[2] + lam[3] * ev[3];
        const T W = T(c_tq_w[q]) * vol * hr * hr * hr * sqrt(sc * etaq);
        T phi[10];
        p2_values_at<T>(lam, phi);
        if (DIAG) {
          for (int a = 0; a < 10; ++a) acc[a] += W * phi[a] * phi[a];
        } else {
          T v = T(0);
          for (int a = 0; a < 10; ++a) v += phi[a] * xv[a];
          v *= W;
          for (int a = 0; a < 10; ++a) acc[a] += v * phi[a];
        }
      }
      for (int a = 0; a < 10; ++a) atomicAdd(&ys[slot[a]], acc[a]);
    }
    __syncthreads();
    for (int s = threadIdx.x; s < NSLOT2; s += blockDim.x) {
      const int code = tab2[s];
      if (code < 0) continue;
      atomicAdd(&y[c * n_p2 + slot_node(code)], ys[s]);
    }
  }
}

// ------------------------------------------------------------------------- MMOC
struct MmocArgs {
  const MacroGeom<double>* geom;
  const MacroTopo* topo;
  Numbering nb2;
  int n, n_p2, blending;
  double r_cmb, r_surf;
  const double* xyz;   // [3][n_p2] physical node positions
};

// P2 node ids and barycentrics of the micro-tet holding X (X first moved radially into the
// shell; a point just outside a macro is projected onto its Kuhn simplex)
__host__ __device__ void mmoc_locate(const MmocArgs& A, const double Xin[3], int ids[10], double lam[4]) {
  const double R0 = sqrt(Xin[0] * Xin[0] + Xin[1] * Xin[1] + Xin[2] * Xin[2]);
  const double e[3] = {Xin[0] / R0, Xin[1] / R0, Xin[2] / R0};
  double dmax = -2.0, dl = 1.0;   // the prism the direction points through: its face alignment, offset
  for (int m = 0; m < 60; ++m) {
    const double* nh = A.geom[m].nh;
    const double d = e[0] * nh[0] + e[1] * nh[1] + e[2] * nh[2];
    if (d > dmax) {
      dmax = d;
      dl = A.geom[m].delta;
    }
  }
  // radially onto the shell: between the spheres (blended), between the prism's inner and
  // outer face planes nh.x = r delta (polyhedral)
  const double R = A.blending ? fmin(fmax(R0, A.r_cmb), A.r_surf)
                              : fmin(fmax(R0 * dmax, A.r_cmb * dl), A.r_surf * dl) / dmax;
  const double X[3] = {R * e[0], R * e[1], R * e[2]};
  int bm = 0;
  double best = -1e300, bxi[3] = {0, 0, 0};
  for (int m = 0; m < 60; ++m) {
    const MacroGeom<double>& G = A.geom[m];
    const double d = e[0] * G.nh[0] + e[1] * G.nh[1] + e[2] * G.nh[2];
    if (d < dmax - 1e-12) continue;
    double xt[3];
    const double sc = A.blending ? R * G.delta / d : 1.0;
    for (int r = 0; r < 3; ++r) xt[r] = A.blending ? sc * e[r] : X[r];
    double z[3];
    for (int r = 0; r < 3; ++r)
      z[r] = G.Jinv[3 * r] * (xt[0] - G.v0[0]) + G.Jinv[3 * r + 1] * (xt[1] - G.v0[1]) + G.Jinv[3 * r + 2] * (xt[2] - G.v0[2]);
    const double sc4 = fmin(fmin(1.0 - z[0], z[0] - z[1]), fmin(z[1] - z[2], z[2]));
    if (sc4 > best) {
      best = sc4;
      bm = m;
      bxi[0] = z[0];
      bxi[1] = z[1];
      bxi[2] = z[2];
    }
  }
  const int n = A.n;
  const double x0 = fmin(fmax(bxi[0], 0.0), 1.0);
  const double x1 = fmin(fmax(bxi[1], 0.0), x0);
  const double x2 = fmin(fmax(bxi[2], 0.0), x1);
  const double C3[3] = {n * x0, n * x1, n * x2};
  int cb[3];
  double fr[3];
  for (int d = 0; d < 3; ++d) {
    int c = (int)floor(C3[d]);
    c = c < 0 ? 0 : (c > n - 1 ? n - 1 : c);
    cb[d] = c;
    fr[d] = fmin(fmax(C3[d] - c, 0.0), 1.0);
  }
  // Freudenthal type: coordinates by decreasing fractional part, ties by index
  int p[3] = {0, 1, 2};
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2 - i; ++j)
      if (fr[p[j + 1]] > fr[p[j]]) {
        const int t = p[j];
        p[j] = p[j + 1];
        p[j + 1] = t;
      }
  lam[0] = 1.0 - fr[p[0]];
  lam[1] = fr[p[0]] - fr[p[1]];
  lam[2] = fr[p[1]] - fr[p[2]];
  lam[3] = fr[p[2]];
  int v[4][3];
  for (int d = 0; d < 3; ++d) {
    v[0][d] = cb[d];
    v[1][d] = cb[d] + (d == p[0]);
    v[2][d] = v[1][d] + (d == p[1]);
    v[3][d] = cb[d] + 1;
  }
  const int N2 = 2 * n;
  const MacroTopo& t = A.topo[bm];
  for (int a = 0; a < 10; ++a) {
    int F[3];
    if (a < 4) {
      for (int d = 0; d < 3; ++d) F[d] = 2 * v[a][d];
    } else {
      const int e2 = a - 4;
      const int i0 = e2 < 3 ? 0 : (e2 < 5 ? 1 : 2);
      const int i1 = e2 < 3 ? e2 + 1 : (e2 < 5 ? e2 - 1 : 3);
      for (int d = 0; d < 3; ++d) F[d] = v[i0][d] + v[i1][d];
    }
    ids[a] = lattice_id(t, A.nb2, bm, N2 - F[0], F[0] - F[1], F[1] - F[2], F[2]);
  }
}

__host__ __device__ __forceinline__ double p2_eval(const double* f, const int ids[10], const double phi[10]) {
  double s = 0.0;
  for (int a = 0; a < 10; ++a) s += phi[a] * f[ids[a]];
  return s;
}

// u(X) = wn u_new(X) + wo u_old(X)
__host__ __device__ void velocity_at(const MmocArgs& A, const double* un, const double* uo, double wn, double wo, const double X[3],
                            double out[3]) {
  int ids[10];
  double lam[4], phi[10];
  mmoc_locate(A, X, ids, lam);
  p2_values_at<double>(lam, phi);
  const int64_t n2 = A.n_p2;
  for (int c = 0; c < 3; ++c) {
    double s = 0.0;
    if (wn != 0.0) s += wn * p2_eval(un + c * n2, ids, phi);
    if (wo != 0.0) s += wo * p2_eval(uo + c * n2, ids, phi);
    out[c] = s;
  }
}

// One particle (Sec. 3): departure point X of the particle at x after one classical RK4 step
// backwards over tau, u linear in time from u_old (start) to u_new (end), and T there.  The
// same code runs in k_mmoc and, on the host, in mfs_mmoc_host.
__host__ __device__ void mmoc_particle(const MmocArgs& A, const double x[3], const double* T, const double* un,
                                       const double* uo, double tau, double* That, double X[3]) {
  double k1[3], k2[3], k3[3], k4[3], y[3];
  velocity_at(A, un, uo, 1.0, 0.0, x, k1);
  for (int c = 0; c < 3; ++c) y[c] = x[c] - 0.5 * tau * k1[c];
  velocity_at(A, un, uo, 0.5, 0.5, y, k2);
  for (int c = 0; c < 3; ++c) y[c] = x[c] - 0.5 * tau * k2[c];
  velocity_at(A, un, uo, 0.5, 0.5, y, k3);
  for (int c = 0; c < 3; ++c) y[c] = x[c] - tau * k3[c];
  velocity_at(A, un, uo, 0.0, 1.0, y, k4);
  for (int c = 0; c < 3; ++c) X[c] = x[c] - tau / 6.0 * (k1[c] + 2.0 * k2[c] + 2.0 * k3[c] + k4[c]);
  int ids[10];
  double lam[4], phi[10];
  mmoc_locate(A, X, ids, lam);
  p2_values_at<double>(lam, phi);
  *That = p2_eval(T, ids, phi);
}

// particle i starts at node i (Xin = null) or at Xin[:, i]
__global__ void k_mmoc(const MmocArgs A, const double* __restrict__ Xin, const double* __restrict__ T,
                       const double* __restrict__ un, const double* __restrict__ uo, double tau,
                       double* __restrict__ That, double* __restrict__ Xout) {
  TM_STRIDE(i, A.n_p2) {
    const int64_t n2 = A.n_p2;
    const double* X0 = Xin ? Xin : A.xyz;
    const double x[3] = {X0[i], X0[n2 + i], X0[2 * n2 + i]};
    double X[3];
    mmoc_particle(A, x, T, un, uo, tau, &That[i], X);
    if (Xout)
      for (int c = 0; c < 3; ++c) Xout[c * n2 + i] = X[c];
  }
}

// ------------------------------------------------------------------------- small kernels
__global__ void k_set_at(int nb, const int* __restrict__ ids, const double* __restrict__ src, double* __restrict__ dst) {
  TM_STRIDE(k, nb) dst[ids[k]] = src ? src[ids[k]] : 0.0;
}
template <typename T>
__global__ void k_identity_rows(int nb, const int* __restrict__ ids, const T* __restrict__ x, T* __restrict__ y) {
  TM_STRIDE(k, nb) y[ids[k]] = x[ids[k]];
}
template <typename T>
__global__ void k_one_at(int nb, const int* __restrict__ ids, T* __restrict__ d) {
  TM_STRIDE(k, nb) d[ids[k]] = T(1);
}

// ------------------------------------------------------------------------- host side
struct TempWork {
  int n2 = 0, nb = 0, m = 0;
  int* bids = nullptr;           // boundary P2 node ids (both spheres)
  double* xyz = nullptr;         // [3][n2] node positions
  double *ustar = nullptr, *Tstar = nullptr, *T0h = nullptr, *Tmh = nullptr, *tmp = nullptr;
  double *b = nullptr, *xb = nullptr, *w = nullptr, *sol = nullptr;
  std::vector<double*> V, Z;     // FGMRES basis (FP64)
  float *r32 = nullptr, *z32 = nullptr, *p32 = nullptr, *q32 = nullptr, *x32 = nullptr, *d32 = nullptr;
  double* red = nullptr;
  double* hpin = nullptr;
  std::vector<void*> owned;
};

// the rule's constant-memory copy, uploaded once per device
static std::mutex g_rule_mutex;
static std::vector<char> g_rule_ready;

static mfs_status ensure_rule() {
  int dev = 0;
  MFS_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lock(g_rule_mutex);
  if ((int)g_rule_ready.size() > dev && g_rule_ready[dev]) return MFS_OK;
  double lam[kTQ][4], w[kTQ];
  if (!conical_rule27(lam, w)) {
    set_error("the conical quadrature rule failed its exactness check");
    return MFS_EINVAL;
  }
  MFS_CUDA(cudaMemcpyToSymbol(c_tq_lam, lam, sizeof(lam)));
  MFS_CUDA(cudaMemcpyToSymbol(c_tq_w, w, sizeof(w)));
  if ((int)g_rule_ready.size() <= dev) g_rule_ready.resize(dev + 1, 0);
  g_rule_ready[dev] = 1;
  return MFS_OK;
}

// y = M_{sqrt(eta_a)} x on the three components of the finest level ([3][n_p2]); diag: the
// diagonal, [n_p2] (x unused)
template <typename T>
mfs_status wmass_apply(mfs_problem* Pb, double a, const T* x, T* y, int diag) {
  MFS_TRY(ensure_rule());
  mfs_mesh* M = Pb->mesh;
  const int L = M->l_max;
  const LevelData& Lv = M->levels[L];
  cudaStream_t s = M->ctx->stream;
  const int64_t n2 = Lv.nb2.total;
  MFS_CUDA(cudaMemsetAsync(y, 0, sizeof(T) * (size_t)n2 * (diag ? 1 : 3), s));
  const ApplyParams<T> prm = sweep_params<T>(Pb, L);
  const dim3 grid(Lv.n_tiles, kMacroCells);
  const T a2 = T(a * a);
  if (M->host.blending) {
    if (diag) k_wmass<T, true, true><<<grid, 128, 0, s>>>(prm, a2, n2, nullptr, y);
    else k_wmass<T, true, false><<<grid, 128, 0, s>>>(prm, a2, n2, x, y);
  } else {
    if (diag) k_wmass<T, false, true><<<grid, 128, 0, s>>>(prm, a2, n2, nullptr, y);
    else k_wmass<T, false, false><<<grid, 128, 0, s>>>(prm, a2, n2, x, y);
  }
  MFS_CUDA(cudaGetLastError());
  return MFS_OK;
}
template mfs_status wmass_apply<double>(mfs_problem*, double, const double*, double*, int);
template mfs_status wmass_apply<float>(mfs_problem*, double, const float*, float*, int);

template <typename T>
static mfs_status talloc(TempWork* W, T** p, int64_t n, cudaStream_t s) {
  const size_t bytes = sizeof(T) * (size_t)(n > 0 ? n : 1);
  cudaError_t e = cudaMalloc((void**)p, bytes);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(temperature workspace)");
  W->owned.push_back(*p);
  MFS_CUDA(cudaMemsetAsync(*p, 0, bytes, s));
  return MFS_OK;
}

void temp_destroy(TempWork* W) {
  if (!W) return;
  for (void* p : W->owned) cudaFree(p);
  if (W->hpin) cudaFreeHost(W->hpin);
  delete W;
}

static mfs_status temp_work(mfs_problem* Pb, int m, TempWork** out) {
  MFS_TRY(ensure_rule());
  mfs_mesh* M = Pb->mesh;
  const int L = M->l_max;
  const int n2 = M->levels[L].nb2.total;
  TempWork* W = Pb->tw;
  if (W && W->n2 == n2 && W->m >= m) {
    *out = W;
    return MFS_OK;
  }
  if (W) temp_destroy(W);
  W = new TempWork;
  Pb->tw = W;
  cudaStream_t s = M->ctx->stream;
  W->n2 = n2;
  W->m = m;
  // node positions and the boundary list, from the host numbering
  const int N = 2 << L;
  std::vector<double> xyz(3 * (size_t)n2);
  std::vector<int> bids;
  for_each_point(M, N, [&](int mc, const int* i, int id) {
    double xs[3], x[3];
    M->host.straight_point(mc, i, N, xs);
    if (M->host.blending) M->host.blend_point(mc, xs, x);
    else for (int r = 0; r < 3; ++r) x[r] = xs[r];
    for (int r = 0; r < 3; ++r) xyz[r * (size_t)n2 + id] = x[r];
  });
  std::vector<char> seen(n2, 0);
  for_each_point(M, N, [&](int mc, const int* i, int id) {
    const int mask = (i[0] > 0) | ((i[1] > 0) << 1) | ((i[2] > 0) << 2) | ((i[3] > 0) << 3);
    const MacroTopo& t = M->host.topo[mc];
    const bool on = ((mask & ~t.topmask & 15) == 0) || ((mask & ~t.botmask & 15) == 0);
    if (on && !seen[id]) {
      seen[id] = 1;
      bids.push_back(id);
    }
  });
  W->nb = (int)bids.size();
  MFS_TRY(talloc(W, &W->xyz, 3 * (int64_t)n2, s));
  MFS_TRY(talloc(W, &W->bids, W->nb, s));
  MFS_CUDA(cudaMemcpyAsync(W->xyz, xyz.data(), sizeof(double) * xyz.size(), cudaMemcpyHostToDevice, s));
  MFS_CUDA(cudaMemcpyAsync(W->bids, bids.data(), sizeof(int) * bids.size(), cudaMemcpyHostToDevice, s));
  for (double** v : {&W->ustar, &W->tmp}) MFS_TRY(talloc(W, v, 3 * (int64_t)n2, s));
  for (double** v : {&W->Tstar, &W->T0h, &W->Tmh, &W->b, &W->xb, &W->w, &W->sol}) MFS_TRY(talloc(W, v, n2, s));
  for (float** v : {&W->r32, &W->z32, &W->p32, &W->q32, &W->x32, &W->d32}) MFS_TRY(talloc(W, v, n2, s));
  W->V.assign(m + 1, nullptr);
  W->Z.assign(m, nullptr);
  for (auto& v : W->V) MFS_TRY(talloc(W, &v, n2, s));
  for (auto& v : W->Z) MFS_TRY(talloc(W, &v, n2, s));
  MFS_TRY(talloc(W, &W->red, kRedBlocks + 16, s));
  MFS_CUDA(cudaMallocHost((void**)&W->hpin, 8 * sizeof(double)));
  MFS_CUDA(cudaStreamSynchronize(s));
  *out = W;
  return MFS_OK;
}

template <typename T>
static TempArgs<T> temp_args(mfs_problem* Pb) {
  mfs_mesh* M = Pb->mesh;
  const int L = M->l_max;
  const LevelData& Lv = M->levels[L];
  TempArgs<T> a{};
  a.geom = lvl_geom<T>(M);
  a.tiles = Lv.d_tiles;
  a.tets = Lv.d_tets;
  a.classes = Lv.d_classes;
  a.ids2 = Lv.d_ids2;
  a.n = Lv.n;
  a.n_p2 = Lv.nb2.total;
  a.dlnrho = Pb->d_dlnrho64;
  a.n_dlnrho = Pb->n_dlnrho;
  a.r_cmb = M->host.r_cmb;
  a.r_surf = M->host.r_surf;
  return a;
}

// y = (cM M + cC C(u) + cD D + cR R(u)) x on the finest level; constrained: identity on the
// boundary rows and columns; diag: the diagonal of cM M + cD D (x unused)
template <typename T>
static mfs_status temp_apply(mfs_problem* Pb, TempWork* W, T cM, T cC, T cD, T cR, int sym, int constrained,
                             const T* u, const T* x, T* y, int diag) {
  mfs_mesh* M = Pb->mesh;
  const LevelData& Lv = M->levels[M->l_max];
  cudaStream_t s = M->ctx->stream;
  MFS_CUDA(cudaMemsetAsync(y, 0, sizeof(T) * (size_t)Lv.nb2.total, s));
  TempArgs<T> a = temp_args<T>(Pb);
  a.cM = cM;
  a.cC = cC;
  a.cD = cD;
  a.cR = cR;
  a.u = u;
  a.x = x;
  a.y = y;
  a.constrained = constrained;
  const bool vel = u != nullptr && (cC != T(0) || cR != T(0));
  const bool bl = M->host.blending != 0;
  dim3 grid(Lv.n_tiles, kMacroCells);
#define TEMP_LAUNCH(B, S, V, D) k_temp_apply<T, B, S, V, D><<<grid, 128, 0, s>>>(a)
  if (diag) {
    if (bl) { if (sym) TEMP_LAUNCH(true, true, false, true); else TEMP_LAUNCH(true, false, false, true); }
    else { if (sym) TEMP_LAUNCH(false, true, false, true); else TEMP_LAUNCH(false, false, false, true); }
  } else if (vel) {
    if (bl) { if (sym) TEMP_LAUNCH(true, true, true, false); else TEMP_LAUNCH(true, false, true, false); }
    else { if (sym) TEMP_LAUNCH(false, true, true, false); else TEMP_LAUNCH(false, false, true, false); }
  } else {
    if (bl) { if (sym) TEMP_LAUNCH(true, true, false, false); else TEMP_LAUNCH(true, false, false, false); }
    else { if (sym) TEMP_LAUNCH(false, true, false, false); else TEMP_LAUNCH(false, false, false, false); }
  }
#undef TEMP_LAUNCH
  MFS_CUDA(cudaGetLastError());
  if (constrained && W->nb) {
    if (diag) k_one_at<T><<<tblk(W->nb), 256, 0, s>>>(W->nb, W->bids, y);
    else k_identity_rows<T><<<tblk(W->nb), 256, 0, s>>>(W->nb, W->bids, x, y);
  }
  MFS_CUDA(cudaGetLastError());
  return MFS_OK;
}

static mfs_status temp_rhs(mfs_problem* Pb, const mfs_temp_params& tp, const double* T0h, const double* Tmh,
                           const double* ustar, const double* Tstar, double tau1, double tau0, double* b) {
  mfs_mesh* M = Pb->mesh;
  const LevelData& Lv = M->levels[M->l_max];
  cudaStream_t s = M->ctx->stream;
  const double s0 = (tau1 + tau0) / tau0, sm = tau1 * tau1 / (tau0 * (tau1 + tau0));
  RhsArgs a{};
  a.geom = M->d_geom64;
  a.tiles = Lv.d_tiles;
  a.tets = Lv.d_tets;
  a.classes = Lv.d_classes;
  a.ids2 = Lv.d_ids2;
  a.n = Lv.n;
  a.n_p2 = Lv.nb2.total;
  a.dlnrho = Pb->d_dlnrho64;
  a.n_dlnrho = Pb->n_dlnrho;
  a.r_cmb = M->host.r_cmb;
  a.r_surf = M->host.r_surf;
  a.T0 = T0h;
  a.Tm = Tmh;
  a.us = ustar;
  a.Ts = Tstar;
  a.s0 = s0;
  a.sm = sm;
  a.cH = tau1 * tp.H / tp.Cp;
  a.cS = tau1 * tp.Pe * tp.Di / (tp.Ra * tp.Cp);
  a.lbase = Pb->d_lbase64;
  a.n_lbase = (int)Pb->lbase_host.size();
  a.E_A = Pb->E_A;
  a.V_A = Pb->V_A;
  a.b = b;
  const bool shear = a.cS != 0.0;
  if (shear && (!Pb->d_lbase64 || !ustar || !Tstar)) {
    set_error("shear heating (Di != 0) needs the viscosity law (mfs_set_viscosity_law), u* and T*");
    return MFS_EINVAL;
  }
  MFS_CUDA(cudaMemsetAsync(b, 0, sizeof(double) * (size_t)Lv.nb2.total, s));
  dim3 grid(Lv.n_tiles, kMacroCells);
  const bool bl = M->host.blending != 0;
  if (bl) {
    if (shear) k_temp_rhs<true, true><<<grid, 128, 0, s>>>(a);
    else k_temp_rhs<true, false><<<grid, 128, 0, s>>>(a);
  } else {
    if (shear) k_temp_rhs<false, true><<<grid, 128, 0, s>>>(a);
    else k_temp_rhs<false, false><<<grid, 128, 0, s>>>(a);
  }
  MFS_CUDA(cudaGetLastError());
  return MFS_OK;
}

static mfs_status temp_mmoc(mfs_problem* Pb, TempWork* W, const double* Xin, const double* T, const double* un,
                            const double* uo, double tau, double* That, double* Xout) {
  mfs_mesh* M = Pb->mesh;
  const LevelData& Lv = M->levels[M->l_max];
  MmocArgs a{};
  a.geom = M->d_geom64;
  a.topo = M->d_topo;
  a.nb2 = Lv.nb2;
  a.n = Lv.n;
  a.n_p2 = Lv.nb2.total;
  a.blending = M->host.blending;
  a.r_cmb = M->host.r_cmb;
  a.r_surf = M->host.r_surf;
  a.xyz = W->xyz;
  k_mmoc<<<tblk(a.n_p2, 128), 128, 0, M->ctx->stream>>>(a, Xin, T, un, uo, tau, That, Xout);
  MFS_CUDA(cudaGetLastError());
  return MFS_OK;
}

static double tdot(TempWork* W, int64_t n, const double* x, const double* y, cudaStream_t s) {
  Blas<double>::dot_async(n, x, y, W->red, W->red + kRedBlocks, s);
  cudaMemcpyAsync(W->hpin, W->red + kRedBlocks, sizeof(double), cudaMemcpyDeviceToHost, s);
  cudaStreamSynchronize(s);
  return W->hpin[0];
}
static double tdot32(TempWork* W, int64_t n, const float* x, const float* y, cudaStream_t s) {
  Blas<float>::dot_async(n, x, y, W->red, W->red + kRedBlocks, s);
  cudaMemcpyAsync(W->hpin, W->red + kRedBlocks, sizeof(double), cudaMemcpyDeviceToHost, s);
  cudaStreamSynchronize(s);
  return W->hpin[0];
}

// z = P^-1 v: Jacobi-CG in FP32 on the constrained symmetric part s1 M + cD D_s
static mfs_status temp_precondition(mfs_problem* Pb, TempWork* W, float s1, float cD, double rtol, int maxit,
                                    const double* v, double* z, int* iters) {
  cudaStream_t s = Pb->mesh->ctx->stream;
  const int64_t n = W->n2;
  Blas<float>::convert_from_f64(n, v, W->r32, s);
  Blas<float>::fill(n, 0.f, W->x32, s);
  const double rr0 = tdot32(W, n, W->r32, W->r32, s);
  if (!std::isfinite(rr0)) {
    set_error("NaN/Inf in the temperature preconditioner");
    return MFS_ENAN;
  }
  if (rr0 > 0.0) {
    Blas<float>::mul(n, W->r32, W->d32, W->z32, s);
    Blas<float>::axpby(n, 1.f, W->z32, 0.f, W->p32, s);
    double rz = tdot32(W, n, W->r32, W->z32, s);
    for (int it = 0; it < maxit; ++it) {
      MFS_TRY(temp_apply<float>(Pb, W, s1, 0.f, cD, 0.f, 1, 1, nullptr, W->p32, W->q32, 0));
      const double pq = tdot32(W, n, W->p32, W->q32, s);
      if (!(pq > 0.0)) break;
      const double alpha = rz / pq;
      Blas<float>::axpby(n, (float)alpha, W->p32, 1.f, W->x32, s);
      Blas<float>::axpby(n, (float)-alpha, W->q32, 1.f, W->r32, s);
      ++*iters;
      const double rr = tdot32(W, n, W->r32, W->r32, s);
      if (!std::isfinite(rr)) {
        set_error("NaN/Inf in the temperature preconditioner");
        return MFS_ENAN;
      }
      if (std::sqrt(rr) <= rtol * std::sqrt(rr0)) break;
      Blas<float>::mul(n, W->r32, W->d32, W->z32, s);
      const double rz2 = tdot32(W, n, W->r32, W->z32, s);
      Blas<float>::axpby(n, 1.f, W->z32, (float)(rz2 / rz), W->p32, s);
      rz = rz2;
    }
  }
  Blas<float>::convert_to_f64(n, W->x32, z, s);
  return MFS_OK;
}

// d solves the constrained system L d = b (b zero on the boundary) by right-preconditioned
// FGMRES(m) from d = 0, to ||b - L d|| <= max(rtol ||b||, atol)
static mfs_status temp_fgmres(mfs_problem* Pb, TempWork* W, const mfs_temp_params& tp, double s1, double tau,
                              const double* b, double* d, mfs_temp_stats& st) {
  cudaStream_t s = Pb->mesh->ctx->stream;
  const int64_t n = W->n2;
  const int m = tp.restart;
  // the solve has no advection block: the MMOC history values carry the advection
  const double cC = 0.0, cD = tau * tp.k / (tp.Pe * tp.Cp), cR = -tau * tp.Di * tp.alpha / tp.Cp;
  // Jacobi diagonal of the preconditioner's operator (FP32)
  MFS_TRY(temp_apply<float>(Pb, W, (float)s1, 0.f, (float)cD, 0.f, 1, 1, nullptr, nullptr, W->d32, 1));
  Blas<float>::recip(n, W->d32, s);
  Blas<double>::fill(n, 0.0, d, s);
  const double beta0 = std::sqrt(tdot(W, n, b, b, s));
  st.r0_norm = beta0;
  st.r_norm = beta0;
  if (!std::isfinite(beta0)) {
    set_error("NaN/Inf in the temperature right-hand side");
    return MFS_ENAN;
  }
  const double target = std::max(tp.rtol * beta0, tp.tol_T);
  if (beta0 <= target) return MFS_OK;
  std::vector<double> H((size_t)(m + 1) * m), cs(m), sn(m), g(m + 1), y(m);
  Blas<double>::axpby(n, 1.0, b, 0.0, W->V[0], s);
  double beta = beta0;
  while (st.fgmres_iters < tp.max_iters) {
    Blas<double>::axpby(n, 1.0 / beta, W->V[0], 0.0, W->V[0], s);
    std::fill(g.begin(), g.end(), 0.0);
    g[0] = beta;
    int k = 0;
    bool done = false;
    for (; k < m; ++k) {
      MFS_TRY(temp_precondition(Pb, W, (float)s1, (float)cD, tp.cg_rtol, tp.max_cg, W->V[k], W->Z[k], &st.cg_iters));
      MFS_TRY(temp_apply<double>(Pb, W, s1, cC, cD, cR, 0, 1, W->ustar, W->Z[k], W->V[k + 1], 0));
      for (int i = 0; i <= k; ++i) {
        const double hik = tdot(W, n, W->V[k + 1], W->V[i], s);
        H[(size_t)i * m + k] = hik;
        Blas<double>::axpby(n, -hik, W->V[i], 1.0, W->V[k + 1], s);
      }
      const double hn = std::sqrt(tdot(W, n, W->V[k + 1], W->V[k + 1], s));
      if (!std::isfinite(hn)) {
        set_error("NaN/Inf in the temperature FGMRES");
        return MFS_ENAN;
      }
      H[(size_t)(k + 1) * m + k] = hn;
      if (hn > 0.0) Blas<double>::axpby(n, 1.0 / hn, W->V[k + 1], 0.0, W->V[k + 1], s);
      for (int i = 0; i < k; ++i) {
        const double a = H[(size_t)i * m + k], bb = H[(size_t)(i + 1) * m + k];
        H[(size_t)i * m + k] = cs[i] * a + sn[i] * bb;
        H[(size_t)(i + 1) * m + k] = -sn[i] * a + cs[i] * bb;
      }
      const double a = H[(size_t)k * m + k], bb = H[(size_t)(k + 1) * m + k];
      const double den = std::hypot(a, bb);
      cs[k] = den > 0 ? a / den : 1.0;
      sn[k] = den > 0 ? bb / den : 0.0;
      H[(size_t)k * m + k] = den;
      H[(size_t)(k + 1) * m + k] = 0.0;
      g[k + 1] = -sn[k] * g[k];
      g[k] = cs[k] * g[k];
      st.fgmres_iters++;
      if (std::fabs(g[k + 1]) <= target || st.fgmres_iters >= tp.max_iters || hn == 0.0) {
        ++k;
        done = true;
        break;
      }
    }
    const int kk = k;
    for (int i = kk - 1; i >= 0; --i) {
      double t = g[i];
      for (int j = i + 1; j < kk; ++j) t -= H[(size_t)i * m + j] * y[j];
      y[i] = t / H[(size_t)i * m + i];
    }
    for (int i = 0; i < kk; ++i) Blas<double>::axpby(n, y[i], W->Z[i], 1.0, d, s);
    MFS_TRY(temp_apply<double>(Pb, W, s1, cC, cD, cR, 0, 1, W->ustar, d, W->w, 0));
    Blas<double>::axpbypcz(n, 1.0, b, -1.0, W->w, 0.0, W->V[0], s);
    beta = std::sqrt(tdot(W, n, W->V[0], W->V[0], s));
    st.r_norm = beta;
    if (beta <= target || done) break;
  }
  if (st.r_norm > target) {
    set_error("temperature solve not converged: residual %.3e > %.3e after %d FGMRES iterations", st.r_norm, target,
              st.fgmres_iters);
    return MFS_ENOTCONV;
  }
  return MFS_OK;
}

static mfs_status check_temp_params(const mfs_temp_params& tp) {
  if (!(tp.Pe > 0) || !(tp.Cp > 0) || !(tp.Ra > 0) || !(tp.k >= 0) || tp.restart < 1 || tp.restart > 200 ||
      tp.max_iters < 1 || tp.max_cg < 1 || !(tp.rtol >= 0) || !(tp.tol_T >= 0) || !(tp.rtol > 0 || tp.tol_T > 0)) {
    set_error("invalid temperature parameters");
    return MFS_EINVAL;
  }
  return MFS_OK;
}

}  // namespace mfs

using namespace mfs;

// ------------------------------------------------------------------------- C ABI (part)
void mfs_temp_params_default(mfs_temp_params* p) {
  if (!p) return;
  p->k = 1.0;
  p->Pe = 1.0;
  p->Cp = 1.0;
  p->Di = 0.0;
  p->alpha = 1.0;
  p->H = 0.0;
  p->Ra = 1.0;
  p->tol_T = 1e-10;
  p->rtol = 0.0;
  p->restart = 30;
  p->max_iters = 300;
  p->max_cg = 200;
  p->cg_rtol = 1e-6;
}

static mfs_status temp_check(mfs_problem* Pb) {
  if (!Pb) {
    set_error("null problem");
    return MFS_EINVAL;
  }
  if (!Pb->d_dlnrho64) {
    set_error("density table not set");
    return MFS_EINVAL;
  }
  return MFS_OK;
}

mfs_status mfs_temp_apply(mfs_problem* Pb, mfs_prec prec, double cM, double cC, double cD, double cR, int sym,
                          int constrained, const void* u, const void* x, void* y) {
  MFS_TRY(temp_check(Pb));
  if (!x || !y || ((cC != 0.0 || cR != 0.0) && !u)) {
    set_error("null vector");
    return MFS_EINVAL;
  }
  TempWork* W = nullptr;
  MFS_TRY(temp_work(Pb, 1, &W));
  if (prec == MFS_F64)
    return temp_apply<double>(Pb, W, cM, cC, cD, cR, sym, constrained, (const double*)u, (const double*)x, (double*)y, 0);
  return temp_apply<float>(Pb, W, (float)cM, (float)cC, (float)cD, (float)cR, sym, constrained, (const float*)u,
                           (const float*)x, (float*)y, 0);
}

mfs_status mfs_temp_rhs(mfs_problem* Pb, const mfs_temp_params* params, const double* T0_hat, const double* Tm_hat,
                        const double* u_star, const double* T_star, double tau_np1, double tau_n, double* b) {
  MFS_TRY(temp_check(Pb));
  mfs_temp_params tp;
  if (params) tp = *params;
  else mfs_temp_params_default(&tp);
  MFS_TRY(check_temp_params(tp));
  if (!T0_hat || !Tm_hat || !b || !(tau_np1 > 0) || !(tau_n > 0)) {
    set_error("null vector or non-positive step");
    return MFS_EINVAL;
  }
  TempWork* W = nullptr;
  MFS_TRY(temp_work(Pb, 1, &W));
  return temp_rhs(Pb, tp, T0_hat, Tm_hat, u_star, T_star, tau_np1, tau_n, b);
}

mfs_status mfs_mmoc(mfs_problem* Pb, const double* T, const double* u_new, const double* u_old, double tau,
                    const double* X_start, double* T_hat, double* X_dep) {
  MFS_TRY(temp_check(Pb));
  if (!T || !u_new || !u_old || !T_hat || !std::isfinite(tau)) {
    set_error("null vector or invalid step");
    return MFS_EINVAL;
  }
  TempWork* W = nullptr;
  MFS_TRY(temp_work(Pb, 1, &W));
  if (X_start && (X_start == X_dep)) {
    set_error("X_start and X_dep must be distinct");
    return MFS_EINVAL;
  }
  return temp_mmoc(Pb, W, X_start, T, u_new, u_old, tau, T_hat, X_dep);
}

mfs_status mfs_temperature_step(mfs_problem* Pb, const mfs_temp_params* params, const double* T_n,
                                const double* T_nm1, const double* u_n, const double* u_nm1, double tau_np1,
                                double tau_n, const double* T_bc, double* T_np1, mfs_temp_stats* stats) {
  MFS_TRY(temp_check(Pb));
  mfs_temp_params tp;
  if (params) tp = *params;
  else mfs_temp_params_default(&tp);
  MFS_TRY(check_temp_params(tp));
  if (!T_n || !T_nm1 || !u_n || !u_nm1 || !T_bc || !T_np1 || !(tau_np1 > 0) || !(tau_n > 0)) {
    set_error("null vector or non-positive step");
    return MFS_EINVAL;
  }
  mfs_temp_stats st;
  std::memset(&st, 0, sizeof(st));
  const auto t0 = std::chrono::steady_clock::now();
  TempWork* W = nullptr;
  MFS_TRY(temp_work(Pb, tp.restart, &W));
  cudaStream_t s = Pb->mesh->ctx->stream;
  const int64_t n = W->n2;
  const double r = tau_np1 / tau_n;
  // extrapolations (Eq. Extrapolation)
  Blas<double>::axpbypcz(3 * n, 1.0 + r, u_n, -r, u_nm1, 0.0, W->ustar, s);
  Blas<double>::axpbypcz(n, 1.0 + r, T_n, -r, T_nm1, 0.0, W->Tstar, s);
  // MMOC for the two history values
  // the particles leave the nodes at t^{n+1} and reach Y = W->tmp at t^n; the same particles
  // are traced on to t^{n-1}, where T^{n-1} is read (the characteristic X(t^{n+1}, t^{n-1}, x))
  MFS_TRY(temp_mmoc(Pb, W, nullptr, T_n, W->ustar, u_n, tau_np1, W->T0h, W->tmp));
  MFS_TRY(temp_mmoc(Pb, W, W->tmp, T_nm1, u_n, u_nm1, tau_n, W->Tmh, nullptr));
  // right-hand side, then the Dirichlet values moved to it
  MFS_TRY(temp_rhs(Pb, tp, W->T0h, W->Tmh, W->ustar, W->Tstar, tau_np1, tau_n, W->b));
  const double s1 = (2 * tau_np1 + tau_n) / (tau_np1 + tau_n);
  const double cC = 0.0, cD = tau_np1 * tp.k / (tp.Pe * tp.Cp), cR = -tau_np1 * tp.Di * tp.alpha / tp.Cp;
  Blas<double>::fill(n, 0.0, W->xb, s);
  if (W->nb) k_set_at<<<tblk(W->nb), 256, 0, s>>>(W->nb, W->bids, T_bc, W->xb);
  MFS_TRY(temp_apply<double>(Pb, W, s1, cC, cD, cR, 0, 0, W->ustar, W->xb, W->w, 0));
  Blas<double>::axpby(n, -1.0, W->w, 1.0, W->b, s);
  if (W->nb) k_set_at<<<tblk(W->nb), 256, 0, s>>>(W->nb, W->bids, nullptr, W->b);
  MFS_CUDA(cudaGetLastError());
  mfs_status rc = temp_fgmres(Pb, W, tp, s1, tau_np1, W->b, W->sol, st);
  if (rc == MFS_OK || rc == MFS_ENOTCONV) {
    Blas<double>::axpbypcz(n, 1.0, W->sol, 1.0, W->xb, 0.0, T_np1, s);
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) rc = cuda_fail(e, "mfs_temperature_step");
  }
  st.time_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  if (stats) *stats = st;
  return rc;
}

mfs_status mfs_temp_rule(double* lam, double* w) {
  if (!lam || !w) {
    set_error("null argument");
    return MFS_EINVAL;
  }
  double l[kTQ][4], ww[kTQ];
  if (!conical_rule27(l, ww)) {
    set_error("the conical quadrature rule failed its exactness check");
    return MFS_EINVAL;
  }
  std::memcpy(lam, l, sizeof(l));
  std::memcpy(w, ww, sizeof(ww));
  return MFS_OK;
}

mfs_status mfs_mmoc_host(const mfs_mesh* M, int n, const double* X_start, const double* T, const double* u_new,
                         const double* u_old, double tau, double* T_hat, double* X_out) {
  if (!M || n < 0 || (n > 0 && (!X_start || !T || !u_new || !u_old || !T_hat)) || !std::isfinite(tau)) {
    set_error("null mesh or field, negative particle count or non-finite tau");
    return MFS_EINVAL;
  }
  const int nl = 1 << M->l_max;
  MmocArgs a{};
  a.geom = M->host.geom;
  a.topo = M->host.topo;
  a.nb2 = make_numbering(2 * nl);
  a.n = nl;
  a.n_p2 = a.nb2.total;
  a.blending = M->host.blending;
  a.r_cmb = M->host.r_cmb;
  a.r_surf = M->host.r_surf;
  a.xyz = nullptr;
  for (int i = 0; i < n; ++i) {
    const double x[3] = {X_start[i], X_start[(size_t)n + i], X_start[2 * (size_t)n + i]};
    double X[3];
    mmoc_particle(a, x, T, u_new, u_old, tau, &T_hat[i], X);
    if (X_out)
      for (int c = 0; c < 3; ++c) X_out[(size_t)c * n + i] = X[c];
  }
  return MFS_OK;
}

mfs_status mfs_apply_vmass(mfs_problem* Pb, mfs_prec prec, double a, const void* x, void* y) {
  if (!Pb || !x || !y) {
    set_error("null argument");
    return MFS_EINVAL;
  }
  if (!Pb->has_eta) {
    set_error("viscosity not set");
    return MFS_EINVAL;
  }
  if (!(a > 0.0) || !std::isfinite(a)) {
    set_error("the weighted-BFBT surface scaling must be positive and finite");
    return MFS_EINVAL;
  }
  if (x == y) {
    set_error("mfs_apply_vmass: x and y must be distinct");
    return MFS_EINVAL;
  }
  if (prec == MFS_F64) return wmass_apply<double>(Pb, a, (const double*)x, (double*)y, 0);
  if (prec == MFS_F32) return wmass_apply<float>(Pb, a, (const float*)x, (float*)y, 0);
  set_error("unknown precision");
  return MFS_EINVAL;
}
