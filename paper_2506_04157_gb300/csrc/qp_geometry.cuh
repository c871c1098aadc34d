// Per-quadrature-point geometry of the blended micro-tets shared by the setup and
// auxiliary sweeps (diag(A), mass weights, gradient, buoyancy, weighted-BFBT operators):
// the lattice-frame gradients of the P2 basis and the rows K of the pulled-back inverse
// Jacobian with the blending scalings (arxiv 2506.04157, Sec. 4.1).
#pragma once

#include "apply.cuh"

namespace mfs {

// lattice gradient (permuted frame) of the P2 basis function a at barycentrics lam
__device__ __forceinline__ void p2_lat_grad(int a, const double lam[4], double g[3]) {
  // grad lambda_0 = (-1,0,0), grad lambda_1 = (1,-1,0), grad lambda_2 = (0,1,-1), grad lambda_3 = (0,0,1)
  const double GL[4][3] = {{-1, 0, 0}, {1, -1, 0}, {0, 1, -1}, {0, 0, 1}};
  if (a < 4) {
    for (int j = 0; j < 3; ++j) g[j] = (4 * lam[a] - 1) * GL[a][j];
  } else {
    const int e = a - 4;
    const int i0 = e < 3 ? 0 : (e < 5 ? 1 : 2);
    const int i1 = e < 3 ? e + 1 : (e < 5 ? e - 1 : 3);
    for (int j = 0; j < 3; ++j) g[j] = 4 * (lam[i1] * GL[i0][j] + lam[i0] * GL[i1][j]);
  }
}

// geometry at the point with lattice coordinates xi (units of micro-cubes, macro Kuhn frame)
// of a tet of Freudenthal type (p0, p1, p2): K rows (permuted lattice frame: the physical
// gradient of a function with lattice-frame gradient g is (g K) / hr), the blending scaling
// hr (w|det J| = (w absdet / n^3) hr^3), 1/|x~| and the straight position x~
template <typename T, bool BLEND>
__device__ __forceinline__ void lattice_geometry(const MacroGeom<T>& G, int n, int p0, int p1, int p2, T xi0, T xi1,
                                                 T xi2, T K[3][3], T& hr, T& rinv, T x[3]) {
  for (int r = 0; r < 3; ++r)
    x[r] = G.v0[r] + (G.Jm[3 * r] * xi0 + G.Jm[3 * r + 1] * xi1 + G.Jm[3 * r + 2] * xi2) / T(n);
  const T r2 = x[0] * x[0] + x[1] * x[1] + x[2] * x[2];
  rinv = T(1) / sqrt(r2);
  const int pr[3] = {p0, p1, p2};
  T Mp[3][3];
  for (int j = 0; j < 3; ++j)
    for (int d = 0; d < 3; ++d) Mp[j][d] = T(n) * G.Jinv[3 * pr[j] + d];
  hr = T(1);
  if (BLEND) {
    const T h = x[0] * G.nh[0] + x[1] * G.nh[1] + x[2] * G.nh[2];
    hr = h * rinv / G.delta;
    T v[3];
    for (int d = 0; d < 3; ++d) v[d] = G.nh[d] / h - x[d] * rinv * rinv;
    for (int j = 0; j < 3; ++j) {
      const T tj = Mp[j][0] * x[0] + Mp[j][1] * x[1] + Mp[j][2] * x[2];
      for (int d = 0; d < 3; ++d) K[j][d] = Mp[j][d] - tj * v[d];
    }
  } else {
    for (int j = 0; j < 3; ++j)
      for (int d = 0; d < 3; ++d) K[j][d] = Mp[j][d];
  }
}

// geometry of qp q of the 4-point rule (see lattice_geometry)
template <typename T, bool BLEND>
__device__ __forceinline__ void qp_geometry(const MacroGeom<T>& G, int n, int p0, int p1, int p2, int q, T qx, T qy,
                                            T qz, T K[3][3], T& hr, T& rinv, T x[3]) {
  const T QA = T(MFS_QA), QB = T(MFS_QB);
  const int S1 = 1 << p0, S2 = S1 | (1 << p1);
  const int Sq = q == 0 ? 0 : (q == 1 ? S1 : (q == 2 ? S2 : 7));
  const T xi0 = qx + QB * T(3 * (p0 == 0) + 2 * (p1 == 0) + (p2 == 0)) + (QA - QB) * T(Sq & 1);
  const T xi1 = qy + QB * T(3 * (p0 == 1) + 2 * (p1 == 1) + (p2 == 1)) + (QA - QB) * T((Sq >> 1) & 1);
  const T xi2 = qz + QB * T(3 * (p0 == 2) + 2 * (p1 == 2) + (p2 == 2)) + (QA - QB) * T(Sq >> 2);
  lattice_geometry<T, BLEND>(G, n, p0, p1, p2, xi0, xi1, xi2, K, hr, rinv, x);
}

// rho(r) = exp(int_{r1}^{r} d ln rho/dr) for the piecewise-linear table on a uniform grid over
// [r0, r1] (rho(r1) = 1), integrated exactly
__device__ __forceinline__ double rho_of(const double* tab, int nt, double r, double r0, double r1) {
  if (nt <= 1) return exp(tab[0] * (r - r1));
  const double h = (r1 - r0) / (nt - 1);
  double s = (r - r0) / h;
  s = s < 0 ? 0 : (s > nt - 1 ? nt - 1 : s);
  int i = (int)s;
  i = i > nt - 2 ? nt - 2 : i;
  const double f = s - i;
  // integral of g from r to r1: the part of cell i above r, then the full cells above
  const double gr = (1 - f) * tab[i] + f * tab[i + 1];
  double integ = 0.5 * (gr + tab[i + 1]) * (1 - f) * h;
  for (int k = i + 1; k < nt - 1; ++k) integ += 0.5 * (tab[k] + tab[k + 1]) * h;
  return exp(-integ);
}

}  // namespace mfs
