// Matrix-free sweep over the micro-tets of one refinement level: applies any
// combination of A(eta), B^T / (B+C)^T and B / (B+C) of the P2-P1 Taylor-Hood Stokes
// system (arxiv 2506.04157, Sec. 5.1, Eq. SaddlePointStructure) in one pass.
//
// Work decomposition: one CTA per tile of TT^3 lattice cubes of one macro-tet
// (Freudenthal cubes (a,b,c) with n > a >= b >= c >= 0).  The CTA stages the tile's
// (2TT+1)^3 block of P2 nodes and (TT+1)^3 block of P1 vertices in shared memory
// (coalesced along the macro lattice rows), one thread per micro-tet computes the
// element contribution at the 4 quadrature points with the blending Jacobian evaluated
// at each of them, accumulates into shared memory, and the block is added to the global
// result with one atomic add per node and component.
//
// Per-quadrature-point algebra (all derived from Sec. 4.1's pulled-back integrals):
//  * straight position x~ = v0 + Jm xi / n, xi the lattice coordinate of the point;
//  * blending map B(x~) = (h/delta) x~/|x~|, h = x~.nh.  Its Jacobian is
//    J_B = s (I - e e^T) + e nh^T / delta (s = h/(delta rho), rho = |x~|, e = x~/rho), with
//      J_B^{-1} = (delta rho / h) (I - x~ (nh/h - x~/rho^2)^T),  det J_B = h^3/(delta rho)^3;
//  * lattice gradient of u from the barycentric form of the P2 gradient
//      grad u = sum_a c_a (x) grad lambda_a,  c_a = (4 lambda_a - 1) u_a + 4 sum_b lambda_b u_ab;
//  * physical gradient grad_x u = (grad_lat u) n Jm^{-1} J_B^{-1};
//  * tau = 2 eta eps(u) - p I, test side R = w |det J| tau K^T, distributed back to the
//    10 nodes through the same barycentric form.
#pragma once

#include "mfs_internal.h"

namespace mfs {


template <typename T>
struct ApplyParams {
  const T* u;        // [3][n_p2] (OP_A, OP_B)
  const T* p;        // [n_p1]    (OP_BT)
  T* yu;             // [3][n_p2] (OP_A, OP_BT), accumulated atomically: zeroed by the launcher
  T* yp;             // [n_p1]    (OP_B), accumulated atomically: zeroed by the launcher
  const T* eta;      // [n_p1] nodal viscosity of this level
  const T* dlnrho;   // radial table of d ln rho / dr (n_dlnrho entries)
  const T* psum;     // device scalar: sum of p; p - psum/n_p1 is used (P_p), or nullptr
  const MacroGeom<T>* geom;
  const MacroTopo* topo;
  const Tile* tiles;
  const uint16_t* tets;   // packed local tets (perm<<12 | k<<8 | j<<4 | i)
  const int2* classes;    // (offset, count) into tets per tile class
  Numbering nb2, nb1;
  int n;                  // cubes per macro edge
  int n_dlnrho;
  T r_cmb, r_surf;
  int blending;
  int constrained;
  int withc_b;            // OP_B computes (B + C) u
  int bc_surface, bc_cmb;
};

// symmetric 4-point degree-2 rule: barycentrics (QA,QB,QB,QB) and permutations, w = 1/24
#define MFS_QA 0.58541019662496845446
#define MFS_QB 0.13819660112501051518

__device__ __forceinline__ constexpr int edge_of(int a, int b) {
  return (a < b ? a : b) == 0 ? (a > b ? a : b) - 1
                              : ((a < b ? a : b) == 1 ? (a > b ? a : b) + 1 : 5);
}
// node (0..9) carrying u_{a,q}: the vertex a itself if a == q, else the edge (a,q)
__device__ __forceinline__ constexpr int wnode(int a, int q) { return a == q ? a : 4 + edge_of(a, q); }

template <typename T>
__device__ __forceinline__ T rsqrt_t(T x);
template <>
__device__ __forceinline__ float rsqrt_t<float>(float x) { return rsqrtf(x); }
template <>
__device__ __forceinline__ double rsqrt_t<double>(double x) { return rsqrt(x); }

template <typename T>
__device__ __forceinline__ T interp_table(const T* tab, int nt, T r, T r0, T r1) {
  if (nt <= 1) return tab[0];
  T s = (r - r0) / (r1 - r0) * T(nt - 1);
  s = s < T(0) ? T(0) : (s > T(nt - 1) ? T(nt - 1) : s);
  int i = (int)s;
  i = i > nt - 2 ? nt - 2 : i;
  const T f = s - T(i);
  return (T(1) - f) * tab[i] + f * tab[i + 1];
}

template <typename T, int OP>
__global__ void __launch_bounds__(256) stokes_tile_kernel(const ApplyParams<T> P) {
  constexpr bool HAS_U = (OP & (OP_A | OP_B)) != 0;
  constexpr bool HAS_P = (OP & OP_BT) != 0;
  constexpr bool OUT_U = (OP & (OP_A | OP_BT)) != 0;
  constexpr bool OUT_P = (OP & OP_B) != 0;
  constexpr bool HAS_CT = (OP & OP_CT) != 0;

  __shared__ T us[HAS_U ? 3 * NSLOT2 : 1];
  __shared__ T ys[OUT_U ? 3 * NSLOT2 : 1];
  __shared__ int gid2[NSLOT2];
  __shared__ int8_t cls2[NSLOT2];
  __shared__ T eta_s[NSLOT1];
  __shared__ T p_s[HAS_P ? NSLOT1 : 1];
  __shared__ T yp_s[OUT_P ? NSLOT1 : 1];
  __shared__ int gid1[NSLOT1];
  __shared__ T cM[9], cJn[9], cv0[3], cnh[3];

  const int m = blockIdx.y;
  const Tile tile = P.tiles[blockIdx.x];
  const MacroTopo topo = P.topo[m];
  const MacroGeom<T>& G = P.geom[m];
  const int a0 = tile.ta * TT, b0 = tile.tb * TT, c0 = tile.tc * TT;
  const int N = P.nb2.N, n = P.n;
  const int tid = threadIdx.x;

  if (tid < 9) {
    cM[tid] = T(n) * G.Jinv[tid];
    cJn[tid] = G.Jm[tid] / T(n);
  }
  if (tid < 3) {
    cv0[tid] = G.v0[tid];
    cnh[tid] = G.nh[tid];
  }

  // ---- stage the P2 node block (u, with the input-side projections) ----
  for (int s = tid; s < NSLOT2; s += blockDim.x) {
    const int dA = s % NB2, dB = (s / NB2) % NB2, dC = s / (NB2 * NB2);
    const int A = 2 * a0 + dA, B = 2 * b0 + dB, C = 2 * c0 + dC;
    int id = -1, cl = NODE_FREE;
    T v0 = 0, v1 = 0, v2 = 0;
    if (A <= N && A >= B && B >= C) {
      const int i0 = N - A, i1 = A - B, i2 = B - C, i3 = C;
      id = lattice_id(topo, P.nb2, m, i0, i1, i2, i3);
      const int mask = (i0 > 0) | ((i1 > 0) << 1) | ((i2 > 0) << 2) | ((i3 > 0) << 3);
      if (P.constrained) cl = node_class(topo, mask, P.bc_surface, P.bc_cmb);
      if (HAS_U) {
        const int nn = P.nb2.total;
        v0 = P.u[id];
        v1 = P.u[nn + id];
        v2 = P.u[2 * nn + id];
        if (cl == NODE_DIRICHLET) {
          v0 = v1 = v2 = T(0);
        } else if (cl == NODE_FREESLIP) {
          const T xa = T(A) / T(N), xb = T(B) / T(N), xc = T(C) / T(N);
          T x[3];
#pragma unroll
          for (int r = 0; r < 3; ++r)
            x[r] = G.v0[r] + G.Jm[3 * r] * xa + G.Jm[3 * r + 1] * xb + G.Jm[3 * r + 2] * xc;
          const T ri = rsqrt_t<T>(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
          const T nx = x[0] * ri, ny = x[1] * ri, nz = x[2] * ri;
          const T un = v0 * nx + v1 * ny + v2 * nz;
          v0 -= un * nx;
          v1 -= un * ny;
          v2 -= un * nz;
        }
      }
    }
    gid2[s] = id;
    cls2[s] = (int8_t)cl;
    if (HAS_U) {
      us[s] = v0;
      us[NSLOT2 + s] = v1;
      us[2 * NSLOT2 + s] = v2;
    }
    if (OUT_U) {
      ys[s] = T(0);
      ys[NSLOT2 + s] = T(0);
      ys[2 * NSLOT2 + s] = T(0);
    }
  }
  // ---- stage the P1 vertex block (eta, p) ----
  const T pm = (HAS_P && P.psum) ? *P.psum / T(P.nb1.total) : T(0);
  for (int s = tid; s < NSLOT1; s += blockDim.x) {
    const int da = s % NB1, db = (s / NB1) % NB1, dc = s / (NB1 * NB1);
    const int a = a0 + da, b = b0 + db, c = c0 + dc;
    int id = -1;
    T e = T(1), pv = T(0);
    if (a <= n && a >= b && b >= c) {
      id = lattice_id(topo, P.nb1, m, n - a, a - b, b - c, c);
      e = P.eta[id];
      if (HAS_P) pv = P.p[id] - pm;
    }
    gid1[s] = id;
    eta_s[s] = e;
    if (HAS_P) p_s[s] = pv;
    if (OUT_P) yp_s[s] = T(0);
  }
  __syncthreads();

  // ---- element sweep: one thread per micro-tet ----
  const T QA = T(MFS_QA), QB = T(MFS_QB);
  const T dq = T(4) * (QA - QB);           // 4(alpha - beta)
  const T bq1 = T(4) * QB - T(1);          // 4 beta - 1
  const T b4 = T(4) * QB;                  // 4 beta
  const T C0 = G.absdet / (T(24) * T(n) * T(n) * T(n));
  const T dinv = T(1) / G.delta;
  const T delta = G.delta;
  const int2 cinfo = P.classes[tile.cls];

  for (int t = tid; t < cinfo.y; t += blockDim.x) {
    const int code = P.tets[cinfo.x + t];
    const int ci = code & 15, cj = (code >> 4) & 15, ck = (code >> 8) & 15, pmu = code >> 12;
    const int p0 = (0x221100 >> (4 * pmu)) & 3;
    const int p1 = (0x102021 >> (4 * pmu)) & 3;
    const int p2 = (0x010212 >> (4 * pmu)) & 3;
    // shared-memory slots of the 10 P2 nodes and 4 P1 vertices
    const int w2p0 = p0 == 0 ? 1 : (p0 == 1 ? NB2 : NB2 * NB2);
    const int w2p1 = p1 == 0 ? 1 : (p1 == 1 ? NB2 : NB2 * NB2);
    const int w1p0 = p0 == 0 ? 1 : (p0 == 1 ? NB1 : NB1 * NB1);
    const int w1p1 = p1 == 0 ? 1 : (p1 == 1 ? NB1 : NB1 * NB1);
    int o2[4], o1[4];
    o2[0] = 0;
    o2[1] = w2p0;
    o2[2] = w2p0 + w2p1;
    o2[3] = 1 + NB2 + NB2 * NB2;
    o1[0] = 0;
    o1[1] = w1p0;
    o1[2] = w1p0 + w1p1;
    o1[3] = 1 + NB1 + NB1 * NB1;
    const int base2 = (2 * ck * NB2 + 2 * cj) * NB2 + 2 * ci;
    const int base1 = (ck * NB1 + cj) * NB1 + ci;
    int slot[10];
#pragma unroll
    for (int a = 0; a < 4; ++a) slot[a] = base2 + 2 * o2[a];
    slot[4] = base2 + o2[0] + o2[1];
    slot[5] = base2 + o2[0] + o2[2];
    slot[6] = base2 + o2[0] + o2[3];
    slot[7] = base2 + o2[1] + o2[2];
    slot[8] = base2 + o2[1] + o2[3];
    slot[9] = base2 + o2[2] + o2[3];

    T eta_v[4], p_v[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      eta_v[a] = eta_s[base1 + o1[a]];
      if (HAS_P) p_v[a] = p_s[base1 + o1[a]];
    }
    const T eta_sum = eta_v[0] + eta_v[1] + eta_v[2] + eta_v[3];
    T p_sum = T(0);
    if (HAS_P) p_sum = p_v[0] + p_v[1] + p_v[2] + p_v[3];

    // nodal values and the qp-independent parts of the barycentric gradient
    T uu[10][3];
    T baseg[4][3];
    if (HAS_U) {
#pragma unroll
      for (int a = 0; a < 10; ++a)
#pragma unroll
        for (int c = 0; c < 3; ++c) uu[a][c] = us[c * NSLOT2 + slot[a]];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          T sa = T(0);
#pragma unroll
          for (int b = 0; b < 4; ++b)
            if (b != a) sa += uu[4 + edge_of(a, b)][c];
          baseg[a][c] = bq1 * uu[a][c] + b4 * sa;
        }
    }

    // lattice coordinates: cube corner and Freudenthal vertex offsets
    const T qx = T(a0 + ci), qy = T(b0 + cj), qz = T(c0 + ck);
    // centroid offset beta*(3 e_p0 + 2 e_p1 + e_p2)
    T cofs[3];
#pragma unroll
    for (int d = 0; d < 3; ++d)
      cofs[d] = QB * T(3 * (p0 == d) + 2 * (p1 == d) + (p2 == d));
    // Mpi rows: rows p0,p1,p2 of M = n Jm^{-1}
    T Mp[3][3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      Mp[0][d] = cM[3 * p0 + d];
      Mp[1][d] = cM[3 * p1 + d];
      Mp[2][d] = cM[3 * p2 + d];
    }

    // test-side accumulators
    T Tacc[4][3], Vd[4][3], Eacc[6][3];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int c = 0; c < 3; ++c) Tacc[a][c] = Vd[a][c] = T(0);
#pragma unroll
    for (int e = 0; e < 6; ++e)
#pragma unroll
      for (int c = 0; c < 3; ++c) Eacc[e][c] = T(0);
    T bq[4];
    T Zsum[3] = {T(0), T(0), T(0)};
    T Zv[4][3];
#pragma unroll
    for (int a = 0; a < 4; ++a) Zv[a][0] = Zv[a][1] = Zv[a][2] = T(0);

#pragma unroll
    for (int q = 0; q < 4; ++q) {
      // lattice position of the quadrature point: q + cofs + (alpha-beta) S_q
      const T sq0 = (q >= 1 && p0 == 0) || (q >= 2 && p1 == 0) || q == 3 ? T(1) : T(0);
      const T sq1 = (q >= 1 && p0 == 1) || (q >= 2 && p1 == 1) || q == 3 ? T(1) : T(0);
      const T sq2 = (q >= 1 && p0 == 2) || (q >= 2 && p1 == 2) || q == 3 ? T(1) : T(0);
      const T xi0 = qx + cofs[0] + (QA - QB) * sq0;
      const T xi1 = qy + cofs[1] + (QA - QB) * sq1;
      const T xi2 = qz + cofs[2] + (QA - QB) * sq2;
      T x[3];
#pragma unroll
      for (int r = 0; r < 3; ++r) x[r] = cv0[r] + cJn[3 * r] * xi0 + cJn[3 * r + 1] * xi1 + cJn[3 * r + 2] * xi2;
      const T r2 = x[0] * x[0] + x[1] * x[1] + x[2] * x[2];
      const T rinv = rsqrt_t<T>(r2);
      T K[3][3];
      T hr = T(1);
      if (P.blending) {
        const T h = x[0] * cnh[0] + x[1] * cnh[1] + x[2] * cnh[2];
        const T hinv = T(1) / h;
        hr = h * rinv * dinv;                  // 1 / s  with s = delta rho / h
        const T ri2 = rinv * rinv;
        T v[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) v[d] = cnh[d] * hinv - x[d] * ri2;
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          const T tj = Mp[j][0] * x[0] + Mp[j][1] * x[1] + Mp[j][2] * x[2];
#pragma unroll
          for (int d = 0; d < 3; ++d) K[j][d] = Mp[j][d] - tj * v[d];
        }
      } else {
#pragma unroll
        for (int j = 0; j < 3; ++j)
#pragma unroll
          for (int d = 0; d < 3; ++d) K[j][d] = Mp[j][d];
      }
      const T coefB = C0 * hr * hr;   // w |det J| s
      const T Wq = coefB * hr;        // w |det J|
      const T etaq = QB * eta_sum + (QA - QB) * eta_v[q];

      // lattice gradient differences D_j = c_{j+1} - c_j at this qp, and grad' = D K
      T trace = T(0);
      T Gp[3][3];
      if (HAS_U) {
        T D[3][3];
#pragma unroll
        for (int j = 0; j < 3; ++j)
#pragma unroll
          for (int c = 0; c < 3; ++c)
            D[j][c] = (baseg[j + 1][c] - baseg[j][c]) + dq * (uu[wnode(j + 1, q)][c] - uu[wnode(j, q)][c]);
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
          for (int d = 0; d < 3; ++d) Gp[c][d] = D[0][c] * K[0][d] + D[1][c] * K[1][d] + D[2][c] * K[2][d];
        trace = Gp[0][0] + Gp[1][1] + Gp[2][2];
      }

      // B: div u + grad ln rho . u
      if (OUT_P) {
        T b = coefB * trace;
        if (P.withc_b) {
          const T rad = P.blending ? (x[0] * cnh[0] + x[1] * cnh[1] + x[2] * cnh[2]) * dinv : r2 * rinv;
          const T g = interp_table<T>(P.dlnrho, P.n_dlnrho, rad, P.r_cmb, P.r_surf);
          // u at the qp: P2 values beta(2beta-1), alpha(2alpha-1) at vertices, 4beta^2, 4 alpha beta at edges
          const T fvb = QB * (T(2) * QB - T(1)), fva = QA * (T(2) * QA - T(1));
          const T feo = T(4) * QB * QB, fei = T(4) * QA * QB;
          T eu = T(0);
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            T sv = uu[0][c] + uu[1][c] + uu[2][c] + uu[3][c];
            T se = uu[4][c] + uu[5][c] + uu[6][c] + uu[7][c] + uu[8][c] + uu[9][c];
            T sqe = T(0);
#pragma unroll
            for (int b2 = 0; b2 < 4; ++b2)
              if (b2 != q) sqe += uu[4 + edge_of(q, b2)][c];
            const T uq = fvb * sv + (fva - fvb) * uu[q][c] + feo * se + (fei - feo) * sqe;
            eu += uq * x[c];
          }
          b += Wq * g * eu * rinv;
        }
        bq[q] = b;
      }

      if (OUT_U) {
        // stress (scaled): sigma = coefA eps(G') - coefB p_q I
        T S[3][3];
        if (OP & OP_A) {
          const T coefA = T(2) * etaq * C0 * hr;
          const T t3 = trace * (T(1) / T(3));
          S[0][0] = coefA * (Gp[0][0] - t3);
          S[1][1] = coefA * (Gp[1][1] - t3);
          S[2][2] = coefA * (Gp[2][2] - t3);
          S[0][1] = S[1][0] = T(0.5) * coefA * (Gp[0][1] + Gp[1][0]);
          S[0][2] = S[2][0] = T(0.5) * coefA * (Gp[0][2] + Gp[2][0]);
          S[1][2] = S[2][1] = T(0.5) * coefA * (Gp[1][2] + Gp[2][1]);
        } else {
#pragma unroll
          for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int d = 0; d < 3; ++d) S[c][d] = T(0);
        }
        if (HAS_P) {
          const T pq = QB * p_sum + (QA - QB) * p_v[q];
          const T sp = coefB * pq;
          S[0][0] -= sp;
          S[1][1] -= sp;
          S[2][2] -= sp;
        }
        // R = S K^T (columns in permuted lattice order), s_a = R grad_lat lambda_a
        T Rm[3][3];
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
          for (int j = 0; j < 3; ++j) Rm[c][j] = S[c][0] * K[j][0] + S[c][1] * K[j][1] + S[c][2] * K[j][2];
        T sv[4][3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          sv[0][c] = -Rm[c][0];
          sv[1][c] = Rm[c][0] - Rm[c][1];
          sv[2][c] = Rm[c][1] - Rm[c][2];
          sv[3][c] = Rm[c][2];
        }
        // (B+C)^T: the C part -W p_q g (x/|x|) . phi_i, distributed through the P2 values
        if (HAS_CT) {
          const T rad = P.blending ? (x[0] * cnh[0] + x[1] * cnh[1] + x[2] * cnh[2]) * dinv : r2 * rinv;
          const T g = interp_table<T>(P.dlnrho, P.n_dlnrho, rad, P.r_cmb, P.r_surf);
          const T pq = QB * p_sum + (QA - QB) * p_v[q];
          const T zc = -Wq * pq * g * rinv;
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            Zsum[c] += zc * x[c];
            Zv[q][c] = zc * x[c];
          }
        }
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            Tacc[a][c] += sv[a][c];
            if (a == q) Vd[a][c] = sv[a][c];
            else Eacc[edge_of(a, q)][c] += sv[a][c];
          }
      }
    }  // qp loop

    if (OUT_U) {
      // P2 basis values at the qps: vertex beta(2beta-1) (alpha(2alpha-1) at its own qp),
      // edge 4 beta^2 (4 alpha beta at the qps of its two vertices)
      const T fvb = QB * (T(2) * QB - T(1)), fva = QA * (T(2) * QA - T(1));
      const T feo = T(4) * QB * QB, fei = T(4) * QA * QB;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        T* y = ys + c * NSLOT2;
#pragma unroll
        for (int a = 0; a < 4; ++a) {
          T val = bq1 * Tacc[a][c] + dq * Vd[a][c];
          if (HAS_CT) val += fvb * Zsum[c] + (fva - fvb) * Zv[a][c];
          atomicAdd(&y[slot[a]], val);
        }
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b = a + 1; b < 4; ++b) {
            const int e = edge_of(a, b);
            T val = b4 * (Tacc[a][c] + Tacc[b][c]) + dq * Eacc[e][c];
            if (HAS_CT) val += feo * Zsum[c] + (fei - feo) * (Zv[a][c] + Zv[b][c]);
            atomicAdd(&y[slot[4 + e]], val);
          }
      }
    }
    if (OUT_P) {
      const T sb = bq[0] + bq[1] + bq[2] + bq[3];
#pragma unroll
      for (int a = 0; a < 4; ++a) atomicAdd(&yp_s[base1 + o1[a]], -(QB * sb + (QA - QB) * bq[a]));
    }
  }
  __syncthreads();

  // ---- add the block to the global result (output-side projections) ----
  if (OUT_U) {
    const int nn = P.nb2.total;
    for (int s = tid; s < NSLOT2; s += blockDim.x) {
      const int id = gid2[s];
      if (id < 0) continue;
      const int cl = cls2[s];
      if (cl == NODE_DIRICHLET) {
        // identity rows of the constrained operator (A part); B^T rows stay zero
        if (OP & OP_A) {
          P.yu[id] = P.u[id];
          P.yu[nn + id] = P.u[nn + id];
          P.yu[2 * nn + id] = P.u[2 * nn + id];
        }
        continue;
      }
      T v0 = ys[s], v1 = ys[NSLOT2 + s], v2 = ys[2 * NSLOT2 + s];
      if (cl == NODE_FREESLIP) {
        const int dA = s % NB2, dB = (s / NB2) % NB2, dC = s / (NB2 * NB2);
        const T xa = T(2 * a0 + dA) / T(N), xb = T(2 * b0 + dB) / T(N), xc = T(2 * c0 + dC) / T(N);
        T x[3];
#pragma unroll
        for (int r = 0; r < 3; ++r)
          x[r] = G.v0[r] + G.Jm[3 * r] * xa + G.Jm[3 * r + 1] * xb + G.Jm[3 * r + 2] * xc;
        const T ri = rsqrt_t<T>(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
        const T nx = x[0] * ri, ny = x[1] * ri, nz = x[2] * ri;
        const T un = v0 * nx + v1 * ny + v2 * nz;
        v0 -= un * nx;
        v1 -= un * ny;
        v2 -= un * nz;
      }
      atomicAdd(&P.yu[id], v0);
      atomicAdd(&P.yu[nn + id], v1);
      atomicAdd(&P.yu[2 * nn + id], v2);
    }
  }
  if (OUT_P) {
    for (int s = tid; s < NSLOT1; s += blockDim.x) {
      const int id = gid1[s];
      if (id >= 0) atomicAdd(&P.yp[id], yp_s[s]);
    }
  }
}

}  // namespace mfs
