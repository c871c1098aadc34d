// Matrix-free sweep over the micro-tets of one refinement level: applies any
// combination of A(eta), B^T / (B+C)^T and B / (B+C) of the P2-P1 Taylor-Hood Stokes
// system (arxiv 2506.04157, Sec. 5.1, Eq. SaddlePointStructure) in one pass.
//
// Work decomposition: one CTA per tile of TT^3 lattice cubes of one macro-tet
// (Freudenthal cubes (a,b,c) with n > a >= b >= c >= 0).  The CTA stages the tile's
// (2TT+1)^3 block of P2 nodes and (TT+1)^3 block of P1 vertices in shared memory
// (global ids from a per-tile table built once per level), one thread per micro-tet
// computes the element contribution at the 4 quadrature points with the blending
// Jacobian evaluated at each of them, accumulates into shared memory, and the block is
// added to the global result with one atomic add per node and component.
//
// Shared-memory layout: nodes are split into the 8 parity classes of their local fine
// coordinates (A&1, B&1, C&1), each a 5x5x5 sub-block.  The threads of a warp process
// the same Freudenthal type in different cubes, so "node k of my tet" lies in one parity
// class at sub-index i + 5j + 25k + const: at most 2-way bank conflicts.
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

#ifndef MFS_EDGE_ACC_REGS
#define MFS_EDGE_ACC_REGS 1   // 1: edge contributions accumulated in registers over the qps
#endif
#ifndef MFS_SLOT_TABLE
#define MFS_SLOT_TABLE 0      // 1: slot offsets from a constant table, 0: computed
#endif
#ifndef MFS_SWEEP_THREADS
#define MFS_SWEEP_THREADS 192   // threads per sweep CTA (micro-tets per round)
#endif
#ifndef MFS_SWEEP_MINBLOCKS
#define MFS_SWEEP_MINBLOCKS (768 / MFS_SWEEP_THREADS)   // resident CTAs per SM the registers target
#endif
constexpr int kSweepThreads = MFS_SWEEP_THREADS;
constexpr int kSub = 125;   // 5x5x5 parity sub-block

template <typename T>
struct ApplyParams {
  const T* u;        // [3][n_p2] (OP_A, OP_B)
  const T* p;        // [n_p1]    (OP_BT)
  T* yu;             // [3][n_p2] (OP_A, OP_BT), accumulated atomically: zeroed by the launcher
  T* yp;             // [n_p1]    (OP_B), accumulated atomically: zeroed by the launcher
  const T* eta;      // [n_p1] nodal viscosity of this level
  const T* dlnrho;   // radial table of d ln rho / dr (n_dlnrho entries)
  const T* dlnrho_int;   // OP_RHO: its integral from r_cmb to each table node (n_dlnrho entries)
  const T* psum;     // device scalar: sum of p; p - psum/n_p1 is used (P_p), or nullptr
  const MacroGeom<T>* geom;
  const Tile* tiles;
  const uint16_t* tets;   // packed local tets (perm<<12 | k<<8 | j<<4 | i)
  const int2* classes;    // (offset, count) into tets per tile class
  const int* ids2;        // [60*tiles][NSLOT2]: global P2 id | geometric class << 29, or -1
  const int* ids1;        // [60*tiles][NSLOT1]: global P1 id, or -1
  int n_p2, n_p1;
  int n;                  // cubes per macro edge
  int n_dlnrho;
  T r_cmb, inv_dr;        // table grid: s = (r - r_cmb) * inv_dr * (n_dlnrho - 1)
  // OP_ETAQ: eta(x, T) = 10^lbase(|x|) exp(-E_A T + V_A (r_surf - |x|)) at the qps
  const T* temp;          // [n_p2] P2 temperature of this level
  const T* lbase;         // log10 eta_base on a uniform radial grid over [r_cmb, r_surf]
  int n_lbase;
  T E_A, V_A, r_surf;
  int constrained;
  int bc_surface, bc_cmb;
  int m0;                 // first macro-tet of the launch (grid.y macros from m0; 0 = all 60)
};

// symmetric 4-point degree-2 rule: barycentrics (QA,QB,QB,QB) and permutations, w = 1/24
#define MFS_QA 0.58541019662496845446
#define MFS_QB 0.13819660112501051518

__host__ __device__ __forceinline__ constexpr int edge_of(int a, int b) {
  return (a < b ? a : b) == 0 ? (a > b ? a : b) - 1
                              : ((a < b ? a : b) == 1 ? (a > b ? a : b) + 1 : 5);
}
// node (0..9) carrying u_{a,q}: the vertex a itself if a == q, else the edge (a,q)
__host__ __device__ __forceinline__ constexpr int wnode(int a, int q) { return a == q ? a : 4 + edge_of(a, q); }

template <typename T>
__device__ __forceinline__ T rsqrt_t(T x);
template <>
__device__ __forceinline__ float rsqrt_t<float>(float x) { return rsqrtf(x); }
template <>
__device__ __forceinline__ double rsqrt_t<double>(double x) { return rsqrt(x); }
template <typename T>
__device__ __forceinline__ T rcp_t(T x);
template <>
__device__ __forceinline__ float rcp_t<float>(float x) { return __frcp_rn(x); }
template <>
__device__ __forceinline__ double rcp_t<double>(double x) { return 1.0 / x; }

// offset inside a 5x5x5 parity sub-block of a 3-bit corner mask (x = bit 0)
__host__ __device__ __forceinline__ constexpr int sub_off(int m) {
  return (m & 1) + 5 * ((m >> 1) & 1) + 25 * ((m >> 2) & 1);
}

// local fine coordinates (0..2TT) of a P2 slot; returns false for padding slots
__host__ __device__ __forceinline__ bool slot_coords(int s, int& dA, int& dB, int& dC) {
  const int cls = s / kSub, sub = s - cls * kSub;
  dA = 2 * (sub % 5) + (cls & 1);
  dB = 2 * ((sub / 5) % 5) + ((cls >> 1) & 1);
  dC = 2 * (sub / 25) + (cls >> 2);
  return dA <= 2 * TT && dB <= 2 * TT && dC <= 2 * TT;
}

template <typename T>
__device__ __forceinline__ T dlnrho_at(const ApplyParams<T>& P, T r) {
  if (P.n_dlnrho <= 1) return P.dlnrho[0];
  const T top = T(P.n_dlnrho - 1);
  T s = (r - P.r_cmb) * P.inv_dr * top;
  s = s < T(0) ? T(0) : (s > top ? top : s);
  int i = (int)s;
  i = i > P.n_dlnrho - 2 ? P.n_dlnrho - 2 : i;
  const T f = s - T(i);
  return (T(1) - f) * P.dlnrho[i] + f * P.dlnrho[i + 1];
}

// rho(r) = exp(int_{r_surf}^{r} d ln rho/dr), rho(r_surf) = 1, for the piecewise-linear table
// (integrated exactly: the node integrals from the table plus one trapezoid inside the cell)
template <typename T>
__device__ __forceinline__ T rho_bar(const ApplyParams<T>& P, T rad) {
  if (P.n_dlnrho <= 1) return exp(P.dlnrho[0] * (rad - P.r_surf));
  const int nt = P.n_dlnrho;
  const T top = T(nt - 1);
  T s = (rad - P.r_cmb) * P.inv_dr * top;
  s = s < T(0) ? T(0) : (s > top ? top : s);
  int i = (int)s;
  i = i > nt - 2 ? nt - 2 : i;
  const T f = s - T(i);
  const T hcell = T(1) / (P.inv_dr * top);
  const T g = (T(1) - f) * P.dlnrho[i] + f * P.dlnrho[i + 1];
  const T G = P.dlnrho_int[i] + T(0.5) * (P.dlnrho[i] + g) * f * hcell;
  return exp(G - P.dlnrho_int[nt - 1]);
}

// outward radial unit vector at a lattice point (Kuhn coordinates A,B,C of N)
template <typename T>
__device__ __forceinline__ void lattice_normal(const MacroGeom<T>& G, int A, int B, int C, int N, T nrm[3]) {
  const T inv = T(1) / T(N);
  const T xa = T(A) * inv, xb = T(B) * inv, xc = T(C) * inv;
  T x[3];
#pragma unroll
  for (int r = 0; r < 3; ++r) x[r] = G.v0[r] + G.Jm[3 * r] * xa + G.Jm[3 * r + 1] * xb + G.Jm[3 * r + 2] * xc;
  const T ri = rsqrt_t<T>(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
  nrm[0] = x[0] * ri;
  nrm[1] = x[1] * ri;
  nrm[2] = x[2] * ri;
}

// Slot offsets (relative to the cube base i + 5j + 25k) of the 10 P2 nodes of each of
// the 6 Freudenthal types (vertices of the path 0, e_p0, e_p0+e_p1, (1,1,1), then the
// edges 01,02,03,12,13,23 in their parity classes).
struct SlotTable {
  int off[6][10];
};
__host__ __device__ constexpr int perm_at(int pm, int k) {
  return k == 0 ? (0x221100 >> (4 * pm)) & 3 : (k == 1 ? (0x102021 >> (4 * pm)) & 3 : (0x010212 >> (4 * pm)) & 3);
}
__host__ __device__ constexpr int slot_off(int pm, int a) {
  return a == 0 ? 0
         : a == 1 ? sub_off(1 << perm_at(pm, 0))
         : a == 2 ? sub_off((1 << perm_at(pm, 0)) | (1 << perm_at(pm, 1)))
         : a == 3 ? sub_off(7)
         : a == 4 ? (1 << perm_at(pm, 0)) * kSub
         : a == 5 ? ((1 << perm_at(pm, 0)) | (1 << perm_at(pm, 1))) * kSub
         : a == 6 ? 7 * kSub
         : a == 7 ? ((1 << perm_at(pm, 1))) * kSub + sub_off(1 << perm_at(pm, 0))
         : a == 8 ? ((1 << perm_at(pm, 0)) ^ 7) * kSub + sub_off(1 << perm_at(pm, 0))
                  : (((1 << perm_at(pm, 0)) | (1 << perm_at(pm, 1))) ^ 7) * kSub +
                        sub_off((1 << perm_at(pm, 0)) | (1 << perm_at(pm, 1)));
}
static __constant__ SlotTable c_slots = {{
#define MFS_ROW(pm) {slot_off(pm, 0), slot_off(pm, 1), slot_off(pm, 2), slot_off(pm, 3), slot_off(pm, 4), \
                     slot_off(pm, 5), slot_off(pm, 6), slot_off(pm, 7), slot_off(pm, 8), slot_off(pm, 9)}
    MFS_ROW(0), MFS_ROW(1), MFS_ROW(2), MFS_ROW(3), MFS_ROW(4), MFS_ROW(5)
#undef MFS_ROW
}};

// bytes of dynamic shared memory of one sweep CTA
// (NR: copies of the output block, one per round of the fixed-point body, else 1)
template <typename T, int OP, int NR = 1>
constexpr size_t sweep_smem_bytes() {
  return sizeof(T) * ((((OP & (OP_A | OP_B)) != 0) ? 3 * NSLOT2 : 0) +
                      (((OP & (OP_A | OP_BT)) != 0) ? NR * 3 * NSLOT2 : 0) + NSLOT1 +
                      (((OP & OP_BT) != 0) ? NSLOT1 : 0) + (((OP & OP_B) != 0) ? NR * NSLOT1 : 0) +
                      (((OP & OP_ETAQ) != 0) ? NSLOT2 : 0)) +
         sizeof(int) * (NSLOT2 + NSLOT1);
}

template <typename T>
__device__ __forceinline__ T exp_t(T x);
template <>
__device__ __forceinline__ float exp_t<float>(float x) { return expf(x); }
template <>
__device__ __forceinline__ double exp_t<double>(double x) { return exp(x); }

// linear interpolation of a table on a uniform grid over [r0, r1] (clamped)
template <typename T>
__device__ __forceinline__ T radial_table(const T* tab, int n, T r, T r0, T r1) {
  if (n <= 1) return tab[0];
  const T top = T(n - 1);
  T s = (r - r0) / (r1 - r0) * top;
  s = s < T(0) ? T(0) : (s > top ? top : s);
  int i = (int)s;
  i = i > n - 2 ? n - 2 : i;
  const T f = s - T(i);
  return (T(1) - f) * tab[i] + f * tab[i + 1];
}

// One micro-tet of the register-resident sweep: its 30 velocity and 4 pressure outputs
// (node order: vertices 0-3, then edges 01, 02, 03, 12, 13, 23) from the staged tile block.
// Same arithmetic as the shared-memory body of sweep_tile (Sec. 4.1 geometry, Sec. 5.1
// forms); only the storage of intermediates differs.
template <typename T, int OP, bool BLEND>
__device__ __forceinline__ void tet_element(const ApplyParams<T>& P, const MacroGeom<T>& G, const int code,
                                            const int a0, const int b0, const int c0, const T* us,
                                            const T* eta_s, const T* p_s, const T* cM, const T* cJn,
                                            const T (&v0)[3], const T (&Jn)[9], const T (&csum)[3],
                                            const T (&nh)[3], const T* dtab, T (&yv)[3][10], T (&ypv)[4]) {
  constexpr bool HAS_U = (OP & (OP_A | OP_B)) != 0;
  constexpr bool HAS_P = (OP & OP_BT) != 0;
  constexpr bool OUT_U = (OP & (OP_A | OP_BT)) != 0;
  constexpr bool OUT_P = (OP & OP_B) != 0;
  constexpr bool HAS_CT = (OP & OP_CT) != 0;
  constexpr bool HAS_BC = (OP & OP_BC) != 0;
  constexpr bool NEED_GR = (OUT_P && HAS_BC) || HAS_CT;
  constexpr bool RHO = (OP & OP_RHO) != 0;
  const T QA = T(MFS_QA), QB = T(MFS_QB);
  const T dd = QA - QB;
  const T dq = T(4) * dd;                  // 4(alpha - beta)
  const T bq1 = T(4) * QB - T(1);          // 4 beta - 1
  const T b4 = T(4) * QB;                  // 4 beta
  const T fvb = QB * (T(2) * QB - T(1)), fva = QA * (T(2) * QA - T(1));
  const T feo = T(4) * QB * QB, fei = T(4) * QA * QB;
  const int n = P.n;
  const T C0 = G.absdet / (T(24) * T(n) * T(n) * T(n));
  const T dinv = T(1) / G.delta;
  const int ci = code & 15, cj = (code >> 4) & 15, ck = (code >> 8) & 15, pmu = code >> 12;
  const int p0 = perm_at(pmu, 0), p1 = perm_at(pmu, 1), p2 = perm_at(pmu, 2);
  const int base = ci + 5 * cj + 25 * ck;

  // nodal values of the micro-tet
  T u[3][10];
  if (HAS_U) {
#pragma unroll
    for (int a = 0; a < 10; ++a) {
      const int sa = base + slot_off(pmu, a);
#pragma unroll
      for (int c = 0; c < 3; ++c) u[c][a] = us[c * NSLOT2 + sa];
    }
  }
  T ev[4], pv[4];
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    ev[a] = eta_s[base + slot_off(pmu, a)];
    pv[a] = HAS_P ? p_s[base + slot_off(pmu, a)] : T(0);
  }
  const T eta_sum = ev[0] + ev[1] + ev[2] + ev[3];
  const T p_sum = pv[0] + pv[1] + pv[2] + pv[3];

  // geometry rows of this Freudenthal type: Mp = n Jm^-1 rows in permuted lattice order,
  // and the lattice steps e_p0, e_p1, e_p2 mapped by Jm/n
  T Mp[3][3], cp[3][3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    Mp[0][d] = cM[3 * p0 + d];
    Mp[1][d] = cM[3 * p1 + d];
    Mp[2][d] = cM[3 * p2 + d];
  }
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    cp[0][r] = cJn[3 * r + p0];
    cp[1][r] = cJn[3 * r + p1];
    cp[2][r] = csum[r] - cp[0][r] - cp[1][r];
  }
  // quadrature point 0: cube corner + beta (3 e_p0 + 2 e_p1 + e_p2); the next points add
  // (alpha - beta) e_p0, e_p1, e_p2 in turn
  const T qx = T(a0 + ci), qy = T(b0 + cj), qz = T(c0 + ck);
  T x[3];
#pragma unroll
  for (int r = 0; r < 3; ++r)
    x[r] = v0[r] + Jn[3 * r] * qx + Jn[3 * r + 1] * qy + Jn[3 * r + 2] * qz +
           QB * (T(3) * cp[0][r] + T(2) * cp[1][r] + cp[2][r]);

  // qp-independent parts of the lattice gradient: dbase_j = base_{j+1} - base_j
  T dbase[3][3], U0[3];
  if (HAS_U) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const T bs0 = bq1 * u[c][0] + b4 * (u[c][4] + u[c][5] + u[c][6]);
      const T bs1 = bq1 * u[c][1] + b4 * (u[c][4] + u[c][7] + u[c][8]);
      const T bs2 = bq1 * u[c][2] + b4 * (u[c][5] + u[c][7] + u[c][9]);
      const T bs3 = bq1 * u[c][3] + b4 * (u[c][6] + u[c][8] + u[c][9]);
      dbase[0][c] = bs1 - bs0;
      dbase[1][c] = bs2 - bs1;
      dbase[2][c] = bs3 - bs2;
      if (HAS_BC)
        U0[c] = fvb * (u[c][0] + u[c][1] + u[c][2] + u[c][3]) +
                feo * (u[c][4] + u[c][5] + u[c][6] + u[c][7] + u[c][8] + u[c][9]);
    }
  }

  T Rs[3][3], Vq[4][3], Ea[6][3], Zs[3], bq[4];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    Zs[c] = T(0);
#pragma unroll
    for (int j = 0; j < 3; ++j) Rs[c][j] = T(0);
#pragma unroll
    for (int e = 0; e < 6; ++e) Ea[e][c] = T(0);
  }

#pragma unroll
  for (int q = 0; q < 4; ++q) {
    if (q > 0) {
#pragma unroll
      for (int r = 0; r < 3; ++r) x[r] += dd * cp[q - 1][r];
    }
    const T r2 = x[0] * x[0] + x[1] * x[1] + x[2] * x[2];
    const T rinv = rsqrt_t<T>(r2);
    T K[3][3];
    T hr = T(1), h = T(0);
    if (BLEND) {
      h = x[0] * nh[0] + x[1] * nh[1] + x[2] * nh[2];
      const T hinv = rcp_t<T>(h);
      hr = h * rinv * dinv;
      const T ri2 = rinv * rinv;
      T v[3];
#pragma unroll
      for (int d = 0; d < 3; ++d) v[d] = nh[d] * hinv - x[d] * ri2;
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
    const T coefB = C0 * hr * hr;
    const T Wq = coefB * hr;

    T trace = T(0), Gp[3][3], wsum[3], wq[3];
    if (HAS_U) {
      T D[3][3];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        T w[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) w[a] = u[c][wnode(a, q)];
#pragma unroll
        for (int j = 0; j < 3; ++j) D[j][c] = dbase[j][c] + dq * (w[j + 1] - w[j]);
        wq[c] = w[q];
        wsum[c] = w[0] + w[1] + w[2] + w[3] - w[q];
      }
#pragma unroll
      for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int d = 0; d < 3; ++d) Gp[c][d] = D[0][c] * K[0][d] + D[1][c] * K[1][d] + D[2][c] * K[2][d];
      trace = Gp[0][0] + Gp[1][1] + Gp[2][2];
    }

    T gr = T(0);
    if (NEED_GR) {
      const T rad = BLEND ? h * dinv : r2 * rinv;
      if (P.n_dlnrho <= 1) {
        gr = dtab[0];
      } else {
        const T top = T(P.n_dlnrho - 1);
        T sg = (rad - P.r_cmb) * P.inv_dr * top;
        sg = sg < T(0) ? T(0) : (sg > top ? top : sg);
        int ig = (int)sg;
        ig = ig > P.n_dlnrho - 2 ? P.n_dlnrho - 2 : ig;
        const T fg = sg - T(ig);
        gr = (ig + 1 < 64) ? (T(1) - fg) * dtab[ig] + fg * dtab[ig + 1]
                           : (T(1) - fg) * P.dlnrho[ig] + fg * P.dlnrho[ig + 1];
      }
    }

    const T rq = RHO ? rho_bar<T>(P, BLEND ? h * dinv : r2 * rinv) : T(1);
    if (OUT_P) {
      T b = coefB * trace;
      if (HAS_BC) {
        T eu = T(0);
#pragma unroll
        for (int c = 0; c < 3; ++c) eu += (U0[c] + (fva - fvb) * wq[c] + (fei - feo) * wsum[c]) * x[c];
        b += Wq * gr * eu * rinv;
        if (RHO) b *= rq;
      }
      bq[q] = b;
    }

    if (OUT_U) {
      T S[3][3];
      if (OP & OP_A) {
        const T etaq = QB * eta_sum + dd * ev[q];
        const T coefA = T(2) * etaq * C0 * hr;
        const T hA = T(0.5) * coefA;
        const T t3 = trace * T(1.0 / 3.0);
        S[0][0] = coefA * (Gp[0][0] - t3);
        S[1][1] = coefA * (Gp[1][1] - t3);
        S[2][2] = coefA * (Gp[2][2] - t3);
        S[0][1] = S[1][0] = hA * (Gp[0][1] + Gp[1][0]);
        S[0][2] = S[2][0] = hA * (Gp[0][2] + Gp[2][0]);
        S[1][2] = S[2][1] = hA * (Gp[1][2] + Gp[2][1]);
      } else {
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
          for (int d = 0; d < 3; ++d) S[c][d] = T(0);
      }
      T pq = T(0);
      if (HAS_P) {
        pq = QB * p_sum + dd * pv[q];
        if (RHO && HAS_CT) pq *= rq;   // the transposed density-weighted constraint
        const T sp = coefB * pq;
        S[0][0] -= sp;
        S[1][1] -= sp;
        S[2][2] -= sp;
      }
      T zq[3] = {T(0), T(0), T(0)};
      if (HAS_CT) {
        const T zc = -Wq * pq * gr * rinv;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          zq[c] = zc * x[c];
          Zs[c] += zq[c];
        }
      }
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const T r0 = S[c][0] * K[0][0] + S[c][1] * K[0][1] + S[c][2] * K[0][2];
        const T r1 = S[c][0] * K[1][0] + S[c][1] * K[1][1] + S[c][2] * K[1][2];
        const T r2c = S[c][0] * K[2][0] + S[c][1] * K[2][1] + S[c][2] * K[2][2];
        Rs[c][0] += r0;
        Rs[c][1] += r1;
        Rs[c][2] += r2c;
        T sv[4];
        sv[0] = -r0;
        sv[1] = r0 - r1;
        sv[2] = r1 - r2c;
        sv[3] = r2c;
        Vq[q][c] = dq * sv[q] + (HAS_CT ? (fva - fvb) * zq[c] : T(0));
#pragma unroll
        for (int a = 0; a < 4; ++a)
          if (a != q) Ea[edge_of(a, q)][c] += sv[a] + (HAS_CT ? ((fei - feo) / dq) * zq[c] : T(0));
      }
    }
  }  // qp loop

  if (OUT_U) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      T Tacc[4];
      Tacc[0] = -Rs[c][0];
      Tacc[1] = Rs[c][0] - Rs[c][1];
      Tacc[2] = Rs[c][1] - Rs[c][2];
      Tacc[3] = Rs[c][2];
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        yv[c][a] = bq1 * Tacc[a] + Vq[a][c];
        if (HAS_CT) yv[c][a] += fvb * Zs[c];
      }
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = a + 1; b < 4; ++b) {
          T val = b4 * (Tacc[a] + Tacc[b]) + dq * Ea[edge_of(a, b)][c];
          if (HAS_CT) val += feo * Zs[c];
          yv[c][4 + edge_of(a, b)] = val;
        }
    }
  }
  if (OUT_P) {
    const T sb = bq[0] + bq[1] + bq[2] + bq[3];
#pragma unroll
    for (int a = 0; a < 4; ++a) ypv[a] = -(QB * sb + dd * bq[a]);
  }
}

// ---- packed FP32 pairs (sm_100+ fma.rn.f32x2 / add / mul): two quadrature points per op ----
__device__ __forceinline__ float2 bc2(float s) { return make_float2(s, s); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

// One micro-tet of the FP32 register-resident sweep with the quadrature points processed in
// pairs (0, 1) and (2, 3): every per-point quantity is a float2 holding the two points, and
// the per-point algebra runs on packed FP32 instructions (one instruction, two points).  Same
// arithmetic, outputs and node order as tet_element.
template <int OP, bool BLEND>
__device__ __forceinline__ void tet_element_x2(const ApplyParams<float>& P, const MacroGeom<float>& G, const int code,
                                               const int a0, const int b0, const int c0, const float* us,
                                               const float* eta_s, const float* p_s, const float* cM,
                                               const float* cJn, const float (&v0)[3], const float (&Jn)[9],
                                               const float (&csum)[3], const float (&nh)[3], const float* dtab,
                                               float (&yv)[3][10], float (&ypv)[4]) {
  using T = float;
  constexpr bool HAS_U = (OP & (OP_A | OP_B)) != 0;
  constexpr bool HAS_P = (OP & OP_BT) != 0;
  constexpr bool OUT_U = (OP & (OP_A | OP_BT)) != 0;
  constexpr bool OUT_P = (OP & OP_B) != 0;
  constexpr bool HAS_CT = (OP & OP_CT) != 0;
  constexpr bool HAS_BC = (OP & OP_BC) != 0;
  constexpr bool NEED_GR = (OUT_P && HAS_BC) || HAS_CT;
  constexpr bool RHO = (OP & OP_RHO) != 0;
  const T QA = T(MFS_QA), QB = T(MFS_QB);
  const T dd = QA - QB;
  const T dq = T(4) * dd;
  const T bq1 = T(4) * QB - T(1);
  const T b4 = T(4) * QB;
  const T fvb = QB * (T(2) * QB - T(1)), fva = QA * (T(2) * QA - T(1));
  const T feo = T(4) * QB * QB, fei = T(4) * QA * QB;
  const int n = P.n;
  const T C0 = G.absdet / (T(24) * T(n) * T(n) * T(n));
  const T dinv = T(1) / G.delta;
  const int ci = code & 15, cj = (code >> 4) & 15, ck = (code >> 8) & 15, pmu = code >> 12;
  const int p0 = perm_at(pmu, 0), p1 = perm_at(pmu, 1), p2 = perm_at(pmu, 2);
  const int base = ci + 5 * cj + 25 * ck;

  T u[3][10];
  if (HAS_U) {
#pragma unroll
    for (int a = 0; a < 10; ++a) {
      const int sa = base + slot_off(pmu, a);
#pragma unroll
      for (int c = 0; c < 3; ++c) u[c][a] = us[c * NSLOT2 + sa];
    }
  }
  T ev[4], pv[4];
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    ev[a] = eta_s[base + slot_off(pmu, a)];
    pv[a] = HAS_P ? p_s[base + slot_off(pmu, a)] : T(0);
  }
  const T eta_sum = ev[0] + ev[1] + ev[2] + ev[3];
  const T p_sum = pv[0] + pv[1] + pv[2] + pv[3];

  T Mp[3][3], cp[3][3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    Mp[0][d] = cM[3 * p0 + d];
    Mp[1][d] = cM[3 * p1 + d];
    Mp[2][d] = cM[3 * p2 + d];
  }
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    cp[0][r] = cJn[3 * r + p0];
    cp[1][r] = cJn[3 * r + p1];
    cp[2][r] = csum[r] - cp[0][r] - cp[1][r];
  }
  // positions of the four quadrature points: cube corner + beta (3 e_p0 + 2 e_p1 + e_p2), then
  // (alpha - beta) e_p0, e_p1, e_p2 added in turn
  const T qx = T(a0 + ci), qy = T(b0 + cj), qz = T(c0 + ck);
  T xs[4][3];
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    xs[0][r] = v0[r] + Jn[3 * r] * qx + Jn[3 * r + 1] * qy + Jn[3 * r + 2] * qz +
               QB * (T(3) * cp[0][r] + T(2) * cp[1][r] + cp[2][r]);
    xs[1][r] = xs[0][r] + dd * cp[0][r];
    xs[2][r] = xs[1][r] + dd * cp[1][r];
    xs[3][r] = xs[2][r] + dd * cp[2][r];
  }

  // qp-independent parts of the lattice gradient: dbase_j = base_{j+1} - base_j
  T dbase[3][3], U0[3];
  if (HAS_U) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const T bs0 = bq1 * u[c][0] + b4 * (u[c][4] + u[c][5] + u[c][6]);
      const T bs1 = bq1 * u[c][1] + b4 * (u[c][4] + u[c][7] + u[c][8]);
      const T bs2 = bq1 * u[c][2] + b4 * (u[c][5] + u[c][7] + u[c][9]);
      const T bs3 = bq1 * u[c][3] + b4 * (u[c][6] + u[c][8] + u[c][9]);
      dbase[0][c] = bs1 - bs0;
      dbase[1][c] = bs2 - bs1;
      dbase[2][c] = bs3 - bs2;
      if (HAS_BC)
        U0[c] = fvb * (u[c][0] + u[c][1] + u[c][2] + u[c][3]) +
                feo * (u[c][4] + u[c][5] + u[c][6] + u[c][7] + u[c][8] + u[c][9]);
    }
  }

  float2 Rs[3][3], Zs[3];
  T Vq[4][3], Ea[6][3], bq[4];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    Zs[c] = bc2(0.f);
#pragma unroll
    for (int j = 0; j < 3; ++j) Rs[c][j] = bc2(0.f);
#pragma unroll
    for (int e = 0; e < 6; ++e) Ea[e][c] = T(0);
  }

#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const int qa = 2 * k, qb = 2 * k + 1;
    float2 x[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) x[r] = make_float2(xs[qa][r], xs[qb][r]);
    const float2 r2 = fma2(x[2], x[2], fma2(x[1], x[1], mul2(x[0], x[0])));
    const float2 rinv = make_float2(rsqrtf(r2.x), rsqrtf(r2.y));
    float2 K[3][3];
    float2 hr = bc2(1.f), h = bc2(0.f);
    if (BLEND) {
      h = fma2(x[2], bc2(nh[2]), fma2(x[1], bc2(nh[1]), mul2(x[0], bc2(nh[0]))));
      const float2 hinv = make_float2(__frcp_rn(h.x), __frcp_rn(h.y));
      hr = mul2(mul2(h, rinv), bc2(dinv));
      const float2 nri2 = mul2(rinv, make_float2(-rinv.x, -rinv.y));   // -1/|x|^2
      float2 v[3];
#pragma unroll
      for (int d = 0; d < 3; ++d) v[d] = fma2(x[d], nri2, mul2(bc2(nh[d]), hinv));
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        const float2 tj = fma2(bc2(Mp[j][2]), x[2], fma2(bc2(Mp[j][1]), x[1], mul2(bc2(Mp[j][0]), x[0])));
        const float2 ntj = make_float2(-tj.x, -tj.y);
#pragma unroll
        for (int d = 0; d < 3; ++d) K[j][d] = fma2(ntj, v[d], bc2(Mp[j][d]));
      }
    } else {
#pragma unroll
      for (int j = 0; j < 3; ++j)
#pragma unroll
        for (int d = 0; d < 3; ++d) K[j][d] = bc2(Mp[j][d]);
    }
    const float2 coefB = mul2(mul2(bc2(C0), hr), hr);
    const float2 Wq = mul2(coefB, hr);

    float2 trace = bc2(0.f), Gp[3][3], wsum[3], wq[3];
    if (HAS_U) {
      float2 D[3][3];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        float2 w[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) w[a] = make_float2(u[c][wnode(a, qa)], u[c][wnode(a, qb)]);
#pragma unroll
        for (int j = 0; j < 3; ++j) D[j][c] = fma2(bc2(dq), sub2(w[j + 1], w[j]), bc2(dbase[j][c]));
        wq[c] = make_float2(u[c][qa], u[c][qb]);
        wsum[c] = sub2(add2(add2(w[0], w[1]), add2(w[2], w[3])), wq[c]);
      }
#pragma unroll
      for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int d = 0; d < 3; ++d) Gp[c][d] = fma2(D[2][c], K[2][d], fma2(D[1][c], K[1][d], mul2(D[0][c], K[0][d])));
      trace = add2(add2(Gp[0][0], Gp[1][1]), Gp[2][2]);
    }

    float2 gr = bc2(0.f);
    if (NEED_GR) {
      if (P.n_dlnrho <= 1) {
        gr = bc2(dtab[0]);
      } else {
        const T top = T(P.n_dlnrho - 1);
        T gg[2];
#pragma unroll
        for (int l = 0; l < 2; ++l) {
          const T rad = BLEND ? (l ? h.y : h.x) * dinv : (l ? r2.y * rinv.y : r2.x * rinv.x);
          T sg = (rad - P.r_cmb) * P.inv_dr * top;
          sg = sg < T(0) ? T(0) : (sg > top ? top : sg);
          int ig = (int)sg;
          ig = ig > P.n_dlnrho - 2 ? P.n_dlnrho - 2 : ig;
          const T fg = sg - T(ig);
          gg[l] = (ig + 1 < 64) ? (T(1) - fg) * dtab[ig] + fg * dtab[ig + 1]
                                : (T(1) - fg) * P.dlnrho[ig] + fg * P.dlnrho[ig + 1];
        }
        gr = make_float2(gg[0], gg[1]);
      }
    }
    float2 rq = bc2(1.f);
    if (RHO) {
      rq = make_float2(rho_bar<T>(P, BLEND ? h.x * dinv : r2.x * rinv.x),
                       rho_bar<T>(P, BLEND ? h.y * dinv : r2.y * rinv.y));
    }

    if (OUT_P) {
      float2 b = mul2(coefB, trace);
      if (HAS_BC) {
        float2 eu = bc2(0.f);
#pragma unroll
        for (int c = 0; c < 3; ++c)
          eu = fma2(fma2(bc2(fei - feo), wsum[c], fma2(bc2(fva - fvb), wq[c], bc2(U0[c]))), x[c], eu);
        b = fma2(mul2(mul2(Wq, gr), rinv), eu, b);
        if (RHO) b = mul2(b, rq);
      }
      bq[qa] = b.x;
      bq[qb] = b.y;
    }

    if (OUT_U) {
      float2 S[3][3];
      if (OP & OP_A) {
        const float2 etaq = fma2(bc2(dd), make_float2(ev[qa], ev[qb]), bc2(QB * eta_sum));
        const float2 coefA = mul2(mul2(bc2(2.f * C0), etaq), hr);
        const float2 hA = mul2(bc2(0.5f), coefA);
        const float2 nt3 = mul2(trace, bc2(-1.0f / 3.0f));
        S[0][0] = mul2(coefA, add2(Gp[0][0], nt3));
        S[1][1] = mul2(coefA, add2(Gp[1][1], nt3));
        S[2][2] = mul2(coefA, add2(Gp[2][2], nt3));
        S[0][1] = S[1][0] = mul2(hA, add2(Gp[0][1], Gp[1][0]));
        S[0][2] = S[2][0] = mul2(hA, add2(Gp[0][2], Gp[2][0]));
        S[1][2] = S[2][1] = mul2(hA, add2(Gp[1][2], Gp[2][1]));
      } else {
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
          for (int d = 0; d < 3; ++d) S[c][d] = bc2(0.f);
      }
      float2 pq = bc2(0.f);
      if (HAS_P) {
        pq = fma2(bc2(dd), make_float2(pv[qa], pv[qb]), bc2(QB * p_sum));
        if (RHO && HAS_CT) pq = mul2(pq, rq);   // the transposed density-weighted constraint
        const float2 sp = mul2(coefB, pq);
        S[0][0] = sub2(S[0][0], sp);
        S[1][1] = sub2(S[1][1], sp);
        S[2][2] = sub2(S[2][2], sp);
      }
      float2 zq[3] = {bc2(0.f), bc2(0.f), bc2(0.f)};
      if (HAS_CT) {
        const float2 zc = mul2(mul2(mul2(Wq, pq), gr), make_float2(-rinv.x, -rinv.y));
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          zq[c] = mul2(zc, x[c]);
          Zs[c] = add2(Zs[c], zq[c]);
        }
      }
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const float2 r0 = fma2(S[c][2], K[0][2], fma2(S[c][1], K[0][1], mul2(S[c][0], K[0][0])));
        const float2 r1 = fma2(S[c][2], K[1][2], fma2(S[c][1], K[1][1], mul2(S[c][0], K[1][0])));
        const float2 r2c = fma2(S[c][2], K[2][2], fma2(S[c][1], K[2][1], mul2(S[c][0], K[2][0])));
        Rs[c][0] = add2(Rs[c][0], r0);
        Rs[c][1] = add2(Rs[c][1], r1);
        Rs[c][2] = add2(Rs[c][2], r2c);
        float2 sv[4];
        sv[0] = make_float2(-r0.x, -r0.y);
        sv[1] = sub2(r0, r1);
        sv[2] = sub2(r1, r2c);
        sv[3] = r2c;
        Vq[qa][c] = dq * sv[qa].x + (HAS_CT ? (fva - fvb) * zq[c].x : T(0));
        Vq[qb][c] = dq * sv[qb].y + (HAS_CT ? (fva - fvb) * zq[c].y : T(0));
#pragma unroll
        for (int a = 0; a < 4; ++a) {
          if (a != qa) Ea[edge_of(a, qa)][c] += sv[a].x + (HAS_CT ? ((fei - feo) / dq) * zq[c].x : T(0));
          if (a != qb) Ea[edge_of(a, qb)][c] += sv[a].y + (HAS_CT ? ((fei - feo) / dq) * zq[c].y : T(0));
        }
      }
    }
  }  // pairs

  if (OUT_U) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const T R0 = Rs[c][0].x + Rs[c][0].y, R1 = Rs[c][1].x + Rs[c][1].y, R2 = Rs[c][2].x + Rs[c][2].y;
      const T Z = Zs[c].x + Zs[c].y;
      T Tacc[4];
      Tacc[0] = -R0;
      Tacc[1] = R0 - R1;
      Tacc[2] = R1 - R2;
      Tacc[3] = R2;
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        yv[c][a] = bq1 * Tacc[a] + Vq[a][c];
        if (HAS_CT) yv[c][a] += fvb * Z;
      }
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = a + 1; b < 4; ++b) {
          T val = b4 * (Tacc[a] + Tacc[b]) + dq * Ea[edge_of(a, b)][c];
          if (HAS_CT) val += feo * Z;
          yv[c][4 + edge_of(a, b)] = val;
        }
    }
  }
  if (OUT_P) {
    const T sb = bq[0] + bq[1] + bq[2] + bq[3];
#pragma unroll
    for (int a = 0; a < 4; ++a) ypv[a] = -(QB * sb + dd * bq[a]);
  }
}

// CTA-uniform geometry of the register-resident sweep, held in registers
template <typename T>
__device__ __forceinline__ void tile_uniforms(const T* cJn, const T* cv0, const T* cnh, T (&v0)[3], T (&Jn)[9],
                                              T (&csum)[3], T (&nh)[3]) {
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    nh[r] = cnh[r];
    v0[r] = cv0[r];
#pragma unroll
    for (int d = 0; d < 3; ++d) Jn[3 * r + d] = cJn[3 * r + d];
    csum[r] = Jn[3 * r] + Jn[3 * r + 1] + Jn[3 * r + 2];
  }
}

// Fixed-point accumulation (FP32 sweeps): the micro-tets of a tile are processed in NR rounds
// of NT; each round has its own int32 copy of the tile block and its own power-of-two scale
// 2^k_r, chosen after the round's outputs are known so that |output| * 2^k_r < 2^25 for every
// output of the round.  A slot receives at most 24 contributions per round (the micro-tets
// around a P2 node), so its integer sum stays below 2^30: no partial or final sum can overflow,
// the per-add rounding error is at most 2^-26 of the round's largest output, and the sums
// inside a tile are exact integer additions (native shared-memory reductions, no retry loop,
// independent of the order of the adds).  The flush converts back: y = sum_r Y_r 2^-k_r.
// Velocity and pressure outputs have separate scales.  A non-finite output (or one of
// magnitude >= 2^120) marks the round, and the flush then writes NaN for the whole tile so that
// the callers' NaN checks still see it.
constexpr int kFixedMaxRounds = 3;
__device__ __forceinline__ unsigned abs_bits(float x) { return __float_as_uint(x) & 0x7fffffffu; }
// max(m, |x|), NaN if either is NaN
__device__ __forceinline__ float max_nan_abs(float m, float x) {
  float r;
  asm("max.NaN.f32 %0, %1, %2;" : "=f"(r) : "f"(m), "f"(fabsf(x)));
  return r;
}
// scale exponent k of a round from the largest |output| bits; 255 marks a bad round
__device__ __forceinline__ int fixed_scale_exp(unsigned maxbits) {
  const int e = (int)(maxbits >> 23) - 127;   // floor(log2 max|out|); -127 for zero / denormals
  if (maxbits >= 0x7f800000u || e >= 120) return 255;
  const int k = 24 - e;
  return k > 100 ? 100 : k;
}
__device__ __forceinline__ float exp2_int(int k) { return __int_as_float((k + 127) << 23); }   // |k| <= 126
__device__ __forceinline__ void red_shared_s32(int* addr, int v) {
  asm volatile("red.shared.add.s32 [%0], %1;" ::"r"((unsigned)__cvta_generic_to_shared(addr)), "r"(v) : "memory");
}

template <int OP, bool BLEND, int NT, int NR, bool PAIR>
__device__ __forceinline__ void tet_sweep_fixed(const ApplyParams<float>& P, const MacroGeom<float>& G, const Tile tile,
                                                const float* us, int* ysi, const float* eta_s, const float* p_s,
                                                int* ypi, const float* cM, const float* cJn, const float* cv0,
                                                const float* cnh, const float* dtab, unsigned* rmax, const int tid) {
  constexpr bool OUT_U = (OP & (OP_A | OP_BT)) != 0;
  constexpr bool OUT_P = (OP & OP_B) != 0;
  float v0[3], Jn[9], csum[3], nh[3];
  tile_uniforms<float>(cJn, cv0, cnh, v0, Jn, csum, nh);
  const int a0 = tile.ta * TT, b0 = tile.tb * TT, c0 = tile.tc * TT;
  const int2 cinfo = P.classes[tile.cls];
#pragma unroll 1
  for (int r = 0; r < NR && r * NT < cinfo.y; ++r) {   // uniform over the CTA
    const int t = r * NT + tid;
    const bool active = t < cinfo.y;
    float yv[3][10], ypv[4];
    int code = 0;
    if (active) {
      code = P.tets[cinfo.x + t];
      if constexpr (PAIR)
        tet_element_x2<OP, BLEND>(P, G, code, a0, b0, c0, us, eta_s, p_s, cM, cJn, v0, Jn, csum, nh, dtab, yv, ypv);
      else
        tet_element<float, OP, BLEND>(P, G, code, a0, b0, c0, us, eta_s, p_s, cM, cJn, v0, Jn, csum, nh, dtab, yv, ypv);
    } else {
#pragma unroll
      for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int a = 0; a < 10; ++a) yv[c][a] = 0.f;
#pragma unroll
      for (int a = 0; a < 4; ++a) ypv[a] = 0.f;
    }
    // largest |output| of the thread (a NaN propagates: max.NaN), then of the warp as float bits
    unsigned mu = 0u, mp = 0u;
    if (OUT_U) {
      float m = 0.f;
#pragma unroll
      for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int a = 0; a < 10; ++a) m = max_nan_abs(m, yv[c][a]);
      mu = __reduce_max_sync(0xffffffffu, abs_bits(m));
    }
    if (OUT_P) {
      float m = 0.f;
#pragma unroll
      for (int a = 0; a < 4; ++a) m = max_nan_abs(m, ypv[a]);
      mp = __reduce_max_sync(0xffffffffu, abs_bits(m));
    }
    if ((tid & 31) == 0) {
      if (OUT_U) atomicMax(&rmax[2 * r], mu);
      if (OUT_P) atomicMax(&rmax[2 * r + 1], mp);
    }
    __syncthreads();
    if (active) {
      const int pmu = code >> 12;
      const int base = (code & 15) + 5 * ((code >> 4) & 15) + 25 * ((code >> 8) & 15);
      if (OUT_U) {
        const int k = fixed_scale_exp(rmax[2 * r]);
        if (k != 255) {
          const float S = exp2_int(k);
          int* y = ysi + r * 3 * NSLOT2;
#pragma unroll
          for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int a = 0; a < 10; ++a)
              red_shared_s32(&y[c * NSLOT2 + base + slot_off(pmu, a)], __float2int_rn(yv[c][a] * S));
        }
      }
      if (OUT_P) {
        const int k = fixed_scale_exp(rmax[2 * r + 1]);
        if (k != 255) {
          const float S = exp2_int(k);
          int* y = ypi + r * NSLOT1;
#pragma unroll
          for (int a = 0; a < 4; ++a) red_shared_s32(&y[base + slot_off(pmu, a)], __float2int_rn(ypv[a] * S));
        }
      }
    }
  }
}

// BODY 0: shared-memory element body (float atomics, also inside the quadrature loop);
// BODY 2: register-resident element body (tet_element) with fixed-point accumulation in NR
// rounds (FP32 only); BODY 3: BODY 2 with the quadrature points processed in packed FP32
// pairs (tet_element_x2).  (A register-resident body with float atomics, once BODY 1, was
// slower than BODY 0 and is gone.)
template <typename T, int OP, bool BLEND, int BODY = 0, int NT = kSweepThreads, int NR = 1>
__device__ __forceinline__ void sweep_tile(const ApplyParams<T>& P, const int m, const int tidx, const int n_tiles) {
  constexpr bool HAS_U = (OP & (OP_A | OP_B)) != 0;
  constexpr bool HAS_P = (OP & OP_BT) != 0;
  constexpr bool OUT_U = (OP & (OP_A | OP_BT)) != 0;
  constexpr bool OUT_P = (OP & OP_B) != 0;
  constexpr bool HAS_CT = (OP & OP_CT) != 0;
  constexpr bool HAS_BC = (OP & OP_BC) != 0;
  constexpr bool ETAQ = (OP & OP_ETAQ) != 0;
  static_assert(!ETAQ || OP == (OP_A | OP_ETAQ), "the quadrature-point viscosity serves A alone");
  static_assert(BODY < 2 || (sizeof(T) == 4 && !ETAQ && NR >= 1 && NR <= kFixedMaxRounds && NR * NT >= 384),
                "the fixed-point body is FP32, without quadrature-point viscosity, and covers a full tile");
  constexpr int NCOPY = BODY >= 2 ? NR : 1;

  // dynamic shared memory, layout of sweep_smem_bytes(): us, ys, eta_s, p_s, yp_s, ts, gid2, gid1
  // (BODY 2: ys and yp_s hold NR int32 copies)
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* us = reinterpret_cast<T*>(smem_raw);
  T* ys = us + (HAS_U ? 3 * NSLOT2 : 0);
  T* eta_s = ys + (OUT_U ? NCOPY * 3 * NSLOT2 : 0);
  T* p_s = eta_s + NSLOT1;
  T* yp_s = p_s + (HAS_P ? NSLOT1 : 0);
  T* ts = yp_s + (OUT_P ? NCOPY * NSLOT1 : 0);   // ETAQ: P2 temperature of the tile
  __shared__ unsigned rmax[2 * kFixedMaxRounds];   // BODY 2: largest |output| bits per round
  int* gid2 = reinterpret_cast<int*>(ts + (ETAQ ? NSLOT2 : 0));
  int* gid1 = gid2 + NSLOT2;
  __shared__ T cM[9], cJn[9], cv0[3], cnh[3];
  __shared__ T qpo[6][4][3];      // physical offset of qp q of type pm from the cube corner
  __shared__ T dtab[64];          // d ln rho / dr table (first 64 entries)

  const size_t tile_lin = (size_t)m * n_tiles + tidx;
  const Tile tile = P.tiles[tidx];
  const MacroGeom<T>& G = P.geom[m];
  const int a0 = tile.ta * TT, b0 = tile.tb * TT, c0 = tile.tc * TT;
  const int n = P.n, N = 2 * n;
  const int tid = threadIdx.x;

  if (BODY >= 2 && tid < 2 * kFixedMaxRounds) rmax[tid] = 0u;
  if (tid < 9) {
    cM[tid] = T(n) * G.Jinv[tid];
    cJn[tid] = G.Jm[tid] / T(n);
  }
  if (tid < 3) {
    cv0[tid] = G.v0[tid];
    cnh[tid] = G.nh[tid];
  }
  if (BODY == 0 && tid < 72) {
    // lattice offset of qp q of type pm: beta (3 e_p0 + 2 e_p1 + e_p2) + (alpha - beta) S_q
    const int pm = tid / 12, q = (tid / 3) % 4, r = tid % 3;
    const int p0 = perm_at(pm, 0), p1 = perm_at(pm, 1), p2 = perm_at(pm, 2);
    const int S1 = 1 << p0, S2 = S1 | (1 << p1);
    const int Sq = q == 0 ? 0 : (q == 1 ? S1 : (q == 2 ? S2 : 7));
    const T QA = T(MFS_QA), QB = T(MFS_QB);
    T o = T(0);
    for (int d = 0; d < 3; ++d) {
      const T lat = QB * T(3 * (p0 == d) + 2 * (p1 == d) + (p2 == d)) + (QA - QB) * T((Sq >> d) & 1);
      o += G.Jm[3 * r + d] * lat;
    }
    qpo[pm][q][r] = o / T(n);
  }
  if (tid < 64 && tid < P.n_dlnrho) dtab[tid] = P.dlnrho[tid];
  __shared__ T lbt[64];   // ETAQ: ln eta_base table (first 64 entries)
  if (ETAQ && tid < 64 && tid < P.n_lbase) lbt[tid] = T(2.302585092994045684) * P.lbase[tid];

  // ---- stage the P2 node block (u, with the input-side projections) and the P1 vertex
  // block (eta, p) ----
  // All table entries of this thread (both blocks) first, then all node values: the loads of
  // each kind are independent and in flight together (two memory latencies per tile).
  constexpr int kG = (NSLOT2 + NT - 1) / NT;
  constexpr int kG1 = (NSLOT1 + NT - 1) / NT;
  const int* tab2 = P.ids2 + tile_lin * NSLOT2;
  const int* tab1 = P.ids1 + tile_lin * NSLOT1;
  int codes[kG], ids1v[kG1];
#pragma unroll
  for (int k = 0; k < kG; ++k) {
    const int s = tid + k * NT;
    codes[k] = s < NSLOT2 ? __ldg(tab2 + s) : -1;
  }
#pragma unroll
  for (int k = 0; k < kG1; ++k) {
    const int s = tid + k * NT;
    ids1v[k] = s < NSLOT1 ? __ldg(tab1 + s) : -1;
  }
  const T psum = (HAS_P && P.psum) ? *P.psum : T(0);
  T uv[kG][3];
#pragma unroll
  for (int k = 0; k < kG; ++k) {
    uv[k][0] = uv[k][1] = uv[k][2] = T(0);
    if (HAS_U && codes[k] >= 0) {
      const int id = slot_node(codes[k]);
      uv[k][0] = __ldg(P.u + id);
      uv[k][1] = __ldg(P.u + P.n_p2 + id);
      uv[k][2] = __ldg(P.u + 2 * P.n_p2 + id);
    }
  }
  T ev1[kG1], pv1[kG1];
#pragma unroll
  for (int k = 0; k < kG1; ++k) {
    ev1[k] = T(1);
    pv1[k] = T(0);
    if (ids1v[k] >= 0) {
      ev1[k] = __ldg(P.eta + ids1v[k]);
      if (HAS_P) pv1[k] = __ldg(P.p + ids1v[k]);
    }
  }
  if (ETAQ) {
#pragma unroll
    for (int k = 0; k < kG; ++k) {
      const int s = tid + k * NT;
      if (s < NSLOT2) ts[s] = codes[k] >= 0 ? __ldg(P.temp + slot_node(codes[k])) : T(0);
    }
  }
#pragma unroll
  for (int k = 0; k < kG; ++k) {
    const int s = tid + k * NT;
    if (s >= NSLOT2) break;
    const int code = codes[k];
    gid2[s] = code;
    T v0 = uv[k][0], v1 = uv[k][1], v2 = uv[k][2];
    if (HAS_U && code >= 0 && P.constrained && slot_class(code) != 0) {
      const int gc = slot_class(code);     // 1 surface, 2 CMB
      const int bc = gc == 1 ? P.bc_surface : P.bc_cmb;
      if (bc == BC_DIRICHLET) {
        v0 = v1 = v2 = T(0);
      } else {
        int dA, dB, dC;
        slot_coords(s, dA, dB, dC);
        T nr[3];
        lattice_normal<T>(G, 2 * a0 + dA, 2 * b0 + dB, 2 * c0 + dC, N, nr);
        const T un = v0 * nr[0] + v1 * nr[1] + v2 * nr[2];
        v0 -= un * nr[0];
        v1 -= un * nr[1];
        v2 -= un * nr[2];
      }
    }
    if (HAS_U) {
      us[s] = v0;
      us[NSLOT2 + s] = v1;
      us[2 * NSLOT2 + s] = v2;
    }
  }
  if (OUT_U) {   // zero the output block(s), 16 bytes per store
    static_assert((3 * NSLOT2 * sizeof(T)) % 16 == 0 && ((HAS_U ? 3 * NSLOT2 : 0) * sizeof(T)) % 16 == 0,
                  "the output block is 16-byte aligned and sized");
    constexpr int n4 = NCOPY * 3 * NSLOT2 * (int)sizeof(T) / 16;
    int4* y4 = reinterpret_cast<int4*>(ys);
    for (int i = tid; i < n4; i += NT) y4[i] = make_int4(0, 0, 0, 0);
  }
  const T pm = psum / T(P.n_p1);
#pragma unroll
  for (int k = 0; k < kG1; ++k) {
    const int s = tid + k * NT;
    if (s >= NSLOT1) break;
    eta_s[s] = ev1[k];
    if (HAS_P) p_s[s] = ids1v[k] >= 0 ? pv1[k] - pm : T(0);
    if (OUT_P) {
#pragma unroll
      for (int r = 0; r < NCOPY; ++r) yp_s[r * NSLOT1 + s] = T(0);
      gid1[s] = ids1v[k];
    }
  }
  __syncthreads();

  if constexpr (BODY >= 2) {
    tet_sweep_fixed<OP, BLEND, NT, NR, BODY == 3>(P, G, tile, us, reinterpret_cast<int*>(ys), eta_s, p_s,
                                       reinterpret_cast<int*>(yp_s), cM, cJn, cv0, cnh, dtab, rmax, tid);
  } else {
  // ---- element sweep: one thread per micro-tet ----
  const T QA = T(MFS_QA), QB = T(MFS_QB);
  const T dq = T(4) * (QA - QB);           // 4(alpha - beta)
  const T bq1 = T(4) * QB - T(1);          // 4 beta - 1
  const T b4 = T(4) * QB;                  // 4 beta
  // P2 basis values at the qps: vertex beta(2beta-1) (alpha(2alpha-1) at its own qp),
  // edge 4 beta^2 (4 alpha beta at the qps of its two vertices)
  const T fvb = QB * (T(2) * QB - T(1)), fva = QA * (T(2) * QA - T(1));
  const T feo = T(4) * QB * QB, fei = T(4) * QA * QB;
  const T C0 = G.absdet / (T(24) * T(n) * T(n) * T(n));
  const T dinv = T(1) / G.delta;
  const int2 cinfo = P.classes[tile.cls];

  for (int t = tid; t < cinfo.y; t += NT) {
    const int code = P.tets[cinfo.x + t];
    const int ci = code & 15, cj = (code >> 4) & 15, ck = (code >> 8) & 15, pmu = code >> 12;
    const int p0 = perm_at(pmu, 0), p1 = perm_at(pmu, 1), p2 = perm_at(pmu, 2);
    const int base = ci + 5 * cj + 25 * ck;
#if MFS_SLOT_TABLE
    const int* soff = c_slots.off[pmu];
#define SLOT(a) (base + soff[a])
#else
#define SLOT(a) (base + slot_off(pmu, (a)))
#endif

    T eta_v[4], p_v[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      eta_v[a] = eta_s[SLOT(a)];          // P1 block uses the vertex sub-block indexing
      if (HAS_P) p_v[a] = p_s[SLOT(a)];
    }
    const T eta_sum = eta_v[0] + eta_v[1] + eta_v[2] + eta_v[3];
    // ETAQ: sums of the P2 temperature over the tet's vertices and edges (the P2 value at a
    // qp is fvb Tv + feo Te + (fva - fvb) T_q + (fei - feo) (edges at q))
    T Tv = T(0), Te = T(0);
    if (ETAQ) {
#pragma unroll
      for (int a = 0; a < 4; ++a) Tv += ts[SLOT(a)];
#pragma unroll
      for (int e = 4; e < 10; ++e) Te += ts[SLOT(e)];
    }
    T p_sum = T(0);
    if (HAS_P) p_sum = p_v[0] + p_v[1] + p_v[2] + p_v[3];

    // qp-independent parts: dbase_j = base_{j+1} - base_j, base_a = (4b-1) u_a + 4b sum_b u_ab,
    // and U0 = fvb sum u_v + feo sum u_e for the P2 value at the qps
    T dbase[3][3], U0[3];
    if (HAS_U) {
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const T* uc = us + c * NSLOT2;
        const T u0 = uc[SLOT(0)], u1 = uc[SLOT(1)], u2 = uc[SLOT(2)], u3 = uc[SLOT(3)];
        const T e01 = uc[SLOT(4)], e02 = uc[SLOT(5)], e03 = uc[SLOT(6)];
        const T e12 = uc[SLOT(7)], e13 = uc[SLOT(8)], e23 = uc[SLOT(9)];
        const T bs0 = bq1 * u0 + b4 * (e01 + e02 + e03);
        const T bs1 = bq1 * u1 + b4 * (e01 + e12 + e13);
        const T bs2 = bq1 * u2 + b4 * (e02 + e12 + e23);
        const T bs3 = bq1 * u3 + b4 * (e03 + e13 + e23);
        dbase[0][c] = bs1 - bs0;
        dbase[1][c] = bs2 - bs1;
        dbase[2][c] = bs3 - bs2;
        if (HAS_BC) U0[c] = fvb * (u0 + u1 + u2 + u3) + feo * (e01 + e02 + e03 + e12 + e13 + e23);
      }
    }

    // cube corner position
    const T qx = T(a0 + ci), qy = T(b0 + cj), qz = T(c0 + ck);
    T xc[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) xc[r] = cv0[r] + cJn[3 * r] * qx + cJn[3 * r + 1] * qy + cJn[3 * r + 2] * qz;

    // Rsum = sum_q R^q: since grad lambda_a is constant on the tet, T_a = sum_q s_a^q = Rsum grad lambda_a
    T Rsum[3][3], Zsum[3];
#if MFS_EDGE_ACC_REGS
    T Eacc[6][3];   // E_ab = s_a^b + s_b^a (+ the C-part of (B+C)^T), times dq at the end
#pragma unroll
    for (int e = 0; e < 6; ++e) Eacc[e][0] = Eacc[e][1] = Eacc[e][2] = T(0);
#endif
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      Zsum[c] = T(0);
#pragma unroll
      for (int j = 0; j < 3; ++j) Rsum[c][j] = T(0);
    }
    T bq[4];

#pragma unroll
    for (int q = 0; q < 4; ++q) {
      T x[3];
#pragma unroll
      for (int r = 0; r < 3; ++r) x[r] = xc[r] + qpo[pmu][q][r];
      const T r2 = x[0] * x[0] + x[1] * x[1] + x[2] * x[2];
      const T rinv = rsqrt_t<T>(r2);
      T K[3][3];
      T hr = T(1), h = T(0);
      if (BLEND) {
        h = x[0] * cnh[0] + x[1] * cnh[1] + x[2] * cnh[2];
        const T hinv = rcp_t<T>(h);
        hr = h * rinv * dinv;                  // 1/s, s = delta rho / h
        const T ri2 = rinv * rinv;
        T v[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) v[d] = cnh[d] * hinv - x[d] * ri2;
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          const int pj = j == 0 ? p0 : (j == 1 ? p1 : p2);
          const T m0 = cM[3 * pj], m1 = cM[3 * pj + 1], m2 = cM[3 * pj + 2];
          const T tj = m0 * x[0] + m1 * x[1] + m2 * x[2];
          K[j][0] = m0 - tj * v[0];
          K[j][1] = m1 - tj * v[1];
          K[j][2] = m2 - tj * v[2];
        }
      } else {
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          const int pj = j == 0 ? p0 : (j == 1 ? p1 : p2);
#pragma unroll
          for (int d = 0; d < 3; ++d) K[j][d] = cM[3 * pj + d];
        }
      }
      const T coefB = C0 * hr * hr;   // w |det J| s
      const T Wq = coefB * hr;        // w |det J|

      // nodal values u_{a,q} at this qp (vertex q and the three edges (a,q))
      T trace = T(0);
      T Gp[3][3];
      T wsum[3], wq[3];
      if (HAS_U) {
        T D[3][3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const T* uc = us + c * NSLOT2;
          T w[4];
#pragma unroll
          for (int a = 0; a < 4; ++a) w[a] = uc[SLOT(wnode(a, q))];
#pragma unroll
          for (int j = 0; j < 3; ++j) D[j][c] = dbase[j][c] + dq * (w[j + 1] - w[j]);
          wq[c] = w[q];
          wsum[c] = w[0] + w[1] + w[2] + w[3] - w[q];
        }
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
          for (int d = 0; d < 3; ++d) Gp[c][d] = D[0][c] * K[0][d] + D[1][c] * K[1][d] + D[2][c] * K[2][d];
        trace = Gp[0][0] + Gp[1][1] + Gp[2][2];
      }

      T gr = T(0);
      if ((OUT_P && HAS_BC) || HAS_CT) {
        const T rad = BLEND ? h * dinv : r2 * rinv;
        if (P.n_dlnrho <= 1) {
          gr = dtab[0];
        } else {
          const T top = T(P.n_dlnrho - 1);
          T sg = (rad - P.r_cmb) * P.inv_dr * top;
          sg = sg < T(0) ? T(0) : (sg > top ? top : sg);
          int ig = (int)sg;
          ig = ig > P.n_dlnrho - 2 ? P.n_dlnrho - 2 : ig;
          const T fg = sg - T(ig);
          gr = (ig + 1 < 64) ? (T(1) - fg) * dtab[ig] + fg * dtab[ig + 1]
                             : (T(1) - fg) * P.dlnrho[ig] + fg * P.dlnrho[ig + 1];
        }
      }

      // B: weights of -(div u + grad ln rho . u); OP_RHO: times rho at the point
      constexpr bool RHO = (OP & OP_RHO) != 0;
      const T rq = RHO ? rho_bar<T>(P, BLEND ? h * dinv : r2 * rinv) : T(1);
      if (OUT_P) {
        T b = coefB * trace;
        if (HAS_BC) {
          T eu = T(0);
#pragma unroll
          for (int c = 0; c < 3; ++c) eu += (U0[c] + (fva - fvb) * wq[c] + (fei - feo) * wsum[c]) * x[c];
          b += Wq * gr * eu * rinv;
          if (RHO) b *= rq;
        }
        bq[q] = b;
      }

      if (OUT_U) {
        // stress (scaled): sigma = coefA eps(G') - coefB p_q I
        T S[3][3];
        if (OP & OP_A) {
          T etaq;
          if (ETAQ) {
            T Tq = fvb * Tv + feo * Te + (fva - fvb) * ts[SLOT(q)];
            T te = T(0);
#pragma unroll
            for (int a = 0; a < 4; ++a)
              if (a != q) te += ts[SLOT(wnode(a, q))];
            Tq += (fei - feo) * te;
            const T rad = BLEND ? h * dinv : r2 * rinv;
            etaq = exp_t<T>(radial_table<T>(lbt, P.n_lbase, rad, P.r_cmb, P.r_surf) - P.E_A * Tq +
                            P.V_A * (P.r_surf - rad));
          } else {
            etaq = QB * eta_sum + (QA - QB) * eta_v[q];
          }
          const T coefA = T(2) * etaq * C0 * hr;
          const T t3 = trace * T(1.0 / 3.0);
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
        T pq = T(0);
        if (HAS_P) {
          pq = QB * p_sum + (QA - QB) * p_v[q];
          if (RHO && HAS_CT) pq *= rq;   // the transposed density-weighted constraint
          const T sp = coefB * pq;
          S[0][0] -= sp;
          S[1][1] -= sp;
          S[2][2] -= sp;
        }
        // R = S K^T (columns in permuted lattice order), s_a = R grad_lat lambda_a; the
        // qp-specific terms dq s_a^q go to vertex q (a == q) and to the edges (a, q)
        T zq[3] = {T(0), T(0), T(0)};
        if (HAS_CT) {
          const T zc = -Wq * pq * gr * rinv;   // (B+C)^T: the C part through the P2 values
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            zq[c] = zc * x[c];
            Zsum[c] += zq[c];
          }
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const T r0 = S[c][0] * K[0][0] + S[c][1] * K[0][1] + S[c][2] * K[0][2];
          const T r1 = S[c][0] * K[1][0] + S[c][1] * K[1][1] + S[c][2] * K[1][2];
          const T r2c = S[c][0] * K[2][0] + S[c][1] * K[2][1] + S[c][2] * K[2][2];
          Rsum[c][0] += r0;
          Rsum[c][1] += r1;
          Rsum[c][2] += r2c;
          T sv[4];
          sv[0] = -r0;
          sv[1] = r0 - r1;
          sv[2] = r1 - r2c;
          sv[3] = r2c;
          T* y = ys + c * NSLOT2;
#if MFS_EDGE_ACC_REGS
          {
            T val = dq * sv[q];
            if (HAS_CT) val += (fva - fvb) * zq[c];
            atomicAdd(&y[SLOT(q)], val);
          }
#pragma unroll
          for (int a = 0; a < 4; ++a)
            if (a != q) {
              Eacc[edge_of(a, q)][c] += sv[a];
              if (HAS_CT) Eacc[edge_of(a, q)][c] += ((fei - feo) / dq) * zq[c];
            }
#else
#pragma unroll
          for (int a = 0; a < 4; ++a) {
            T val = dq * sv[a];
            if (HAS_CT) val += (a == q ? (fva - fvb) : (fei - feo)) * zq[c];
            atomicAdd(&y[SLOT(wnode(a, q))], val);
          }
#endif
        }
      }
    }  // qp loop

    if (OUT_U) {
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        T* y = ys + c * NSLOT2;
        T Tacc[4];
        Tacc[0] = -Rsum[c][0];
        Tacc[1] = Rsum[c][0] - Rsum[c][1];
        Tacc[2] = Rsum[c][1] - Rsum[c][2];
        Tacc[3] = Rsum[c][2];
#pragma unroll
        for (int a = 0; a < 4; ++a) {
          T val = bq1 * Tacc[a];
          if (HAS_CT) val += fvb * Zsum[c];
          atomicAdd(&y[SLOT(a)], val);
        }
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b = a + 1; b < 4; ++b) {
            T val = b4 * (Tacc[a] + Tacc[b]);
#if MFS_EDGE_ACC_REGS
            val += dq * Eacc[edge_of(a, b)][c];
#endif
            if (HAS_CT) val += feo * Zsum[c];
            atomicAdd(&y[SLOT(4 + edge_of(a, b))], val);
          }
      }
    }
    if (OUT_P) {
      const T sb = bq[0] + bq[1] + bq[2] + bq[3];
#pragma unroll
      for (int a = 0; a < 4; ++a) atomicAdd(&yp_s[SLOT(a)], -(QB * sb + (QA - QB) * bq[a]));
    }
#undef SLOT
  }
  }   // BODY
  __syncthreads();

  // ---- add the block to the global result (output-side projections) ----
  // fixed-point bodies: 2^-k_r of each round (NaN for a marked round)
  T inv_u[NR], inv_p[NR];
#pragma unroll
  for (int r = 0; r < NR; ++r) {
    inv_u[r] = inv_p[r] = T(0);
    if constexpr (BODY >= 2) {
      const int ku = fixed_scale_exp(rmax[2 * r]), kp = fixed_scale_exp(rmax[2 * r + 1]);
      inv_u[r] = ku == 255 ? T(__int_as_float(0x7fc00000)) : T(exp2_int(-ku));
      inv_p[r] = kp == 255 ? T(__int_as_float(0x7fc00000)) : T(exp2_int(-kp));
    }
  }
  if (OUT_U) {
    const int nn = P.n_p2;
    for (int s = tid; s < NSLOT2; s += NT) {
      const int code = gid2[s];
      if (code < 0) continue;
      const int id = slot_node(code);
      const int gc = slot_class(code);
      int cl = NODE_FREE;
      if (P.constrained && gc != 0) {
        const int bc = gc == 1 ? P.bc_surface : P.bc_cmb;
        cl = bc == BC_DIRICHLET ? NODE_DIRICHLET : NODE_FREESLIP;
      }
      if (cl == NODE_DIRICHLET) {
        // identity rows of the constrained operator (A part); B^T rows stay zero
        if (OP & OP_A) {
          P.yu[id] = P.u[id];
          P.yu[nn + id] = P.u[nn + id];
          P.yu[2 * nn + id] = P.u[2 * nn + id];
        }
        continue;
      }
      T v0, v1, v2;
      if constexpr (BODY >= 2) {
        const int* yi = reinterpret_cast<const int*>(ys);
        v0 = v1 = v2 = T(0);
#pragma unroll
        for (int r = 0; r < NR; ++r) {
          const T inv = inv_u[r];
          v0 += T(yi[r * 3 * NSLOT2 + s]) * inv;
          v1 += T(yi[r * 3 * NSLOT2 + NSLOT2 + s]) * inv;
          v2 += T(yi[r * 3 * NSLOT2 + 2 * NSLOT2 + s]) * inv;
        }
      } else {
        v0 = ys[s];
        v1 = ys[NSLOT2 + s];
        v2 = ys[2 * NSLOT2 + s];
      }
      if (cl == NODE_FREESLIP) {
        int dA, dB, dC;
        slot_coords(s, dA, dB, dC);
        T nr[3];
        lattice_normal<T>(G, 2 * a0 + dA, 2 * b0 + dB, 2 * c0 + dC, N, nr);
        const T un = v0 * nr[0] + v1 * nr[1] + v2 * nr[2];
        v0 -= un * nr[0];
        v1 -= un * nr[1];
        v2 -= un * nr[2];
      }
      atomicAdd(&P.yu[id], v0);
      atomicAdd(&P.yu[nn + id], v1);
      atomicAdd(&P.yu[2 * nn + id], v2);
    }
  }
  if (OUT_P) {
    for (int s = tid; s < NSLOT1; s += NT) {
      const int id = gid1[s];
      if (id < 0) continue;
      T v = T(0);
      if constexpr (BODY >= 2) {
        const int* yi = reinterpret_cast<const int*>(yp_s);
#pragma unroll
        for (int r = 0; r < NR; ++r) v += T(yi[r * NSLOT1 + s]) * inv_p[r];
      } else {
        v = yp_s[s];
      }
      atomicAdd(&P.yp[id], v);
    }
  }
}

// one problem: grid (tiles, 60 macros)
template <typename T, int OP, bool BLEND>
__global__ void __launch_bounds__(kSweepThreads, MFS_SWEEP_MINBLOCKS) stokes_tile_kernel(const ApplyParams<T> P) {
  sweep_tile<T, OP, BLEND>(P, P.m0 + blockIdx.y, blockIdx.x, gridDim.x);
}
// the register-resident element body with fixed-point accumulation in ceil(384 / NT) rounds
template <typename T, int OP, bool BLEND, int NT, int MINB>
__global__ void __launch_bounds__(NT, MINB) stokes_tile_kernel_fixed(const ApplyParams<T> P) {
  sweep_tile<T, OP, BLEND, 2, NT, (384 + NT - 1) / NT>(P, P.m0 + blockIdx.y, blockIdx.x, gridDim.x);
}
// the same with the packed-pair element body
template <typename T, int OP, bool BLEND, int NT, int MINB>
__global__ void __launch_bounds__(NT, MINB) stokes_tile_kernel_fixed_x2(const ApplyParams<T> P) {
  sweep_tile<T, OP, BLEND, 3, NT, (384 + NT - 1) / NT>(P, P.m0 + blockIdx.y, blockIdx.x, gridDim.x);
}
// the same sweep compiled for one fewer resident CTA per SM (more registers per thread);
// the autotuner picks between the two per level
template <typename T, int OP, bool BLEND>
__global__ void __launch_bounds__(kSweepThreads, MFS_SWEEP_MINBLOCKS - 1)
    stokes_tile_kernel_wide(const ApplyParams<T> P) {
  sweep_tile<T, OP, BLEND>(P, P.m0 + blockIdx.y, blockIdx.x, gridDim.x);
}

// an ensemble in one persistent launch: CTA c works on the tiles map[c], map[c + grid], ...
// with map[b] = (problem, macro * 65536 + tile)
template <typename T, int OP, bool BLEND>
__global__ void __launch_bounds__(kSweepThreads, MFS_SWEEP_MINBLOCKS)
    stokes_tile_batch_kernel(const ApplyParams<T>* __restrict__ params, const int2* __restrict__ map,
                             const int* __restrict__ n_tiles, int n_items) {
  for (int b = blockIdx.x; b < n_items; b += gridDim.x) {
    const int2 w = map[b];
    sweep_tile<T, OP, BLEND>(params[w.x], w.y >> 16, w.y & 0xffff, n_tiles[w.x]);
    __syncthreads();   // the next tile's staging reuses the shared memory
  }
}

}  // namespace mfs
