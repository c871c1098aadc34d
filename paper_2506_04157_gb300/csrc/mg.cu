// Kernels of the multigrid and Krylov layers (arxiv 2506.04157, Sec. 5.2):
//  * BLAS-1 on velocity / pressure / saddle-point vectors, dot products accumulated in
//    FP64 with a deterministic two-pass reduction;
//  * Jacobi scaling and the boundary projections (Dirichlet zeroing, free-slip P_v);
//  * P2 prolongation / restriction as CSR products (exact P2 interpolation, Sec. 5.2.2);
//  * diag(A) without the free-slip projection (Sec. 5.2.2) and the inverse-viscosity P1
//    mass M_{1/eta} with its diagonal (Sec. 5.2.3), both as micro-tet sweeps;
//  * the coarsest-level operator: assembled column by column, inverted once per
//    viscosity in FP64 by Gauss-Jordan elimination, applied as a GEMV.
#include "apply.cuh"
#include "library.h"
#include "qp_geometry.cuh"
#include "solver.h"
#include "sweep_params.cuh"

namespace mfs {

static inline int blocks_for(int64_t n, int threads = 256, int cap = 8192) {
  int64_t b = (n + threads - 1) / threads;
  if (b < 1) b = 1;
  return (int)(b < cap ? b : cap);
}

#define GRID_STRIDE(i, n) \
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (n); i += (int64_t)gridDim.x * blockDim.x)

// ------------------------------------------------------------------------- BLAS-1
template <typename T>
__global__ void k_axpby(int64_t n, T a, const T* __restrict__ x, T b, T* __restrict__ y) {
  if (b == T(0)) {
    GRID_STRIDE(i, n) y[i] = a * x[i];
  } else {
    GRID_STRIDE(i, n) y[i] = a * x[i] + b * y[i];
  }
}
template <typename T>
__global__ void k_axpbypcz(int64_t n, T a, const T* __restrict__ x, T b, const T* __restrict__ y, T c,
                           T* __restrict__ z) {
  if (c == T(0)) {
    GRID_STRIDE(i, n) z[i] = a * x[i] + b * y[i];
  } else {
    GRID_STRIDE(i, n) z[i] = a * x[i] + b * y[i] + c * z[i];
  }
}
template <typename T>
__global__ void k_fill(int64_t n, T v, T* __restrict__ y) {
  GRID_STRIDE(i, n) y[i] = v;
}
template <typename T, typename S>
__global__ void k_convert(int64_t n, const S* __restrict__ x, T* __restrict__ y) {
  GRID_STRIDE(i, n) y[i] = (T)x[i];
}
template <typename T>
__global__ void k_mul(int64_t n, const T* __restrict__ x, const T* __restrict__ d, T* __restrict__ z) {
  GRID_STRIDE(i, n) z[i] = x[i] * d[i];
}
template <typename T>
__global__ void k_recip(int64_t n, T* __restrict__ x) {
  GRID_STRIDE(i, n) x[i] = T(1) / x[i];
}

__device__ __forceinline__ double dwarp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double dblock_sum(double v) {
  __shared__ double red[32];
  v = dwarp_sum(v);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  const int nw = (blockDim.x + 31) >> 5;
  v = threadIdx.x < nw ? red[threadIdx.x] : 0.0;
  if (w == 0) v = dwarp_sum(v);
  return v;
}

// Block sum of per-thread partials held in T: the warp stage adds in T (FP32 lanes are
// 64x the FP64 rate on this part), the across-warp stage in FP64; thread 0 gets the sum.
template <typename T>
__device__ __forceinline__ double block_sum_mixed(T v) {
  __shared__ double red[32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[w] = (double)v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int k = 0; k < (int)((blockDim.x + 31) >> 5); ++k) s += red[k];
  return s;
}

// per-thread partial in T over a fixed stride pattern, block and final sums in FP64
template <typename T>
__global__ void k_dot_part(int64_t n, const T* __restrict__ x, const T* __restrict__ y, double* __restrict__ part) {
  T acc = T(0);
  GRID_STRIDE(i, n) acc += x[i] * y[i];
  const double s = block_sum_mixed(acc);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}
__global__ void k_dot_final(const double* __restrict__ part, int np, double* __restrict__ out) {
  double acc = 0.0;
  for (int i = threadIdx.x; i < np; i += blockDim.x) acc += part[i];
  acc = dblock_sum(acc);
  if (threadIdx.x == 0) *out = acc;
}

// ------------------------------------------------------------------------- projections
// kind: 1 = Dirichlet (zero the node), 2 = free slip (remove the normal component)
template <typename T>
__global__ void k_bproject(int nb, const int* __restrict__ ids, const int8_t* __restrict__ kind,
                           const T* __restrict__ nrm, int64_t n_p2, T* __restrict__ v) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nb; k += gridDim.x * blockDim.x) {
    const int64_t id = ids[k];
    if (kind[k] == 1) {
      v[id] = T(0);
      v[n_p2 + id] = T(0);
      v[2 * n_p2 + id] = T(0);
    } else {
      const T nx = nrm[3 * k], ny = nrm[3 * k + 1], nz = nrm[3 * k + 2];
      const T un = v[id] * nx + v[n_p2 + id] * ny + v[2 * n_p2 + id] * nz;
      v[id] -= un * nx;
      v[n_p2 + id] -= un * ny;
      v[2 * n_p2 + id] -= un * nz;
    }
  }
}
// Dirichlet rows of diag(A) are 1 (identity rows of the constrained operator)
template <typename T>
__global__ void k_diag_dirichlet(int nb, const int* __restrict__ ids, const int8_t* __restrict__ kind, int64_t n_p2,
                                 T* __restrict__ d) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nb; k += gridDim.x * blockDim.x)
    if (kind[k] == 1) {
      const int64_t id = ids[k];
      d[id] = d[n_p2 + id] = d[2 * n_p2 + id] = T(1);
    }
}
// coarse matrix: add n n^T on free-slip nodes (regularises the projected-out directions)
__global__ void k_regularise_normals(int nb, const int* __restrict__ ids, const int8_t* __restrict__ kind,
                                     const double* __restrict__ nrm, int64_t n_p2, double* __restrict__ A) {
  const int64_t N = 3 * n_p2;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nb; k += gridDim.x * blockDim.x) {
    if (kind[k] != 2) continue;
    const int64_t id = ids[k];
    for (int c = 0; c < 3; ++c)
      for (int d = 0; d < 3; ++d) A[(c * n_p2 + id) * N + d * n_p2 + id] += nrm[3 * k + c] * nrm[3 * k + d];
  }
}

// ------------------------------------------------------------------------- transfers
// y[c] = alpha * P x[c] + beta * y[c] for the three components (SoA), P in CSR
template <typename T>
__global__ void k_spmv3(int nrows, const int* __restrict__ rp, const int* __restrict__ ci, const T* __restrict__ w,
                        int64_t ncols, const T* __restrict__ x, T alpha, T beta, T* __restrict__ y) {
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < nrows; r += gridDim.x * blockDim.x) {
    T s0 = T(0), s1 = T(0), s2 = T(0);
    for (int k = rp[r]; k < rp[r + 1]; ++k) {
      const int64_t j = ci[k];
      const T wk = w[k];
      s0 += wk * x[j];
      s1 += wk * x[ncols + j];
      s2 += wk * x[2 * ncols + j];
    }
    const int64_t nr = nrows;
    if (beta == T(0)) {
      y[r] = alpha * s0;
      y[nr + r] = alpha * s1;
      y[2 * nr + r] = alpha * s2;
    } else {
      y[r] = alpha * s0 + beta * y[r];
      y[nr + r] = alpha * s1 + beta * y[nr + r];
      y[2 * nr + r] = alpha * s2 + beta * y[2 * nr + r];
    }
  }
}

// projection of one node's velocity: zero at Dirichlet nodes, normal component removed at
// free-slip nodes (k = position in the boundary list)
template <typename T>
__device__ __forceinline__ void project_node(int k, const int8_t* __restrict__ kind, const T* __restrict__ nrm, T& v0,
                                             T& v1, T& v2) {
  if (kind[k] == 1) {
    v0 = v1 = v2 = T(0);
  } else {
    const T nx = nrm[3 * k], ny = nrm[3 * k + 1], nz = nrm[3 * k + 2];
    const T un = v0 * nx + v1 * ny + v2 * nz;
    v0 -= un * nx;
    v1 -= un * ny;
    v2 -= un * nz;
  }
}

// one warp per coarse row: lanes split the row's entries, a shuffle tree adds them
template <typename T>
__global__ void k_restrict_residual(int nrows, const int* __restrict__ rp, const int* __restrict__ ci,
                                    const T* __restrict__ w, int64_t ncols, const T* __restrict__ b,
                                    const T* __restrict__ t, T* __restrict__ y, const int* __restrict__ cmap,
                                    const int8_t* __restrict__ kind, const T* __restrict__ nrm) {
  const int lane = threadIdx.x & 31;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < nrows; r += nw) {
    T s0 = T(0), s1 = T(0), s2 = T(0);
    for (int k = rp[r] + lane; k < rp[r + 1]; k += 32) {
      const int64_t j = ci[k];
      const T wk = w[k];
      s0 += wk * (b[j] - t[j]);
      s1 += wk * (b[ncols + j] - t[ncols + j]);
      s2 += wk * (b[2 * ncols + j] - t[2 * ncols + j]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      s0 += __shfl_xor_sync(0xffffffffu, s0, o);
      s1 += __shfl_xor_sync(0xffffffffu, s1, o);
      s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    }
    if (lane == 0) {
      const int kb = cmap[r];
      if (kb >= 0) project_node(kb, kind, nrm, s0, s1, s2);
      const int64_t nr = nrows;
      y[r] = s0;
      y[nr + r] = s1;
      y[2 * nr + r] = s2;
    }
  }
}
template <typename T>
__global__ void k_prolong_add(int nrows, const int* __restrict__ rp, const int* __restrict__ ci,
                              const T* __restrict__ w, int64_t ncols, const T* __restrict__ xc, T* __restrict__ x,
                              T* __restrict__ t, const int* __restrict__ fmap, const int8_t* __restrict__ kind,
                              const T* __restrict__ nrm) {
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < nrows; r += gridDim.x * blockDim.x) {
    T s0 = T(0), s1 = T(0), s2 = T(0);
    for (int k = rp[r]; k < rp[r + 1]; ++k) {
      const int64_t j = ci[k];
      const T wk = w[k];
      s0 += wk * xc[j];
      s1 += wk * xc[ncols + j];
      s2 += wk * xc[2 * ncols + j];
    }
    const int64_t nr = nrows;
    T x0 = x[r] + s0, x1 = x[nr + r] + s1, x2 = x[2 * nr + r] + s2;
    const int kb = fmap[r];
    if (kb >= 0) project_node(kb, kind, nrm, x0, x1, x2);
    x[r] = x0;
    x[nr + r] = x1;
    x[2 * nr + r] = x2;
    t[r] = t[nr + r] = t[2 * nr + r] = T(0);
  }
}
// Jacobi-preconditioned Chebyshev update of one smoothing application (see Blas::cheb_update),
// one thread per node with its three components
template <typename T>
__global__ void k_cheb_update(int64_t n2, int mode, const T* __restrict__ b, T* __restrict__ t, T* __restrict__ r,
                              const T* __restrict__ dinv, T* __restrict__ d, T* __restrict__ x, T cz, T cd,
                              const int* __restrict__ nmap, const int8_t* __restrict__ kind,
                              const T* __restrict__ nrm) {
  GRID_STRIDE(i, n2) {
    T bv[3], tv[3], rv[3], iv[3], dv[3], xv[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const int64_t k = c * n2 + i;
      iv[c] = dinv[k];
      if (mode != 2) bv[c] = b[k];
      if (mode != 0) tv[c] = t[k];
      if (mode == 2) rv[c] = r[k];
      if (cd != T(0)) dv[c] = d[k];
      if (mode != 0) xv[c] = x[k];
    }
    const int kb = nmap[i];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const T rk = mode == 0 ? bv[c] : (mode == 1 ? bv[c] : rv[c]) - tv[c];
      rv[c] = rk;
      T dk = cz * iv[c] * rk;
      if (cd != T(0)) dk += cd * dv[c];
      dv[c] = dk;
      xv[c] = mode == 0 ? dk : xv[c] + dk;
    }
    if (kb >= 0) {
      project_node(kb, kind, nrm, dv[0], dv[1], dv[2]);
      project_node(kb, kind, nrm, xv[0], xv[1], xv[2]);
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const int64_t k = c * n2 + i;
      t[k] = T(0);
      r[k] = rv[c];
      d[k] = dv[c];
      x[k] = xv[c];
    }
  }
}

// ------------------------------------------------------------------------- coarse solve
// x = Ainv b, FP64 accumulation; one warp per row
template <typename T>
__global__ void k_gemv_f64(int n, const double* __restrict__ A, const T* __restrict__ b, T* __restrict__ x) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int r = warp; r < n; r += nw) {
    double s = 0.0;
    const double* row = A + (int64_t)r * n;
    for (int j = lane; j < n; j += 32) s += row[j] * (double)b[j];
    s = dwarp_sum(s);
    if (lane == 0) x[r] = (T)s;
  }
}

// Gauss-Jordan inversion in place, no pivoting (the regularised coarse operator is SPD).
// step k, part 1 (one block): save column k, scale row k by 1/a_kk, a_kk <- 1/a_kk
__global__ void k_gj_row(int n, int k, double* __restrict__ A, double* __restrict__ colk) {
  const double piv = A[(int64_t)k * n + k];
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x) colk[i] = A[(int64_t)i * n + k];
  __syncthreads();
  const double inv = 1.0 / piv;
  for (int j = threadIdx.x; j < n; j += blockDim.x) A[(int64_t)k * n + j] = (j == k ? 1.0 : A[(int64_t)k * n + j]) * inv;
}
// part 2: eliminate column k from every other row
__global__ void k_gj_elim(int n, int k, double* __restrict__ A, const double* __restrict__ colk) {
  const int64_t total = (int64_t)n * n;
  GRID_STRIDE(t, total) {
    const int i = (int)(t / n), j = (int)(t - (int64_t)i * n);
    if (i == k) continue;
    const double f = colk[i];
    const double akj = A[(int64_t)k * n + j];
    A[t] = (j == k ? 0.0 : A[t]) - f * akj;
  }
}
__global__ void k_unit(int64_t n, int64_t j, double* __restrict__ e) {
  GRID_STRIDE(i, n) e[i] = (i == j) ? 1.0 : 0.0;
}

void gj_invert(int n, double* A, double* colk, cudaStream_t s) {
  for (int k = 0; k < n; ++k) {
    k_gj_row<<<1, 512, 0, s>>>(n, k, A, colk);
    k_gj_elim<<<blocks_for((int64_t)n * n, 256, 4096), 256, 0, s>>>(n, k, A, colk);
  }
}

void unit_vector(int64_t n, int64_t j, double* e, cudaStream_t s) { k_unit<<<blocks_for(n), 256, 0, s>>>(n, j, e); }

// ------------------------------------------------------------------------- diag(A), M_{1/eta}
// diag(A) (raw, no projection): sum over tets and qps of 2 eta W (|g|^2/2 + g_c^2/6);
// ETAQ: eta from the viscosity law at the quadrature points (levels up to l_eta)
template <typename T, bool BLEND, bool ETAQ>
__global__ void __launch_bounds__(128) k_diag_sweep(const ApplyParams<T> P, T* __restrict__ diag) {
  __shared__ T ds[3 * NSLOT2];
  __shared__ T eta_s[NSLOT1];
  __shared__ T tsm[ETAQ ? NSLOT2 : 1];   // ETAQ: P2 temperature of the tile
  const int m = blockIdx.y, tidx = blockIdx.x;
  const size_t lin = (size_t)m * gridDim.x + tidx;
  const Tile tile = P.tiles[tidx];
  const MacroGeom<T>& G = P.geom[m];
  const int n = P.n;
  for (int s = threadIdx.x; s < 3 * NSLOT2; s += blockDim.x) ds[s] = T(0);
  for (int s = threadIdx.x; s < NSLOT1; s += blockDim.x) {
    const int id = P.ids1[lin * NSLOT1 + s];
    eta_s[s] = id >= 0 ? P.eta[id] : T(1);
  }
  if (ETAQ)
    for (int s = threadIdx.x; s < NSLOT2; s += blockDim.x) {
      const int code = P.ids2[lin * NSLOT2 + s];
      tsm[s] = code >= 0 ? P.temp[slot_node(code)] : T(0);
    }
  __syncthreads();
  const double QA = MFS_QA, QB = MFS_QB;
  const T C0 = G.absdet / (T(24) * T(n) * T(n) * T(n));
  const int2 cinfo = P.classes[tile.cls];
  for (int t = threadIdx.x; t < cinfo.y; t += blockDim.x) {
    const int code = P.tets[cinfo.x + t];
    const int ci = code & 15, cj = (code >> 4) & 15, ck = (code >> 8) & 15, pmu = code >> 12;
    const int p0 = (0x221100 >> (4 * pmu)) & 3, p1 = (0x102021 >> (4 * pmu)) & 3, p2 = (0x010212 >> (4 * pmu)) & 3;
    const int S1 = 1 << p0, S2 = S1 | (1 << p1);
    const int base = ci + 5 * cj + 25 * ck;
    int slot[10];
    slot[0] = base;
    slot[1] = base + sub_off(S1);
    slot[2] = base + sub_off(S2);
    slot[3] = base + sub_off(7);
    slot[4] = S1 * kSub + base;
    slot[5] = S2 * kSub + base;
    slot[6] = 7 * kSub + base;
    slot[7] = (S1 ^ S2) * kSub + base + sub_off(S1);
    slot[8] = (S1 ^ 7) * kSub + base + sub_off(S1);
    slot[9] = (S2 ^ 7) * kSub + base + sub_off(S2);
    T eta_v[4];
    for (int a = 0; a < 4; ++a) eta_v[a] = eta_s[slot[a]];
    const T qx = T(tile.ta * TT + ci), qy = T(tile.tb * TT + cj), qz = T(tile.tc * TT + ck);
    T acc[10][3];
    for (int a = 0; a < 10; ++a) acc[a][0] = acc[a][1] = acc[a][2] = T(0);
    for (int q = 0; q < 4; ++q) {
      T K[3][3], hr, rinv, x[3];
      qp_geometry<T, BLEND>(G, n, p0, p1, p2, q, qx, qy, qz, K, hr, rinv, x);
      const double lam[4] = {q == 0 ? QA : QB, q == 1 ? QA : QB, q == 2 ? QA : QB, q == 3 ? QA : QB};
      T etaq;
      if (ETAQ) {   // eta(x_q, T(x_q)), T the P2 interpolant
        T Tq = T(0);
        for (int a = 0; a < 4; ++a) Tq += T(lam[a] * (2 * lam[a] - 1)) * tsm[slot[a]];
        for (int e = 0; e < 6; ++e) {
          const int i0 = e < 3 ? 0 : (e < 5 ? 1 : 2);
          const int i1 = e < 3 ? e + 1 : (e < 5 ? e - 1 : 3);
          Tq += T(4 * lam[i0] * lam[i1]) * tsm[slot[4 + e]];
        }
        const T h = x[0] * G.nh[0] + x[1] * G.nh[1] + x[2] * G.nh[2];
        const T rad = BLEND ? h / G.delta : T(1) / rinv;
        etaq = exp_t<T>(T(2.302585092994045684) * radial_table<T>(P.lbase, P.n_lbase, rad, P.r_cmb, P.r_surf) -
                        P.E_A * Tq + P.V_A * (P.r_surf - rad));
      } else {
        etaq = T(lam[0]) * eta_v[0] + T(lam[1]) * eta_v[1] + T(lam[2]) * eta_v[2] + T(lam[3]) * eta_v[3];
      }
      const T coefA = T(2) * etaq * C0 * hr;
      for (int a = 0; a < 10; ++a) {
        double gl[3];
        p2_lat_grad(a, lam, gl);
        T g[3];
        for (int d = 0; d < 3; ++d) g[d] = T(gl[0]) * K[0][d] + T(gl[1]) * K[1][d] + T(gl[2]) * K[2][d];
        const T g2 = g[0] * g[0] + g[1] * g[1] + g[2] * g[2];
        for (int c = 0; c < 3; ++c) acc[a][c] += coefA * (T(0.5) * g2 + g[c] * g[c] / T(6));
      }
    }
    for (int a = 0; a < 10; ++a)
      for (int c = 0; c < 3; ++c) atomicAdd(&ds[c * NSLOT2 + slot[a]], acc[a][c]);
  }
  __syncthreads();
  for (int s = threadIdx.x; s < NSLOT2; s += blockDim.x) {
    const int code = P.ids2[lin * NSLOT2 + s];
    if (code < 0) continue;
    const int64_t id = slot_node(code);
    for (int c = 0; c < 3; ++c) atomicAdd(&diag[c * (int64_t)P.n_p2 + id], ds[c * NSLOT2 + s]);
  }
}

// y += M_{1/eta} p (DIAG: y += diag(M_{1/eta})): int (1/eta_q) psi_j psi_k over blended tets
template <typename T, bool BLEND, bool DIAG>
__global__ void __launch_bounds__(128) k_mass_sweep(const ApplyParams<T> P, const T* __restrict__ pin, T* __restrict__ y,
                                                     const double* __restrict__ active) {
  if (active && !(*active > 0.0)) return;
  __shared__ T ps[NSLOT1], ys[NSLOT1], eta_s[NSLOT1];
  __shared__ int gid[NSLOT1];
  const int m = blockIdx.y, tidx = blockIdx.x;
  const size_t lin = (size_t)m * gridDim.x + tidx;
  const Tile tile = P.tiles[tidx];
  const MacroGeom<T>& G = P.geom[m];
  const int n = P.n;
  for (int s = threadIdx.x; s < NSLOT1; s += blockDim.x) {
    const int id = P.ids1[lin * NSLOT1 + s];
    gid[s] = id;
    eta_s[s] = id >= 0 ? P.eta[id] : T(1);
    ps[s] = (!DIAG && id >= 0) ? pin[id] : T(0);
    ys[s] = T(0);
  }
  __syncthreads();
  const double QA = MFS_QA, QB = MFS_QB;
  const T C0 = G.absdet / (T(24) * T(n) * T(n) * T(n));
  const int2 cinfo = P.classes[tile.cls];
  for (int t = threadIdx.x; t < cinfo.y; t += blockDim.x) {
    const int code = P.tets[cinfo.x + t];
    const int ci = code & 15, cj = (code >> 4) & 15, ck = (code >> 8) & 15, pmu = code >> 12;
    const int p0 = (0x221100 >> (4 * pmu)) & 3, p1 = (0x102021 >> (4 * pmu)) & 3, p2 = (0x010212 >> (4 * pmu)) & 3;
    const int S1 = 1 << p0, S2 = S1 | (1 << p1);
    const int base = ci + 5 * cj + 25 * ck;
    const int sl[4] = {base, base + sub_off(S1), base + sub_off(S2), base + sub_off(7)};
    T ev[4], pv[4], out[4] = {T(0), T(0), T(0), T(0)};
    for (int a = 0; a < 4; ++a) {
      ev[a] = eta_s[sl[a]];
      pv[a] = ps[sl[a]];
    }
    const T qx = T(tile.ta * TT + ci), qy = T(tile.tb * TT + cj), qz = T(tile.tc * TT + ck);
    for (int q = 0; q < 4; ++q) {
      T K[3][3], hr, rinv, x[3];
      qp_geometry<T, BLEND>(G, n, p0, p1, p2, q, qx, qy, qz, K, hr, rinv, x);
      const T W = C0 * hr * hr * hr;
      T lam[4];
      for (int a = 0; a < 4; ++a) lam[a] = T(a == q ? QA : QB);
      const T etaq = lam[0] * ev[0] + lam[1] * ev[1] + lam[2] * ev[2] + lam[3] * ev[3];
      const T wq = W / etaq;
      if (DIAG) {
        for (int a = 0; a < 4; ++a) out[a] += wq * lam[a] * lam[a];
      } else {
        const T pq = lam[0] * pv[0] + lam[1] * pv[1] + lam[2] * pv[2] + lam[3] * pv[3];
        for (int a = 0; a < 4; ++a) out[a] += wq * lam[a] * pq;
      }
    }
    for (int a = 0; a < 4; ++a) atomicAdd(&ys[sl[a]], out[a]);
  }
  __syncthreads();
  for (int s = threadIdx.x; s < NSLOT1; s += blockDim.x)
    if (gid[s] >= 0) atomicAdd(&y[gid[s]], ys[s]);
}

// ------------------------------------------------------------------------- host wrappers
template <typename T>
void Blas<T>::axpby(int64_t n, T a, const T* x, T b, T* y, cudaStream_t s) {
  k_axpby<T><<<blocks_for(n), 256, 0, s>>>(n, a, x, b, y);
}
template <typename T>
void Blas<T>::axpbypcz(int64_t n, T a, const T* x, T b, const T* y, T c, T* z, cudaStream_t s) {
  k_axpbypcz<T><<<blocks_for(n), 256, 0, s>>>(n, a, x, b, y, c, z);
}
template <typename T>
void Blas<T>::fill(int64_t n, T v, T* y, cudaStream_t s) {
  k_fill<T><<<blocks_for(n), 256, 0, s>>>(n, v, y);
}
template <typename T>
void Blas<T>::mul(int64_t n, const T* x, const T* d, T* z, cudaStream_t s) {
  k_mul<T><<<blocks_for(n), 256, 0, s>>>(n, x, d, z);
}
template <typename T>
void Blas<T>::recip(int64_t n, T* x, cudaStream_t s) {
  k_recip<T><<<blocks_for(n), 256, 0, s>>>(n, x);
}
template <typename T>
void Blas<T>::dot_async(int64_t n, const T* x, const T* y, double* part, double* out, cudaStream_t s) {
  const int nb = blocks_for(n, 256, kRedBlocks);
  k_dot_part<T><<<nb, 256, 0, s>>>(n, x, y, part);
  k_dot_final<<<1, 512, 0, s>>>(part, nb, out);
}
template <typename T>
void Blas<T>::bproject(const BoundaryList& B, int64_t n_p2, T* v, cudaStream_t s) {
  if (B.nb == 0) return;
  k_bproject<T><<<blocks_for(B.nb), 256, 0, s>>>(B.nb, B.ids, B.kind, B.template normals<T>(), n_p2, v);
}
template <typename T>
void Blas<T>::spmv3(const Csr& P, int64_t ncols, const T* x, T alpha, T beta, T* y, cudaStream_t s) {
  k_spmv3<T><<<blocks_for(P.nrows), 256, 0, s>>>(P.nrows, P.rp, P.ci, P.template w<T>(), ncols, x, alpha, beta, y);
}
template <typename T>
void Blas<T>::cheb_update(int64_t n2, int mode, const T* b, T* t, T* r, const T* dinv, T* d, T* x, T cz, T cd,
                          const BoundaryList& B, cudaStream_t s) {
  k_cheb_update<T><<<blocks_for(n2), 256, 0, s>>>(n2, mode, b, t, r, dinv, d, x, cz, cd, B.nodemap, B.kind,
                                                  B.template normals<T>());
}
template <typename T>
void Blas<T>::restrict_residual(const Csr& R, int64_t ncols, const T* b, const T* t, T* y, const BoundaryList& Bc,
                                cudaStream_t s) {
  k_restrict_residual<T><<<blocks_for((int64_t)R.nrows * 32, 256, 16384), 256, 0, s>>>(
      R.nrows, R.rp, R.ci, R.template w<T>(), ncols, b, t, y, Bc.nodemap, Bc.kind, Bc.template normals<T>());
}
template <typename T>
void Blas<T>::prolong_add(const Csr& P, int64_t ncols, const T* xc, T* x, T* t, const BoundaryList& Bf,
                          cudaStream_t s) {
  k_prolong_add<T><<<blocks_for(P.nrows), 256, 0, s>>>(P.nrows, P.rp, P.ci, P.template w<T>(), ncols, xc, x, t,
                                                       Bf.nodemap, Bf.kind, Bf.template normals<T>());
}
template <typename T>
void Blas<T>::gemv_f64(int n, const double* A, const T* b, T* x, cudaStream_t s) {
  k_gemv_f64<T><<<blocks_for((int64_t)n * 32, 256, 4096), 256, 0, s>>>(n, A, b, x);
}
template <>
void Blas<float>::convert_from_f64(int64_t n, const double* x, float* y, cudaStream_t s) {
  k_convert<float, double><<<blocks_for(n), 256, 0, s>>>(n, x, y);
}
template <>
void Blas<double>::convert_from_f64(int64_t n, const double* x, double* y, cudaStream_t s) {
  cudaMemcpyAsync(y, x, sizeof(double) * n, cudaMemcpyDeviceToDevice, s);
}
template <>
void Blas<float>::convert_to_f64(int64_t n, const float* x, double* y, cudaStream_t s) {
  k_convert<double, float><<<blocks_for(n), 256, 0, s>>>(n, x, y);
}
template <>
void Blas<double>::convert_to_f64(int64_t n, const double* x, double* y, cudaStream_t s) {
  cudaMemcpyAsync(y, x, sizeof(double) * n, cudaMemcpyDeviceToDevice, s);
}

template struct Blas<float>;
template struct Blas<double>;


template <typename T>
mfs_status diag_A(mfs_problem* P, int lvl, const BoundaryList& B, T* diag) {
  mfs_mesh* M = P->mesh;
  const LevelData& L = M->levels[lvl];
  cudaStream_t s = M->ctx->stream;
  MFS_CUDA(cudaMemsetAsync(diag, 0, sizeof(T) * 3 * (size_t)L.nb2.total, s));
  dim3 grid(L.n_tiles, kMacroCells);
  ApplyParams<T> prm = sweep_params<T>(P, lvl);
  if (lvl <= P->l_eta) {
    if (M->host.blending) k_diag_sweep<T, true, true><<<grid, 128, 0, s>>>(prm, diag);
    else k_diag_sweep<T, false, true><<<grid, 128, 0, s>>>(prm, diag);
  } else {
    if (M->host.blending) k_diag_sweep<T, true, false><<<grid, 128, 0, s>>>(prm, diag);
    else k_diag_sweep<T, false, false><<<grid, 128, 0, s>>>(prm, diag);
  }
  if (B.nb) k_diag_dirichlet<T><<<blocks_for(B.nb), 256, 0, s>>>(B.nb, B.ids, B.kind, L.nb2.total, diag);
  MFS_CUDA(cudaGetLastError());
  return MFS_OK;
}

template <typename T>
mfs_status mass_apply(mfs_problem* P, int lvl, const T* pin, T* y, int diag_only, const double* active, int zero_out) {
  mfs_mesh* M = P->mesh;
  const LevelData& L = M->levels[lvl];
  cudaStream_t s = M->ctx->stream;
  if (zero_out) MFS_CUDA(cudaMemsetAsync(y, 0, sizeof(T) * (size_t)L.nb1.total, s));
  dim3 grid(L.n_tiles, kMacroCells);
  ApplyParams<T> prm = sweep_params<T>(P, lvl);
  const bool bl = M->host.blending != 0;
  if (diag_only) {
    if (bl) k_mass_sweep<T, true, true><<<grid, 128, 0, s>>>(prm, pin, y, active);
    else k_mass_sweep<T, false, true><<<grid, 128, 0, s>>>(prm, pin, y, active);
  } else {
    if (bl) k_mass_sweep<T, true, false><<<grid, 128, 0, s>>>(prm, pin, y, active);
    else k_mass_sweep<T, false, false><<<grid, 128, 0, s>>>(prm, pin, y, active);
  }
  MFS_CUDA(cudaGetLastError());
  return MFS_OK;
}

template mfs_status diag_A<float>(mfs_problem*, int, const BoundaryList&, float*);
template mfs_status diag_A<double>(mfs_problem*, int, const BoundaryList&, double*);
// stored quadrature weights of M_{1/eta} (FP64), see mass_weights
template <bool BLEND>
__global__ void __launch_bounds__(128) k_mass_weights(const ApplyParams<double> P, double* __restrict__ w) {
  __shared__ double eta_s[NSLOT1];
  const int m = blockIdx.y, tidx = blockIdx.x;
  const size_t lin = (size_t)m * gridDim.x + tidx;
  const Tile tile = P.tiles[tidx];
  const MacroGeom<double>& G = P.geom[m];
  const int n = P.n;
  for (int s = threadIdx.x; s < NSLOT1; s += blockDim.x) {
    const int id = P.ids1[lin * NSLOT1 + s];
    eta_s[s] = id >= 0 ? P.eta[id] : 1.0;
  }
  __syncthreads();
  const double QA = MFS_QA, QB = MFS_QB;
  const double C0 = G.absdet / (24.0 * n * (double)n * n);
  const int2 cinfo = P.classes[tile.cls];
  for (int t = threadIdx.x; t < cinfo.y; t += blockDim.x) {
    const int code = P.tets[cinfo.x + t];
    const int ci = code & 15, cj = (code >> 4) & 15, ck = (code >> 8) & 15, pmu = code >> 12;
    const int p0 = perm_at(pmu, 0), p1 = perm_at(pmu, 1), p2 = perm_at(pmu, 2);
    const int base = ci + 5 * cj + 25 * ck;
    double ev[4];
    for (int a = 0; a < 4; ++a) ev[a] = eta_s[base + slot_off(pmu, a)];
    const double qx = tile.ta * TT + ci, qy = tile.tb * TT + cj, qz = tile.tc * TT + ck;
    for (int q = 0; q < 4; ++q) {
      double K[3][3], hr, rinv, x[3];
      qp_geometry<double, BLEND>(G, n, p0, p1, p2, q, qx, qy, qz, K, hr, rinv, x);
      double etaq = 0.0;
      for (int a = 0; a < 4; ++a) etaq += (a == q ? QA : QB) * ev[a];
      w[(lin * 4 + q) * kMassSlots + t] = C0 * hr * hr * hr / etaq;
    }
  }
}

mfs_status mass_weights(mfs_problem* P, int lvl, double* w) {
  mfs_mesh* M = P->mesh;
  const LevelData& L = M->levels[lvl];
  cudaStream_t s = M->ctx->stream;
  dim3 grid(L.n_tiles, kMacroCells);
  ApplyParams<double> prm = sweep_params<double>(P, lvl);
  if (M->host.blending) k_mass_weights<true><<<grid, 128, 0, s>>>(prm, w);
  else k_mass_weights<false><<<grid, 128, 0, s>>>(prm, w);
  MFS_CUDA(cudaGetLastError());
  return MFS_OK;
}

// y = M_{1/eta} p from the stored weights: with p(q) = sum_b lambda_b(q) p_b,
// y_a = sum_q w_q lambda_a(q) p(q) (DIAG: sum_q w_q lambda_a(q)^2)
template <typename T, bool DIAG>
__global__ void __launch_bounds__(128) k_mass_sweep_w(const ApplyParams<T> P, const T* __restrict__ w,
                                                      const T* __restrict__ pin, T* __restrict__ y,
                                                      const double* __restrict__ active) {
  if (active && !(*active > 0.0)) return;
  __shared__ T ps[NSLOT1], ys[NSLOT1];
  __shared__ int gid[NSLOT1];
  const int m = blockIdx.y, tidx = blockIdx.x;
  const size_t lin = (size_t)m * gridDim.x + tidx;
  const Tile tile = P.tiles[tidx];
  for (int s = threadIdx.x; s < NSLOT1; s += blockDim.x) {
    const int id = P.ids1[lin * NSLOT1 + s];
    gid[s] = id;
    ps[s] = (!DIAG && id >= 0) ? pin[id] : T(0);
    ys[s] = T(0);
  }
  __syncthreads();
  const T QA = T(MFS_QA), QB = T(MFS_QB);
  const int2 cinfo = P.classes[tile.cls];
  const T* wt = w + lin * 4 * kMassSlots;
  for (int t = threadIdx.x; t < cinfo.y; t += blockDim.x) {
    const int code = P.tets[cinfo.x + t];
    const int ci = code & 15, cj = (code >> 4) & 15, ck = (code >> 8) & 15, pmu = code >> 12;
    const int base = ci + 5 * cj + 25 * ck;
    int sl[4];
    T wq[4], pv[4];
    for (int a = 0; a < 4; ++a) {
      sl[a] = base + slot_off(pmu, a);
      wq[a] = wt[a * kMassSlots + t];
      pv[a] = ps[sl[a]];
    }
    if (DIAG) {
      const T sw = wq[0] + wq[1] + wq[2] + wq[3];
      for (int a = 0; a < 4; ++a) atomicAdd(&ys[sl[a]], QB * QB * sw + (QA * QA - QB * QB) * wq[a]);
    } else {
      const T psum = pv[0] + pv[1] + pv[2] + pv[3];
      T wp[4], swp = T(0);
      for (int q = 0; q < 4; ++q) {
        wp[q] = wq[q] * (QB * psum + (QA - QB) * pv[q]);
        swp += wp[q];
      }
      for (int a = 0; a < 4; ++a) atomicAdd(&ys[sl[a]], QB * swp + (QA - QB) * wp[a]);
    }
  }
  __syncthreads();
  for (int s = threadIdx.x; s < NSLOT1; s += blockDim.x)
    if (gid[s] >= 0) atomicAdd(&y[gid[s]], ys[s]);
}

template <typename T>
mfs_status mass_apply_w(mfs_problem* P, int lvl, const T* w, const T* pin, T* y, int diag_only, const double* active,
                        int zero_out) {
  mfs_mesh* M = P->mesh;
  const LevelData& L = M->levels[lvl];
  cudaStream_t s = M->ctx->stream;
  if (zero_out) MFS_CUDA(cudaMemsetAsync(y, 0, sizeof(T) * (size_t)L.nb1.total, s));
  dim3 grid(L.n_tiles, kMacroCells);
  ApplyParams<T> prm = sweep_params<T>(P, lvl);
  if (diag_only) k_mass_sweep_w<T, true><<<grid, 128, 0, s>>>(prm, w, pin, y, active);
  else k_mass_sweep_w<T, false><<<grid, 128, 0, s>>>(prm, w, pin, y, active);
  MFS_CUDA(cudaGetLastError());
  return MFS_OK;
}
template mfs_status mass_apply_w<float>(mfs_problem*, int, const float*, const float*, float*, int, const double*, int);
template mfs_status mass_apply_w<double>(mfs_problem*, int, const double*, const double*, double*, int,
                                         const double*, int);

template mfs_status mass_apply<float>(mfs_problem*, int, const float*, float*, int, const double*, int);
template mfs_status mass_apply<double>(mfs_problem*, int, const double*, double*, int, const double*, int);

// Coarse operator (A_c + n n^T on free-slip nodes) assembled column by column with the FP64
// sweep, then inverted in place.
mfs_status coarse_inverse(mfs_problem* P, int lvl, const BoundaryList& B, double* A, double* work) {
  mfs_mesh* M = P->mesh;
  const LevelData& L = M->levels[lvl];
  cudaStream_t s = M->ctx->stream;
  const int64_t N = 3 * (int64_t)L.nb2.total;
  double* e = work;
  double* colk = work + N;
  for (int64_t j = 0; j < N; ++j) {
    k_unit<<<blocks_for(N), 256, 0, s>>>(N, j, e);
    MFS_TRY(launch_apply<double>(P, lvl, OP_A, 1, 0, e, nullptr, A + j * N, nullptr, nullptr));
  }
  if (B.nb) k_regularise_normals<<<blocks_for(B.nb), 256, 0, s>>>(B.nb, B.ids, B.kind, B.nrm64, L.nb2.total, A);
  gj_invert((int)N, A, colk, s);
  MFS_CUDA(cudaGetLastError());
  return MFS_OK;
}

}  // namespace mfs

namespace mfs {

// ------------------------------------------------------------------------- device-side CG
// Scalars of a device-resident CG (slots of a double array, see solver.h CG_*).
__global__ void k_cg_init(double* __restrict__ sc) {
  sc[CG_IT] = 0.0;
  sc[CG_ACTIVE] = (sc[CG_RR0] > 0.0 && sc[CG_RZ] > 0.0) ? 1.0 : 0.0;
  sc[CG_ALPHA] = sc[CG_BETA] = 0.0;
}

template <typename T>
void CgDev<T>::init(double* sc, cudaStream_t s) {
  k_cg_init<<<1, 1, 0, s>>>(sc);
}
// Grid-wide sums of K quantities in one pass: per-thread partials in T, warps add in T
// (FP32 lanes are 64x the FP64 rate here), the block's warps and then the grid's blocks
// in FP64; the last block to arrive adds the block partials in a fixed order
// (deterministic).  All K sums share each barrier: one __syncthreads per level.
template <int K, typename T>
__device__ __forceinline__ void block_partials(T (&v)[K], double* part) {
  __shared__ double red[K][32];
#pragma unroll
  for (int k = 0; k < K; ++k)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < K; ++k) red[k][w] = (double)v[k];
  __syncthreads();
  if (threadIdx.x < K) {
    double s = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[threadIdx.x][i];
    part[threadIdx.x * gridDim.x + blockIdx.x] = s;
    __threadfence();
  }
}
// after block_partials: true in the last block to arrive (the counter is left zeroed)
__device__ __forceinline__ bool last_block_arrived(unsigned* counter) {
  __shared__ bool last;
  __syncthreads();
  if (threadIdx.x == 0) {
    last = atomicAdd(counter, 1u) == gridDim.x - 1;
    if (last) *counter = 0u;
  }
  __syncthreads();
  return last;
}
// in the last block: warp k adds quantity k over the blocks; out (shared) gets the K sums
template <int K>
__device__ __forceinline__ void grid_final(const double* part, double* out) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nb = gridDim.x;
  if (w < K) {
    double a = 0.0;
    for (int i = lane; i < nb; i += 32) a += __ldcg(part + w * nb + i);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    if (lane == 0) out[w] = a;
  }
  __syncthreads();
}
template <typename T>
__global__ void k_mcg_dots(int64_t n, const T* __restrict__ p, const T* __restrict__ q, double* __restrict__ part,
                           unsigned* __restrict__ counter, double* __restrict__ sc) {
  if (!(sc[CG_ACTIVE] > 0.0)) return;   // the same for every block: set by earlier launches
  T sq_t = T(0), spq_t = T(0);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i0 < n; i0 += 4 * stride) {
    T pv[4], qv[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int64_t i = i0 + k * stride;
      pv[k] = i < n ? p[i] : T(0);
      qv[k] = i < n ? q[i] : T(0);
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      sq_t += qv[k];
      spq_t += pv[k] * qv[k];
    }
  }
  T v[2] = {sq_t, spq_t};
  block_partials<2>(v, part);
  if (!last_block_arrived(counter)) return;
  __shared__ double f[2];
  grid_final<2>(part, f);
  if (threadIdx.x == 0) {
    sc[CG_MEANQ] = f[0] / (double)n;
    sc[CG_PQ] = f[1];             // p is mean-free: p.(q - mean q) = p.q
    const bool ok = f[1] > 0.0;
    sc[CG_ALPHA] = ok ? sc[CG_RZ] / f[1] : 0.0;
    if (!ok) sc[CG_ACTIVE] = 0.0;
  }
}
template <typename T>
__global__ void k_mcg_update(int64_t n, const T* __restrict__ p, T* __restrict__ q, T* __restrict__ x,
                             T* __restrict__ r, T* __restrict__ z, const T* __restrict__ dinv,
                             double* __restrict__ part, unsigned* __restrict__ counter, double* __restrict__ sc,
                             double tol2, double maxit) {
  if (!(sc[CG_ACTIVE] > 0.0)) return;
  const T a = (T)sc[CG_ALPHA], mq = (T)sc[CG_MEANQ];
  T srr_t = T(0), srz_t = T(0), sz_t = T(0), sr_t = T(0);
  // four grid-strided elements per round, all loads before the first store: twenty loads
  // in flight per thread instead of one element's latency after another
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i0 < n; i0 += 4 * stride) {
    T pv[4], qv[4], xv[4], rv[4], dv[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int64_t i = i0 + k * stride;
      if (i < n) {
        pv[k] = p[i];
        qv[k] = q[i];
        xv[k] = x[i];
        rv[k] = r[i];
        dv[k] = dinv[i];
      }
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int64_t i = i0 + k * stride;
      if (i < n) {
        x[i] = xv[k] + a * pv[k];
        const T ri = rv[k] - a * (qv[k] - mq);
        q[i] = T(0);
        r[i] = ri;
        const T zi = dv[k] * ri;
        z[i] = zi;
        srr_t += ri * ri;
        srz_t += ri * zi;
        sz_t += zi;
        sr_t += ri;
      }
    }
  }
  T v[4] = {srr_t, srz_t, sz_t, sr_t};
  block_partials<4>(v, part);
  if (!last_block_arrived(counter)) return;
  __shared__ double f[4];
  grid_final<4>(part, f);
  if (threadIdx.x == 0) {
    const double meanz = f[2] / (double)n;
    const double rzn = f[1] - meanz * f[3];   // r . (z - mean z)
    sc[CG_RR] = f[0];
    sc[CG_MEANZ] = meanz;
    sc[CG_RZN] = rzn;
    sc[CG_BETA] = rzn / sc[CG_RZ];
    sc[CG_RZ] = rzn;
    sc[CG_IT] += 1.0;
    if (!(f[0] > tol2 * sc[CG_RR0]) || sc[CG_IT] >= maxit || !(rzn > 0.0)) sc[CG_ACTIVE] = 0.0;
  }
}
template <typename T>
__global__ void k_mcg_p(int64_t n, const T* __restrict__ z, T* __restrict__ p, const double* __restrict__ sc) {
  if (!(sc[CG_ACTIVE] > 0.0)) return;
  const T b = (T)sc[CG_BETA], mz = (T)sc[CG_MEANZ];
  GRID_STRIDE(i, n) p[i] = (z[i] - mz) + b * p[i];
}
template <typename T>
void CgDev<T>::mass_dots(int64_t n, const T* p, const T* q, double* part, unsigned* counter, double* sc,
                         cudaStream_t s) {
  k_mcg_dots<T><<<blocks_for(n, 256, kMassRedBlocks), 256, 0, s>>>(n, p, q, part, counter, sc);
}
template <typename T>
void CgDev<T>::mass_update(int64_t n, const T* p, T* q, T* x, T* r, T* z, const T* dinv, double* part,
                           unsigned* counter, double* sc, double tol2, int maxit, cudaStream_t s) {
  k_mcg_update<T><<<blocks_for(n, 256, kMassRedBlocks), 256, 0, s>>>(n, p, q, x, r, z, dinv, part, counter, sc,
                                                                     tol2, (double)maxit);
}
template <typename T>
void CgDev<T>::mass_pupd(int64_t n, const T* z, T* p, const double* sc, cudaStream_t s) {
  k_mcg_p<T><<<blocks_for(n), 256, 0, s>>>(n, z, p, sc);
}
template struct CgDev<float>;
template struct CgDev<double>;

}  // namespace mfs

namespace mfs {

// ------------------------------------------------------------------------- adjoint gradient
// dJ/d(log eta_k) = -eta_k lam^T (dA/d eta_k) u with A linear in the P1 viscosity:
// (dA/d eta_k)_ij = sum_q 2 w|det J| psi_k(q) eps(phi_j):eps(phi_i).  u is the full forward
// velocity (with its Dirichlet values), lam the constrained adjoint velocity.
__global__ void __launch_bounds__(128) k_grad_sweep(const ApplyParams<double> P, int blend, const double* __restrict__ u,
                                                    const double* __restrict__ lam, double* __restrict__ g) {
  __shared__ double gs[NSLOT1];
  __shared__ int gid1[NSLOT1];
  const int m = blockIdx.y, tidx = blockIdx.x;
  const size_t lin = (size_t)m * gridDim.x + tidx;
  const Tile tile = P.tiles[tidx];
  const MacroGeom<double>& G = P.geom[m];
  const int n = P.n;
  const int64_t n2 = P.n_p2;
  for (int s = threadIdx.x; s < NSLOT1; s += blockDim.x) {
    gs[s] = 0.0;
    gid1[s] = P.ids1[lin * NSLOT1 + s];
  }
  __syncthreads();
  const double QA = MFS_QA, QB = MFS_QB;
  const double C0 = G.absdet / (24.0 * n * (double)n * n);
  const int2 cinfo = P.classes[tile.cls];
  const int* tab2 = P.ids2 + lin * NSLOT2;
  for (int t = threadIdx.x; t < cinfo.y; t += blockDim.x) {
    const int code = P.tets[cinfo.x + t];
    const int ci = code & 15, cj = (code >> 4) & 15, ck = (code >> 8) & 15, pmu = code >> 12;
    const int p0 = (0x221100 >> (4 * pmu)) & 3, p1 = (0x102021 >> (4 * pmu)) & 3, p2 = (0x010212 >> (4 * pmu)) & 3;
    const int S1 = 1 << p0, S2 = S1 | (1 << p1);
    const int base = ci + 5 * cj + 25 * ck;
    int slot[10];
    slot[0] = base;
    slot[1] = base + sub_off(S1);
    slot[2] = base + sub_off(S2);
    slot[3] = base + sub_off(7);
    slot[4] = S1 * kSub + base;
    slot[5] = S2 * kSub + base;
    slot[6] = 7 * kSub + base;
    slot[7] = (S1 ^ S2) * kSub + base + sub_off(S1);
    slot[8] = (S1 ^ 7) * kSub + base + sub_off(S1);
    slot[9] = (S2 ^ 7) * kSub + base + sub_off(S2);
    double uv[10][3], lv[10][3];
    for (int a = 0; a < 10; ++a) {
      const int64_t id = slot_node(tab2[slot[a]]);
      for (int c = 0; c < 3; ++c) {
        uv[a][c] = u[c * n2 + id];
        lv[a][c] = lam[c * n2 + id];
      }
    }
    const double qx = tile.ta * TT + ci, qy = tile.tb * TT + cj, qz = tile.tc * TT + ck;
    double out[4] = {0, 0, 0, 0};
    for (int q = 0; q < 4; ++q) {
      double K[3][3], hr, rinv, x[3];
      if (blend) qp_geometry<double, true>(G, n, p0, p1, p2, q, qx, qy, qz, K, hr, rinv, x);
      else qp_geometry<double, false>(G, n, p0, p1, p2, q, qx, qy, qz, K, hr, rinv, x);
      const double lam_q[4] = {q == 0 ? QA : QB, q == 1 ? QA : QB, q == 2 ? QA : QB, q == 3 ? QA : QB};
      // gradients (scaled) of u and lam: sum_a value_a (x) (lattice grad of phi_a) K
      double Gu[3][3] = {{0}}, Gl[3][3] = {{0}};
      for (int a = 0; a < 10; ++a) {
        double gl[3];
        p2_lat_grad(a, lam_q, gl);
        double gx[3];
        for (int d = 0; d < 3; ++d) gx[d] = gl[0] * K[0][d] + gl[1] * K[1][d] + gl[2] * K[2][d];
        for (int c = 0; c < 3; ++c)
          for (int d = 0; d < 3; ++d) {
            Gu[c][d] += uv[a][c] * gx[d];
            Gl[c][d] += lv[a][c] * gx[d];
          }
      }
      const double tu = (Gu[0][0] + Gu[1][1] + Gu[2][2]) / 3.0, tl = (Gl[0][0] + Gl[1][1] + Gl[2][2]) / 3.0;
      double contr = 0.0;
      for (int c = 0; c < 3; ++c)
        for (int d = 0; d < 3; ++d) {
          const double eu = 0.5 * (Gu[c][d] + Gu[d][c]) - (c == d ? tu : 0.0);
          const double el = 0.5 * (Gl[c][d] + Gl[d][c]) - (c == d ? tl : 0.0);
          contr += eu * el;
        }
      // w|det J| s^2 = C0 hr ; dA/d eta contributes 2 psi_k
      const double wq = 2.0 * C0 * hr * contr;
      for (int k = 0; k < 4; ++k) out[k] += wq * lam_q[k];
    }
    for (int k = 0; k < 4; ++k) atomicAdd(&gs[slot[k]], out[k]);
  }
  __syncthreads();
  for (int s = threadIdx.x; s < NSLOT1; s += blockDim.x)
    if (gid1[s] >= 0) atomicAdd(&g[gid1[s]], gs[s]);
}

__global__ void k_scale_by_minus_eta(int64_t n, const double* __restrict__ eta, double* __restrict__ g) {
  GRID_STRIDE(i, n) g[i] = -eta[i] * g[i];
}

mfs_status grad_log_eta(mfs_problem* P, int lvl, const double* u, const double* lam, double* g) {
  mfs_mesh* M = P->mesh;
  const LevelData& L = M->levels[lvl];
  cudaStream_t s = M->ctx->stream;
  MFS_CUDA(cudaMemsetAsync(g, 0, sizeof(double) * (size_t)L.nb1.total, s));
  dim3 grid(L.n_tiles, kMacroCells);
  ApplyParams<double> prm = sweep_params<double>(P, lvl);
  k_grad_sweep<<<grid, 128, 0, s>>>(prm, M->host.blending, u, lam, g);
  k_scale_by_minus_eta<<<blocks_for(L.nb1.total), 256, 0, s>>>(L.nb1.total, P->eta64[lvl], g);
  MFS_CUDA(cudaGetLastError());
  return MFS_OK;
}

}  // namespace mfs

namespace mfs {

// ------------------------------------------------------------------------- buoyancy load vector
// f_(a,c) = scale sum_q w|det J| rho(r_q) T_q (x_q/|x_q|)_c phi_a(q); T nodal P2 (FP64), rho from
// the d ln rho / dr table integrated exactly (piecewise linear) with rho(r_surf) = 1.
__global__ void __launch_bounds__(128) k_buoyancy_sweep(const ApplyParams<double> P, int blend, const double* __restrict__ T,
                                                        double scale, double r_surf, double* __restrict__ f) {
  __shared__ double fs[3 * NSLOT2];
  const int m = blockIdx.y, tidx = blockIdx.x;
  const size_t lin = (size_t)m * gridDim.x + tidx;
  const Tile tile = P.tiles[tidx];
  const MacroGeom<double>& G = P.geom[m];
  const int n = P.n;
  const int64_t n2 = P.n_p2;
  const int* tab2 = P.ids2 + lin * NSLOT2;
  for (int s = threadIdx.x; s < 3 * NSLOT2; s += blockDim.x) fs[s] = 0.0;
  __syncthreads();
  const double QA = MFS_QA, QB = MFS_QB;
  const double C0 = G.absdet / (24.0 * n * (double)n * n);
  const int2 cinfo = P.classes[tile.cls];
  for (int t = threadIdx.x; t < cinfo.y; t += blockDim.x) {
    const int code = P.tets[cinfo.x + t];
    const int ci = code & 15, cj = (code >> 4) & 15, ck = (code >> 8) & 15, pmu = code >> 12;
    const int p0 = perm_at(pmu, 0), p1 = perm_at(pmu, 1), p2 = perm_at(pmu, 2);
    const int base = ci + 5 * cj + 25 * ck;
    double Tv[10];
    for (int a = 0; a < 10; ++a) Tv[a] = T[slot_node(tab2[base + slot_off(pmu, a)])];
    const double qx = tile.ta * TT + ci, qy = tile.tb * TT + cj, qz = tile.tc * TT + ck;
    double out[10][3];
    for (int a = 0; a < 10; ++a) out[a][0] = out[a][1] = out[a][2] = 0.0;
    for (int q = 0; q < 4; ++q) {
      double K[3][3], hr, rinv, x[3];
      if (blend) qp_geometry<double, true>(G, n, p0, p1, p2, q, qx, qy, qz, K, hr, rinv, x);
      else qp_geometry<double, false>(G, n, p0, p1, p2, q, qx, qy, qz, K, hr, rinv, x);
      const double lam[4] = {q == 0 ? QA : QB, q == 1 ? QA : QB, q == 2 ? QA : QB, q == 3 ? QA : QB};
      double phi[10];
      for (int a = 0; a < 4; ++a) phi[a] = lam[a] * (2 * lam[a] - 1);
      phi[4] = 4 * lam[0] * lam[1];
      phi[5] = 4 * lam[0] * lam[2];
      phi[6] = 4 * lam[0] * lam[3];
      phi[7] = 4 * lam[1] * lam[2];
      phi[8] = 4 * lam[1] * lam[3];
      phi[9] = 4 * lam[2] * lam[3];
      double Tq = 0.0;
      for (int a = 0; a < 10; ++a) Tq += phi[a] * Tv[a];
      const double h = x[0] * G.nh[0] + x[1] * G.nh[1] + x[2] * G.nh[2];
      const double rad = blend ? h / G.delta : 1.0 / rinv;
      const double W = C0 * hr * hr * hr;
      const double rho = rho_of(P.dlnrho, P.n_dlnrho, rad, (double)P.r_cmb, r_surf);
      const double c = scale * W * rho * Tq * rinv;
      for (int a = 0; a < 10; ++a)
        for (int d = 0; d < 3; ++d) out[a][d] += c * x[d] * phi[a];
    }
    for (int a = 0; a < 10; ++a)
      for (int d = 0; d < 3; ++d) atomicAdd(&fs[d * NSLOT2 + base + slot_off(pmu, a)], out[a][d]);
  }
  __syncthreads();
  for (int s = threadIdx.x; s < NSLOT2; s += blockDim.x) {
    const int code = tab2[s];
    if (code < 0) continue;
    const int64_t id = slot_node(code);
    for (int d = 0; d < 3; ++d) atomicAdd(&f[d * n2 + id], fs[d * NSLOT2 + s]);
  }
}

mfs_status rhs_buoyancy(mfs_problem* P, int lvl, const double* T, double scale, double* f) {
  mfs_mesh* M = P->mesh;
  const LevelData& L = M->levels[lvl];
  cudaStream_t s = M->ctx->stream;
  MFS_CUDA(cudaMemsetAsync(f, 0, sizeof(double) * 3 * (size_t)L.nb2.total, s));
  dim3 grid(L.n_tiles, kMacroCells);
  ApplyParams<double> prm = sweep_params<double>(P, lvl);
  prm.dlnrho = P->d_dlnrho64;
  prm.n_dlnrho = P->n_dlnrho;
  prm.r_cmb = M->host.r_cmb;
  k_buoyancy_sweep<<<grid, 128, 0, s>>>(prm, M->host.blending, T, scale, M->host.r_surf, f);
  MFS_CUDA(cudaGetLastError());
  return MFS_OK;
}

}  // namespace mfs

using namespace mfs;

mfs_status mfs_rhs_buoyancy(mfs_problem* P, const double* T_p2, double scale, double* f) {
  if (!P || !T_p2 || !f) {
    set_error("null argument");
    return MFS_EINVAL;
  }
  return rhs_buoyancy(P, P->mesh->l_max, T_p2, scale, f);
}
