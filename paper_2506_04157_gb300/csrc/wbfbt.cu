// Operators of the weighted BFBT Schur approximation (arxiv 2506.04157, Sec. 5.2.3,
// Eq. schurWBFBT in its rescaled form
//     S_w^-1 ~ K_{1/sqrt(eta_l)}^-1 (B M_{sqrt(eta_l)}^-1 A M_{sqrt(eta_r)}^-1 B^T) K_{1/sqrt(eta_r)}^-1,
// eta_{l,r} = a_{l,r}^2 eta on the elements touching the outer surface, eta elsewhere):
//  * K_{1/sqrt(eta_a)}: the P1 Laplacian with coefficient 1/sqrt(eta_a(x_q)) (eta the P1
//    interpolant at the quadrature points) and natural boundary conditions.  Each micro-tet
//    stores the 6 off-diagonal entries of its element matrix, computed once per viscosity
//    in FP64; the diagonal follows from the zero row sums, so constants lie exactly in the
//    kernel of the applied operator in either precision.
//  * its geometric multigrid: P1 interpolation (coincident vertex 1, coarse-edge ends 1/2)
//    and its transpose, Jacobi-preconditioned Chebyshev smoothing with FP64 power-iteration
//    intervals, and the exact FP64 inverse of K_c + (mean diag / n) 1 1^T on the coarsest
//    level (the Neumann operator's constant null space lifted).
//  * the lumped vector mass M_{sqrt(eta_a)}: each element's consistent-mass diagonal
//    (weight sqrt(eta_a)) scaled to the element's total mass (Hinton-Rock-Zienkiewicz
//    lumping), inverted and replicated over the three velocity components.
#include <cmath>
#include <cstring>
#include <vector>

#include "apply.cuh"
#include "library.h"
#include "qp_geometry.cuh"
#include "solver.h"
#include "sweep_params.cuh"

namespace mfs {

constexpr int kPoissonEntries = 6;   // off-diagonal element entries: 01 02 03 12 13 23
constexpr int kMaxSides = 8;

inline int64_t poisson_weight_count(const LevelData& L) {
  return (int64_t)kMacroCells * L.n_tiles * kPoissonEntries * kMassSlots;
}

struct PoissonSide {
  double a = 1.0;
  int version = -1;
  std::vector<double*> kw64, dinv64;   // per level: element entries, inverse diagonal
  std::vector<float*> kw32, dinv32;
  std::vector<double> lo, hi;          // Chebyshev intervals per level
  double* cinv = nullptr;              // coarsest level: (K_c + lift)^-1, nc x nc
  double* minv64 = nullptr;            // lumped M_{sqrt(eta_a)}^-1, [3][n_p2] of the finest level
  float* minv32 = nullptr;
  double* cdinv64 = nullptr;           // consistent M_{sqrt(eta_a)}: inverse diagonal, [3][n_p2]
  float* cdinv32 = nullptr;            // (allocated on first use)
  int cversion = -1;
};

template <typename T>
struct PoissonWork {
  std::vector<T*> b, x, r, t, d;       // per level, n_p1(l) entries
};

struct PoissonMG {
  int l_min = -1, l_max = -1, nc = 0;
  std::vector<Csr> P, R;               // index l: interpolation l-1 -> l (fine rows) and its transpose
  PoissonWork<double> w64;
  PoissonWork<float> w32;
  std::vector<PoissonSide> sides;
  double* red = nullptr;               // [kRedBlocks] partials + result
  double* hpin = nullptr;              // pinned host scalar
  double* colk = nullptr;              // Gauss-Jordan column, nc entries
  double* d2 = nullptr;                // lumped mass diagonal, n_p2 of the finest level
  std::vector<void*> owned;
};

namespace {
inline int nblk(int64_t n, int threads = 256, int cap = 8192) {
  int64_t b = (n + threads - 1) / threads;
  if (b < 1) b = 1;
  return (int)(b < cap ? b : cap);
}
}  // namespace

#define WB_STRIDE(i, n) \
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (n); i += (int64_t)gridDim.x * blockDim.x)

// ------------------------------------------------------------------------- kernels
// Vertex s (< 125) of a tile's P1 block and P2 slot s (parity class 0) are the same lattice
// point, so the P2 table's geometric class marks the vertices on the outer surface.
__device__ __forceinline__ int on_surface(const int* ids2, size_t lin, int s) {
  const int code = ids2[lin * NSLOT2 + s];
  return (code >= 0 && slot_class(code) == 1) ? 1 : 0;
}

// Element entries k_ab (a < b) of K_{1/sqrt(eta_a)}: sum_q w|det J| grad psi_a . grad psi_b
// / sqrt(s eta_q), s = a^2 on tets with a surface vertex.  With the lattice-frame P1
// gradients GL and the rows K of qp_geometry the physical gradients are (GL K) / hr and
// w|det J| = C0 hr^3.
template <bool BLEND>
__global__ void __launch_bounds__(128) k_poisson_weights(const ApplyParams<double> P, double a2,
                                                         double* __restrict__ kw) {
  __shared__ double eta_s[NSLOT1];
  __shared__ int surf_s[NSLOT1];
  const int m = blockIdx.y, tidx = blockIdx.x;
  const size_t lin = (size_t)m * gridDim.x + tidx;
  const Tile tile = P.tiles[tidx];
  const MacroGeom<double>& G = P.geom[m];
  const int n = P.n;
  for (int s = threadIdx.x; s < NSLOT1; s += blockDim.x) {
    const int id = P.ids1[lin * NSLOT1 + s];
    eta_s[s] = id >= 0 ? P.eta[id] : 1.0;
    surf_s[s] = on_surface(P.ids2, lin, s);
  }
  __syncthreads();
  const double QA = MFS_QA, QB = MFS_QB;
  const double C0 = G.absdet / (24.0 * n * (double)n * n);
  const double GL[4][3] = {{-1, 0, 0}, {1, -1, 0}, {0, 1, -1}, {0, 0, 1}};
  const int2 cinfo = P.classes[tile.cls];
  double* out = kw + lin * kPoissonEntries * kMassSlots;
  for (int t = threadIdx.x; t < cinfo.y; t += blockDim.x) {
    const int code = P.tets[cinfo.x + t];
    const int ci = code & 15, cj = (code >> 4) & 15, ck = (code >> 8) & 15, pmu = code >> 12;
    const int p0 = perm_at(pmu, 0), p1 = perm_at(pmu, 1), p2 = perm_at(pmu, 2);
    const int base = ci + 5 * cj + 25 * ck;
    double ev[4];
    int on = 0;
    for (int a = 0; a < 4; ++a) {
      const int sl = base + slot_off(pmu, a);
      ev[a] = eta_s[sl];
      on |= surf_s[sl];
    }
    const double sc = on ? a2 : 1.0;
    const double qx = tile.ta * TT + ci, qy = tile.tb * TT + cj, qz = tile.tc * TT + ck;
    double kab[kPoissonEntries] = {0, 0, 0, 0, 0, 0};
    for (int q = 0; q < 4; ++q) {
      double K[3][3], hr, rinv, x[3];
      qp_geometry<double, BLEND>(G, n, p0, p1, p2, q, qx, qy, qz, K, hr, rinv, x);
      double etaq = 0.0;
      for (int a = 0; a < 4; ++a) etaq += (a == q ? QA : QB) * ev[a];
      const double wq = C0 * hr / sqrt(sc * etaq);
      double g[4][3];
      for (int a = 0; a < 4; ++a)
        for (int d = 0; d < 3; ++d) g[a][d] = GL[a][0] * K[0][d] + GL[a][1] * K[1][d] + GL[a][2] * K[2][d];
      int e = 0;
      for (int a = 0; a < 4; ++a)
        for (int b = a + 1; b < 4; ++b, ++e) kab[e] += wq * (g[a][0] * g[b][0] + g[a][1] * g[b][1] + g[a][2] * g[b][2]);
    }
    for (int e = 0; e < kPoissonEntries; ++e) out[e * kMassSlots + t] = kab[e];
  }
}

// y += K p from the stored entries: y_a = sum_{b != a} k_ab (p_b - p_a)
// (DIAG: y += diag(K), diag_a = -sum_{b != a} k_ab)
template <typename T, bool DIAG>
__global__ void __launch_bounds__(128) k_poisson_sweep(const ApplyParams<T> P, const T* __restrict__ kw,
                                                       const T* __restrict__ pin, T* __restrict__ y) {
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
  const int2 cinfo = P.classes[tile.cls];
  const T* wt = kw + lin * kPoissonEntries * kMassSlots;
  for (int t = threadIdx.x; t < cinfo.y; t += blockDim.x) {
    const int code = P.tets[cinfo.x + t];
    const int ci = code & 15, cj = (code >> 4) & 15, ck = (code >> 8) & 15, pmu = code >> 12;
    const int base = ci + 5 * cj + 25 * ck;
    int sl[4];
    for (int a = 0; a < 4; ++a) sl[a] = base + slot_off(pmu, a);
    T k[kPoissonEntries];
    for (int e = 0; e < kPoissonEntries; ++e) k[e] = wt[e * kMassSlots + t];
    T y0, y1, y2, y3;
    if (DIAG) {
      y0 = -(k[0] + k[1] + k[2]);
      y1 = -(k[0] + k[3] + k[4]);
      y2 = -(k[1] + k[3] + k[5]);
      y3 = -(k[2] + k[4] + k[5]);
    } else {
      const T p0 = ps[sl[0]], p1 = ps[sl[1]], p2 = ps[sl[2]], p3 = ps[sl[3]];
      const T d01 = p1 - p0, d02 = p2 - p0, d03 = p3 - p0, d12 = p2 - p1, d13 = p3 - p1, d23 = p3 - p2;
      y0 = k[0] * d01 + k[1] * d02 + k[2] * d03;
      y1 = -k[0] * d01 + k[3] * d12 + k[4] * d13;
      y2 = -k[1] * d02 - k[3] * d12 + k[5] * d23;
      y3 = -k[2] * d03 - k[4] * d13 - k[5] * d23;
    }
    atomicAdd(&ys[sl[0]], y0);
    atomicAdd(&ys[sl[1]], y1);
    atomicAdd(&ys[sl[2]], y2);
    atomicAdd(&ys[sl[3]], y3);
  }
  __syncthreads();
  for (int s = threadIdx.x; s < NSLOT1; s += blockDim.x)
    if (gid[s] >= 0) atomicAdd(&y[gid[s]], ys[s]);
}

// d += HRZ-lumped P2 mass of weight sqrt(s eta_q): per tet m_aa = sum_q w|det J| sqrt(s eta_q)
// phi_a(q)^2, scaled by (sum_q w|det J| sqrt(s eta_q)) / (sum_a m_aa)
template <bool BLEND>
__global__ void __launch_bounds__(128) k_vmass_lumped(const ApplyParams<double> P, double a2,
                                                      double* __restrict__ d) {
  __shared__ double ds[NSLOT2];
  __shared__ double eta_s[NSLOT1];
  __shared__ int surf_s[NSLOT1];
  const int m = blockIdx.y, tidx = blockIdx.x;
  const size_t lin = (size_t)m * gridDim.x + tidx;
  const Tile tile = P.tiles[tidx];
  const MacroGeom<double>& G = P.geom[m];
  const int n = P.n;
  for (int s = threadIdx.x; s < NSLOT2; s += blockDim.x) ds[s] = 0.0;
  for (int s = threadIdx.x; s < NSLOT1; s += blockDim.x) {
    const int id = P.ids1[lin * NSLOT1 + s];
    eta_s[s] = id >= 0 ? P.eta[id] : 1.0;
    surf_s[s] = on_surface(P.ids2, lin, s);
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
    int slot[10];
    for (int a = 0; a < 10; ++a) slot[a] = base + slot_off(pmu, a);
    double ev[4];
    int on = 0;
    for (int a = 0; a < 4; ++a) {
      ev[a] = eta_s[slot[a]];      // vertex slots lie in parity class 0: P1 slot = P2 slot
      on |= surf_s[slot[a]];
    }
    const double sc = on ? a2 : 1.0;
    const double qx = tile.ta * TT + ci, qy = tile.tb * TT + cj, qz = tile.tc * TT + ck;
    double acc[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    double tot = 0.0;
    for (int q = 0; q < 4; ++q) {
      double K[3][3], hr, rinv, x[3];
      qp_geometry<double, BLEND>(G, n, p0, p1, p2, q, qx, qy, qz, K, hr, rinv, x);
      double etaq = 0.0;
      for (int a = 0; a < 4; ++a) etaq += (a == q ? QA : QB) * ev[a];
      const double wq = C0 * hr * hr * hr * sqrt(sc * etaq);
      double lam[4];
      for (int a = 0; a < 4; ++a) lam[a] = a == q ? QA : QB;
      double phi[10];
      for (int a = 0; a < 4; ++a) phi[a] = lam[a] * (2.0 * lam[a] - 1.0);
      for (int e = 0; e < 6; ++e) {
        const int i0 = e < 3 ? 0 : (e < 5 ? 1 : 2);
        const int i1 = e < 3 ? e + 1 : (e < 5 ? e - 1 : 3);
        phi[4 + e] = 4.0 * lam[i0] * lam[i1];
      }
      for (int a = 0; a < 10; ++a) acc[a] += wq * phi[a] * phi[a];
      tot += wq;
    }
    double tr = 0.0;
    for (int a = 0; a < 10; ++a) tr += acc[a];
    const double f = tot / tr;
    for (int a = 0; a < 10; ++a) atomicAdd(&ds[slot[a]], acc[a] * f);
  }
  __syncthreads();
  for (int s = threadIdx.x; s < NSLOT2; s += blockDim.x) {
    const int code = P.ids2[lin * NSLOT2 + s];
    if (code < 0) continue;
    atomicAdd(&d[slot_node(code)], ds[s]);
  }
}

// m[c][i] = 1 / d[i] for the three velocity components
__global__ void k_minv_expand(int64_t n2, const double* __restrict__ d, double* __restrict__ m64,
                              float* __restrict__ m32) {
  WB_STRIDE(i, n2) {
    const double v = 1.0 / d[i];
    for (int c = 0; c < 3; ++c) {
      m64[c * n2 + i] = v;
      m32[c * n2 + i] = (float)v;
    }
  }
}

__global__ void k_add_scalar(int64_t n, double a, double* __restrict__ x) { WB_STRIDE(i, n) x[i] += a; }

__global__ void k_wb_seed(int64_t n, double* __restrict__ v) {
  WB_STRIDE(i, n) {
    uint64_t z = (uint64_t)i * 0x9E3779B97F4A7C15ull + 0x2545F4914F6CDD1Dull;   // splitmix64 finaliser
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    v[i] = (double)(z >> 11) * (1.0 / 9007199254740992.0) - 0.5;
  }
}

// y = R (b - t): restriction of a residual (R: coarse rows)
template <typename T>
__global__ void k_p1_restrict(int nrows, const int* __restrict__ rp, const int* __restrict__ ci,
                              const T* __restrict__ w, const T* __restrict__ b, const T* __restrict__ t,
                              T* __restrict__ y) {
  WB_STRIDE(r, nrows) {
    T s = T(0);
    for (int k = rp[r]; k < rp[r + 1]; ++k) s += w[k] * (b[ci[k]] - t[ci[k]]);
    y[r] = s;
  }
}

// x += P xc (P: fine rows)
template <typename T>
__global__ void k_p1_prolong_add(int nrows, const int* __restrict__ rp, const int* __restrict__ ci,
                                 const T* __restrict__ w, const T* __restrict__ xc, T* __restrict__ x) {
  WB_STRIDE(r, nrows) {
    T s = T(0);
    for (int k = rp[r]; k < rp[r + 1]; ++k) s += w[k] * xc[ci[k]];
    x[r] += s;
  }
}

// first degree of a Chebyshev step: r = b (mode 0) or b - t (mode 1); d = cz dinv r;
// x = (mode 0 ? 0 : x) + d
template <typename T>
__global__ void k_pcheb_first(int64_t n, int mode, const T* __restrict__ b, const T* __restrict__ t,
                              T* __restrict__ r, const T* __restrict__ dinv, T* __restrict__ d, T* __restrict__ x,
                              T cz) {
  WB_STRIDE(i, n) {
    const T ri = mode ? b[i] - t[i] : b[i];
    const T di = cz * dinv[i] * ri;
    r[i] = ri;
    d[i] = di;
    x[i] = (mode ? x[i] : T(0)) + di;
  }
}
// later degrees: r -= t; d = cd d + cz dinv r; x += d
template <typename T>
__global__ void k_pcheb_next(int64_t n, const T* __restrict__ t, T* __restrict__ r, const T* __restrict__ dinv,
                             T* __restrict__ d, T* __restrict__ x, T cz, T cd) {
  WB_STRIDE(i, n) {
    const T ri = r[i] - t[i];
    const T di = cd * d[i] + cz * dinv[i] * ri;
    r[i] = ri;
    d[i] = di;
    x[i] += di;
  }
}

// ------------------------------------------------------------------------- host side

template <typename T>
static PoissonWork<T>& pwork(PoissonMG* W);
template <>
PoissonWork<double>& pwork<double>(PoissonMG* W) { return W->w64; }
template <>
PoissonWork<float>& pwork<float>(PoissonMG* W) { return W->w32; }
template <typename T>
static const T* side_kw(const PoissonSide& S, int l);
template <>
const double* side_kw<double>(const PoissonSide& S, int l) { return S.kw64[l]; }
template <>
const float* side_kw<float>(const PoissonSide& S, int l) { return S.kw32[l]; }
template <typename T>
static const T* side_dinv(const PoissonSide& S, int l);
template <>
const double* side_dinv<double>(const PoissonSide& S, int l) { return S.dinv64[l]; }
template <>
const float* side_dinv<float>(const PoissonSide& S, int l) { return S.dinv32[l]; }

template <typename T>
static mfs_status palloc(PoissonMG* W, T** p, int64_t n, cudaStream_t s) {
  const size_t bytes = sizeof(T) * (size_t)(n > 0 ? n : 1);
  cudaError_t e = cudaMalloc((void**)p, bytes);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(weighted-BFBT operators)");
  W->owned.push_back(*p);
  MFS_CUDA(cudaMemsetAsync(*p, 0, bytes, s));
  return MFS_OK;
}

void pmg_destroy(PoissonMG* W) {
  if (!W) return;
  for (void* p : W->owned) cudaFree(p);
  if (W->hpin) cudaFreeHost(W->hpin);
  delete W;
}

static double pdot(PoissonMG* W, int64_t n, const double* x, const double* y, cudaStream_t s) {
  Blas<double>::dot_async(n, x, y, W->red, W->red + kRedBlocks, s);
  cudaMemcpyAsync(W->hpin, W->red + kRedBlocks, sizeof(double), cudaMemcpyDeviceToHost, s);
  cudaStreamSynchronize(s);
  return W->hpin[0];
}

// CSR upload of (row, col, weight) triplets
static mfs_status upload_csr(PoissonMG* W, int nrows, int ncols, const std::vector<int>& rows,
                             const std::vector<int>& cols, const std::vector<double>& vals, Csr& C, cudaStream_t s) {
  std::vector<int> rp(nrows + 1, 0), ci(rows.size());
  std::vector<double> w(rows.size());
  std::vector<float> w32(rows.size());
  for (int r : rows) rp[r + 1]++;
  for (int i = 0; i < nrows; ++i) rp[i + 1] += rp[i];
  std::vector<int> pos(rp.begin(), rp.end() - 1);
  for (size_t k = 0; k < rows.size(); ++k) {
    const int at = pos[rows[k]]++;
    ci[at] = cols[k];
    w[at] = vals[k];
    w32[at] = (float)vals[k];
  }
  C.nrows = nrows;
  C.ncols = ncols;
  MFS_TRY(palloc(W, &C.rp, nrows + 1, s));
  MFS_TRY(palloc(W, &C.ci, (int64_t)ci.size(), s));
  MFS_TRY(palloc(W, &C.w64, (int64_t)w.size(), s));
  MFS_TRY(palloc(W, &C.w32, (int64_t)w32.size(), s));
  MFS_CUDA(cudaMemcpyAsync(C.rp, rp.data(), sizeof(int) * rp.size(), cudaMemcpyHostToDevice, s));
  MFS_CUDA(cudaMemcpyAsync(C.ci, ci.data(), sizeof(int) * ci.size(), cudaMemcpyHostToDevice, s));
  MFS_CUDA(cudaMemcpyAsync(C.w64, w.data(), sizeof(double) * w.size(), cudaMemcpyHostToDevice, s));
  MFS_CUDA(cudaMemcpyAsync(C.w32, w32.data(), sizeof(float) * w32.size(), cudaMemcpyHostToDevice, s));
  MFS_CUDA(cudaStreamSynchronize(s));   // the host vectors go out of scope
  return MFS_OK;
}

// transfers and work vectors for the multigrid range of the problem's hierarchy
static mfs_status pmg_structure(mfs_problem* Pb) {
  const int l_min = mg_lmin(Pb);
  if (l_min < 0) {
    set_error("multigrid not set up (call mfs_setup_multigrid after mfs_set_viscosity)");
    return MFS_EINVAL;
  }
  if (Pb->pmg && Pb->pmg->l_min == l_min) return MFS_OK;
  if (Pb->pmg) {
    pmg_destroy(Pb->pmg);
    Pb->pmg = nullptr;
  }
  mfs_mesh* M = Pb->mesh;
  cudaStream_t s = M->ctx->stream;
  PoissonMG* W = new PoissonMG;
  Pb->pmg = W;
  const int L = M->l_max;
  W->l_min = l_min;
  W->l_max = L;
  W->nc = M->levels[l_min].nb1.total;
  W->P.resize(L + 1);
  W->R.resize(L + 1);
  for (int l = l_min + 1; l <= L; ++l) {
    std::vector<int> tv, tj;
    std::vector<double> tw;
    p1_transfer_triplets(M, l, tv, tj, tw);
    const int nf = M->levels[l].nb1.total, nc = M->levels[l - 1].nb1.total;
    MFS_TRY(upload_csr(W, nf, nc, tj, tv, tw, W->P[l], s));
    MFS_TRY(upload_csr(W, nc, nf, tv, tj, tw, W->R[l], s));
  }
  auto grow = [&](auto& V, int l, int64_t n) -> mfs_status {
    V.resize(L + 1, nullptr);
    return palloc(W, &V[l], n, s);
  };
  for (int l = l_min; l <= L; ++l) {
    const int64_t n1 = M->levels[l].nb1.total;
    for (auto* V : {&W->w64.b, &W->w64.x, &W->w64.r, &W->w64.t, &W->w64.d}) MFS_TRY(grow(*V, l, n1));
    for (auto* V : {&W->w32.b, &W->w32.x, &W->w32.r, &W->w32.t, &W->w32.d}) MFS_TRY(grow(*V, l, n1));
  }
  MFS_TRY(palloc(W, &W->red, kRedBlocks + 16, s));
  MFS_TRY(palloc(W, &W->colk, W->nc, s));
  MFS_TRY(palloc(W, &W->d2, M->levels[L].nb2.total, s));
  MFS_CUDA(cudaMallocHost((void**)&W->hpin, 8 * sizeof(double)));
  return MFS_OK;
}

template <typename T>
mfs_status poisson_apply(mfs_problem* Pb, int side, int lvl, const T* p, T* y) {
  PoissonMG* W = Pb->pmg;
  const PoissonSide& S = W->sides[side];
  const LevelData& Lv = Pb->mesh->levels[lvl];
  cudaStream_t s = Pb->mesh->ctx->stream;
  MFS_CUDA(cudaMemsetAsync(y, 0, sizeof(T) * (size_t)Lv.nb1.total, s));
  dim3 grid(Lv.n_tiles, kMacroCells);
  k_poisson_sweep<T, false><<<grid, 128, 0, s>>>(sweep_params<T>(Pb, lvl), side_kw<T>(S, lvl), p, y);
  MFS_CUDA(cudaGetLastError());
  return MFS_OK;
}

static mfs_status lumped_into(mfs_problem* Pb, double a, double* d) {
  mfs_mesh* M = Pb->mesh;
  const int L = M->l_max;
  const LevelData& Lv = M->levels[L];
  cudaStream_t s = M->ctx->stream;
  MFS_CUDA(cudaMemsetAsync(d, 0, sizeof(double) * (size_t)Lv.nb2.total, s));
  dim3 grid(Lv.n_tiles, kMacroCells);
  const ApplyParams<double> prm = sweep_params<double>(Pb, L);
  if (M->host.blending) k_vmass_lumped<true><<<grid, 128, 0, s>>>(prm, a * a, d);
  else k_vmass_lumped<false><<<grid, 128, 0, s>>>(prm, a * a, d);
  MFS_CUDA(cudaGetLastError());
  return MFS_OK;
}

// element entries, Jacobi diagonals, Chebyshev intervals, coarse inverse and lumped mass
static mfs_status side_numeric(mfs_problem* Pb, int side) {
  PoissonMG* W = Pb->pmg;
  PoissonSide& S = W->sides[side];
  mfs_mesh* M = Pb->mesh;
  cudaStream_t s = M->ctx->stream;
  const int L = W->l_max;
  std::vector<double> cdiag;
  for (int l = W->l_min; l <= L; ++l) {
    const LevelData& Lv = M->levels[l];
    const int64_t n1 = Lv.nb1.total, cnt = poisson_weight_count(Lv);
    dim3 grid(Lv.n_tiles, kMacroCells);
    const ApplyParams<double> prm = sweep_params<double>(Pb, l);
    MFS_CUDA(cudaMemsetAsync(S.kw64[l], 0, sizeof(double) * (size_t)cnt, s));
    if (M->host.blending) k_poisson_weights<true><<<grid, 128, 0, s>>>(prm, S.a * S.a, S.kw64[l]);
    else k_poisson_weights<false><<<grid, 128, 0, s>>>(prm, S.a * S.a, S.kw64[l]);
    MFS_CUDA(cudaGetLastError());
    Blas<float>::convert_from_f64(cnt, S.kw64[l], S.kw32[l], s);
    MFS_CUDA(cudaMemsetAsync(S.dinv64[l], 0, sizeof(double) * (size_t)n1, s));
    k_poisson_sweep<double, true><<<grid, 128, 0, s>>>(prm, S.kw64[l], nullptr, S.dinv64[l]);
    MFS_CUDA(cudaGetLastError());
    if (l == W->l_min) {
      cdiag.resize(n1);
      MFS_CUDA(cudaMemcpyAsync(cdiag.data(), S.dinv64[l], sizeof(double) * n1, cudaMemcpyDeviceToHost, s));
    }
    Blas<float>::convert_from_f64(n1, S.dinv64[l], S.dinv32[l], s);
    Blas<double>::recip(n1, S.dinv64[l], s);
    Blas<float>::recip(n1, S.dinv32[l], s);
    if (l > W->l_min) {
      // largest eigenvalue of D^-1 K: 15 FP64 power iterations from a seeded vector
      double* x = W->w64.x[l];
      double* t = W->w64.t[l];
      k_wb_seed<<<nblk(n1), 256, 0, s>>>(n1, x);
      double lam = 0.0;
      for (int it = 0; it < 15; ++it) {
        const double nv = std::sqrt(pdot(W, n1, x, x, s));
        if (!(nv > 0.0) || !std::isfinite(nv)) {
          set_error("power iteration on K_{1/sqrt(eta)} broke down on level %d", l);
          return MFS_ENAN;
        }
        Blas<double>::axpby(n1, 1.0 / nv, x, 0.0, x, s);
        MFS_TRY(poisson_apply<double>(Pb, side, l, x, t));
        Blas<double>::mul(n1, t, S.dinv64[l], x, s);
        lam = std::sqrt(pdot(W, n1, x, x, s));
      }
      S.hi[l] = 1.2 * lam;
      S.lo[l] = S.hi[l] / 20.0;
    }
  }
  // coarsest level: K_c column by column, lifted along the constants, inverted in FP64
  const int nc = W->nc;
  double* e = W->w64.x[W->l_min];
  for (int j = 0; j < nc; ++j) {
    unit_vector(nc, j, e, s);
    MFS_TRY(poisson_apply<double>(Pb, side, W->l_min, e, S.cinv + (int64_t)j * nc));
  }
  MFS_CUDA(cudaStreamSynchronize(s));
  double tr = 0.0;
  for (double v : cdiag) tr += v;
  k_add_scalar<<<nblk((int64_t)nc * nc), 256, 0, s>>>((int64_t)nc * nc, tr / nc / nc, S.cinv);
  gj_invert(nc, S.cinv, W->colk, s);
  // lumped M_{sqrt(eta_a)} on the finest level
  MFS_TRY(lumped_into(Pb, S.a, W->d2));
  const int64_t n2 = M->levels[L].nb2.total;
  k_minv_expand<<<nblk(n2), 256, 0, s>>>(n2, W->d2, S.minv64, S.minv32);
  MFS_CUDA(cudaStreamSynchronize(s));
  MFS_CUDA(cudaGetLastError());
  S.version = Pb->version;
  return MFS_OK;
}

mfs_status pmg_side(mfs_problem* Pb, double a, int* side) {
  if (!(a > 0.0) || !std::isfinite(a)) {
    set_error("the weighted-BFBT surface scaling must be positive and finite");
    return MFS_EINVAL;
  }
  MFS_TRY(pmg_structure(Pb));
  PoissonMG* W = Pb->pmg;
  for (size_t i = 0; i < W->sides.size(); ++i)
    if (W->sides[i].a == a) {
      *side = (int)i;
      if (W->sides[i].version != Pb->version) return side_numeric(Pb, (int)i);
      return MFS_OK;
    }
  if ((int)W->sides.size() >= kMaxSides) {
    set_error("at most %d distinct weighted-BFBT surface scalings per problem", kMaxSides);
    return MFS_EINVAL;
  }
  mfs_mesh* M = Pb->mesh;
  cudaStream_t s = M->ctx->stream;
  const int L = W->l_max;
  PoissonSide S;
  S.a = a;
  S.kw64.assign(L + 1, nullptr);
  S.kw32.assign(L + 1, nullptr);
  S.dinv64.assign(L + 1, nullptr);
  S.dinv32.assign(L + 1, nullptr);
  S.lo.assign(L + 1, 0.0);
  S.hi.assign(L + 1, 0.0);
  for (int l = W->l_min; l <= L; ++l) {
    const int64_t cnt = poisson_weight_count(M->levels[l]), n1 = M->levels[l].nb1.total;
    MFS_TRY(palloc(W, &S.kw64[l], cnt, s));
    MFS_TRY(palloc(W, &S.kw32[l], cnt, s));
    MFS_TRY(palloc(W, &S.dinv64[l], n1, s));
    MFS_TRY(palloc(W, &S.dinv32[l], n1, s));
  }
  MFS_TRY(palloc(W, &S.cinv, (int64_t)W->nc * W->nc, s));
  MFS_TRY(palloc(W, &S.minv64, 3 * (int64_t)M->levels[L].nb2.total, s));
  MFS_TRY(palloc(W, &S.minv32, 3 * (int64_t)M->levels[L].nb2.total, s));
  W->sides.push_back(S);
  *side = (int)W->sides.size() - 1;
  return side_numeric(Pb, *side);
}

// Jacobi-preconditioned Chebyshev smoothing of K x = b on level l (the iteration of the
// A-block smoother): `steps` steps of `deg` applications each; x_zero: x = 0 on entry.
template <typename T>
static mfs_status pcheb(mfs_problem* Pb, int side, int l, T* x, const T* b, int steps, int deg, bool x_zero) {
  PoissonMG* W = Pb->pmg;
  const PoissonSide& S = W->sides[side];
  PoissonWork<T>& Wk = pwork<T>(W);
  cudaStream_t s = Pb->mesh->ctx->stream;
  const int64_t n = Pb->mesh->levels[l].nb1.total;
  const double lo = S.lo[l], hi = S.hi[l];
  const double theta = 0.5 * (hi + lo), delta = 0.5 * (hi - lo), sigma1 = theta / delta;
  const T* dinv = side_dinv<T>(S, l);
  for (int st = 0; st < steps; ++st) {
    int mode = 0;
    if (st > 0 || !x_zero) {
      MFS_TRY(poisson_apply<T>(Pb, side, l, x, Wk.t[l]));
      mode = 1;
    }
    k_pcheb_first<T><<<nblk(n), 256, 0, s>>>(n, mode, b, Wk.t[l], Wk.r[l], dinv, Wk.d[l], x, T(1.0 / theta));
    double rho = 1.0 / sigma1;
    for (int k = 2; k <= deg; ++k) {
      MFS_TRY(poisson_apply<T>(Pb, side, l, Wk.d[l], Wk.t[l]));
      const double rho_new = 1.0 / (2.0 * sigma1 - rho);
      k_pcheb_next<T><<<nblk(n), 256, 0, s>>>(n, Wk.t[l], Wk.r[l], dinv, Wk.d[l], x, T(2.0 * rho_new / delta),
                                              T(rho_new * rho));
      rho = rho_new;
    }
  }
  MFS_CUDA(cudaGetLastError());
  return MFS_OK;
}

template <typename T>
static mfs_status pvcycle(mfs_problem* Pb, int side, int l, T* x, const T* b, int m, int deg) {
  PoissonMG* W = Pb->pmg;
  const PoissonSide& S = W->sides[side];
  PoissonWork<T>& Wk = pwork<T>(W);
  cudaStream_t s = Pb->mesh->ctx->stream;
  if (l == W->l_min) {
    Blas<T>::gemv_f64(W->nc, S.cinv, b, x, s);
    return MFS_OK;
  }
  const int n = Pb->mesh->levels[l].nb1.total, nc = Pb->mesh->levels[l - 1].nb1.total;
  if (m == 0) Blas<T>::fill(n, T(0), x, s);
  MFS_TRY(pcheb<T>(Pb, side, l, x, b, m, deg, true));
  MFS_TRY(poisson_apply<T>(Pb, side, l, x, Wk.t[l]));
  const Csr& R = W->R[l];
  k_p1_restrict<T><<<nblk(nc), 256, 0, s>>>(nc, R.rp, R.ci, R.w<T>(), b, Wk.t[l], Wk.b[l - 1]);
  MFS_TRY(pvcycle<T>(Pb, side, l - 1, Wk.x[l - 1], Wk.b[l - 1], m, deg));
  const Csr& P = W->P[l];
  k_p1_prolong_add<T><<<nblk(n), 256, 0, s>>>(n, P.rp, P.ci, P.w<T>(), Wk.x[l - 1], x);
  MFS_TRY(pcheb<T>(Pb, side, l, x, b, m, deg, false));
  MFS_CUDA(cudaGetLastError());
  return MFS_OK;
}

template <typename T>
mfs_status poisson_vcycle(mfs_problem* Pb, int side, T* x, const T* b, int m, int deg) {
  return pvcycle<T>(Pb, side, Pb->pmg->l_max, x, b, m, deg);
}

template <>
const double* poisson_minv<double>(mfs_problem* Pb, int side) { return Pb->pmg->sides[side].minv64; }
template <>
const float* poisson_minv<float>(mfs_problem* Pb, int side) { return Pb->pmg->sides[side].minv32; }

mfs_status lumped_vmass(mfs_problem* Pb, double a, double* d) { return lumped_into(Pb, a, d); }

// Jacobi scaling of the consistent-mass CG: 1 / diag(M_{sqrt(eta_a)}) per velocity component
static mfs_status cmass_dinv(mfs_problem* Pb, int side) {
  PoissonMG* W = Pb->pmg;
  PoissonSide& S = W->sides[side];
  if (S.cversion == Pb->version) return MFS_OK;
  mfs_mesh* M = Pb->mesh;
  cudaStream_t s = M->ctx->stream;
  const int64_t n2 = M->levels[W->l_max].nb2.total;
  if (!S.cdinv64) {
    MFS_TRY(palloc(W, &S.cdinv64, 3 * n2, s));
    MFS_TRY(palloc(W, &S.cdinv32, 3 * n2, s));
  }
  MFS_TRY(wmass_apply<double>(Pb, S.a, nullptr, W->d2, 1));
  k_minv_expand<<<nblk(n2), 256, 0, s>>>(n2, W->d2, S.cdinv64, S.cdinv32);
  MFS_CUDA(cudaGetLastError());
  S.cversion = Pb->version;
  return MFS_OK;
}
template <>
mfs_status poisson_cmass_dinv<double>(mfs_problem* Pb, int side, const double** out) {
  MFS_TRY(cmass_dinv(Pb, side));
  *out = Pb->pmg->sides[side].cdinv64;
  return MFS_OK;
}
template <>
mfs_status poisson_cmass_dinv<float>(mfs_problem* Pb, int side, const float** out) {
  MFS_TRY(cmass_dinv(Pb, side));
  *out = Pb->pmg->sides[side].cdinv32;
  return MFS_OK;
}

template mfs_status poisson_apply<double>(mfs_problem*, int, int, const double*, double*);
template mfs_status poisson_apply<float>(mfs_problem*, int, int, const float*, float*);
template mfs_status poisson_vcycle<double>(mfs_problem*, int, double*, const double*, int, int);
template mfs_status poisson_vcycle<float>(mfs_problem*, int, float*, const float*, int, int);

}  // namespace mfs

using namespace mfs;

// ------------------------------------------------------------------------- C ABI (part)
mfs_status mfs_apply_poisson(mfs_problem* Pb, int lvl, mfs_prec prec, double a, const void* p, void* y) {
  if (!Pb || !p || !y) {
    set_error("null argument");
    return MFS_EINVAL;
  }
  const int l_min = mg_lmin(Pb);
  if (l_min < 0) {
    set_error("multigrid not set up (call mfs_setup_multigrid after mfs_set_viscosity)");
    return MFS_EINVAL;
  }
  if (lvl < l_min || lvl > Pb->mesh->l_max) {
    set_error("level %d outside the multigrid range [%d, %d]", lvl, l_min, Pb->mesh->l_max);
    return MFS_EINVAL;
  }
  int side = 0;
  MFS_TRY(pmg_side(Pb, a, &side));
  if (prec == MFS_F64) return poisson_apply<double>(Pb, side, lvl, (const double*)p, (double*)y);
  return poisson_apply<float>(Pb, side, lvl, (const float*)p, (float*)y);
}

mfs_status mfs_lumped_vmass(mfs_problem* Pb, double a, double* d) {
  if (!Pb || !d) {
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
  return lumped_vmass(Pb, a, d);
}
