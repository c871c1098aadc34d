// Multigrid hierarchy and Stokes solver (arxiv 2506.04157, Sec. 5.2):
//   * Sec. 5.2.2: CG on A preconditioned by a GMG V-cycle with Jacobi-preconditioned
//     Chebyshev smoothing (m pre/post steps of degree deg), diag(A) without P_v;
//   * Sec. 5.2.3, Eq. (schurV): V-cycle BFBT Schur approximation, its inner CG on
//     X = B A_C^-1 B^T preconditioned by CG on M_{1/eta};
//   * Sec. 5.2.1, Eq. (SymmetricUzawaStep1): symmetric Uzawa block preconditioner with
//     B + C in the pressure update;
//   * Sec. 5.2.4: FGMRES outer solver; FP32 inner solves wrapped in FP64 iterative
//     refinement (mixed = 1), an FP64 FGMRES preconditioned by the FP32 Uzawa step
//     (mixed = 2), or everything in FP64 (mixed = 0).
// Host code orchestrates the CUDA kernels; every vector operation runs on the device.
#include <algorithm>
#include <array>
#include <chrono>
#include <cmath>
#include <cstring>
#include <memory>
#include <new>

#include "apply.cuh"
#include "solver.h"

namespace mfs {

template <typename T>
struct Work {
  T *dinv = nullptr, *r = nullptr, *z = nullptr, *d = nullptr, *t = nullptr, *b = nullptr, *x = nullptr;
};

template <typename T>
struct Krylov {           // FGMRES / CG / Uzawa storage at the finest level
  int64_t N = 0;
  int m = 0;
  std::vector<T*> V, Z;
  T *w = nullptr, *ua = nullptr, *ub = nullptr, *uc = nullptr, *ud = nullptr;  // velocity temporaries
  T *pa = nullptr, *pb = nullptr, *pc = nullptr, *pd = nullptr, *pe = nullptr, *pf = nullptr;
  T *cg_r = nullptr, *cg_z = nullptr, *cg_p = nullptr, *cg_q = nullptr;        // velocity CG
  T *cgp_r = nullptr, *cgp_z = nullptr, *cgp_p = nullptr, *cgp_q = nullptr;    // pressure CG (X)
  T *cgm_r = nullptr, *cgm_z = nullptr, *cgm_p = nullptr, *cgm_q = nullptr;    // pressure CG (M)
  T *tmpu = nullptr, *tmpp = nullptr;
  T *rhs = nullptr, *sol = nullptr;                                             // FGMRES b and x
  T *ir_r = nullptr, *ir_y = nullptr, *ir_p = nullptr;                          // refinement (FP64)
};

struct MG {
  int l_min = 1, l_max = 0;
  std::vector<BoundaryList> bnd;
  std::vector<Csr> P, R;
  std::vector<double> lo, hi;
  std::vector<int> have_bounds;
  double* Ainv = nullptr;
  double* ainv_work = nullptr;
  int ncoarse = 0;
  std::vector<Work<float>> w32;
  std::vector<Work<double>> w64;
  double* mw64 = nullptr;       // stored quadrature weights of M_{1/eta} on the finest level
  float* mw32 = nullptr;
  double* mdinv64 = nullptr;
  float* mdinv32 = nullptr;
  double* red = nullptr;        // [kRedBlocks] partials + 8 scalars
  double* hpin = nullptr;       // pinned host scalar
  bool structure = false, numeric = false;
  Krylov<float> k32;
  Krylov<double> k64;
  std::vector<void*> owned;     // device allocations to free
  // device-resident CG: scalar slots, a capture stream and cached graphs of CG chunks
  double* cgsc = nullptr;
  double* mcg_part = nullptr;   // [4 * kMassRedBlocks] block partials of the mass CG
  unsigned* mcg_counter = nullptr;
  cudaStream_t cap = nullptr;
  struct Graph {
    int prec;
    const void* x;
    double tol;
    int maxit;
    cudaGraphExec_t exec;
  };
  std::vector<Graph> graphs;
  // captured V-cycles, keyed by precision, level, smoother shape and buffers; dropped
  // whenever the Chebyshev intervals change, stale when the sweep tuning changes
  struct VGraph {
    int prec, l, steps, deg;
    const void* x;
    const void* b;
    int tuning_gen, uses;
    cudaGraphExec_t exec;
  };
  std::vector<VGraph> vgraphs;
};

static void drop_vgraphs(MG* G) {
  for (auto& g : G->vgraphs)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  G->vgraphs.clear();
}

static mfs_status dalloc(MG* G, void** p, size_t bytes) {
  cudaError_t e = cudaMalloc(p, bytes ? bytes : 16);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(solver workspace)");
  G->owned.push_back(*p);
  return MFS_OK;
}
template <typename T>
static mfs_status dalloc_zero(MG* G, T** p, int64_t n, cudaStream_t s) {
  MFS_TRY(dalloc(G, (void**)p, sizeof(T) * (size_t)n));
  MFS_CUDA(cudaMemsetAsync(*p, 0, sizeof(T) * (size_t)n, s));
  return MFS_OK;
}

void mg_destroy(MG* G) {
  if (!G) return;
  for (auto& g : G->graphs) cudaGraphExecDestroy(g.exec);
  drop_vgraphs(G);
  if (G->cap) cudaStreamDestroy(G->cap);
  for (void* p : G->owned) cudaFree(p);
  if (G->hpin) cudaFreeHost(G->hpin);
  delete G;
}

// ------------------------------------------------------------------------- structure
static void kuhn_bary(int A, int B, int C, int N, int i[4]) {
  i[0] = N - A;
  i[1] = A - B;
  i[2] = B - C;
  i[3] = C;
}

static mfs_status build_boundary(mfs_problem* Pb, int l, BoundaryList& BL, cudaStream_t s, MG* G) {
  const mfs_mesh* M = Pb->mesh;
  const int N = 2 << l;
  const Numbering nb = make_numbering(N);
  std::vector<char> seen(nb.total, 0);
  std::vector<int> ids;
  std::vector<int8_t> kind;
  std::vector<double> nrm;
  for (int m = 0; m < 60; ++m) {
    const MacroTopo& t = M->host.topo[m];
    for (int side = 0; side < 2; ++side) {
      const int mask = side == 0 ? t.topmask : t.botmask;
      const int bc = side == 0 ? Pb->bc_surface : Pb->bc_cmb;
      for (int i3 = 0; i3 <= N; ++i3)
        for (int i2 = 0; i2 <= N - i3; ++i2)
          for (int i1 = 0; i1 <= N - i3 - i2; ++i1) {
            const int i[4] = {N - i1 - i2 - i3, i1, i2, i3};
            bool on = true;
            for (int k = 0; k < 4; ++k)
              if (i[k] > 0 && !(mask >> k & 1)) on = false;
            if (!on) continue;
            const int id = lattice_id(t, nb, m, i[0], i[1], i[2], i[3]);
            if (seen[id]) continue;
            seen[id] = 1;
            double x[3];
            M->host.straight_point(m, i, N, x);
            const double r = std::sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
            ids.push_back(id);
            kind.push_back(bc == BC_DIRICHLET ? 1 : 2);
            for (int c = 0; c < 3; ++c) nrm.push_back(x[c] / r);
          }
    }
  }
  BL.nb = (int)ids.size();
  std::vector<float> n32(nrm.begin(), nrm.end());
  std::vector<int> nodemap(nb.total, -1);
  for (size_t k = 0; k < ids.size(); ++k) nodemap[ids[k]] = (int)k;
  MFS_TRY(dalloc(G, (void**)&BL.nodemap, sizeof(int) * nodemap.size()));
  MFS_CUDA(cudaMemcpyAsync(BL.nodemap, nodemap.data(), sizeof(int) * nodemap.size(), cudaMemcpyHostToDevice, s));
  MFS_TRY(dalloc(G, (void**)&BL.ids, sizeof(int) * ids.size()));
  MFS_TRY(dalloc(G, (void**)&BL.kind, ids.size()));
  MFS_TRY(dalloc(G, (void**)&BL.nrm64, sizeof(double) * nrm.size()));
  MFS_TRY(dalloc(G, (void**)&BL.nrm32, sizeof(float) * nrm.size()));
  MFS_CUDA(cudaMemcpyAsync(BL.ids, ids.data(), sizeof(int) * ids.size(), cudaMemcpyHostToDevice, s));
  MFS_CUDA(cudaMemcpyAsync(BL.kind, kind.data(), kind.size(), cudaMemcpyHostToDevice, s));
  MFS_CUDA(cudaMemcpyAsync(BL.nrm64, nrm.data(), sizeof(double) * nrm.size(), cudaMemcpyHostToDevice, s));
  MFS_CUDA(cudaMemcpyAsync(BL.nrm32, n32.data(), sizeof(float) * n32.size(), cudaMemcpyHostToDevice, s));
  MFS_CUDA(cudaStreamSynchronize(s));
  return MFS_OK;
}

// Prolongation from level l-1 to level l (P2 nodes): every fine node is a quarter point
// (barycentrics s/4, sum s = 4) of a coarse micro-tet; its value is the coarse P2
// interpolant there.  The first coarse tet met defines the row (all give the same value).
// CSR (host) of the P2 prolongation from level l-1 to level l: every fine P2 node (a quarter
// point of a coarse micro-tet) takes the coarse P2 interpolant there, the nonzero basis values
static mfs_status prolongation_csr(const mfs_mesh* M, int l, std::vector<int>& rp, std::vector<int>& ci,
                                   std::vector<double>& w) {
  static const int PERM[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
  static const int LE[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}};
  const int n = 1 << (l - 1);          // coarse micro-tets per macro edge
  const int Nc = 2 * n, Nf = 4 * n;
  const Numbering nbc = make_numbering(Nc), nbf = make_numbering(Nf);
  // quarter points and the 10 P2 basis values there
  std::vector<std::array<int, 4>> sub;
  std::vector<std::array<double, 10>> phi;
  for (int s3 = 0; s3 <= 4; ++s3)
    for (int s2 = 0; s2 <= 4 - s3; ++s2)
      for (int s1 = 0; s1 <= 4 - s3 - s2; ++s1) {
        const std::array<int, 4> sp = {4 - s1 - s2 - s3, s1, s2, s3};
        std::array<double, 10> ph;
        double lam[4];
        for (int a = 0; a < 4; ++a) lam[a] = sp[a] / 4.0;
        for (int a = 0; a < 4; ++a) ph[a] = lam[a] * (2 * lam[a] - 1);
        for (int e = 0; e < 6; ++e) ph[4 + e] = 4 * lam[LE[e][0]] * lam[LE[e][1]];
        sub.push_back(sp);
        phi.push_back(ph);
      }
  std::vector<int> cnt(nbf.total, 0);
  std::vector<int> cols((size_t)nbf.total * 10, -1);
  std::vector<double> vals((size_t)nbf.total * 10, 0.0);
  std::vector<char> seen(nbf.total, 0);
  for (int m = 0; m < 60; ++m) {
    const MacroTopo& t = M->host.topo[m];
    for (int a = 0; a < n; ++a)
      for (int b = 0; b <= a; ++b)
        for (int c = 0; c <= b; ++c)
          for (int pm = 0; pm < 6; ++pm) {
            int K[4][3];
            K[0][0] = a;
            K[0][1] = b;
            K[0][2] = c;
            bool ok = true;
            for (int k = 1; k < 4; ++k) {
              for (int d = 0; d < 3; ++d) K[k][d] = K[k - 1][d];
              K[k][PERM[pm][k - 1]] += 1;
              if (!(K[k][0] >= K[k][1] && K[k][1] >= K[k][2])) ok = false;
            }
            if (!ok) continue;
            int cid[10];
            for (int v = 0; v < 4; ++v) {
              int i[4];
              kuhn_bary(2 * K[v][0], 2 * K[v][1], 2 * K[v][2], Nc, i);
              cid[v] = lattice_id(t, nbc, m, i[0], i[1], i[2], i[3]);
            }
            for (int e = 0; e < 6; ++e) {
              const int u = LE[e][0], v = LE[e][1];
              int i[4];
              kuhn_bary(K[u][0] + K[v][0], K[u][1] + K[v][1], K[u][2] + K[v][2], Nc, i);
              cid[4 + e] = lattice_id(t, nbc, m, i[0], i[1], i[2], i[3]);
            }
            for (size_t q = 0; q < sub.size(); ++q) {
              int F[3] = {0, 0, 0};
              for (int v = 0; v < 4; ++v)
                for (int d = 0; d < 3; ++d) F[d] += sub[q][v] * K[v][d];
              int i[4];
              kuhn_bary(F[0], F[1], F[2], Nf, i);
              const int fid = lattice_id(t, nbf, m, i[0], i[1], i[2], i[3]);
              if (seen[fid]) continue;
              seen[fid] = 1;
              int k = 0;
              for (int z = 0; z < 10; ++z)
                if (phi[q][z] != 0.0) {
                  cols[(size_t)fid * 10 + k] = cid[z];
                  vals[(size_t)fid * 10 + k] = phi[q][z];
                  ++k;
                }
              cnt[fid] = k;
            }
          }
  }
  for (int i = 0; i < nbf.total; ++i)
    if (!seen[i]) {
      set_error("internal: prolongation misses fine node %d on level %d", i, l);
      return MFS_EINVAL;
    }
  // CSR of P
  rp.assign(nbf.total + 1, 0);
  for (int i = 0; i < nbf.total; ++i) rp[i + 1] = rp[i] + cnt[i];
  const int nnz = rp[nbf.total];
  ci.assign(nnz, 0);
  w.assign(nnz, 0.0);
  for (int i = 0; i < nbf.total; ++i)
    for (int k = 0; k < cnt[i]; ++k) {
      ci[rp[i] + k] = cols[(size_t)i * 10 + k];
      w[rp[i] + k] = vals[(size_t)i * 10 + k];
    }
  return MFS_OK;
}

static mfs_status build_transfer(mfs_problem* Pb, int l, Csr& P, Csr& R, cudaStream_t s, MG* G) {
  const mfs_mesh* M = Pb->mesh;
  const Numbering nbc = make_numbering(2 << (l - 1)), nbf = make_numbering(4 << (l - 1));
  std::vector<int> rp, ci;
  std::vector<double> w;
  MFS_TRY(prolongation_csr(M, l, rp, ci, w));
  const int nnz = rp[nbf.total];
  // CSR of P^T (restriction), rows in increasing fine index per coarse row
  std::vector<int> rrp(nbc.total + 1, 0);
  for (int k = 0; k < nnz; ++k) rrp[ci[k] + 1]++;
  for (int i = 0; i < nbc.total; ++i) rrp[i + 1] += rrp[i];
  std::vector<int> pos(rrp.begin(), rrp.end() - 1);
  std::vector<int> rci(nnz);
  std::vector<double> rw(nnz);
  for (int i = 0; i < nbf.total; ++i)
    for (int k = rp[i]; k < rp[i + 1]; ++k) {
      const int c = ci[k];
      rci[pos[c]] = i;
      rw[pos[c]] = w[k];
      pos[c]++;
    }
  auto upload = [&](Csr& X, int nrows, int ncols, const std::vector<int>& xrp, const std::vector<int>& xci,
                    const std::vector<double>& xw) -> mfs_status {
    X.nrows = nrows;
    X.ncols = ncols;
    std::vector<float> w32(xw.begin(), xw.end());
    MFS_TRY(dalloc(G, (void**)&X.rp, sizeof(int) * xrp.size()));
    MFS_TRY(dalloc(G, (void**)&X.ci, sizeof(int) * xci.size()));
    MFS_TRY(dalloc(G, (void**)&X.w64, sizeof(double) * xw.size()));
    MFS_TRY(dalloc(G, (void**)&X.w32, sizeof(float) * xw.size()));
    MFS_CUDA(cudaMemcpyAsync(X.rp, xrp.data(), sizeof(int) * xrp.size(), cudaMemcpyHostToDevice, s));
    MFS_CUDA(cudaMemcpyAsync(X.ci, xci.data(), sizeof(int) * xci.size(), cudaMemcpyHostToDevice, s));
    MFS_CUDA(cudaMemcpyAsync(X.w64, xw.data(), sizeof(double) * xw.size(), cudaMemcpyHostToDevice, s));
    MFS_CUDA(cudaMemcpyAsync(X.w32, w32.data(), sizeof(float) * w32.size(), cudaMemcpyHostToDevice, s));
    MFS_CUDA(cudaStreamSynchronize(s));
    return MFS_OK;
  };
  MFS_TRY(upload(P, nbf.total, nbc.total, rp, ci, w));
  MFS_TRY(upload(R, nbc.total, nbf.total, rrp, rci, rw));
  return MFS_OK;
}

template <typename T>
static mfs_status alloc_work(MG* G, Work<T>& W, int64_t n3, cudaStream_t s) {
  MFS_TRY(dalloc_zero(G, &W.dinv, n3, s));
  MFS_TRY(dalloc_zero(G, &W.r, n3, s));
  MFS_TRY(dalloc_zero(G, &W.z, n3, s));
  MFS_TRY(dalloc_zero(G, &W.d, n3, s));
  MFS_TRY(dalloc_zero(G, &W.t, n3, s));
  MFS_TRY(dalloc_zero(G, &W.b, n3, s));
  MFS_TRY(dalloc_zero(G, &W.x, n3, s));
  return MFS_OK;
}

static mfs_status mg_structure(mfs_problem* Pb, int l_min) {
  mfs_mesh* M = Pb->mesh;
  cudaStream_t s = M->ctx->stream;
  if (Pb->mg && Pb->mg->structure && Pb->mg->l_min == l_min) return MFS_OK;
  if (Pb->mg) {
    mg_destroy(Pb->mg);
    Pb->mg = nullptr;
  }
  if (l_min < 0 || l_min > M->l_max) {
    set_error("l_min %d outside [0, l_max = %d]", l_min, M->l_max);
    return MFS_EINVAL;
  }
  MG* G = new (std::nothrow) MG;
  if (!G) {
    set_error("host allocation failed");
    return MFS_ENOMEM;
  }
  Pb->mg = G;
  G->l_min = l_min;
  G->l_max = M->l_max;
  const int L = M->l_max;
  G->bnd.resize(L + 1);
  G->P.resize(L + 1);
  G->R.resize(L + 1);
  G->lo.assign(L + 1, 0.0);
  G->hi.assign(L + 1, 0.0);
  G->have_bounds.assign(L + 1, 0);
  G->w32.resize(L + 1);
  G->w64.resize(L + 1);
  for (int l = l_min; l <= L; ++l) {
    MFS_TRY(build_boundary(Pb, l, G->bnd[l], s, G));
    if (l > l_min) MFS_TRY(build_transfer(Pb, l, G->P[l], G->R[l], s, G));
    const int64_t n3 = 3 * (int64_t)M->levels[l].nb2.total;
    MFS_TRY(alloc_work<float>(G, G->w32[l], n3, s));
    MFS_TRY(alloc_work<double>(G, G->w64[l], n3, s));
  }
  G->ncoarse = 3 * M->levels[l_min].nb2.total;
  MFS_TRY(dalloc(G, (void**)&G->Ainv, sizeof(double) * (size_t)G->ncoarse * G->ncoarse));
  MFS_TRY(dalloc(G, (void**)&G->ainv_work, sizeof(double) * 2 * (size_t)G->ncoarse));
  MFS_TRY(dalloc_zero(G, &G->mw64, mass_weight_count(M->levels[L]), s));
  MFS_TRY(dalloc_zero(G, &G->mw32, mass_weight_count(M->levels[L]), s));
  MFS_TRY(dalloc_zero(G, &G->mdinv64, M->levels[L].nb1.total, s));
  MFS_TRY(dalloc_zero(G, &G->mdinv32, M->levels[L].nb1.total, s));
  MFS_TRY(dalloc_zero(G, &G->red, kRedBlocks + 16, s));
  MFS_TRY(dalloc_zero(G, &G->cgsc, CG_NSLOTS, s));
  MFS_TRY(dalloc_zero(G, &G->mcg_part, 4 * kMassRedBlocks, s));
  MFS_TRY(dalloc_zero(G, &G->mcg_counter, 4, s));
  MFS_CUDA(cudaStreamCreateWithFlags(&G->cap, cudaStreamNonBlocking));
  MFS_CUDA(cudaMallocHost((void**)&G->hpin, 16 * sizeof(double)));
  G->structure = true;
  return MFS_OK;
}

// ------------------------------------------------------------------------- operators
template <typename T>
static Work<T>& work(MG* G, int l);
template <>
Work<float>& work<float>(MG* G, int l) { return G->w32[l]; }
template <>
Work<double>& work<double>(MG* G, int l) { return G->w64[l]; }

static double host_dot_result(MG* G, cudaStream_t s) {
  cudaMemcpyAsync(G->hpin, G->red + kRedBlocks, sizeof(double), cudaMemcpyDeviceToHost, s);
  cudaStreamSynchronize(s);
  return G->hpin[0];
}

template <typename T>
static double dot(MG* G, int64_t n, const T* x, const T* y, cudaStream_t s) {
  Blas<T>::dot_async(n, x, y, G->red, G->red + kRedBlocks, s);
  return host_dot_result(G, s);
}

// constrained A on level l
template <typename T>
static mfs_status applyA(mfs_problem* Pb, int l, const T* x, T* y) {
  return launch_apply<T>(Pb, l, OP_A, 1, 0, x, nullptr, y, nullptr, nullptr);
}
// the same into a buffer known to hold zeros
template <typename T>
static mfs_status applyA_acc(mfs_problem* Pb, int l, const T* x, T* y) {
  return launch_apply<T>(Pb, l, OP_A, 1, 0, x, nullptr, y, nullptr, nullptr, 0);
}

template <typename T>
static T* red_scalar(mfs_problem* Pb);
template <>
double* red_scalar<double>(mfs_problem* Pb) { return Pb->d_red64; }
template <>
float* red_scalar<float>(mfs_problem* Pb) { return Pb->d_red32; }

// P_p: subtract the arithmetic mean
template <typename T>
static mfs_status mean_free(mfs_problem* Pb, T* p, int64_t n) {
  cudaStream_t s = Pb->mesh->ctx->stream;
  T* red = red_scalar<T>(Pb);
  MFS_TRY(vec_sum<T>(p, n, red, red + kRedBlocks + 4, s));
  MFS_TRY(vec_sub_mean<T>(p, n, red + kRedBlocks + 4, s));
  return MFS_OK;
}

// adds the wall time of its scope to a millisecond counter
struct WallTimer {
  double& acc;
  std::chrono::steady_clock::time_point t0 = std::chrono::steady_clock::now();
  explicit WallTimer(double& a) : acc(a) {}
  ~WallTimer() { acc += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count(); }
};

// ------------------------------------------------------------------------- smoother / V-cycle
// Jacobi-preconditioned Chebyshev iteration (Saad, Iterative Methods, Alg. 12.1), `steps`
// steps of `deg` applications of A each.  Every application is one sweep into the level's
// buffer t (kept zeroed between uses) and one fused per-node update of r, d and x that also
// applies the boundary projections to d and x (the update is linear and x stays in the
// projected space).  x_zero: x = 0 on entry, so the first step needs no apply.
template <typename T>
static mfs_status chebyshev(mfs_problem* Pb, MG* G, int l, T* x, const T* b, int steps, int deg, bool x_zero) {
  cudaStream_t s = Pb->mesh->ctx->stream;
  Work<T>& W = work<T>(G, l);
  const int64_t n2 = Pb->mesh->levels[l].nb2.total;
  const double lo = G->lo[l], hi = G->hi[l];
  const double theta = 0.5 * (hi + lo), delta = 0.5 * (hi - lo), sigma1 = theta / delta;
  for (int st = 0; st < steps; ++st) {
    int mode = 0;                                                    // r = b
    if (st > 0 || !x_zero) {
      MFS_TRY(applyA_acc<T>(Pb, l, x, W.t));
      mode = 1;                                                      // r = b - A x
    }
    Blas<T>::cheb_update(n2, mode, b, W.t, W.r, W.dinv, W.d, x, T(1.0 / theta), T(0), G->bnd[l], s);   // d = z / theta
    double rho = 1.0 / sigma1;
    for (int k = 2; k <= deg; ++k) {
      MFS_TRY(applyA_acc<T>(Pb, l, W.d, W.t));
      const double rho_new = 1.0 / (2.0 * sigma1 - rho);
      Blas<T>::cheb_update(n2, 2, b, W.t, W.r, W.dinv, W.d, x, T(2.0 * rho_new / delta), T(rho_new * rho),
                           G->bnd[l], s);
      rho = rho_new;
    }
  }
  return MFS_OK;
}

// One V-cycle for A_c x = b on level l from x = 0; x is overwritten.
template <typename T>
static mfs_status vcycle_launch(mfs_problem* Pb, MG* G, int l, T* x, const T* b, int steps, int deg) {
  mfs_mesh* M = Pb->mesh;
  cudaStream_t s = M->ctx->stream;
  const int64_t n2 = M->levels[l].nb2.total;
  if (l == G->l_min) {
    Blas<T>::gemv_f64((int)(3 * n2), G->Ainv, b, x, s);
    Blas<T>::bproject(G->bnd[l], n2, x, s);
    return MFS_OK;
  }
  Work<T>& W = work<T>(G, l);
  Work<T>& C = work<T>(G, l - 1);
  const int64_t nc2 = M->levels[l - 1].nb2.total;
  MFS_TRY(chebyshev<T>(Pb, G, l, x, b, steps, deg, true));
  MFS_TRY(applyA_acc<T>(Pb, l, x, W.t));
  Blas<T>::restrict_residual(G->R[l], n2, b, W.t, C.b, G->bnd[l - 1], s);   // P_c P^T (b - A x)
  MFS_TRY(vcycle_launch<T>(Pb, G, l - 1, C.x, C.b, steps, deg));
  Blas<T>::prolong_add(G->P[l], nc2, C.x, x, W.t, G->bnd[l], s);   // x += P x_c, projected; t = 0
  MFS_TRY(chebyshev<T>(Pb, G, l, x, b, steps, deg, false));
  return MFS_OK;
}

// A V-cycle is a fixed launch sequence: from its second use on (the first one runs the
// kernels' lazy setup) it is replayed from a captured CUDA graph.  With per-sweep timing
// on, it is always launched eagerly.
template <typename T>
static mfs_status vcycle(mfs_problem* Pb, MG* G, int l, T* x, const T* b, int steps, int deg) {
  mfs_mesh* M = Pb->mesh;
  mfs_ctx* C = M->ctx;
  if (C->timing) return vcycle_launch<T>(Pb, G, l, x, b, steps, deg);
  const int prec = sizeof(T) == 8 ? 0 : 1;
  size_t k = 0;
  for (; k < G->vgraphs.size(); ++k) {
    const MG::VGraph& g = G->vgraphs[k];
    if (g.prec == prec && g.l == l && g.steps == steps && g.deg == deg && g.x == x && g.b == b) break;
  }
  if (k == G->vgraphs.size()) {
    if (G->vgraphs.size() >= 64) {   // many distinct caller buffers: start over
      drop_vgraphs(G);
      k = 0;
    }
    G->vgraphs.push_back({prec, l, steps, deg, x, b, M->tuning_gen, 0, nullptr});
  }
  MG::VGraph& g = G->vgraphs[k];
  if (g.exec && g.tuning_gen != M->tuning_gen) {
    cudaGraphExecDestroy(g.exec);
    g.exec = nullptr;
    g.uses = 0;
  }
  if (!g.exec) {
    if (g.uses++ == 0) return vcycle_launch<T>(Pb, G, l, x, b, steps, deg);
    cudaStream_t saved = C->stream;
    C->stream = G->cap;
    cudaError_t e = cudaStreamBeginCapture(G->cap, cudaStreamCaptureModeThreadLocal);
    mfs_status st = MFS_OK;
    if (e == cudaSuccess) st = vcycle_launch<T>(Pb, G, l, x, b, steps, deg);
    cudaGraph_t graph = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(G->cap, &graph);
    C->stream = saved;
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamBeginCapture");
    if (st != MFS_OK) {
      if (graph) cudaGraphDestroy(graph);
      return st;
    }
    if (e2 != cudaSuccess) return cuda_fail(e2, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&g.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      g.exec = nullptr;
      return cuda_fail(e, "cudaGraphInstantiate");
    }
    g.tuning_gen = M->tuning_gen;
  }
  MFS_CUDA(cudaGraphLaunch(g.exec, C->stream));
  return MFS_OK;
}

// ------------------------------------------------------------------------- numeric setup
__global__ void k_seed_vector(int64_t n, double* v) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    uint64_t z = (uint64_t)i + 0x9E3779B97F4A7C15ull;   // splitmix64
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    v[i] = (double)(z >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0;
  }
}

// Chebyshev interval of level l (reading of Sec. 5.2: [b/20, b], b = 1.2 lambda_max(D^-1 A_c)):
// 15 FP64 power iterations on D^-1 A_c from the start vector held in the level's work vector
// x (projected first; its scale does not matter).  Needs the level's inverse diagonal.
static mfs_status power_bound(mfs_problem* Pb, int l, double* lam_out) {
  MG* G = Pb->mg;
  mfs_mesh* M = Pb->mesh;
  cudaStream_t s = M->ctx->stream;
  const int64_t n2 = M->levels[l].nb2.total, n3 = 3 * n2;
  Work<double>& W = G->w64[l];
  Blas<double>::bproject(G->bnd[l], n2, W.x, s);
  double lam = 0.0;
  for (int it = 0; it < 15; ++it) {
    const double nv = std::sqrt(dot<double>(G, n3, W.x, W.x, s));
    if (!(nv > 0.0) || !std::isfinite(nv)) {
      set_error("power iteration broke down on level %d", l);
      return MFS_ENAN;
    }
    Blas<double>::axpby(n3, 1.0 / nv, W.x, 0.0, W.x, s);
    MFS_TRY(applyA<double>(Pb, l, W.x, W.t));
    Blas<double>::mul(n3, W.t, W.dinv, W.x, s);
    Blas<double>::bproject(G->bnd[l], n2, W.x, s);
    lam = std::sqrt(dot<double>(G, n3, W.x, W.x, s));
  }
  G->hi[l] = 1.2 * lam;
  G->lo[l] = G->hi[l] / 20.0;
  *lam_out = lam;
  return MFS_OK;
}

static mfs_status mg_numeric(mfs_problem* Pb) {
  MG* G = Pb->mg;
  mfs_mesh* M = Pb->mesh;
  cudaStream_t s = M->ctx->stream;
  const int L = M->l_max;
  for (int l = G->l_min; l <= L; ++l) {
    const int64_t n2 = M->levels[l].nb2.total, n3 = 3 * n2;
    Work<double>& W = G->w64[l];
    MFS_TRY(diag_A<double>(Pb, l, G->bnd[l], W.dinv));
    Blas<float>::convert_from_f64(n3, W.dinv, G->w32[l].dinv, s);
    Blas<double>::recip(n3, W.dinv, s);
    Blas<float>::recip(n3, G->w32[l].dinv, s);
    if (l > G->l_min && !G->have_bounds[l]) {
      k_seed_vector<<<1024, 256, 0, s>>>(n3, W.x);
      double lam = 0.0;
      MFS_TRY(power_bound(Pb, l, &lam));
    }
  }
  MFS_TRY(coarse_inverse(Pb, G->l_min, G->bnd[G->l_min], G->Ainv, G->ainv_work));
  // inverse diagonal of M_{1/eta} on the finest level
  MFS_TRY(mass_weights(Pb, L, G->mw64));
  Blas<float>::convert_from_f64(mass_weight_count(M->levels[L]), G->mw64, G->mw32, s);
  MFS_TRY(mass_apply_w<double>(Pb, L, G->mw64, nullptr, G->mdinv64, 1));
  Blas<float>::convert_from_f64(M->levels[L].nb1.total, G->mdinv64, G->mdinv32, s);
  Blas<double>::recip(M->levels[L].nb1.total, G->mdinv64, s);
  Blas<float>::recip(M->levels[L].nb1.total, G->mdinv32, s);
  MFS_CUDA(cudaStreamSynchronize(s));
  MFS_CUDA(cudaGetLastError());
  drop_vgraphs(G);   // new Chebyshev intervals
  G->numeric = true;
  return MFS_OK;
}

}  // namespace mfs

using namespace mfs;

// ------------------------------------------------------------------------- C ABI (part)
static mfs_status need_mg(mfs_problem* Pb, int lvl) {
  if (!Pb) {
    set_error("null problem");
    return MFS_EINVAL;
  }
  if (!Pb->mg || !Pb->mg->structure || !Pb->mg->numeric) {
    set_error("multigrid not set up (call mfs_setup_multigrid after mfs_set_viscosity)");
    return MFS_EINVAL;
  }
  if (lvl < Pb->mg->l_min || lvl > Pb->mg->l_max) {
    set_error("level %d outside the multigrid range [%d, %d]", lvl, Pb->mg->l_min, Pb->mg->l_max);
    return MFS_EINVAL;
  }
  return MFS_OK;
}

mfs_status mfs_setup_multigrid(mfs_problem* Pb, int l_min) {
  if (!Pb) {
    set_error("null problem");
    return MFS_EINVAL;
  }
  if (!Pb->has_eta) {
    set_error("viscosity not set (call mfs_set_viscosity first)");
    return MFS_EINVAL;
  }
  MFS_TRY(mg_structure(Pb, l_min));
  return mg_numeric(Pb);
}

mfs_status mfs_set_cheb_bounds(mfs_problem* Pb, int lvl, double lo, double hi) {
  if (!Pb || !Pb->mg || !Pb->mg->structure) {
    set_error("multigrid not set up");
    return MFS_EINVAL;
  }
  if (lvl <= Pb->mg->l_min || lvl > Pb->mg->l_max || !(hi > lo) || !(lo > 0.0)) {
    set_error("invalid Chebyshev interval or level");
    return MFS_EINVAL;
  }
  Pb->mg->lo[lvl] = lo;
  Pb->mg->hi[lvl] = hi;
  Pb->mg->have_bounds[lvl] = 1;
  drop_vgraphs(Pb->mg);
  return MFS_OK;
}

// ------------------------------------------------------------------------- checkpoint
// The viscosity-dependent state of the hierarchy, copied on the device: per level the nodal
// viscosity (FP64, FP32) and the inverse diagonal of A (FP64, FP32), the Chebyshev intervals,
// the coarse-level inverse, and the finest level's M_{1/eta} quadrature weights and inverse
// diagonal.
struct mfs_mg_state {
  mfs_problem* prob = nullptr;
  int l_min = 0, l_max = 0;
  std::vector<std::pair<void*, size_t>> blocks;   // device copies in a fixed order
  std::vector<double> lo, hi;
  std::vector<int> have_bounds;
};

namespace mfs {
// the device arrays of the state, in the order of mfs_mg_state::blocks
static std::vector<std::pair<void*, size_t>> mg_state_arrays(mfs_problem* Pb) {
  MG* G = Pb->mg;
  mfs_mesh* M = Pb->mesh;
  std::vector<std::pair<void*, size_t>> a;
  for (int l = 0; l <= M->l_max; ++l) {
    const size_t n1 = (size_t)M->levels[l].nb1.total;
    a.push_back({Pb->eta64[l], sizeof(double) * n1});
    a.push_back({Pb->eta32[l], sizeof(float) * n1});
  }
  for (int l = G->l_min; l <= G->l_max; ++l) {
    const size_t n3 = 3 * (size_t)M->levels[l].nb2.total;
    a.push_back({G->w64[l].dinv, sizeof(double) * n3});
    a.push_back({G->w32[l].dinv, sizeof(float) * n3});
  }
  a.push_back({G->Ainv, sizeof(double) * (size_t)G->ncoarse * G->ncoarse});
  const size_t nw = (size_t)mass_weight_count(M->levels[M->l_max]);
  const size_t n1 = (size_t)M->levels[M->l_max].nb1.total;
  a.push_back({G->mw64, sizeof(double) * nw});
  a.push_back({G->mw32, sizeof(float) * nw});
  a.push_back({G->mdinv64, sizeof(double) * n1});
  a.push_back({G->mdinv32, sizeof(float) * n1});
  return a;
}
}  // namespace mfs

mfs_status mfs_mg_state_destroy(mfs_mg_state* S) {
  if (!S) return MFS_OK;
  for (auto& b : S->blocks) cudaFree(b.first);
  delete S;
  return MFS_OK;
}

mfs_status mfs_mg_checkpoint(mfs_problem* Pb, mfs_mg_state** out) {
  if (!out) {
    set_error("null output");
    return MFS_EINVAL;
  }
  *out = nullptr;
  MFS_TRY(need_mg(Pb, Pb ? (Pb->mg ? Pb->mg->l_max : 0) : 0));
  if (Pb->l_eta >= 0) {
    set_error("checkpoint of a hierarchy with quadrature-point viscosity (l_eta >= 0) is not supported");
    return MFS_EINVAL;
  }
  mfs_mg_state* S = new (std::nothrow) mfs_mg_state;
  if (!S) {
    set_error("host allocation failed");
    return MFS_ENOMEM;
  }
  S->prob = Pb;
  S->l_min = Pb->mg->l_min;
  S->l_max = Pb->mg->l_max;
  S->lo = Pb->mg->lo;
  S->hi = Pb->mg->hi;
  S->have_bounds = Pb->mg->have_bounds;
  cudaStream_t s = Pb->mesh->ctx->stream;
  for (auto& a : mg_state_arrays(Pb)) {
    void* d = nullptr;
    cudaError_t e = cudaMalloc(&d, a.second ? a.second : 16);
    if (e == cudaSuccess) {
      S->blocks.push_back({d, a.second});
      e = cudaMemcpyAsync(d, a.first, a.second, cudaMemcpyDeviceToDevice, s);
    }
    if (e != cudaSuccess) {
      mfs_mg_state_destroy(S);
      return cuda_fail(e, "mfs_mg_checkpoint");
    }
  }
  const cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    mfs_mg_state_destroy(S);
    return cuda_fail(e, "mfs_mg_checkpoint");
  }
  *out = S;
  return MFS_OK;
}

mfs_status mfs_mg_restore(mfs_problem* Pb, const mfs_mg_state* S) {
  if (!S || S->prob != Pb) {
    set_error("null state or a state of another problem");
    return MFS_EINVAL;
  }
  MFS_TRY(need_mg(Pb, S->l_max));
  if (Pb->mg->l_min != S->l_min || Pb->mg->l_max != S->l_max || Pb->l_eta >= 0) {
    set_error("the hierarchy's level range or viscosity mode changed since the checkpoint");
    return MFS_EINVAL;
  }
  const auto arrays = mg_state_arrays(Pb);
  if (arrays.size() != S->blocks.size()) {
    set_error("internal: checkpoint layout mismatch");
    return MFS_EINVAL;
  }
  cudaStream_t s = Pb->mesh->ctx->stream;
  for (size_t k = 0; k < arrays.size(); ++k)
    MFS_CUDA(cudaMemcpyAsync(arrays[k].first, S->blocks[k].first, S->blocks[k].second, cudaMemcpyDeviceToDevice, s));
  Pb->mg->lo = S->lo;
  Pb->mg->hi = S->hi;
  Pb->mg->have_bounds = S->have_bounds;
  Pb->has_eta = true;
  Pb->version++;        // coefficient-keyed caches (ensembles, weighted-BFBT operators) rebuild
  drop_vgraphs(Pb->mg);  // the intervals may differ
  MFS_CUDA(cudaStreamSynchronize(s));
  return MFS_OK;
}

mfs_status mfs_estimate_cheb_bounds(mfs_problem* Pb, int lvl, const double* x0, double* lam_max) {
  MFS_TRY(need_mg(Pb, lvl));
  if (!x0 || !lam_max) {
    set_error("null start vector or output");
    return MFS_EINVAL;
  }
  if (lvl <= Pb->mg->l_min) {
    set_error("level %d has no smoother", lvl);
    return MFS_EINVAL;
  }
  mfs_mesh* M = Pb->mesh;
  const int64_t n3 = 3 * (int64_t)M->levels[lvl].nb2.total;
  MFS_CUDA(cudaMemcpyAsync(Pb->mg->w64[lvl].x, x0, sizeof(double) * n3, cudaMemcpyDeviceToDevice, M->ctx->stream));
  MFS_TRY(power_bound(Pb, lvl, lam_max));
  Pb->mg->have_bounds[lvl] = 1;
  drop_vgraphs(Pb->mg);
  return MFS_OK;
}

mfs_status mfs_get_cheb_bounds(const mfs_problem* Pb, int lvl, double* lo, double* hi) {
  if (!Pb || !Pb->mg || !Pb->mg->structure || !lo || !hi) {
    set_error("multigrid not set up or null output");
    return MFS_EINVAL;
  }
  if (lvl <= Pb->mg->l_min || lvl > Pb->mg->l_max) {
    set_error("level %d has no smoother", lvl);
    return MFS_EINVAL;
  }
  *lo = Pb->mg->lo[lvl];
  *hi = Pb->mg->hi[lvl];
  return MFS_OK;
}

mfs_status mfs_diag_A(mfs_problem* Pb, int lvl, mfs_prec prec, void* y) {
  MFS_TRY(need_mg(Pb, lvl));
  if (!y) {
    set_error("null output");
    return MFS_EINVAL;
  }
  if (prec == MFS_F64) return diag_A<double>(Pb, lvl, Pb->mg->bnd[lvl], (double*)y);
  return diag_A<float>(Pb, lvl, Pb->mg->bnd[lvl], (float*)y);
}

mfs_status mfs_apply_mass(mfs_problem* Pb, int lvl, mfs_prec prec, const void* p, void* y) {
  if (!Pb || !Pb->has_eta) {
    set_error("null problem or viscosity not set");
    return MFS_EINVAL;
  }
  if (lvl < 0 || lvl > Pb->mesh->l_max || !p || !y) {
    set_error("invalid level or null vector");
    return MFS_EINVAL;
  }
  MG* G = Pb->mg;
  if (G && G->numeric && lvl == G->l_max) {   // stored weights on the finest level
    if (prec == MFS_F64) return mass_apply_w<double>(Pb, lvl, G->mw64, (const double*)p, (double*)y, 0);
    return mass_apply_w<float>(Pb, lvl, G->mw32, (const float*)p, (float*)y, 0);
  }
  if (prec == MFS_F64) return mass_apply<double>(Pb, lvl, (const double*)p, (double*)y, 0);
  return mass_apply<float>(Pb, lvl, (const float*)p, (float*)y, 0);
}

mfs_status mfs_prolongate(mfs_problem* Pb, int lvl, mfs_prec prec, const void* xc, void* xf) {
  MFS_TRY(need_mg(Pb, lvl));
  if (lvl == Pb->mg->l_min || !xc || !xf) {
    set_error("prolongation needs l_min < lvl and non-null vectors");
    return MFS_EINVAL;
  }
  MG* G = Pb->mg;
  cudaStream_t s = Pb->mesh->ctx->stream;
  const int64_t nc = Pb->mesh->levels[lvl - 1].nb2.total, nf = Pb->mesh->levels[lvl].nb2.total;
  if (prec == MFS_F64) {
    Blas<double>::spmv3(G->P[lvl], nc, (const double*)xc, 1.0, 0.0, (double*)xf, s);
    Blas<double>::bproject(G->bnd[lvl], nf, (double*)xf, s);
  } else {
    Blas<float>::spmv3(G->P[lvl], nc, (const float*)xc, 1.f, 0.f, (float*)xf, s);
    Blas<float>::bproject(G->bnd[lvl], nf, (float*)xf, s);
  }
  MFS_CUDA(cudaGetLastError());
  return MFS_OK;
}

mfs_status mfs_project(mfs_problem* Pb, int lvl, mfs_prec prec, void* x) {
  MFS_TRY(need_mg(Pb, lvl));
  if (!x || (prec != MFS_F64 && prec != MFS_F32)) {
    set_error("null vector or invalid precision");
    return MFS_EINVAL;
  }
  cudaStream_t s = Pb->mesh->ctx->stream;
  const int64_t n2 = Pb->mesh->levels[lvl].nb2.total;
  if (prec == MFS_F64) Blas<double>::bproject(Pb->mg->bnd[lvl], n2, (double*)x, s);
  else Blas<float>::bproject(Pb->mg->bnd[lvl], n2, (float*)x, s);
  MFS_CUDA(cudaGetLastError());
  return MFS_OK;
}

mfs_status mfs_restrict(mfs_problem* Pb, int lvl, mfs_prec prec, const void* rf, void* rc) {
  MFS_TRY(need_mg(Pb, lvl));
  if (lvl == Pb->mg->l_min || !rf || !rc) {
    set_error("restriction needs l_min < lvl and non-null vectors");
    return MFS_EINVAL;
  }
  MG* G = Pb->mg;
  cudaStream_t s = Pb->mesh->ctx->stream;
  const int64_t nc = Pb->mesh->levels[lvl - 1].nb2.total, nf = Pb->mesh->levels[lvl].nb2.total;
  if (prec == MFS_F64) {
    Blas<double>::spmv3(G->R[lvl], nf, (const double*)rf, 1.0, 0.0, (double*)rc, s);
    Blas<double>::bproject(G->bnd[lvl - 1], nc, (double*)rc, s);
  } else {
    Blas<float>::spmv3(G->R[lvl], nf, (const float*)rf, 1.f, 0.f, (float*)rc, s);
    Blas<float>::bproject(G->bnd[lvl - 1], nc, (float*)rc, s);
  }
  MFS_CUDA(cudaGetLastError());
  return MFS_OK;
}

mfs_status mfs_vcycle(mfs_problem* Pb, int lvl, mfs_prec prec, int steps, int degree, const void* f, void* u) {
  MFS_TRY(need_mg(Pb, lvl));
  if (!f || !u || steps < 0 || degree < 1) {
    set_error("invalid V-cycle arguments");
    return MFS_EINVAL;
  }
  if (prec == MFS_F64) return vcycle<double>(Pb, Pb->mg, lvl, (double*)u, (const double*)f, steps, degree);
  return vcycle<float>(Pb, Pb->mg, lvl, (float*)u, (const float*)f, steps, degree);
}

namespace mfs {
int mg_lmin(const mfs_problem* Pb) {
  return (Pb && Pb->mg && Pb->mg->structure && Pb->mg->numeric) ? Pb->mg->l_min : -1;
}

void problem_release_solver(mfs_problem* Pb) {
  if (Pb && Pb->tw) {
    temp_destroy(Pb->tw);
    Pb->tw = nullptr;
  }
  if (Pb && Pb->pmg) {
    pmg_destroy(Pb->pmg);
    Pb->pmg = nullptr;
  }
  if (Pb && Pb->mg) {
    mg_destroy(Pb->mg);
    Pb->mg = nullptr;
  }
}
}  // namespace mfs

// ========================================================================= Stokes solver
namespace mfs {

template <typename T>
static Krylov<T>& kry(MG* G);
template <>
Krylov<float>& kry<float>(MG* G) { return G->k32; }
template <>
Krylov<double>& kry<double>(MG* G) { return G->k64; }

template <typename T>
static mfs_status ensure_krylov(MG* G, int64_t nu, int64_t np, int m, cudaStream_t s) {
  Krylov<T>& K = kry<T>(G);
  const int64_t N = nu + np;
  if (K.N == N && K.m >= m) return MFS_OK;
  if (K.N != 0 && K.N != N) {
    set_error("internal: Krylov storage of another size");
    return MFS_EINVAL;
  }
  if (K.N == 0) {
    T** uvecs[] = {&K.w, &K.ua, &K.ub, &K.uc, &K.ud, &K.cg_r, &K.cg_z, &K.cg_p, &K.cg_q, &K.tmpu,
                   &K.rhs, &K.sol, &K.ir_r, &K.ir_y};
    for (T** v : uvecs) MFS_TRY(dalloc_zero(G, v, N, s));   // N-sized: also used for combined vectors
    T** pvecs[] = {&K.pa, &K.pb, &K.pc, &K.pd, &K.pe, &K.pf, &K.cgp_r, &K.cgp_z, &K.cgp_p, &K.cgp_q,
                   &K.cgm_r, &K.cgm_z, &K.cgm_p, &K.cgm_q, &K.tmpp, &K.ir_p};
    for (T** v : pvecs) MFS_TRY(dalloc_zero(G, v, np, s));
    K.N = N;
  }
  // grow the Krylov basis to m (+1) vectors
  while ((int)K.V.size() < m + 1) {
    T* v = nullptr;
    MFS_TRY(dalloc_zero(G, &v, N, s));
    K.V.push_back(v);
  }
  while ((int)K.Z.size() < m) {
    T* v = nullptr;
    MFS_TRY(dalloc_zero(G, &v, N, s));
    K.Z.push_back(v);
  }
  K.m = m;
  return MFS_OK;
}

template <typename T>
static const T* mass_dinv(MG* G);
template <>
const float* mass_dinv<float>(MG* G) { return G->mdinv32; }
template <>
const double* mass_dinv<double>(MG* G) { return G->mdinv64; }
template <typename T>
static const T* mass_w(MG* G);
template <>
const float* mass_w<float>(MG* G) { return G->mw32; }
template <>
const double* mass_w<double>(MG* G) { return G->mw64; }

template <typename T>
struct Stokes {
  mfs_problem* Pb;
  MG* G;
  const mfs_solve_opts& o;
  mfs_solve_stats& st;
  int L;
  int64_t n2, nu, np, N;
  cudaStream_t s;
  Krylov<T>& K;
  double tolM, tolW;
  int transpose;   // 1: the adjoint operator [A (B+C)^T; B 0]
  // FP64 outer Krylov with an FP32 preconditioner (mixed = 2): the preconditioner of this
  // (FP64) instance is the FP32 instance's Uzawa step, through FP32 copies of its vectors
  Stokes<float>* inner = nullptr;

  Stokes(mfs_problem* P, const mfs_solve_opts& opts, mfs_solve_stats& stats, int transp = 0)
      : Pb(P), G(P->mg), o(opts), st(stats), L(P->mesh->l_max), n2(P->mesh->levels[L].nb2.total), nu(3 * n2),
        np(P->mesh->levels[L].nb1.total), N(nu + np), s(P->mesh->ctx->stream), K(kry<T>(P->mg)),
        transpose(transp) {
    tolM = o.tol_invMass;
    if (sizeof(T) == 4 && tolM < 1e-5) tolM = 1e-5;   // FP32 CG stagnates near 1e-6
    tolW = o.tol_wBFBT;
    if (sizeof(T) == 4 && tolW < 1e-5) tolW = 1e-5;
  }

  double dotn(int64_t n, const T* x, const T* y) { return dot<T>(G, n, x, y, s); }

  // ---- blocks of the constrained system
  mfs_status A(const T* u, T* y) {
    st.applies++;
    return applyA<T>(Pb, L, u, y);
  }
  mfs_status BT(const T* p, T* y) { return apply_constrained<T>(Pb, L, OP_BT, 1, 0, nullptr, p, y, nullptr); }
  mfs_status Bop(const T* u, T* q, int withc) {
    return apply_constrained<T>(Pb, L, OP_B, 1, withc, u, nullptr, nullptr, q);
  }
  // the momentum row's pressure block: B^T, or (B+C)^T in the adjoint operator
  mfs_status BTrow(const T* p, T* y) {
    const int op = (transpose && o.with_C) ? (OP_BT | OP_CT) : OP_BT;
    return apply_constrained<T>(Pb, L, op, 1, 0, nullptr, p, y, nullptr);
  }
  // the constraint row: (B+C), or B in the adjoint operator
  int withc_row() const { return transpose ? 0 : o.with_C; }
  mfs_status Kop(const T* x, T* y) {
    st.applies++;
    if (transpose && o.with_C)
      return apply_constrained<T>(Pb, L, OP_A | OP_BT | OP_CT | OP_B, 1, 0, x, x + nu, y, y + nu);
    return apply_constrained<T>(Pb, L, OP_A | OP_BT | OP_B, 1, withc_row(), x, x + nu, y, y + nu);
  }

  // generic preconditioned CG on n entries; op/pre write their output vector
  template <typename Op, typename Pre>
  mfs_status cg(int64_t n, Op op, Pre pre, const T* b, T* x, double rtol, int maxit, T* r, T* z, T* p, T* q,
                int* iters, int proj = 0, double atol = 0.0) {
    // proj: 1 keeps a pressure residual mean-free, 2 keeps a velocity residual in the
    // constrained space (FP32 rounding leaves residue in directions the operator ignores);
    // stops at ||r|| <= max(rtol ||r0||, atol)
    Blas<T>::axpby(n, T(1), b, T(0), r, s);
    if (proj == 1) MFS_TRY(mean_free<T>(Pb, r, n));
    if (proj == 2) Blas<T>::bproject(G->bnd[L], n2, r, s);
    Blas<T>::fill(n, T(0), x, s);
    *iters = 0;
    const double rr0 = dotn(n, r, r);
    if (!std::isfinite(rr0)) {
      set_error("NaN/Inf in a CG right-hand side");
      return MFS_ENAN;
    }
    if (rr0 == 0.0) return MFS_OK;
    MFS_TRY(pre(r, z));
    Blas<T>::axpby(n, T(1), z, T(0), p, s);
    double rz = dotn(n, r, z);
    for (int it = 0; it < maxit; ++it) {
      MFS_TRY(op(p, q));
      const double pq = dotn(n, p, q);
      if (!std::isfinite(pq)) {
        set_error("NaN/Inf in CG");
        return MFS_ENAN;
      }
      if (pq <= 0.0) break;   // loss of positivity (inexact inner solves): keep the iterate
      const double alpha = rz / pq;
      Blas<T>::axpby(n, T(alpha), p, T(1), x, s);
      Blas<T>::axpby(n, T(-alpha), q, T(1), r, s);
      if (proj == 1) MFS_TRY(mean_free<T>(Pb, r, n));
      if (proj == 2) Blas<T>::bproject(G->bnd[L], n2, r, s);
      ++*iters;
      const double rr = dotn(n, r, r);
      if (!std::isfinite(rr)) {
        set_error("NaN/Inf in CG residual");
        return MFS_ENAN;
      }
      if (std::sqrt(rr) <= rtol * std::sqrt(rr0) || std::sqrt(rr) <= atol) break;
      MFS_TRY(pre(r, z));
      const double rz_new = dotn(n, r, z);
      Blas<T>::axpby(n, T(1), z, T(rz_new / rz), p, s);
      rz = rz_new;
    }
    return MFS_OK;
  }

  // ---- A-block: CG on A preconditioned by a V-cycle (m_A, deg_A) to tol_A
  mfs_status Ahat_inv(const T* r, T* x) {
    WallTimer tm(st.time_Ahat_ms);
    int it = 0;
    auto op = [&](const T* v, T* y) { return A(v, y); };
    auto pre = [&](const T* v, T* y) {
      st.vcycles++;
      return vcycle<T>(Pb, G, L, y, v, o.m_A, o.deg_A);
    };
    MFS_TRY(cg(nu, op, pre, r, x, o.tol_A, o.max_cg, K.cg_r, K.cg_z, K.cg_p, K.cg_q, &it, 2));
    st.cg_A_iters += it;
    st.cg_A_calls++;
    st.cg_A_max = it > st.cg_A_max ? it : st.cg_A_max;
    return MFS_OK;
  }
  // cheap V-cycle A_C^-1 (m_V, deg_V)
  mfs_status Ac_inv(const T* r, T* x) {
    st.vcycles++;
    return vcycle<T>(Pb, G, L, x, r, o.m_V, o.deg_V);
  }
  // M_{1/eta}^-1 by CG (P_p M P_p, Jacobi) to tol_invMass, run on the device: the scalars
  // stay in device memory and chunks of kChunk iterations replay a captured CUDA graph
  // (finished iterations are no-ops); the host reads one flag per chunk.
  static constexpr int kChunk = 8;
  void mass_iteration(cudaStream_t cs, T* x) {
    const double tol2 = tolM * tolM;
    mass_apply_w<T>(Pb, L, mass_w<T>(G), K.cgm_p, K.cgm_q, 0, G->cgsc + CG_ACTIVE, 0);   // q = M p (q held 0)
    CgDev<T>::mass_dots(np, K.cgm_p, K.cgm_q, G->mcg_part, G->mcg_counter, G->cgsc, cs);
    CgDev<T>::mass_update(np, K.cgm_p, K.cgm_q, x, K.cgm_r, K.cgm_z, mass_dinv<T>(G), G->mcg_part, G->mcg_counter,
                          G->cgsc, tol2, o.max_cg, cs);
    CgDev<T>::mass_pupd(np, K.cgm_z, K.cgm_p, G->cgsc, cs);
  }
  mfs_status mass_graph(T* x, cudaGraphExec_t* out) {
    const int prec = sizeof(T) == 8 ? 0 : 1;
    for (auto& g : G->graphs)
      if (g.prec == prec && g.x == x && g.tol == tolM && g.maxit == o.max_cg) {
        *out = g.exec;
        return MFS_OK;
      }
    mfs_ctx* C = Pb->mesh->ctx;
    cudaStream_t saved = C->stream;
    C->stream = G->cap;
    cudaError_t e = cudaStreamBeginCapture(G->cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      for (int k = 0; k < kChunk; ++k) mass_iteration(G->cap, x);
    }
    cudaGraph_t graph = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(G->cap, &graph);
    C->stream = saved;
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamBeginCapture");
    if (e2 != cudaSuccess) return cuda_fail(e2, "cudaStreamEndCapture");
    cudaGraphExec_t exec;
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
    G->graphs.push_back({prec, x, tolM, o.max_cg, exec});
    *out = exec;
    return MFS_OK;
  }
  mfs_status M_inv(const T* r, T* x) {
    WallTimer tm(st.time_Minv_ms);
    cudaGraphExec_t exec;
    MFS_TRY(mass_graph(x, &exec));
    Blas<T>::axpby(np, T(1), r, T(0), K.cgm_r, s);
    MFS_TRY(mean_free<T>(Pb, K.cgm_r, np));
    Blas<T>::fill(np, T(0), x, s);
    Blas<T>::fill(np, T(0), K.cgm_q, s);
    Blas<T>::mul(np, K.cgm_r, mass_dinv<T>(G), K.cgm_z, s);
    MFS_TRY(mean_free<T>(Pb, K.cgm_z, np));
    Blas<T>::axpby(np, T(1), K.cgm_z, T(0), K.cgm_p, s);
    Blas<T>::dot_async(np, K.cgm_r, K.cgm_z, G->red, G->cgsc + CG_RZ, s);
    Blas<T>::dot_async(np, K.cgm_r, K.cgm_r, G->red, G->cgsc + CG_RR0, s);
    CgDev<T>::init(G->cgsc, s);
    double flags[CG_NSLOTS];
    for (int it = 0; it < o.max_cg; it += kChunk) {
      MFS_CUDA(cudaGraphLaunch(exec, s));
      MFS_CUDA(cudaMemcpyAsync(G->hpin, G->cgsc, sizeof(double) * CG_NSLOTS, cudaMemcpyDeviceToHost, s));
      MFS_CUDA(cudaStreamSynchronize(s));
      std::memcpy(flags, G->hpin, sizeof(flags));
      if (!std::isfinite(flags[CG_RR])) {
        set_error("NaN/Inf in the mass-matrix CG");
        return MFS_ENAN;
      }
      if (!(flags[CG_ACTIVE] > 0.0)) break;
    }
    const int it = (int)flags[CG_IT];
    st.cg_M_iters += it;
    st.cg_M_calls++;
    st.cg_M_max = it > st.cg_M_max ? it : st.cg_M_max;
    return mean_free<T>(Pb, x, np);
  }
  // diag(A)^-1 on the constrained velocity space (finest level)
  mfs_status D_inv(const T* r, T* x) {
    Blas<T>::mul(nu, r, work<T>(G, L).dinv, x, s);
    Blas<T>::bproject(G->bnd[L], n2, x, s);
    return MFS_OK;
  }
  // the C^-1 of the BFBT approximation: the cheap V-cycle (V-cycle BFBT) or diag(A)^-1
  mfs_status C_inv(const T* r, T* x) { return o.schur == 2 ? D_inv(r, x) : Ac_inv(r, x); }
  // X q = B C^-1 B^T q
  mfs_status X(const T* q, T* y) {
    MFS_TRY(BT(q, K.ua));
    MFS_TRY(C_inv(K.ua, K.ub));
    return Bop(K.ub, y, 0);
  }
  // V-cycle BFBT: X^-1 (B A_C^-1 A A_C^-1 B^T) X^-1 r
  // K_{1/sqrt(eta_a)}^-1 r by CG preconditioned with its V-cycle (the A-block smoother
  // shape), to tol_wBFBT relative or absolute, whichever is reached first
  mfs_status K_inv(int side, const T* r, T* x) {
    int it = 0;
    auto op = [&](const T* v, T* y) { return poisson_apply<T>(Pb, side, L, v, y); };
    auto pre = [&](const T* v, T* y) { return poisson_vcycle<T>(Pb, side, y, v, o.m_A, o.deg_A); };
    MFS_TRY(cg(np, op, pre, r, x, tolW, o.max_cg, K.cgp_r, K.cgp_z, K.cgp_p, K.cgp_q, &it, 1, tolW));
    st.cg_X_iters += it;
    st.cg_X_calls++;
    st.cg_X_max = it > st.cg_X_max ? it : st.cg_X_max;
    return mean_free<T>(Pb, x, np);
  }
  // M_{sqrt(eta_a)}^-1 r on the constrained velocity space: the lumped inverse (vmass = 0), or
  // CG on P_v M P_v with the consistent mass, Jacobi-preconditioned, to tol_VectorMass
  // relative (vmass = 1; Sec. 5.2.3); x and r distinct
  mfs_status Mw_inv(int side, double a, const T* r, T* x) {
    if (o.vmass == 0) {
      Blas<T>::mul(nu, r, poisson_minv<T>(Pb, side), x, s);
      Blas<T>::bproject(G->bnd[L], n2, x, s);
      return MFS_OK;
    }
    WallTimer tm(st.time_Minv_ms);
    const T* dinv = nullptr;
    MFS_TRY(poisson_cmass_dinv<T>(Pb, side, &dinv));
    int it = 0;
    auto op = [&](const T* v, T* y) {
      MFS_TRY(wmass_apply<T>(Pb, a, v, y, 0));
      Blas<T>::bproject(G->bnd[L], n2, y, s);
      return MFS_OK;
    };
    auto pre = [&](const T* v, T* y) {
      Blas<T>::mul(nu, v, dinv, y, s);
      Blas<T>::bproject(G->bnd[L], n2, y, s);
      return MFS_OK;
    };
    MFS_TRY(cg(nu, op, pre, r, x, o.tol_VectorMass, o.max_cg, K.cg_r, K.cg_z, K.cg_p, K.cg_q, &it, 2));
    st.cg_M_iters += it;
    st.cg_M_calls++;
    st.cg_M_max = it > st.cg_M_max ? it : st.cg_M_max;
    Blas<T>::bproject(G->bnd[L], n2, x, s);
    return MFS_OK;
  }
  // weighted BFBT (Eq. schurWBFBT, rescaled form):
  //   K_{1/sqrt(eta_l)}^-1 (B M_{sqrt(eta_l)}^-1 A M_{sqrt(eta_r)}^-1 B^T) K_{1/sqrt(eta_r)}^-1 r
  mfs_status wbfbt(const T* r, T* z) {
    int sl = 0, sr = 0;
    MFS_TRY(pmg_side(Pb, o.a_l, &sl));
    MFS_TRY(pmg_side(Pb, o.a_r, &sr));
    MFS_TRY(K_inv(sr, r, K.pe));
    MFS_TRY(BT(K.pe, K.uc));
    MFS_TRY(Mw_inv(sr, o.a_r, K.uc, K.ud));
    MFS_TRY(A(K.ud, K.uc));
    MFS_TRY(Mw_inv(sl, o.a_l, K.uc, K.ud));
    MFS_TRY(Bop(K.ud, K.pf, 0));
    return K_inv(sl, K.pf, z);
  }
  mfs_status S_inv(const T* r, T* z) {
    WallTimer tm(st.time_Sinv_ms);
    if (o.schur == 1) return M_inv(r, z);   // Eq. schurMass: M_{1/eta}^-1 (mean-free)
    if (o.schur == 3) return wbfbt(r, z);
    int it = 0;
    auto op = [&](const T* v, T* y) { return X(v, y); };
    auto pre = [&](const T* v, T* y) { return M_inv(v, y); };
    MFS_TRY(cg(np, op, pre, r, K.pe, o.tol_VBFBT, o.max_cg, K.cgp_r, K.cgp_z, K.cgp_p, K.cgp_q, &it, 1));
    st.cg_X_iters += it;
    st.cg_X_calls++;
    st.cg_X_max = it > st.cg_X_max ? it : st.cg_X_max;
    MFS_TRY(BT(K.pe, K.uc));
    MFS_TRY(C_inv(K.uc, K.ud));
    MFS_TRY(A(K.ud, K.uc));
    MFS_TRY(C_inv(K.uc, K.ud));
    MFS_TRY(Bop(K.ud, K.pf, 0));
    MFS_TRY(cg(np, op, pre, K.pf, z, o.tol_VBFBT, o.max_cg, K.cgp_r, K.cgp_z, K.cgp_p, K.cgp_q, &it, 1));
    st.cg_X_iters += it;
    st.cg_X_calls++;
    st.cg_X_max = it > st.cg_X_max ? it : st.cg_X_max;
    return mean_free<T>(Pb, z, np);
  }
  // Uzawa-type step from (0, 0) on r = (r_u, r_p); output z = (u, p).  B + C replaces B
  // in the pressure updates (the adjoint operator swaps the roles, see Bop/BTrow).
  mfs_status uzawa(const T* r, T* z) {
    const T* ru = r;
    const T* rp = r + nu;
    T* zu = z;
    T* zp = z + nu;
    if (o.uzawa == 1) {   // inexact Uzawa, Eq. (InexactUzawaStep1)
      MFS_TRY(Ahat_inv(ru, zu));
      if (o.sigma != 1.0) Blas<T>::axpby(nu, T(o.sigma), zu, T(0), zu, s);
      MFS_TRY(Bop(zu, K.pa, withc_row()));
      Blas<T>::axpbypcz(np, T(1), rp, T(-1), K.pa, T(0), K.pb, s);     // r_p - Bbar u
      MFS_TRY(S_inv(K.pb, zp));
      Blas<T>::axpby(np, T(-o.omega), zp, T(0), zp, s);
      return MFS_OK;
    }
    if (o.uzawa == 2) {   // adjoint inexact Uzawa, Eq. (AdjointInexactUzawaStep1)
      MFS_TRY(S_inv(rp, zp));
      Blas<T>::axpby(np, T(-o.omega), zp, T(0), zp, s);                // p = -omega S^-1 r_p
      MFS_TRY(BTrow(zp, K.ua));
      Blas<T>::axpbypcz(nu, T(1), ru, T(-1), K.ua, T(0), K.ub, s);     // r_u - B^T p
      MFS_TRY(Ahat_inv(K.ub, zu));
      if (o.sigma != 1.0) Blas<T>::axpby(nu, T(o.sigma), zu, T(0), zu, s);
      return MFS_OK;
    }
    T* uh = K.tmpu;       // symmetric Uzawa, Eq. (SymmetricUzawaStep1)
    MFS_TRY(Ahat_inv(ru, uh));
    if (o.sigma != 1.0) Blas<T>::axpby(nu, T(o.sigma), uh, T(0), uh, s);
    MFS_TRY(Bop(uh, K.pa, withc_row()));                               // (B + C) uh (B: adjoint)
    Blas<T>::axpbypcz(np, T(1), rp, T(-1), K.pa, T(0), K.pb, s);       // r_p - Bbar uh
    MFS_TRY(S_inv(K.pb, zp));
    Blas<T>::axpby(np, T(-o.omega), zp, T(0), zp, s);                  // p = -omega S^-1 (...)
    MFS_TRY(A(uh, K.w));
    MFS_TRY(BTrow(zp, K.ua));
    Blas<T>::axpbypcz(nu, T(1), ru, T(-1), K.w, T(0), K.ub, s);
    Blas<T>::axpby(nu, T(-1), K.ua, T(1), K.ub, s);                    // r_u - A uh - B^T p
    MFS_TRY(Ahat_inv(K.ub, zu));
    Blas<T>::axpby(nu, T(1), uh, T(o.sigma), zu, s);                   // u = uh + sigma A^-1 (...)
    return MFS_OK;
  }

  mfs_status precondition(const T* r, T* z) {
    if constexpr (sizeof(T) == 8) {
      if (inner) {
        float* r32 = G->k32.rhs;   // free in this mode: the FP32 FGMRES is not used
        float* z32 = G->k32.sol;
        Blas<float>::convert_from_f64(N, r, r32, s);
        MFS_TRY(inner->uzawa(r32, z32));
        Blas<float>::convert_to_f64(N, z32, z, s);
        return MFS_OK;
      }
    }
    return uzawa(r, z);
  }

  // right-preconditioned flexible GMRES(m) on K x = b from x = 0 (modified Gram-Schmidt,
  // Givens rotations on the host); stops at ||b - K x|| <= rtol ||b||
  mfs_status fgmres(const T* b, T* x, double rtol, int* iters, double* rel_out) {
    const int m = o.restart;
    Blas<T>::fill(N, T(0), x, s);
    const double beta0 = std::sqrt(dotn(N, b, b));
    *iters = 0;
    *rel_out = 0.0;
    if (!std::isfinite(beta0)) {
      set_error("NaN/Inf in the FGMRES right-hand side");
      return MFS_ENAN;
    }
    if (beta0 == 0.0) return MFS_OK;
    std::vector<double> H((size_t)(m + 1) * m), cs(m), sn(m), g(m + 1), y(m);
    T* r = K.V[0];
    Blas<T>::axpby(N, T(1), b, T(0), r, s);
    double beta = beta0;
    bool done = false;
    while (!done) {
      Blas<T>::axpby(N, T(1.0 / beta), r, T(0), K.V[0], s);
      std::fill(g.begin(), g.end(), 0.0);
      g[0] = beta;
      int k = 0;
      for (; k < m; ++k) {
        MFS_TRY(precondition(K.V[k], K.Z[k]));
        MFS_TRY(Kop(K.Z[k], K.V[k + 1]));
        for (int i = 0; i <= k; ++i) {
          const double hik = dotn(N, K.V[k + 1], K.V[i]);
          H[(size_t)i * m + k] = hik;
          Blas<T>::axpby(N, T(-hik), K.V[i], T(1), K.V[k + 1], s);
        }
        const double hn = std::sqrt(dotn(N, K.V[k + 1], K.V[k + 1]));
        if (!std::isfinite(hn)) {
          set_error("NaN/Inf in FGMRES");
          return MFS_ENAN;
        }
        H[(size_t)(k + 1) * m + k] = hn;
        if (hn > 0.0) Blas<T>::axpby(N, T(1.0 / hn), K.V[k + 1], T(0), K.V[k + 1], s);
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
        ++*iters;
        st.fgmres_iters++;
        if (std::fabs(g[k + 1]) <= rtol * beta0 || *iters >= o.max_iters || hn == 0.0) {
          ++k;
          done = true;
          break;
        }
      }
      // solve the triangular system and update x with the preconditioned directions
      const int kk = k;
      for (int i = kk - 1; i >= 0; --i) {
        double t = g[i];
        for (int j = i + 1; j < kk; ++j) t -= H[(size_t)i * m + j] * y[j];
        y[i] = t / H[(size_t)i * m + i];
      }
      for (int i = 0; i < kk; ++i) Blas<T>::axpby(N, T(y[i]), K.Z[i], T(1), x, s);
      // true residual for the restart / final report
      MFS_TRY(Kop(x, K.V[1]));
      r = K.V[0];
      Blas<T>::axpbypcz(N, T(1), b, T(-1), K.V[1], T(0), r, s);
      beta = std::sqrt(dotn(N, r, r));
      *rel_out = beta / beta0;
      if (beta <= rtol * beta0 || *iters >= o.max_iters) done = true;
    }
    return MFS_OK;
  }
};

// remove normal components at free-slip nodes only (Dirichlet values untouched)
__global__ void k_freeslip_only(int nb, const int* __restrict__ ids, const int8_t* __restrict__ kind,
                                const double* __restrict__ nrm, int64_t n_p2, double* __restrict__ v) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nb; k += gridDim.x * blockDim.x) {
    if (kind[k] != 2) continue;
    const int64_t id = ids[k];
    const double nx = nrm[3 * k], ny = nrm[3 * k + 1], nz = nrm[3 * k + 2];
    const double un = v[id] * nx + v[n_p2 + id] * ny + v[2 * n_p2 + id] * nz;
    v[id] -= un * nx;
    v[n_p2 + id] -= un * ny;
    v[2 * n_p2 + id] -= un * nz;
  }
}
static void k_project_freeslip_only(const BoundaryList& B, int64_t n_p2, double* v, cudaStream_t s) {
  if (B.nb) k_freeslip_only<<<(B.nb + 255) / 256, 256, 0, s>>>(B.nb, B.ids, B.kind, B.nrm64, n_p2, v);
}

// FP64 projected residual of the full system: r_u = P0 (f - A u - B^T P_p p),
// r_p = P_p (g - (B + C) u); raw operators so that u carries the Dirichlet values.
static mfs_status residual64(mfs_problem* Pb, const mfs_solve_opts& o, const double* f, const double* g,
                             const double* u, const double* p, double* r, double* ptmp, double* y, int transpose) {
  MG* G = Pb->mg;
  const int L = Pb->mesh->l_max;
  const int64_t n2 = Pb->mesh->levels[L].nb2.total, nu = 3 * n2, np = Pb->mesh->levels[L].nb1.total;
  cudaStream_t s = Pb->mesh->ctx->stream;
  MFS_CUDA(cudaMemcpyAsync(ptmp, p, sizeof(double) * np, cudaMemcpyDeviceToDevice, s));
  MFS_TRY(mean_free<double>(Pb, ptmp, np));
  if (transpose && o.with_C)
    MFS_TRY(launch_apply<double>(Pb, L, OP_A | OP_BT | OP_CT | OP_B, 0, 0, u, ptmp, y, y + nu, nullptr));
  else
    MFS_TRY(launch_apply<double>(Pb, L, OP_A | OP_BT | OP_B, 0, transpose ? 0 : o.with_C, u, ptmp, y, y + nu,
                                 nullptr));
  Blas<double>::axpbypcz(nu, 1.0, f, -1.0, y, 0.0, r, s);
  Blas<double>::bproject(G->bnd[L], n2, r, s);
  Blas<double>::axpbypcz(np, 1.0, g, -1.0, y + nu, 0.0, r + nu, s);
  MFS_TRY(mean_free<double>(Pb, r + nu, np));
  return MFS_OK;
}

static mfs_status check_schur_opts(const mfs_solve_opts& o) {
  if (o.schur < 0 || o.schur > 3) {
    set_error("schur must be 0 (V-cycle BFBT), 1 (mass), 2 (diag(A)-BFBT) or 3 (weighted BFBT)");
    return MFS_EINVAL;
  }
  if (o.schur == 3 && (!(o.a_l > 0.0) || !(o.a_r > 0.0) || !std::isfinite(o.a_l) || !std::isfinite(o.a_r) ||
                       !(o.tol_wBFBT > 0.0))) {
    set_error("weighted BFBT needs positive finite a_l, a_r and a positive tol_wBFBT");
    return MFS_EINVAL;
  }
  if (o.schur == 3 && ((o.vmass != 0 && o.vmass != 1) || (o.vmass == 1 && !(o.tol_VectorMass > 0.0)))) {
    set_error("vmass must be 0 (lumped) or 1 (consistent, with a positive tol_VectorMass)");
    return MFS_EINVAL;
  }
  return MFS_OK;
}

static mfs_status stokes_solve(mfs_problem* Pb, const mfs_solve_opts& o, const double* f, const double* g, double* u,
                               double* p, mfs_solve_stats& st, int transpose) {
  MG* G = Pb->mg;
  const int L = Pb->mesh->l_max;
  const int64_t n2 = Pb->mesh->levels[L].nb2.total, nu = 3 * n2, np = Pb->mesh->levels[L].nb1.total, N = nu + np;
  cudaStream_t s = Pb->mesh->ctx->stream;
  if (o.mixed < 0 || o.mixed > 2) {
    set_error("mixed must be 0 (FP64), 1 (FP32 FGMRES in FP64 refinement) or 2 (FP64 FGMRES, FP32 preconditioner)");
    return MFS_EINVAL;
  }
  MFS_TRY(check_schur_opts(o));
  if (o.uzawa < 0 || o.uzawa > 2) {
    set_error("uzawa must be 0 (symmetric), 1 (inexact) or 2 (adjoint)");
    return MFS_EINVAL;
  }
  MFS_TRY(ensure_krylov<double>(G, nu, np, o.mixed == 1 ? 1 : o.restart, s));
  if (o.mixed) MFS_TRY(ensure_krylov<float>(G, nu, np, o.mixed == 1 ? o.restart : 1, s));
  Krylov<double>& K64 = G->k64;
  double* r = K64.ir_r;      // FP64 projected residual
  double* y = K64.ir_y;      // operator output / scaled residual
  double* ptmp = K64.ir_p;
  double* d = K64.sol;       // correction
  const auto t0 = std::chrono::steady_clock::now();
  // free-slip nodes: the velocity is tangential (the constrained operator cannot see normal
  // components, so they must not enter u); Dirichlet values are kept
  k_project_freeslip_only(G->bnd[L], n2, u, s);
  MFS_TRY(residual64(Pb, o, f, g, u, p, r, ptmp, y, transpose));
  const double r0 = std::sqrt(dot<double>(G, N, r, r, s));
  st.r0_norm = r0;
  st.r_norm = r0;
  st.rel_residual = r0 > 0 ? 1.0 : 0.0;
  if (!std::isfinite(r0)) {
    set_error("NaN/Inf in the initial residual");
    return MFS_ENAN;
  }
  mfs_status status = MFS_OK;
  double rn = r0;
  for (int outer = 0; outer < o.max_outer && rn > o.rtol * r0; ++outer) {
    int its = 0;
    double rel = 0.0;
    if (o.mixed == 2) {
      Stokes<float> S32(Pb, o, st, transpose);
      Stokes<double> S(Pb, o, st, transpose);
      S.inner = &S32;
      Blas<double>::axpby(N, 1.0 / rn, r, 0.0, K64.rhs, s);
      status = S.fgmres(K64.rhs, d, o.rtol * r0 / rn, &its, &rel);
      if (status != MFS_OK) return status;
    } else if (o.mixed) {
      Stokes<float> S(Pb, o, st, transpose);
      float* r32 = G->k32.rhs;
      float* d32 = G->k32.sol;
      // scaled residual to FP32
      Blas<double>::axpby(N, 1.0 / rn, r, 0.0, y, s);
      Blas<float>::convert_from_f64(N, y, r32, s);
      // inner tolerance: inner_rtol, relaxed in the last step to what the target still
      // needs (with a factor 2 margin for the FP32 estimate of the reduction)
      const double tol_k = std::max(o.inner_rtol, 0.5 * o.rtol * r0 / rn);
      status = S.fgmres(r32, d32, tol_k < 0.5 ? tol_k : 0.5, &its, &rel);
      if (status != MFS_OK) return status;
      Blas<float>::convert_to_f64(N, d32, d, s);
    } else {
      Stokes<double> S(Pb, o, st, transpose);
      Blas<double>::axpby(N, 1.0 / rn, r, 0.0, K64.rhs, s);
      status = S.fgmres(K64.rhs, d, o.rtol * r0 / rn, &its, &rel);
      if (status != MFS_OK) return status;
    }
    // corrections live in the constrained space: project in FP64 before the update
    Blas<double>::bproject(G->bnd[L], n2, d, s);
    Blas<double>::axpby(nu, rn, d, 1.0, u, s);
    Blas<double>::axpby(np, rn, d + nu, 1.0, p, s);
    MFS_TRY(residual64(Pb, o, f, g, u, p, r, ptmp, y, transpose));
    rn = std::sqrt(dot<double>(G, N, r, r, s));
    st.outer_iters++;
    if (!std::isfinite(rn)) {
      set_error("NaN/Inf in the refined residual");
      return MFS_ENAN;
    }
    if (st.fgmres_iters >= o.max_iters) break;
  }
  MFS_TRY(mean_free<double>(Pb, p, np));
  MFS_CUDA(cudaStreamSynchronize(s));
  st.r_norm = rn;
  st.rel_residual = r0 > 0 ? rn / r0 : 0.0;
  st.time_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  if (rn > o.rtol * r0) {
    set_error("not converged: relative residual %.3e > %.3e after %d FGMRES iterations", st.rel_residual, o.rtol,
              st.fgmres_iters);
    return MFS_ENOTCONV;
  }
  return MFS_OK;
}

}  // namespace mfs

void mfs_solve_opts_default(mfs_solve_opts* o) {
  if (!o) return;
  o->mixed = 1;
  o->rtol = 1e-8;
  o->restart = 30;
  o->max_iters = 300;
  o->max_outer = 20;
  o->inner_rtol = 1e-4;
  o->sigma = 1.0;
  o->omega = 0.3;
  o->tol_A = 1e-2;
  o->m_A = 3;
  o->deg_A = 2;
  o->tol_VBFBT = 1e-1;
  o->tol_invMass = 1e-10;
  o->m_V = 1;
  o->deg_V = 1;
  o->max_cg = 200;
  o->with_C = 1;
  o->uzawa = 0;
  o->schur = 0;
  o->a_l = 1.0;
  o->a_r = 1.0;
  o->tol_wBFBT = 1e-10;
  o->vmass = 1;   // the consistent vector mass (Sec. 5.2.3), the paper's CG solve
  o->tol_VectorMass = 1e-4;
}

mfs_status mfs_mesh_prolongation(const mfs_mesh* M, int lvl, int* nnz, int* rp, int* ci, double* w) {
  if (!M || !nnz || lvl < 1 || lvl > M->l_max) {
    set_error("null argument or level outside 1..l_max");
    return MFS_EINVAL;
  }
  std::vector<int> r, c;
  std::vector<double> v;
  MFS_TRY(prolongation_csr(M, lvl, r, c, v));
  *nnz = (int)c.size();
  if (rp) std::memcpy(rp, r.data(), sizeof(int) * r.size());
  if (ci) std::memcpy(ci, c.data(), sizeof(int) * c.size());
  if (w) std::memcpy(w, v.data(), sizeof(double) * v.size());
  return MFS_OK;
}

mfs_status mfs_mesh_p1_interpolation(const mfs_mesh* M, int lvl, int* nnz, int* coarse, int* fine, double* w) {
  if (!M || !nnz || lvl < 1 || lvl > M->l_max) {
    set_error("null argument or level outside 1..l_max");
    return MFS_EINVAL;
  }
  std::vector<int> tv, tj;
  std::vector<double> tw;
  p1_transfer_triplets(M, lvl, tv, tj, tw);
  *nnz = (int)tv.size();
  if (coarse) std::memcpy(coarse, tv.data(), sizeof(int) * tv.size());
  if (fine) std::memcpy(fine, tj.data(), sizeof(int) * tj.size());
  if (w) std::memcpy(w, tw.data(), sizeof(double) * tw.size());
  return MFS_OK;
}

mfs_status mfs_apply_schur(mfs_problem* Pb, const mfs_solve_opts* opts, mfs_prec prec, const void* r, void* z,
                           mfs_solve_stats* stats) {
  if (!Pb || !r || !z) {
    set_error("null argument");
    return MFS_EINVAL;
  }
  if (!Pb->mg || !Pb->mg->numeric) {
    set_error("multigrid not set up (call mfs_setup_multigrid after mfs_set_viscosity)");
    return MFS_EINVAL;
  }
  mfs_solve_opts o;
  if (opts) o = *opts;
  else mfs_solve_opts_default(&o);
  MFS_TRY(check_schur_opts(o));
  if (o.m_V < 0 || o.deg_V < 1 || o.m_A < 0 || o.deg_A < 1 || o.max_cg < 1) {
    set_error("invalid solver options");
    return MFS_EINVAL;
  }
  MG* G = Pb->mg;
  const int L = Pb->mesh->l_max;
  const int64_t nu = 3 * (int64_t)Pb->mesh->levels[L].nb2.total, np = Pb->mesh->levels[L].nb1.total;
  cudaStream_t s = Pb->mesh->ctx->stream;
  mfs_solve_stats st;
  std::memset(&st, 0, sizeof(st));
  mfs_status rc;
  if (prec == MFS_F64) {
    MFS_TRY(ensure_krylov<double>(G, nu, np, 1, s));
    Stokes<double> S(Pb, o, st);
    rc = S.S_inv((const double*)r, (double*)z);
  } else {
    MFS_TRY(ensure_krylov<float>(G, nu, np, 1, s));
    Stokes<float> S(Pb, o, st);
    rc = S.S_inv((const float*)r, (float*)z);
  }
  if (rc == MFS_OK) {
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) rc = cuda_fail(e, "mfs_apply_schur");
  }
  if (stats) *stats = st;
  return rc;
}

mfs_status mfs_stokes_solve(mfs_problem* Pb, const mfs_solve_opts* opts, const double* f, const double* g, double* u,
                            double* p, mfs_solve_stats* stats) {
  if (!Pb || !f || !g || !u || !p) {
    set_error("null argument");
    return MFS_EINVAL;
  }
  if (!Pb->mg || !Pb->mg->numeric) {
    set_error("multigrid not set up (call mfs_setup_multigrid after mfs_set_viscosity)");
    return MFS_EINVAL;
  }
  mfs_solve_opts o;
  if (opts) o = *opts;
  else mfs_solve_opts_default(&o);
  if (o.restart < 1 || o.restart > 200 || !(o.rtol > 0) || o.m_A < 0 || o.deg_A < 1 || o.m_V < 0 || o.deg_V < 1) {
    set_error("invalid solver options");
    return MFS_EINVAL;
  }
  mfs_solve_stats st;
  std::memset(&st, 0, sizeof(st));
  const mfs_status rc = stokes_solve(Pb, o, f, g, u, p, st, 0);
  if (stats) *stats = st;
  return rc;
}

mfs_status mfs_adjoint_solve(mfs_problem* Pb, const mfs_solve_opts* opts, const double* ju, const double* jp,
                             double* lam_u, double* lam_p, mfs_solve_stats* stats) {
  if (!Pb || !ju || !jp || !lam_u || !lam_p) {
    set_error("null argument");
    return MFS_EINVAL;
  }
  if (!Pb->mg || !Pb->mg->numeric) {
    set_error("multigrid not set up (call mfs_setup_multigrid after mfs_set_viscosity)");
    return MFS_EINVAL;
  }
  mfs_solve_opts o;
  if (opts) o = *opts;
  else mfs_solve_opts_default(&o);
  mfs_solve_stats st;
  std::memset(&st, 0, sizeof(st));
  // homogeneous constraints for the multiplier: zero its Dirichlet values
  const int L = Pb->mesh->l_max;
  Blas<double>::bproject(Pb->mg->bnd[L], Pb->mesh->levels[L].nb2.total, lam_u, Pb->mesh->ctx->stream);
  const mfs_status rc = stokes_solve(Pb, o, ju, jp, lam_u, lam_p, st, 1);
  if (stats) *stats = st;
  return rc;
}

mfs_status mfs_grad_log_eta(mfs_problem* Pb, const double* u, const double* lam_u, double* g) {
  if (!Pb || !u || !lam_u || !g) {
    set_error("null argument");
    return MFS_EINVAL;
  }
  if (!Pb->has_eta) {
    set_error("viscosity not set");
    return MFS_EINVAL;
  }
  return grad_log_eta(Pb, Pb->mesh->l_max, u, lam_u, g);
}
