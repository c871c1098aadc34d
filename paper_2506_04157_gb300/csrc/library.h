// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/mfs.h"
#include "mfs_internal.h"

namespace mfs {

// ---- error handling ----
void set_error(const char* fmt, ...);
mfs_status cuda_fail(cudaError_t e, const char* what);
#define MFS_CUDA(call)                                   \
  do {                                                   \
    cudaError_t e__ = (call);                            \
    if (e__ != cudaSuccess) return cuda_fail(e__, #call); \
  } while (0)
#define MFS_TRY(call)                   \
  do {                                  \
    mfs_status s__ = (call);            \
    if (s__ != MFS_OK) return s__;      \
  } while (0)

// ---- host macro mesh (Sec. 4.1: icosahedral shell, one radial layer) ----
struct HostMacroMesh {
  double r_cmb = 0.5, r_surf = 1.0;
  int blending = 1;
  double unit[24][3];
  double verts[24][3];
  int layer[24];
  int cells[60][4];       // increasing global vertex ids
  int cell_prism[60];
  int edges[102][2];
  int faces[140][3];
  double prism_nh[20][3];
  double prism_delta[20];
  MacroTopo topo[60];
  MacroGeom<double> geom[60];
  void build(double r_cmb, double r_surf, int blending);
  // position of a lattice point of macro m with integer barycentrics i (sum N)
  void straight_point(int m, const int i[4], int N, double x[3]) const;
  void blend_point(int m, const double xs[3], double x[3]) const;
};

// Tiles and per-class local tet lists of one level.
struct HostTiles {
  std::vector<Tile> tiles;
  std::vector<uint16_t> tets;
  std::vector<int2> classes;
};
HostTiles build_tiles(int n);

// launch variants of the FP32 hot sweeps (element body, threads per CTA, resident CTAs per
// SM), chosen per level by mfs_autotune; apply_launch.cuh lists them.  The defaults are the
// fastest on the GB300, both the register-resident body with the quadrature points in packed
// FP32 pairs and fixed-point accumulation: 128 threads and 4 CTAs per SM for the fused
// operator (and the other operator sets; fastest at levels 5 and 6), 192 threads and 3 CTAs
// per SM for A alone (the smoother's operator, which needs fewer registers; fastest on every
// level).
constexpr int kSweepVariants = 9;
constexpr int kDefaultSweepVariant = 8;
constexpr int kDefaultSweepVariantA = 7;

struct LevelData {
  int l = 0, n = 1;
  Numbering nb2{}, nb1{};
  int n_tiles = 0;
  Tile* d_tiles = nullptr;
  uint16_t* d_tets = nullptr;
  int2* d_classes = nullptr;
  int* d_ids2 = nullptr;     // [60 * n_tiles][NSLOT2] P2 id | geometric class << 29, or -1
  int* d_ids1 = nullptr;     // [60 * n_tiles][NSLOT1] P1 id, or -1
  // P1 full weighting from this level to the next coarser one (rows: coarse vertices)
  int er_rows = 0;
  int* d_er_rp = nullptr;
  int* d_er_ci = nullptr;
  double* d_er_w = nullptr;
  int64_t n_tets = 0, n_surface = 0, n_cmb = 0;
  int variant = kDefaultSweepVariant;   // sweep launch variant (mfs_autotune / mfs_set_tuning)
  int variant_a = kDefaultSweepVariantA;   // the same for the sweep of A alone
  // viscosity law (built on first use): per P1 vertex the finest-level P2 node at the same
  // point and the vertex's radius; per P2 node (levels below the finest) the finest node
  int* d_vfine = nullptr;
  double* d_vrad = nullptr;
  int* d_p2fine = nullptr;
};

template <typename T>
MacroGeom<T> cast_geom(const MacroGeom<double>& g);

}  // namespace mfs

namespace mfs {
struct MG;
struct PoissonMG;
struct TempWork;
void problem_release_solver(mfs_problem* P);
void pmg_destroy(PoissonMG* W);
void temp_destroy(TempWork* W);
}  // namespace mfs

struct mfs_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  // optional CUDA-event timing of the element-sweep kernels
  int timing = 0;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_used;
};

namespace mfs {
// events bracketing one sweep launch when ctx->timing is on (nullptr otherwise)
std::pair<cudaEvent_t, cudaEvent_t> timing_events(mfs_ctx* ctx);
}

struct mfs_mesh {
  mfs_ctx* ctx = nullptr;
  int l_max = 0;
  mfs::HostMacroMesh host;
  mfs::MacroTopo* d_topo = nullptr;
  mfs::MacroGeom<double>* d_geom64 = nullptr;
  mfs::MacroGeom<float>* d_geom32 = nullptr;
  std::vector<mfs::LevelData> levels;
  int tuning_gen = 0;   // bumped when a level's sweep variant changes (captured graphs go stale)
};

namespace mfs {
// Visit every lattice point of every macro at N intervals: f(m, i[4], id) with the point's
// integer barycentrics i (sum N) in macro m and its global id.
template <typename F>
inline void for_each_point(const mfs_mesh* M, int N, F f) {
  const Numbering nb = make_numbering(N);
  for (int m = 0; m < 60; ++m)
    for (int i3 = 0; i3 <= N; ++i3)
      for (int i2 = 0; i2 <= N - i3; ++i2)
        for (int i1 = 0; i1 <= N - i3 - i2; ++i1) {
          const int i[4] = {N - i1 - i2 - i3, i1, i2, i3};
          f(m, i, lattice_id(M->host.topo[m], nb, m, i[0], i[1], i[2], i[3]));
        }
}
}  // namespace mfs

struct mfs_problem {
  mfs_mesh* mesh = nullptr;
  int bc_surface = 0, bc_cmb = 1;
  bool has_eta = false;
  std::vector<double*> eta64;   // per level, [n_p1(l)]
  std::vector<float*> eta32;
  double* d_dlnrho64 = nullptr;
  float* d_dlnrho32 = nullptr;
  double* d_dlnrho_int64 = nullptr;   // integral of the table from r_cmb to each node
  float* d_dlnrho_int32 = nullptr;
  int rho_weighted = 0;             // constraint -int q div(rho u) instead of B + C
  int n_dlnrho = 1;
  // reduction workspace: partial sums and a few device scalars
  double* d_red64 = nullptr;    // [kRedSlots]
  float* d_red32 = nullptr;
  mfs::MG* mg = nullptr;        // multigrid hierarchy and solver workspaces
  mfs::PoissonMG* pmg = nullptr;  // weighted-BFBT operators (K_{1/sqrt(eta)} GMG, lumped mass)
  mfs::TempWork* tw = nullptr;    // temperature-step workspace
  // temperature-dependent viscosity law (mfs_set_viscosity_law / mfs_set_temperature):
  // levels l <= l_eta evaluate eta at the quadrature points from temp64/32[l]
  int l_eta = -1;                  // in effect (set with the temperature)
  int law_l_eta = -1;              // requested by mfs_set_viscosity_law
  double E_A = 0.0, V_A = 0.0;
  std::vector<double> lbase_host;  // log10 eta_base table
  double* d_lbase64 = nullptr;
  float* d_lbase32 = nullptr;
  std::vector<double*> temp64;  // per level, P2 temperature (levels <= l_eta)
  std::vector<float*> temp32;
  int version = 0;              // bumped by every coefficient change (captured graphs go stale)
};

namespace mfs {


constexpr int kRedBlocks = 512;     // partial sums of the two-pass reductions
constexpr int kRedSlots = kRedBlocks + 64;

// ---- launchers (apply.cu) ----
// The sweep adds into yu / yp; they are zeroed first unless zero_out == 0 (the caller
// guarantees zeros, e.g. the smoother's fused update leaves its apply buffer zeroed).
// m0, m1: the launch covers the micro-tets of macros m0 <= m < m1 (all 60 by default).
template <typename T>
mfs_status launch_apply(mfs_problem* P, int lvl, int op, int constrained, int withc_b, const T* u,
                        const T* p, T* yu, T* yp, const T* psum, int zero_out = 1, int m0 = 0,
                        int m1 = kMacroCells);

template <typename T>
struct ApplyParams;
template <typename T>
ApplyParams<T> fill_params(mfs_problem* P, int lvl, int constrained, const T* u, const T* p, T* yu, T* yp,
                           const T* psum);
template <typename T>
mfs_status launch_batch(const ApplyParams<T>* dparams, const int2* map, const int* ntiles, int nblocks, int op,
                        int blending, cudaStream_t s);

// launch_apply plus the pressure projections of the constrained mode
template <typename T>
mfs_status apply_constrained(mfs_problem* P, int lvl, int op, int constrained, int withc_b, const T* u, const T* p,
                             T* yu, T* yp);

// ---- vector kernels (vec.cu) ----
template <typename T>
mfs_status vec_sum(const T* x, int64_t n, T* d_partials, T* d_out, cudaStream_t s);
template <typename T>
mfs_status vec_sub_mean(T* x, int64_t n, const T* d_sum, cudaStream_t s);
mfs_status inject_p1(const mfs_mesh* M, int l_from, int l_to, const double* src, double* dst);
void p1_transfer_triplets(const mfs_mesh* M, int l, std::vector<int>& tv, std::vector<int>& tj,
                          std::vector<double>& tw);
mfs_status build_eta_restriction(mfs_mesh* M, int l);
mfs_status restrict_eta(const mfs_mesh* M, int l, const double* fine, double* coarse);
mfs_status build_id_tables(const mfs_mesh* M, LevelData& L);
mfs_status convert_f64_f32(const double* src, float* dst, int64_t n, cudaStream_t s);
mfs_status exp_inplace(double* x, int64_t n, cudaStream_t s);
// eta[i] = 10^lbase(rad[i]) exp(-E_A T[fine[i]] + V_A (r1 - rad[i])), lbase linear in r on a
// uniform grid of nt entries over [r0, r1] (Eq. ViscosityDef)
mfs_status law_eta(int64_t n, const int* fine, const double* rad, const double* T, const double* lbase, int nt,
                   double E_A, double V_A, double r0, double r1, double* eta, cudaStream_t s);
// dst[i] = src[idx[i]]
mfs_status gather_f64(int64_t n, const int* idx, const double* src, double* dst, cudaStream_t s);

}  // namespace mfs
