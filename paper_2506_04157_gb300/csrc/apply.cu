// Launchers of the fused micro-tet sweep (see apply.cuh).
#include "apply.cuh"
#include "library.h"

namespace mfs {

template <typename T>
static const T* eta_of(mfs_problem* P, int lvl);
template <>
const double* eta_of<double>(mfs_problem* P, int lvl) { return P->eta64[lvl]; }
template <>
const float* eta_of<float>(mfs_problem* P, int lvl) { return P->eta32[lvl]; }

template <typename T>
static const MacroGeom<T>* geom_of(mfs_mesh* M);
template <>
const MacroGeom<double>* geom_of<double>(mfs_mesh* M) { return M->d_geom64; }
template <>
const MacroGeom<float>* geom_of<float>(mfs_mesh* M) { return M->d_geom32; }

template <typename T>
static const T* dlnrho_of(mfs_problem* P);
template <>
const double* dlnrho_of<double>(mfs_problem* P) { return P->d_dlnrho64; }
template <>
const float* dlnrho_of<float>(mfs_problem* P) { return P->d_dlnrho32; }

template <typename T, int OP>
static void run(const ApplyParams<T>& prm, int n_tiles, mfs_ctx* ctx) {
  dim3 grid(n_tiles, kMacroCells);
  auto ev = timing_events(ctx);
  if (ev.first) cudaEventRecord(ev.first, ctx->stream);
  stokes_tile_kernel<T, OP><<<grid, 256, 0, ctx->stream>>>(prm);
  if (ev.second) cudaEventRecord(ev.second, ctx->stream);
}

template <typename T>
mfs_status launch_apply(mfs_problem* P, int lvl, int op, int constrained, int withc_b, const T* u,
                        const T* p, T* yu, T* yp, const T* psum) {
  mfs_mesh* M = P->mesh;
  const LevelData& L = M->levels[lvl];
  cudaStream_t s = M->ctx->stream;
  ApplyParams<T> prm;
  prm.u = u;
  prm.p = p;
  prm.yu = yu;
  prm.yp = yp;
  prm.eta = eta_of<T>(P, lvl);
  prm.dlnrho = dlnrho_of<T>(P);
  prm.n_dlnrho = P->n_dlnrho;
  prm.psum = psum;
  prm.geom = geom_of<T>(M);
  prm.topo = M->d_topo;
  prm.tiles = L.d_tiles;
  prm.tets = L.d_tets;
  prm.classes = L.d_classes;
  prm.nb2 = L.nb2;
  prm.nb1 = L.nb1;
  prm.n = L.n;
  prm.r_cmb = (T)M->host.r_cmb;
  prm.r_surf = (T)M->host.r_surf;
  prm.blending = M->host.blending;
  prm.constrained = constrained;
  prm.withc_b = withc_b;
  prm.bc_surface = P->bc_surface;
  prm.bc_cmb = P->bc_cmb;
  if (op & (OP_A | OP_BT)) MFS_CUDA(cudaMemsetAsync(yu, 0, sizeof(T) * 3 * (size_t)L.nb2.total, s));
  if (op & OP_B) MFS_CUDA(cudaMemsetAsync(yp, 0, sizeof(T) * (size_t)L.nb1.total, s));
  switch (op) {
    case OP_A: run<T, OP_A>(prm, L.n_tiles, M->ctx); break;
    case OP_BT: run<T, OP_BT>(prm, L.n_tiles, M->ctx); break;
    case OP_BT | OP_CT: run<T, OP_BT | OP_CT>(prm, L.n_tiles, M->ctx); break;
    case OP_B: run<T, OP_B>(prm, L.n_tiles, M->ctx); break;
    case OP_A | OP_BT | OP_B: run<T, OP_A | OP_BT | OP_B>(prm, L.n_tiles, M->ctx); break;
    case OP_A | OP_BT | OP_CT | OP_B: run<T, OP_A | OP_BT | OP_CT | OP_B>(prm, L.n_tiles, M->ctx); break;
    default: set_error("internal: unsupported operator combination %d", op); return MFS_EINVAL;
  }
  MFS_CUDA(cudaGetLastError());
  return MFS_OK;
}

template mfs_status launch_apply<double>(mfs_problem*, int, int, int, int, const double*, const double*,
                                         double*, double*, const double*);
template mfs_status launch_apply<float>(mfs_problem*, int, int, int, int, const float*, const float*,
                                        float*, float*, const float*);

}  // namespace mfs
