// Launcher of the fused micro-tet sweep (see apply.cuh); included once per precision.
#pragma once

#include "apply.cuh"
#include "library.h"

namespace mfs {

template <typename T>
struct PrecData;
template <>
struct PrecData<double> {
  static const double* eta(mfs_problem* P, int l) { return P->eta64[l]; }
  static const MacroGeom<double>* geom(mfs_mesh* M) { return M->d_geom64; }
  static const double* dlnrho(mfs_problem* P) { return P->d_dlnrho64; }
};
template <>
struct PrecData<float> {
  static const float* eta(mfs_problem* P, int l) { return P->eta32[l]; }
  static const MacroGeom<float>* geom(mfs_mesh* M) { return M->d_geom32; }
  static const float* dlnrho(mfs_problem* P) { return P->d_dlnrho32; }
};

template <typename T, int OP, bool BLEND>
static cudaError_t sweep_attr() {
  // opt in to more than 48 KB of dynamic shared memory once per instantiation
  static cudaError_t e = cudaFuncSetAttribute(stokes_tile_kernel<T, OP, BLEND>,
                                              cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)sweep_smem_bytes<T, OP>());
  return e;
}

template <typename T, int OP>
static mfs_status run_sweep(const ApplyParams<T>& prm, int n_tiles, int blending, mfs_ctx* ctx) {
  dim3 grid(n_tiles, kMacroCells);
  const size_t smem = sweep_smem_bytes<T, OP>();
  const cudaError_t attr = blending ? sweep_attr<T, OP, true>() : sweep_attr<T, OP, false>();
  MFS_CUDA(attr);
  auto ev = timing_events(ctx);
  if (ev.first) cudaEventRecord(ev.first, ctx->stream);
  if (blending) stokes_tile_kernel<T, OP, true><<<grid, kSweepThreads, smem, ctx->stream>>>(prm);
  else stokes_tile_kernel<T, OP, false><<<grid, kSweepThreads, smem, ctx->stream>>>(prm);
  if (ev.second) cudaEventRecord(ev.second, ctx->stream);
  return MFS_OK;
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
  prm.eta = PrecData<T>::eta(P, lvl);
  prm.dlnrho = PrecData<T>::dlnrho(P);
  prm.n_dlnrho = P->n_dlnrho;
  prm.psum = psum;
  prm.geom = PrecData<T>::geom(M);
  prm.tiles = L.d_tiles;
  prm.tets = L.d_tets;
  prm.classes = L.d_classes;
  prm.ids2 = L.d_ids2;
  prm.ids1 = L.d_ids1;
  prm.n_p2 = L.nb2.total;
  prm.n_p1 = L.nb1.total;
  prm.n = L.n;
  prm.r_cmb = (T)M->host.r_cmb;
  prm.inv_dr = (T)(1.0 / (M->host.r_surf - M->host.r_cmb));
  prm.constrained = constrained;
  prm.bc_surface = P->bc_surface;
  prm.bc_cmb = P->bc_cmb;
  if (op & (OP_A | OP_BT)) MFS_CUDA(cudaMemsetAsync(yu, 0, sizeof(T) * 3 * (size_t)L.nb2.total, s));
  if (op & OP_B) MFS_CUDA(cudaMemsetAsync(yp, 0, sizeof(T) * (size_t)L.nb1.total, s));
  if ((op & OP_B) && withc_b) op |= OP_BC;
  const int bl = M->host.blending;
  switch (op) {
    case OP_A: MFS_TRY((run_sweep<T, OP_A>(prm, L.n_tiles, bl, M->ctx))); break;
    case OP_BT: MFS_TRY((run_sweep<T, OP_BT>(prm, L.n_tiles, bl, M->ctx))); break;
    case OP_BT | OP_CT: MFS_TRY((run_sweep<T, OP_BT | OP_CT>(prm, L.n_tiles, bl, M->ctx))); break;
    case OP_B: MFS_TRY((run_sweep<T, OP_B>(prm, L.n_tiles, bl, M->ctx))); break;
    case OP_B | OP_BC: MFS_TRY((run_sweep<T, OP_B | OP_BC>(prm, L.n_tiles, bl, M->ctx))); break;
    case OP_A | OP_BT | OP_B | OP_BC: MFS_TRY((run_sweep<T, OP_A | OP_BT | OP_B | OP_BC>(prm, L.n_tiles, bl, M->ctx))); break;
    case OP_A | OP_BT | OP_CT | OP_B: MFS_TRY((run_sweep<T, OP_A | OP_BT | OP_CT | OP_B>(prm, L.n_tiles, bl, M->ctx))); break;
    default: set_error("internal: unsupported operator combination %d", op); return MFS_EINVAL;
  }
  MFS_CUDA(cudaGetLastError());
  return MFS_OK;
}

}  // namespace mfs
