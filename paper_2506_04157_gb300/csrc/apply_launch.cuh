// Launcher of the fused micro-tet sweep (see apply.cuh); included once per precision.
#pragma once

#include <mutex>
#include <set>
#include <utility>

#include "apply.cuh"
#include "library.h"

namespace mfs {

template <typename T>
struct PrecData;
template <>
struct PrecData<double> {
  static const double* eta(mfs_problem* P, int l) { return P->eta64[l]; }
  static const double* temp(mfs_problem* P, int l) { return P->temp64[l]; }
  static const double* lbase(mfs_problem* P) { return P->d_lbase64; }
  static const MacroGeom<double>* geom(mfs_mesh* M) { return M->d_geom64; }
  static const double* dlnrho(mfs_problem* P) { return P->d_dlnrho64; }
  static const double* dlnrho_int(mfs_problem* P) { return P->d_dlnrho_int64; }
};
template <>
struct PrecData<float> {
  static const float* eta(mfs_problem* P, int l) { return P->eta32[l]; }
  static const float* temp(mfs_problem* P, int l) { return P->temp32[l]; }
  static const float* lbase(mfs_problem* P) { return P->d_lbase32; }
  static const MacroGeom<float>* geom(mfs_mesh* M) { return M->d_geom32; }
  static const float* dlnrho(mfs_problem* P) { return P->d_dlnrho32; }
  static const float* dlnrho_int(mfs_problem* P) { return P->d_dlnrho_int32; }
};

// Opt a kernel in to its dynamic shared memory once per (kernel, device): the attribute is a
// property of the kernel on the device that is current when it is set.
inline cudaError_t smem_opt_in(const void* func, size_t smem) {
  if (smem <= 48 * 1024) return cudaSuccess;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  static std::mutex mu;
  static std::set<std::pair<const void*, int>> done;
  std::lock_guard<std::mutex> lock(mu);
  if (done.count({func, dev})) return cudaSuccess;
  e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess) done.insert({func, dev});
  return e;
}

// Sweep variants (mfs_autotune chooses one per level for the FP32 hot sweeps):
//   0: shared-memory element body, float atomics, 192 threads, 4 resident CTAs per SM
//   1: the same body with 3 resident CTAs per SM
//   2: register-resident element body, fixed-point accumulation, 192 threads, 2 CTAs per SM
//   3: the same, 128 threads, 3 CTAs per SM
//   4: the same, 128 threads, 4 CTAs per SM (128 registers)
//   5: the same, 256 threads, 2 CTAs per SM (128 registers)
//   6: the same, 192 threads, 3 CTAs per SM (96 registers)
//   7: variant 6 with the packed-pair element body (two quadrature points per FP32x2 op)
//   8: variant 4 with the packed-pair element body
// The FP32 sweeps of A alone (smoothers) and of the forward fused operator (Krylov) are
// tunable over all variants.  The other FP32 operator sets without quadrature-point viscosity
// (B, B^T, their C and density-weighted forms, the transposed fused operator) run the
// packed-pair fixed-point body with 128 threads and 4 CTAs per SM whenever the level's variant
// is a fixed-point one (2-8), else the shared-memory body; FP64 always runs the latter.
template <typename T, int OP>
constexpr bool kTunable = sizeof(T) == 4 && (OP == OP_A || OP == (OP_A | OP_BT | OP_B | OP_BC));
template <typename T, int OP>
constexpr bool kFixedBody = sizeof(T) == 4 && (OP & OP_ETAQ) == 0;

template <typename T, int OP, bool BLEND>
static void (*sweep_kernel(int variant, int* nt, size_t* smem))(const ApplyParams<T>) {
  if constexpr (kTunable<T, OP>) {
    switch (variant) {
      case 2: *nt = 192; *smem = sweep_smem_bytes<T, OP, 2>(); return stokes_tile_kernel_fixed<T, OP, BLEND, 192, 2>;
      case 3: *nt = 128; *smem = sweep_smem_bytes<T, OP, 3>(); return stokes_tile_kernel_fixed<T, OP, BLEND, 128, 3>;
      case 4: *nt = 128; *smem = sweep_smem_bytes<T, OP, 3>(); return stokes_tile_kernel_fixed<T, OP, BLEND, 128, 4>;
      case 5: *nt = 256; *smem = sweep_smem_bytes<T, OP, 2>(); return stokes_tile_kernel_fixed<T, OP, BLEND, 256, 2>;
      case 6: *nt = 192; *smem = sweep_smem_bytes<T, OP, 2>(); return stokes_tile_kernel_fixed<T, OP, BLEND, 192, 3>;
      case 7: *nt = 192; *smem = sweep_smem_bytes<T, OP, 2>(); return stokes_tile_kernel_fixed_x2<T, OP, BLEND, 192, 3>;
      case 8: *nt = 128; *smem = sweep_smem_bytes<T, OP, 3>(); return stokes_tile_kernel_fixed_x2<T, OP, BLEND, 128, 4>;
      default: break;
    }
  } else if constexpr (kFixedBody<T, OP>) {
    if (variant >= 2) {
      *nt = 128;
      *smem = sweep_smem_bytes<T, OP, 3>();
      return stokes_tile_kernel_fixed_x2<T, OP, BLEND, 128, 4>;
    }
  }
  *nt = kSweepThreads;
  *smem = sweep_smem_bytes<T, OP>();
  if (variant == 1) return stokes_tile_kernel_wide<T, OP, BLEND>;
  return stokes_tile_kernel<T, OP, BLEND>;
}

template <typename T, int OP, bool BLEND>
static mfs_status run_sweep_v(const ApplyParams<T>& prm, int n_tiles, mfs_ctx* ctx, int variant, int n_macros) {
  dim3 grid(n_tiles, n_macros);
  size_t smem = 0;
  int nt = kSweepThreads;
  auto k = sweep_kernel<T, OP, BLEND>(variant, &nt, &smem);
  MFS_CUDA(smem_opt_in((const void*)k, smem));
  auto ev = timing_events(ctx);
  if (ev.first) cudaEventRecord(ev.first, ctx->stream);
  k<<<grid, nt, smem, ctx->stream>>>(prm);
  if (ev.second) cudaEventRecord(ev.second, ctx->stream);
  return MFS_OK;
}

// the level's variant selects the kernel of the FP32 sweeps (see kTunable / kFixedBody)
template <typename T, int OP>
static mfs_status run_sweep(const ApplyParams<T>& prm, int n_tiles, int blending, mfs_ctx* ctx, int variant,
                           int n_macros) {
  if constexpr (kTunable<T, OP> || kFixedBody<T, OP>) {
    if (variant > 0 && variant < kSweepVariants)
      return blending ? run_sweep_v<T, OP, true>(prm, n_tiles, ctx, variant, n_macros)
                      : run_sweep_v<T, OP, false>(prm, n_tiles, ctx, variant, n_macros);
  }
  return blending ? run_sweep_v<T, OP, true>(prm, n_tiles, ctx, 0, n_macros)
                  : run_sweep_v<T, OP, false>(prm, n_tiles, ctx, 0, n_macros);
}

template <typename T>
ApplyParams<T> fill_params(mfs_problem* P, int lvl, int constrained, const T* u, const T* p, T* yu, T* yp,
                           const T* psum) {
  mfs_mesh* M = P->mesh;
  const LevelData& L = M->levels[lvl];
  ApplyParams<T> prm{};
  prm.u = u;
  prm.p = p;
  prm.yu = yu;
  prm.yp = yp;
  prm.eta = PrecData<T>::eta(P, lvl);
  prm.dlnrho = PrecData<T>::dlnrho(P);
  prm.dlnrho_int = PrecData<T>::dlnrho_int(P);
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
  prm.r_surf = (T)M->host.r_surf;
  prm.inv_dr = (T)(1.0 / (M->host.r_surf - M->host.r_cmb));
  prm.constrained = constrained;
  prm.bc_surface = P->bc_surface;
  prm.bc_cmb = P->bc_cmb;
  return prm;
}

template <typename T, int OP>
static mfs_status run_batch(const ApplyParams<T>* dparams, const int2* map, const int* ntiles, int nblocks,
                            int blending, cudaStream_t s) {
  const size_t smem = sweep_smem_bytes<T, OP>();
  MFS_CUDA(smem_opt_in((const void*)(blending ? stokes_tile_batch_kernel<T, OP, true>
                                              : stokes_tile_batch_kernel<T, OP, false>), smem));
  // persistent grid: as many CTAs as fit on the device at once
  int cap = 0;
  {
    int dev = 0, sms = 0, per_sm = 0;
    MFS_CUDA(cudaGetDevice(&dev));
    MFS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    if (blending)
      MFS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, stokes_tile_batch_kernel<T, OP, true>,
                                                               kSweepThreads, smem));
    else
      MFS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, stokes_tile_batch_kernel<T, OP, false>,
                                                               kSweepThreads, smem));
    cap = sms * (per_sm > 0 ? per_sm : 1);
  }
  const int grid = nblocks < cap ? nblocks : cap;
  if (blending)
    stokes_tile_batch_kernel<T, OP, true><<<grid, kSweepThreads, smem, s>>>(dparams, map, ntiles, nblocks);
  else
    stokes_tile_batch_kernel<T, OP, false><<<grid, kSweepThreads, smem, s>>>(dparams, map, ntiles, nblocks);
  MFS_CUDA(cudaGetLastError());
  return MFS_OK;
}

// ensemble sweep: op in {forward fused, transposed fused}; params already on the device
template <typename T>
mfs_status launch_batch(const ApplyParams<T>* dparams, const int2* map, const int* ntiles, int nblocks, int op,
                        int blending, cudaStream_t s) {
  switch (op) {
    case OP_A | OP_BT | OP_B | OP_BC:
      return run_batch<T, OP_A | OP_BT | OP_B | OP_BC>(dparams, map, ntiles, nblocks, blending, s);
    case OP_A | OP_BT | OP_B: return run_batch<T, OP_A | OP_BT | OP_B>(dparams, map, ntiles, nblocks, blending, s);
    case OP_A | OP_BT | OP_CT | OP_B:
      return run_batch<T, OP_A | OP_BT | OP_CT | OP_B>(dparams, map, ntiles, nblocks, blending, s);
    default: set_error("internal: unsupported batched operator %d", op); return MFS_EINVAL;
  }
}

template <typename T>
mfs_status launch_apply(mfs_problem* P, int lvl, int op, int constrained, int withc_b, const T* u,
                             const T* p, T* yu, T* yp, const T* psum, int zero_out, int m0, int m1) {
  mfs_mesh* M = P->mesh;
  const LevelData& L = M->levels[lvl];
  cudaStream_t s = M->ctx->stream;
  ApplyParams<T> prm{};
  prm.u = u;
  prm.p = p;
  prm.yu = yu;
  prm.yp = yp;
  prm.eta = PrecData<T>::eta(P, lvl);
  prm.dlnrho = PrecData<T>::dlnrho(P);
  prm.dlnrho_int = PrecData<T>::dlnrho_int(P);
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
  prm.r_surf = (T)M->host.r_surf;
  prm.inv_dr = (T)(1.0 / (M->host.r_surf - M->host.r_cmb));
  prm.constrained = constrained;
  prm.bc_surface = P->bc_surface;
  prm.bc_cmb = P->bc_cmb;
  prm.m0 = m0;
  const int nm = m1 - m0;
  if (lvl <= P->l_eta && (op & OP_A)) {
    // quadrature-point viscosity on this level
    if (op != OP_A) {
      set_error("level %d evaluates the viscosity at quadrature points: only A alone is available there (l_eta = %d)",
                lvl, P->l_eta);
      return MFS_EINVAL;
    }
    op = OP_A | OP_ETAQ;
    prm.temp = PrecData<T>::temp(P, lvl);
    prm.lbase = PrecData<T>::lbase(P);
    prm.n_lbase = (int)P->lbase_host.size();
    prm.E_A = (T)P->E_A;
    prm.V_A = (T)P->V_A;
    prm.r_surf = (T)M->host.r_surf;
  }
  if (zero_out && (op & (OP_A | OP_BT))) MFS_CUDA(cudaMemsetAsync(yu, 0, sizeof(T) * 3 * (size_t)L.nb2.total, s));
  if (zero_out && (op & OP_B)) MFS_CUDA(cudaMemsetAsync(yp, 0, sizeof(T) * (size_t)L.nb1.total, s));
  if ((op & OP_B) && withc_b) op |= OP_BC;
  if (P->rho_weighted && (op & (OP_BC | OP_CT))) op |= OP_RHO;
  const int bl = M->host.blending;
  switch (op) {
    case OP_A: MFS_TRY((run_sweep<T, OP_A>(prm, L.n_tiles, bl, M->ctx, L.variant_a, nm))); break;
    case OP_A | OP_ETAQ: MFS_TRY((run_sweep<T, OP_A | OP_ETAQ>(prm, L.n_tiles, bl, M->ctx, 0, nm))); break;
    case OP_BT: MFS_TRY((run_sweep<T, OP_BT>(prm, L.n_tiles, bl, M->ctx, L.variant, nm))); break;
    case OP_BT | OP_CT: MFS_TRY((run_sweep<T, OP_BT | OP_CT>(prm, L.n_tiles, bl, M->ctx, L.variant, nm))); break;
    case OP_B: MFS_TRY((run_sweep<T, OP_B>(prm, L.n_tiles, bl, M->ctx, L.variant, nm))); break;
    case OP_B | OP_BC: MFS_TRY((run_sweep<T, OP_B | OP_BC>(prm, L.n_tiles, bl, M->ctx, L.variant, nm))); break;
    case OP_A | OP_BT | OP_B | OP_BC: MFS_TRY((run_sweep<T, OP_A | OP_BT | OP_B | OP_BC>(prm, L.n_tiles, bl, M->ctx, L.variant, nm))); break;
    case OP_A | OP_BT | OP_CT | OP_B: MFS_TRY((run_sweep<T, OP_A | OP_BT | OP_CT | OP_B>(prm, L.n_tiles, bl, M->ctx, L.variant, nm))); break;
    case OP_B | OP_BC | OP_RHO: MFS_TRY((run_sweep<T, OP_B | OP_BC | OP_RHO>(prm, L.n_tiles, bl, M->ctx, 0, nm))); break;
    case OP_BT | OP_CT | OP_RHO: MFS_TRY((run_sweep<T, OP_BT | OP_CT | OP_RHO>(prm, L.n_tiles, bl, M->ctx, 0, nm))); break;
    case OP_A | OP_BT | OP_B | OP_BC | OP_RHO:
      MFS_TRY((run_sweep<T, OP_A | OP_BT | OP_B | OP_BC | OP_RHO>(prm, L.n_tiles, bl, M->ctx, 0, nm))); break;
    case OP_A | OP_BT | OP_CT | OP_B | OP_RHO:
      MFS_TRY((run_sweep<T, OP_A | OP_BT | OP_CT | OP_B | OP_RHO>(prm, L.n_tiles, bl, M->ctx, 0, nm))); break;
    default: set_error("internal: unsupported operator combination %d", op); return MFS_EINVAL;
  }
  MFS_CUDA(cudaGetLastError());
  return MFS_OK;
}

}  // namespace mfs
