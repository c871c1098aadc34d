// Autotuner of the sweep launch: per refinement level, the FP32 hot sweeps (fused
// saddle-point apply, A alone) run in one of two register budgets (4 or 3 resident CTAs
// per SM); the faster one, timed with CUDA events on this GPU, is kept.  Choices are
// cached in a small text file so later runs skip the timing.
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "library.h"

namespace mfs {

__global__ void k_fill_pattern(int64_t n, float* v, float scale) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    v[i] = scale * (float)(((i * 2654435761ll) % 2001) - 1000) * 1e-3f;
}

static mfs_status time_variant(mfs_problem* P, int l, int variant, float* u, float* p, float* yu, float* yp,
                               double* ms_out) {
  mfs_mesh* M = P->mesh;
  cudaStream_t s = M->ctx->stream;
  M->levels[l].variant = variant;
  for (int w = 0; w < 2; ++w)
    MFS_TRY(launch_apply<float>(P, l, OP_A | OP_BT | OP_B, 0, 1, u, p, yu, yp, nullptr));
  cudaEvent_t e0, e1;
  MFS_CUDA(cudaEventCreate(&e0));
  MFS_CUDA(cudaEventCreate(&e1));
  const int reps = 5;
  cudaEventRecord(e0, s);
  for (int r = 0; r < reps; ++r) {
    MFS_TRY(launch_apply<float>(P, l, OP_A | OP_BT | OP_B, 0, 1, u, p, yu, yp, nullptr));
    MFS_TRY(launch_apply<float>(P, l, OP_A, 0, 0, u, nullptr, yu, nullptr, nullptr));
  }
  cudaEventRecord(e1, s);
  MFS_CUDA(cudaEventSynchronize(e1));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *ms_out = ms / reps;
  return MFS_OK;
}

}  // namespace mfs

using namespace mfs;

mfs_status mfs_autotune(mfs_problem* P, const char* cache_path) {
  if (!P || !P->has_eta) {
    set_error("null problem or viscosity not set");
    return MFS_EINVAL;
  }
  mfs_mesh* M = P->mesh;
  const int L = M->l_max;
  std::vector<int> chosen(L + 1, -1);
  std::vector<double> t0(L + 1, 0.0), t1(L + 1, 0.0);
  if (cache_path) {
    if (FILE* f = std::fopen(cache_path, "r")) {
      char line[256];
      while (std::fgets(line, sizeof(line), f)) {
        int lv = -1, v = -1;
        if (std::sscanf(line, " {\"level\": %d, \"variant\": %d", &lv, &v) == 2 && lv >= 0 && lv <= L &&
            (v == 0 || v == 1))
          chosen[lv] = v;
      }
      std::fclose(f);
    }
  }
  bool timed = false;
  for (int l = 0; l <= L; ++l) {
    if (chosen[l] >= 0) continue;
    const LevelData& Lv = M->levels[l];
    const int64_t nu = 3 * (int64_t)Lv.nb2.total, np = Lv.nb1.total;
    float *u = nullptr, *yu = nullptr, *p = nullptr, *yp = nullptr;
    cudaError_t e = cudaMalloc((void**)&u, sizeof(float) * nu);
    if (e == cudaSuccess) e = cudaMalloc((void**)&yu, sizeof(float) * nu);
    if (e == cudaSuccess) e = cudaMalloc((void**)&p, sizeof(float) * np);
    if (e == cudaSuccess) e = cudaMalloc((void**)&yp, sizeof(float) * np);
    mfs_status st = e == cudaSuccess ? MFS_OK : cuda_fail(e, "cudaMalloc(autotune)");
    if (st == MFS_OK) {
      k_fill_pattern<<<256, 256, 0, M->ctx->stream>>>(nu, u, 1.0f);
      k_fill_pattern<<<64, 256, 0, M->ctx->stream>>>(np, p, 0.5f);
      st = time_variant(P, l, 0, u, p, yu, yp, &t0[l]);
      if (st == MFS_OK) st = time_variant(P, l, 1, u, p, yu, yp, &t1[l]);
    }
    cudaFree(u);
    cudaFree(yu);
    cudaFree(p);
    cudaFree(yp);
    if (st != MFS_OK) {
      M->levels[l].variant = 0;
      return st;
    }
    chosen[l] = t1[l] < t0[l] ? 1 : 0;
    timed = true;
  }
  for (int l = 0; l <= L; ++l) M->levels[l].variant = chosen[l];
  M->tuning_gen++;
  if (cache_path && timed) {
    if (FILE* f = std::fopen(cache_path, "w")) {
      std::fprintf(f, "[\n");
      for (int l = 0; l <= L; ++l)
        std::fprintf(f, " {\"level\": %d, \"variant\": %d, \"ms_default\": %.6f, \"ms_wide\": %.6f}%s\n", l, chosen[l],
                     t0[l], t1[l], l < L ? "," : "");
      std::fprintf(f, "]\n");
      std::fclose(f);
    }
  }
  return MFS_OK;
}

mfs_status mfs_get_tuning(const mfs_problem* P, int lvl, int* variant) {
  if (!P || !variant || lvl < 0 || lvl > P->mesh->l_max) {
    set_error("invalid arguments");
    return MFS_EINVAL;
  }
  *variant = P->mesh->levels[lvl].variant;
  return MFS_OK;
}
