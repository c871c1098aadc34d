// Autotuner of the sweep launch: per refinement level, the FP32 hot sweeps (fused
// saddle-point apply, A alone) run in one of kSweepVariants launch shapes — the element body
// (shared-memory or register-resident), the threads per CTA and the resident CTAs per SM
// (apply_launch.cuh lists them); the fastest, timed with CUDA events on this GPU, is kept.
// Choices are cached in a small text file so later runs skip the timing.
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
  M->levels[l].variant = M->levels[l].variant_a = variant;
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
  std::vector<std::vector<double>> tv(L + 1, std::vector<double>(kSweepVariants, 0.0));
  if (cache_path) {
    if (FILE* f = std::fopen(cache_path, "r")) {
      char line[512];
      while (std::fgets(line, sizeof(line), f)) {
        int lv = -1, v = -1;
        if (std::sscanf(line, " {\"level\": %d, \"variant\": %d", &lv, &v) == 2 && lv >= 0 && lv <= L && v >= 0 &&
            v < kSweepVariants)
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
      for (int v = 0; v < kSweepVariants && st == MFS_OK; ++v) st = time_variant(P, l, v, u, p, yu, yp, &tv[l][v]);
    }
    cudaFree(u);
    cudaFree(yu);
    cudaFree(p);
    cudaFree(yp);
    if (st != MFS_OK) {
      M->levels[l].variant = kDefaultSweepVariant;
      M->levels[l].variant_a = kDefaultSweepVariantA;
      return st;
    }
    int best = 0;
    for (int v = 1; v < kSweepVariants; ++v)
      if (tv[l][v] < tv[l][best]) best = v;
    chosen[l] = best;
    timed = true;
  }
  for (int l = 0; l <= L; ++l) M->levels[l].variant = M->levels[l].variant_a = chosen[l];
  M->tuning_gen++;
  if (cache_path && timed) {
    if (FILE* f = std::fopen(cache_path, "w")) {
      std::fprintf(f, "[\n");
      for (int l = 0; l <= L; ++l) {
        std::fprintf(f, " {\"level\": %d, \"variant\": %d, \"ms\": [", l, chosen[l]);
        for (int v = 0; v < kSweepVariants; ++v) std::fprintf(f, "%s%.6f", v ? ", " : "", tv[l][v]);
        std::fprintf(f, "]}%s\n", l < L ? "," : "");
      }
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

mfs_status mfs_set_tuning(mfs_problem* P, int lvl, int variant) {
  if (!P || lvl < 0 || lvl > P->mesh->l_max || variant < 0 || variant >= kSweepVariants) {
    set_error("invalid arguments: level outside the mesh or variant outside 0..%d", kSweepVariants - 1);
    return MFS_EINVAL;
  }
  P->mesh->levels[lvl].variant = P->mesh->levels[lvl].variant_a = variant;
  P->mesh->tuning_gen++;
  return MFS_OK;
}
