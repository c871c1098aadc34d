// Throughput of the fused multiply-add pipes of the device: the measured denominators of
// the micro-tet sweeps' ALU roofline (the sweeps are bound by FP32, resp. FP64, arithmetic,
// not by HBM).  Each thread runs kChains independent dependency chains of FMAs whose values
// stay bounded (x <- x * a + b with |a| < 1), so nothing overflows and nothing can be folded
// away; the result is stored so that the chains stay live.
#include <cuda_runtime.h>

#include "library.h"

namespace mfs {

constexpr int kChains = 8;
constexpr int kUnroll = 16;

// kind 0: FP32 fma.rn.f32; kind 1: FP32 packed pair fma.rn.f32x2 (two FMAs per instruction);
// kind 2: FP64 fma.rn.f64
template <int KIND>
__global__ void __launch_bounds__(256) k_fma_chain(float* out32, double* out64, int iters) {
  if (KIND == 0) {
    float x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = 1e-3f * (threadIdx.x + c);
    const float a = 0.999999f, b = 1e-7f;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
      for (int u = 0; u < kUnroll; ++u)
#pragma unroll
        for (int c = 0; c < kChains; ++c) asm volatile("fma.rn.f32 %0, %0, %1, %2;" : "+f"(x[c]) : "f"(a), "f"(b));
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    out32[blockIdx.x * blockDim.x + threadIdx.x] = s;
  } else if (KIND == 1) {
    unsigned long long x[kChains], a2, b2;
    const float a = 0.999999f, b = 1e-7f;
    asm("mov.b64 %0, {%1, %2};" : "=l"(a2) : "f"(a), "f"(a));
    asm("mov.b64 %0, {%1, %2};" : "=l"(b2) : "f"(b), "f"(b));
#pragma unroll
    for (int c = 0; c < kChains; ++c) {
      const float lo = 1e-3f * (threadIdx.x + c), hi = 2e-3f * (threadIdx.x + c);
      asm("mov.b64 %0, {%1, %2};" : "=l"(x[c]) : "f"(lo), "f"(hi));
    }
    for (int i = 0; i < iters; ++i) {
#pragma unroll
      for (int u = 0; u < kUnroll; ++u)
#pragma unroll
        for (int c = 0; c < kChains; ++c) asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(x[c]) : "l"(a2), "l"(b2));
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) {
      float lo, hi;
      asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(x[c]));
      s += lo + hi;
    }
    out32[blockIdx.x * blockDim.x + threadIdx.x] = s;
  } else {
    double x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = 1e-3 * (threadIdx.x + c);
    const double a = 0.999999, b = 1e-7;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
      for (int u = 0; u < kUnroll; ++u)
#pragma unroll
        for (int c = 0; c < kChains; ++c) asm volatile("fma.rn.f64 %0, %0, %1, %2;" : "+d"(x[c]) : "d"(a), "d"(b));
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    out64[blockIdx.x * blockDim.x + threadIdx.x] = s;
  }
}

}  // namespace mfs

using namespace mfs;

extern "C" mfs_status mfs_fma_peak(mfs_ctx* ctx, int kind, int launches, int iters, double* tflops, double* ms) {
  if (!ctx || !tflops || !ms || kind < 0 || kind > 2 || launches < 1 || iters < 1) {
    set_error("mfs_fma_peak: null argument, kind outside 0..2, or launches/iters < 1");
    return MFS_EINVAL;
  }
  int dev = 0, sms = 0;
  MFS_CUDA(cudaGetDevice(&dev));
  MFS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int threads = 256, blocks = sms * 8;   // 64 warps per SM: every FMA pipe fed
  const size_t nout = (size_t)blocks * threads;
  float* o32 = nullptr;
  double* o64 = nullptr;
  MFS_CUDA(cudaMalloc((void**)&o32, nout * sizeof(float)));
  cudaError_t e = cudaMalloc((void**)&o64, nout * sizeof(double));
  if (e != cudaSuccess) {
    cudaFree(o32);
    return cuda_fail(e, "cudaMalloc(fma peak output)");
  }
  cudaStream_t s = ctx->stream;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  auto launch = [&](int it) {
    if (kind == 0) k_fma_chain<0><<<blocks, threads, 0, s>>>(o32, o64, it);
    else if (kind == 1) k_fma_chain<1><<<blocks, threads, 0, s>>>(o32, o64, it);
    else k_fma_chain<2><<<blocks, threads, 0, s>>>(o32, o64, it);
  };
  launch(iters < 64 ? iters : 64);   // warm-up (module load, clocks)
  cudaEventRecord(e0, s);
  for (int k = 0; k < launches; ++k) launch(iters);
  cudaEventRecord(e1, s);
  e = cudaEventSynchronize(e1);
  float t = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
  if (e == cudaSuccess) e = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(o32);
  cudaFree(o64);
  if (e != cudaSuccess) return cuda_fail(e, "mfs_fma_peak");
  const double fma_per_thread = (double)iters * kUnroll * kChains * (kind == 1 ? 2 : 1);
  const double flops = 2.0 * fma_per_thread * (double)nout * launches;
  *ms = (double)t;
  *tflops = flops / ((double)t * 1e-3) / 1e12;
  return MFS_OK;
}
