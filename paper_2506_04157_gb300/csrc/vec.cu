// Vector kernels: deterministic two-pass sums, mean removal (P_p of Sec. 5.1),
// viscosity injection to coarser levels (Sec. 5.2.2: eta as a P1 function on every
// level, coarse vertices are fine vertices), precision conversion.
#include "library.h"

namespace mfs {

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <typename T>
__device__ __forceinline__ T block_sum(T v) {
  __shared__ T red[32];
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  const int nw = (blockDim.x + 31) >> 5;
  v = threadIdx.x < nw ? red[threadIdx.x] : T(0);
  if (w == 0) v = warp_sum(v);
  return v;
}

// pass 1: per-block partial sums over a grid-stride range
template <typename T>
__global__ void sum_partials_kernel(const T* __restrict__ x, int64_t n, T* __restrict__ partials) {
  T acc = T(0);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    acc += x[i];
  acc = block_sum(acc);
  if (threadIdx.x == 0) partials[blockIdx.x] = acc;
}

// pass 2: one block adds the partials in a fixed order
template <typename T>
__global__ void sum_final_kernel(const T* __restrict__ partials, int np, T* __restrict__ out) {
  T acc = T(0);
  for (int i = threadIdx.x; i < np; i += blockDim.x) acc += partials[i];
  acc = block_sum(acc);
  if (threadIdx.x == 0) *out = acc;
}

template <typename T>
mfs_status vec_sum(const T* x, int64_t n, T* d_partials, T* d_out, cudaStream_t s) {
  const int threads = 256;
  int blocks = (int)std::min<int64_t>((n + threads - 1) / threads, kRedBlocks);
  if (blocks < 1) blocks = 1;
  sum_partials_kernel<T><<<blocks, threads, 0, s>>>(x, n, d_partials);
  sum_final_kernel<T><<<1, 512, 0, s>>>(d_partials, blocks, d_out);
  MFS_CUDA(cudaGetLastError());
  return MFS_OK;
}

template <typename T>
__global__ void sub_mean_kernel(T* __restrict__ x, int64_t n, const T* __restrict__ sum) {
  const T mean = *sum / T(n);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x[i] -= mean;
}

template <typename T>
mfs_status vec_sub_mean(T* x, int64_t n, const T* d_sum, cudaStream_t s) {
  const int threads = 256;
  int blocks = (int)std::min<int64_t>((n + threads - 1) / threads, 4096);
  if (blocks < 1) blocks = 1;
  sub_mean_kernel<T><<<blocks, threads, 0, s>>>(x, n, d_sum);
  MFS_CUDA(cudaGetLastError());
  return MFS_OK;
}

template mfs_status vec_sum<double>(const double*, int64_t, double*, double*, cudaStream_t);
template mfs_status vec_sum<float>(const float*, int64_t, float*, float*, cudaStream_t);
template mfs_status vec_sub_mean<double>(double*, int64_t, const double*, cudaStream_t);
template mfs_status vec_sub_mean<float>(float*, int64_t, const float*, cudaStream_t);

// Injection of a P1 field from level l_from (fine) to l_to (coarse): the coarse vertex
// with barycentrics i (sum N_to) is the fine vertex i * 2^(l_from - l_to).
__global__ void inject_kernel(const MacroTopo* __restrict__ topo, Numbering nf, Numbering nc, int shift,
                              const double* __restrict__ src, double* __restrict__ dst) {
  const int m = blockIdx.y;
  const MacroTopo t = topo[m];
  const int N = nc.N;
  const int span = N + 1;
  const int64_t total = (int64_t)span * span * span;
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < total; s += (int64_t)gridDim.x * blockDim.x) {
    const int i1 = (int)(s % span), i2 = (int)((s / span) % span), i3 = (int)(s / ((int64_t)span * span));
    if (i1 + i2 + i3 > N) continue;
    const int i0 = N - i1 - i2 - i3;
    const int idc = lattice_id(t, nc, m, i0, i1, i2, i3);
    const int idf = lattice_id(t, nf, m, i0 << shift, i1 << shift, i2 << shift, i3 << shift);
    dst[idc] = src[idf];
  }
}

mfs_status inject_p1(const mfs_mesh* M, int l_from, int l_to, const double* src, double* dst) {
  const LevelData& Lf = M->levels[l_from];
  const LevelData& Lc = M->levels[l_to];
  const int N = Lc.nb1.N;
  const int64_t total = (int64_t)(N + 1) * (N + 1) * (N + 1);
  int bx = (int)std::min<int64_t>((total + 255) / 256, 1024);
  dim3 grid(bx, kMacroCells);
  inject_kernel<<<grid, 256, 0, M->ctx->stream>>>(M->d_topo, Lf.nb1, Lc.nb1, l_from - l_to, src, dst);
  MFS_CUDA(cudaGetLastError());
  return MFS_OK;
}

__global__ void f64_to_f32_kernel(const double* __restrict__ a, float* __restrict__ b, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = (float)a[i];
}

mfs_status convert_f64_f32(const double* src, float* dst, int64_t n, cudaStream_t s) {
  int blocks = (int)std::min<int64_t>((n + 255) / 256, 4096);
  if (blocks < 1) blocks = 1;
  f64_to_f32_kernel<<<blocks, 256, 0, s>>>(src, dst, n);
  MFS_CUDA(cudaGetLastError());
  return MFS_OK;
}

__global__ void exp_kernel(double* __restrict__ x, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x[i] = exp(x[i]);
}

mfs_status exp_inplace(double* x, int64_t n, cudaStream_t s) {
  int blocks = (int)std::min<int64_t>((n + 255) / 256, 4096);
  if (blocks < 1) blocks = 1;
  exp_kernel<<<blocks, 256, 0, s>>>(x, n);
  MFS_CUDA(cudaGetLastError());
  return MFS_OK;
}

}  // namespace mfs
