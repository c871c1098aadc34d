// Vector kernels: deterministic two-pass sums, mean removal (P_p of Sec. 5.1),
// viscosity injection to coarser levels (Sec. 5.2.2: eta as a P1 function on every
// level, coarse vertices are fine vertices), precision conversion.
#include <algorithm>
#include <vector>

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

__global__ void law_eta_kernel(int64_t n, const int* __restrict__ fine, const double* __restrict__ rad,
                               const double* __restrict__ T, const double* __restrict__ lbase, int nt, double E_A,
                               double V_A, double r0, double r1, double* __restrict__ eta) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double r = rad[i];
    double lb = lbase[0];
    if (nt > 1) {
      double t = (r - r0) / (r1 - r0) * (nt - 1);
      t = t < 0.0 ? 0.0 : (t > nt - 1 ? nt - 1 : t);
      int k = (int)t;
      k = k > nt - 2 ? nt - 2 : k;
      lb = (1.0 - (t - k)) * lbase[k] + (t - k) * lbase[k + 1];
    }
    eta[i] = exp(2.302585092994045684 * lb - E_A * T[fine[i]] + V_A * (r1 - r));
  }
}

mfs_status law_eta(int64_t n, const int* fine, const double* rad, const double* T, const double* lbase, int nt,
                   double E_A, double V_A, double r0, double r1, double* eta, cudaStream_t s) {
  int blocks = (int)std::min<int64_t>((n + 255) / 256, 4096);
  if (blocks < 1) blocks = 1;
  law_eta_kernel<<<blocks, 256, 0, s>>>(n, fine, rad, T, lbase, nt, E_A, V_A, r0, r1, eta);
  MFS_CUDA(cudaGetLastError());
  return MFS_OK;
}

__global__ void gather_f64_kernel(int64_t n, const int* __restrict__ idx, const double* __restrict__ src,
                                  double* __restrict__ dst) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = src[idx[i]];
}

mfs_status gather_f64(int64_t n, const int* idx, const double* src, double* dst, cudaStream_t s) {
  int blocks = (int)std::min<int64_t>((n + 255) / 256, 4096);
  if (blocks < 1) blocks = 1;
  gather_f64_kernel<<<blocks, 256, 0, s>>>(n, idx, src, dst);
  MFS_CUDA(cudaGetLastError());
  return MFS_OK;
}

}  // namespace mfs

namespace mfs {

// Entries (coarse vertex, fine vertex, weight) of the P1 interpolation from level l-1 to
// level l, built from the Freudenthal micro-tets of level l-1 (the P1 vertices of level l
// are the P2 nodes of level l-1, vertices and edge midpoints of its micro-tets): weight 1
// for the coincident vertex, 1/2 for each end of the coarse edge at a midpoint.  Each fine
// vertex appears once.
void p1_transfer_triplets(const mfs_mesh* M, int l, std::vector<int>& tv, std::vector<int>& tj,
                          std::vector<double>& tw) {
  static const int PERM[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
  static const int LE[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}};
  const int n = 1 << (l - 1);
  const Numbering nbf = make_numbering(2 * n);
  const Numbering nbc = make_numbering(n);
  std::vector<char> seen(nbf.total, 0);
  tv.clear();
  tj.clear();
  tw.clear();
  for (int m = 0; m < 60; ++m) {
    const MacroTopo& t = M->host.topo[m];
    for (int a = 0; a < n; ++a)
      for (int b = 0; b <= a; ++b)
        for (int c = 0; c <= b; ++c)
          for (int pm = 0; pm < 6; ++pm) {
            int K[4][3] = {{a, b, c}};
            bool ok = true;
            for (int k = 1; k < 4; ++k) {
              for (int d = 0; d < 3; ++d) K[k][d] = K[k - 1][d];
              K[k][PERM[pm][k - 1]] += 1;
              if (!(K[k][0] >= K[k][1] && K[k][1] >= K[k][2])) ok = false;
            }
            if (!ok) continue;
            int v[4];
            for (int q = 0; q < 4; ++q) {
              v[q] = lattice_id(t, nbc, m, n - K[q][0], K[q][0] - K[q][1], K[q][1] - K[q][2], K[q][2]);
              const int A = 2 * K[q][0], B = 2 * K[q][1], C = 2 * K[q][2];
              const int j = lattice_id(t, nbf, m, 2 * n - A, A - B, B - C, C);
              if (!seen[j]) {
                seen[j] = 1;
                tv.push_back(v[q]);
                tj.push_back(j);
                tw.push_back(1.0);
              }
            }
            for (int e = 0; e < 6; ++e) {
              const int p = LE[e][0], q = LE[e][1];
              const int A = K[p][0] + K[q][0], B = K[p][1] + K[q][1], C = K[p][2] + K[q][2];
              const int j = lattice_id(t, nbf, m, 2 * n - A, A - B, B - C, C);
              if (seen[j]) continue;
              seen[j] = 1;
              tv.push_back(v[p]);
              tj.push_back(j);
              tw.push_back(0.5);
              tv.push_back(v[q]);
              tj.push_back(j);
              tw.push_back(0.5);
            }
          }
  }
}

// P1 full weighting from level l to l-1: the rows of the transposed P1 interpolation,
// normalised to sum one.
mfs_status build_eta_restriction(mfs_mesh* M, int l) {
  LevelData& L = M->levels[l];
  const Numbering nbc = make_numbering(1 << (l - 1));
  std::vector<int> tv, tj;
  std::vector<double> tw;
  p1_transfer_triplets(M, l, tv, tj, tw);
  std::vector<int> rp(nbc.total + 1, 0);
  for (int v : tv) rp[v + 1]++;
  for (int i = 0; i < nbc.total; ++i) rp[i + 1] += rp[i];
  std::vector<int> pos(rp.begin(), rp.end() - 1), ci(tv.size());
  std::vector<double> w(tv.size()), rs(nbc.total, 0.0);
  for (size_t k = 0; k < tv.size(); ++k) rs[tv[k]] += tw[k];
  for (size_t k = 0; k < tv.size(); ++k) {
    const int r = tv[k];
    ci[pos[r]] = tj[k];
    w[pos[r]] = tw[k] / rs[r];
    pos[r]++;
  }
  cudaStream_t s = M->ctx->stream;
  L.er_rows = nbc.total;
  MFS_CUDA(cudaMalloc((void**)&L.d_er_rp, sizeof(int) * rp.size()));
  MFS_CUDA(cudaMalloc((void**)&L.d_er_ci, sizeof(int) * ci.size()));
  MFS_CUDA(cudaMalloc((void**)&L.d_er_w, sizeof(double) * w.size()));
  MFS_CUDA(cudaMemcpyAsync(L.d_er_rp, rp.data(), sizeof(int) * rp.size(), cudaMemcpyHostToDevice, s));
  MFS_CUDA(cudaMemcpyAsync(L.d_er_ci, ci.data(), sizeof(int) * ci.size(), cudaMemcpyHostToDevice, s));
  MFS_CUDA(cudaMemcpyAsync(L.d_er_w, w.data(), sizeof(double) * w.size(), cudaMemcpyHostToDevice, s));
  MFS_CUDA(cudaStreamSynchronize(s));
  return MFS_OK;
}

__global__ void restrict_eta_kernel(int rows, const int* __restrict__ rp, const int* __restrict__ ci,
                                    const double* __restrict__ w, const double* __restrict__ fine,
                                    double* __restrict__ coarse) {
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < rows; r += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int k = rp[r]; k < rp[r + 1]; ++k) s += w[k] * fine[ci[k]];
    coarse[r] = s;
  }
}

mfs_status restrict_eta(const mfs_mesh* M, int l, const double* fine, double* coarse) {
  const LevelData& L = M->levels[l];
  const int blocks = std::max(1, std::min((L.er_rows + 255) / 256, 4096));
  restrict_eta_kernel<<<blocks, 256, 0, M->ctx->stream>>>(L.er_rows, L.d_er_rp, L.d_er_ci, L.d_er_w, fine, coarse);
  MFS_CUDA(cudaGetLastError());
  return MFS_OK;
}

}  // namespace mfs
