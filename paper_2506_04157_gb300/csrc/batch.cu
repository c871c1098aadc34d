// Ensembles of problems (possibly of different refinement levels): the constrained fused
// saddle-point apply of every instance in one sweep launch, with batched zeroing and
// pressure mean removal; a batch solve over the instances; and a concurrent solve of
// problems on several contexts (streams), one host thread per context.
#include <atomic>
#include <cstring>
#include <exception>
#include <new>
#include <string>
#include <system_error>
#include <thread>
#include <vector>

#include "apply.cuh"
#include "library.h"

struct mfs_batch {
  mfs_ctx* ctx = nullptr;
  std::vector<mfs_problem*> probs;
  int blending = 1;
  int nblocks = 0;
  int2* d_map = nullptr;        // block -> (problem, macro << 16 | tile)
  int* d_ntiles = nullptr;      // tiles per macro of each problem's finest level
  void* d_params = nullptr;     // ApplyParams<T>[n] (sized for double)
  void* h_params = nullptr;     // pinned staging
  void** d_ptrs = nullptr;      // [4][n] device pointers u, p, yu, yp
  void** h_ptrs = nullptr;      // pinned staging
  // recorded after the copies out of h_params / h_ptrs: the host waits on it before it
  // rewrites them (a pinned-memory copy reads its source only when the stream reaches it)
  cudaEvent_t staged = nullptr;
  bool staged_pending = false;
  int64_t* d_np2 = nullptr;
  int64_t* d_np1 = nullptr;
  double* d_part = nullptr;     // [n][kBatchRed] partial sums
  double* d_sums = nullptr;     // [2][n] sums (as T)
  // The device work of the last argument set (operator, precision, 4n vector pointers, the
  // members' coefficient versions) is
  // replayed from a captured CUDA graph from its second consecutive use on; the device
  // pointer and parameter arrays always hold that argument set's values.
  std::vector<const void*> key;
  cudaGraphExec_t graph = nullptr;
  cudaStream_t cap = nullptr;
};

namespace mfs {

constexpr int kBatchRed = 64;

template <typename T>
__global__ void k_batch_zero(T* const* __restrict__ ptrs, const int64_t* __restrict__ n, int mult) {
  const int b = blockIdx.y;
  T* x = ptrs[b];
  const int64_t m = n[b] * mult;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
    x[i] = T(0);
}

__device__ __forceinline__ double bwarp(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// partial sums: grid (kBatchRed, n), block b sums a slice of vector ptrs[b]
template <typename T>
__global__ void k_batch_sum_part(T* const* __restrict__ ptrs, const int64_t* __restrict__ n, double* __restrict__ part) {
  __shared__ double red[32];
  const int b = blockIdx.y;
  const T* x = ptrs[b];
  T acc = T(0);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n[b]; i += (int64_t)gridDim.x * blockDim.x)
    acc += x[i];
  double v = bwarp((double)acc);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    v = bwarp(v);
    if (threadIdx.x == 0) part[b * kBatchRed + blockIdx.x] = v;
  }
}
template <typename T>
__global__ void k_batch_sum_final(const double* __restrict__ part, T* __restrict__ sums) {
  const int b = blockIdx.x;
  if (threadIdx.x < 32) {
    double v = part[b * kBatchRed + threadIdx.x] + part[b * kBatchRed + 32 + threadIdx.x];
    v = bwarp(v);
    if (threadIdx.x == 0) sums[b] = (T)v;
  }
}
template <typename T>
__global__ void k_batch_sub_mean(T* const* __restrict__ ptrs, const int64_t* __restrict__ n, const T* __restrict__ sums) {
  const int b = blockIdx.y;
  T* x = ptrs[b];
  const T mean = sums[b] / T(n[b]);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n[b]; i += (int64_t)gridDim.x * blockDim.x)
    x[i] -= mean;
}

// pressure sums, zeroing, the one-launch sweep, output mean removal (device arrays set)
template <typename T>
static mfs_status batch_device_work(mfs_batch* B, int op, cudaStream_t s) {
  const int n = (int)B->probs.size();
  T* const* dp_p = (T* const*)(B->d_ptrs + n);
  T* const* dp_yu = (T* const*)(B->d_ptrs + 2 * n);
  T* const* dp_yp = (T* const*)(B->d_ptrs + 3 * n);
  T* sums = (T*)B->d_sums;               // [0, n): input pressure sums, [n, 2n): output sums
  // P_p on the pressure inputs: per-instance sums, subtracted inside the sweep
  k_batch_sum_part<T><<<dim3(kBatchRed, n), 256, 0, s>>>(dp_p, B->d_np1, B->d_part);
  k_batch_sum_final<T><<<n, 32, 0, s>>>(B->d_part, sums);
  // zero the accumulated outputs
  k_batch_zero<T><<<dim3(512, n), 256, 0, s>>>(dp_yu, B->d_np2, 3);
  k_batch_zero<T><<<dim3(64, n), 256, 0, s>>>(dp_yp, B->d_np1, 1);
  auto ev = timing_events(B->ctx);
  if (ev.first) cudaEventRecord(ev.first, s);
  MFS_TRY(launch_batch<T>((const ApplyParams<T>*)B->d_params, B->d_map, B->d_ntiles, B->nblocks, op, B->blending, s));
  if (ev.second) cudaEventRecord(ev.second, s);
  // P_p on the pressure outputs
  k_batch_sum_part<T><<<dim3(kBatchRed, n), 256, 0, s>>>(dp_yp, B->d_np1, B->d_part);
  k_batch_sum_final<T><<<n, 32, 0, s>>>(B->d_part, sums + n);
  k_batch_sub_mean<T><<<dim3(64, n), 256, 0, s>>>(dp_yp, B->d_np1, sums + n);
  MFS_CUDA(cudaGetLastError());
  return MFS_OK;
}

template <typename T>
static mfs_status batch_apply_typed(mfs_batch* B, int transpose, int with_C, const void* const* u, const void* const* p,
                                    void* const* yu, void* const* yp) {
  const int n = (int)B->probs.size();
  cudaStream_t s = B->ctx->stream;
  const int op = transpose ? (with_C ? OP_A | OP_BT | OP_CT | OP_B : OP_A | OP_BT | OP_B)
                           : (with_C ? OP_A | OP_BT | OP_B | OP_BC : OP_A | OP_BT | OP_B);
  std::vector<const void*> key(5 * n + 1);
  key[0] = reinterpret_cast<const void*>((uintptr_t)(op * 2 + (sizeof(T) == 8 ? 1 : 0)));
  for (int b = 0; b < n; ++b) {
    key[1 + b] = u[b];
    key[1 + n + b] = p[b];
    key[1 + 2 * n + b] = yu[b];
    key[1 + 3 * n + b] = yp[b];
    key[1 + 4 * n + b] = reinterpret_cast<const void*>((uintptr_t)B->probs[b]->version);   // coefficients
  }
  if (key == B->key && !B->ctx->timing) {
    if (!B->graph) {   // second consecutive use of this argument set: capture
      cudaError_t e = cudaStreamBeginCapture(B->cap, cudaStreamCaptureModeThreadLocal);
      mfs_status st = MFS_OK;
      if (e == cudaSuccess) st = batch_device_work<T>(B, op, B->cap);
      cudaGraph_t g = nullptr;
      cudaError_t e2 = cudaStreamEndCapture(B->cap, &g);
      if (e != cudaSuccess) return cuda_fail(e, "cudaStreamBeginCapture");
      if (st != MFS_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
      }
      if (e2 != cudaSuccess) return cuda_fail(e2, "cudaStreamEndCapture");
      e = cudaGraphInstantiate(&B->graph, g, 0);
      cudaGraphDestroy(g);
      if (e != cudaSuccess) {
        B->graph = nullptr;
        return cuda_fail(e, "cudaGraphInstantiate");
      }
    }
    MFS_CUDA(cudaGraphLaunch(B->graph, s));
    return MFS_OK;
  }
  if (B->graph) {
    cudaGraphExecDestroy(B->graph);
    B->graph = nullptr;
  }
  B->key.swap(key);
  // new argument set: device pointer and parameter arrays, then the work eagerly; the
  // staging buffers are reused only after the previous set's copies have read them
  if (B->staged_pending) {
    MFS_CUDA(cudaEventSynchronize(B->staged));
    B->staged_pending = false;
  }
  void** hp = B->h_ptrs;
  for (int b = 0; b < n; ++b) {
    hp[b] = const_cast<void*>(u[b]);
    hp[n + b] = const_cast<void*>(p[b]);
    hp[2 * n + b] = yu[b];
    hp[3 * n + b] = yp[b];
  }
  MFS_CUDA(cudaMemcpyAsync(B->d_ptrs, hp, sizeof(void*) * 4 * n, cudaMemcpyHostToDevice, s));
  T* sums = (T*)B->d_sums;
  ApplyParams<T>* hpar = (ApplyParams<T>*)B->h_params;
  for (int b = 0; b < n; ++b) {
    mfs_problem* P = B->probs[b];
    hpar[b] = fill_params<T>(P, P->mesh->l_max, 1, (const T*)u[b], (const T*)p[b], (T*)yu[b], (T*)yp[b], sums + b);
  }
  MFS_CUDA(cudaMemcpyAsync(B->d_params, hpar, sizeof(ApplyParams<T>) * n, cudaMemcpyHostToDevice, s));
  MFS_CUDA(cudaEventRecord(B->staged, s));
  B->staged_pending = true;
  return batch_device_work<T>(B, op, s);
}

}  // namespace mfs

using namespace mfs;

mfs_status mfs_batch_destroy(mfs_batch* B) {
  if (!B) return MFS_OK;
  if (B->graph) cudaGraphExecDestroy(B->graph);
  if (B->cap) cudaStreamDestroy(B->cap);
  if (B->staged) {
    if (B->staged_pending) cudaEventSynchronize(B->staged);
    cudaEventDestroy(B->staged);
  }
  cudaFree(B->d_map);
  cudaFree(B->d_ntiles);
  cudaFree(B->d_params);
  cudaFree(B->d_ptrs);
  cudaFree(B->d_np2);
  cudaFree(B->d_np1);
  cudaFree(B->d_part);
  cudaFree(B->d_sums);
  if (B->h_params) cudaFreeHost(B->h_params);
  if (B->h_ptrs) cudaFreeHost(B->h_ptrs);
  delete B;
  return MFS_OK;
}

mfs_status mfs_batch_create(mfs_ctx* ctx, int n, mfs_problem* const* probs, mfs_batch** out) {
  if (!ctx || !probs || !out || n < 1 || n > 4096) {
    set_error("invalid batch arguments");
    return MFS_EINVAL;
  }
  for (int b = 0; b < n; ++b) {
    if (!probs[b] || probs[b]->mesh->ctx != ctx || !probs[b]->has_eta) {
      set_error("batch member %d: null, on another context, or without viscosity", b);
      return MFS_EINVAL;
    }
    if (probs[b]->rho_weighted) {
      set_error("batch member %d uses the density-weighted constraint, which the batched sweep does not have", b);
      return MFS_EINVAL;
    }
    if (probs[b]->mesh->host.blending != probs[0]->mesh->host.blending) {
      set_error("batch members must all be blended or all polyhedral");
      return MFS_EINVAL;
    }
  }
  mfs_batch* B = new (std::nothrow) mfs_batch;
  if (!B) {
    set_error("host allocation failed");
    return MFS_ENOMEM;
  }
  B->ctx = ctx;
  B->probs.assign(probs, probs + n);
  B->blending = probs[0]->mesh->host.blending;
  std::vector<int2> map;
  std::vector<int> nt(n);
  std::vector<int64_t> np2(n), np1(n);
  for (int b = 0; b < n; ++b) {
    const LevelData& L = probs[b]->mesh->levels[probs[b]->mesh->l_max];
    nt[b] = L.n_tiles;
    np2[b] = L.nb2.total;
    np1[b] = L.nb1.total;
    for (int m = 0; m < kMacroCells; ++m)
      for (int t = 0; t < L.n_tiles; ++t) map.push_back(make_int2(b, (m << 16) | t));
  }
  B->nblocks = (int)map.size();
  cudaStream_t s = ctx->stream;
  cudaError_t e = cudaSuccess;
  auto chk = [&](cudaError_t x) {
    if (e == cudaSuccess) e = x;
  };
  chk(cudaMalloc((void**)&B->d_map, sizeof(int2) * map.size()));
  chk(cudaMalloc((void**)&B->d_ntiles, sizeof(int) * n));
  chk(cudaMalloc(&B->d_params, sizeof(ApplyParams<double>) * n));
  chk(cudaMalloc((void**)&B->d_ptrs, sizeof(void*) * 4 * n));
  chk(cudaMalloc((void**)&B->d_np2, sizeof(int64_t) * n));
  chk(cudaMalloc((void**)&B->d_np1, sizeof(int64_t) * n));
  chk(cudaMalloc((void**)&B->d_part, sizeof(double) * kBatchRed * n));
  chk(cudaMalloc((void**)&B->d_sums, sizeof(double) * 2 * n));
  chk(cudaMallocHost(&B->h_params, sizeof(ApplyParams<double>) * n));
  chk(cudaMallocHost((void**)&B->h_ptrs, sizeof(void*) * 4 * n));
  chk(cudaStreamCreateWithFlags(&B->cap, cudaStreamNonBlocking));
  chk(cudaEventCreateWithFlags(&B->staged, cudaEventDisableTiming));
  if (e == cudaSuccess) {
    chk(cudaMemcpyAsync(B->d_map, map.data(), sizeof(int2) * map.size(), cudaMemcpyHostToDevice, s));
    chk(cudaMemcpyAsync(B->d_ntiles, nt.data(), sizeof(int) * n, cudaMemcpyHostToDevice, s));
    chk(cudaMemcpyAsync(B->d_np2, np2.data(), sizeof(int64_t) * n, cudaMemcpyHostToDevice, s));
    chk(cudaMemcpyAsync(B->d_np1, np1.data(), sizeof(int64_t) * n, cudaMemcpyHostToDevice, s));
    chk(cudaStreamSynchronize(s));
  }
  if (e != cudaSuccess) {
    mfs_batch_destroy(B);
    return cuda_fail(e, "mfs_batch_create");
  }
  *out = B;
  return MFS_OK;
}

mfs_status mfs_batch_apply_stokes(mfs_batch* B, mfs_prec prec, int transpose, const void* const* u,
                                  const void* const* p, void* const* yu, void* const* yp) {
  if (!B || !u || !p || !yu || !yp) {
    set_error("null argument");
    return MFS_EINVAL;
  }
  for (size_t b = 0; b < B->probs.size(); ++b) {
    if (!u[b] || !p[b] || !yu[b] || !yp[b]) {
      set_error("null vector for batch member %d", (int)b);
      return MFS_EINVAL;
    }
    if (B->probs[b]->rho_weighted) {
      set_error("batch member %d uses the density-weighted constraint, which the batched sweep does not have",
                (int)b);
      return MFS_EINVAL;
    }
  }
  if (prec == MFS_F64) return batch_apply_typed<double>(B, transpose, 1, u, p, yu, yp);
  if (prec == MFS_F32) return batch_apply_typed<float>(B, transpose, 1, u, p, yu, yp);
  set_error("invalid precision");
  return MFS_EINVAL;
}

mfs_status mfs_batch_solve(mfs_batch* B, const mfs_solve_opts* opts, const double* const* f, const double* const* g,
                           double* const* u, double* const* p, mfs_solve_stats* stats) {
  if (!B || !f || !g || !u || !p) {
    set_error("null argument");
    return MFS_EINVAL;
  }
  mfs_status worst = MFS_OK;
  for (size_t b = 0; b < B->probs.size(); ++b) {
    mfs_solve_stats st;
    std::memset(&st, 0, sizeof(st));
    const mfs_status rc = mfs_stokes_solve(B->probs[b], opts, f[b], g[b], u[b], p[b], &st);
    if (stats) stats[b] = st;
    if (rc != MFS_OK && worst == MFS_OK) worst = rc;
    if (rc != MFS_OK && rc != MFS_ENOTCONV) return rc;
  }
  return worst;
}

// Concurrent solve: the problems are grouped by context; one host thread works through a
// group, member after member, on that context's stream, and up to n_threads groups run at the
// same time, so that the many small kernels and host round trips of low-level members of
// different groups overlap on the device.  A worker's errors are recorded per member and the
// first one is reported on the calling thread (the error text is per thread).
mfs_status mfs_solve_concurrent(int n, mfs_problem* const* probs, const mfs_solve_opts* opts, const double* const* f,
                                const double* const* g, double* const* u, double* const* p, mfs_solve_stats* stats,
                                int n_threads) {
  if (n < 0 || (n > 0 && (!probs || !opts || !f || !g || !u || !p)) || n_threads < 0) {
    set_error("invalid arguments: n >= 0, n_threads >= 0 and non-null arrays");
    return MFS_EINVAL;
  }
  std::vector<mfs_ctx*> ctxs;
  std::vector<std::vector<int>> groups;
  for (int b = 0; b < n; ++b) {
    if (!probs[b] || !probs[b]->mesh || !probs[b]->mesh->ctx || !f[b] || !g[b] || !u[b] || !p[b]) {
      set_error("null problem or vector for member %d", b);
      return MFS_EINVAL;
    }
    mfs_ctx* c = probs[b]->mesh->ctx;
    size_t k = 0;
    while (k < ctxs.size() && ctxs[k] != c) ++k;
    if (k == ctxs.size()) {
      for (mfs_ctx* o : ctxs)
        if (o->stream == c->stream && o->device == c->device) {
          set_error("two contexts of the members share one stream: the members would not run concurrently");
          return MFS_EINVAL;
        }
      ctxs.push_back(c);
      groups.emplace_back();
    }
    groups[k].push_back(b);
  }
  if (n == 0) return MFS_OK;
  // inputs written on other streams are complete before any member starts
  {
    int cur = 0;
    MFS_CUDA(cudaGetDevice(&cur));
    std::vector<int> devs;
    for (mfs_ctx* c : ctxs) {
      bool seen = false;
      for (int d : devs) seen = seen || d == c->device;
      if (seen) continue;
      devs.push_back(c->device);
      MFS_CUDA(cudaSetDevice(c->device));
      MFS_CUDA(cudaDeviceSynchronize());
    }
    MFS_CUDA(cudaSetDevice(cur));
  }
  std::vector<mfs_status> rc(n, MFS_OK);
  std::vector<std::string> msg(n);
  std::vector<mfs_solve_stats> st(n);
  std::atomic<int> next{0};
  const int ngroups = (int)groups.size();
  auto worker = [&]() {
    for (int k = next++; k < ngroups; k = next++) {
      const cudaError_t e = cudaSetDevice(ctxs[k]->device);
      for (int b : groups[k]) {
        std::memset(&st[b], 0, sizeof(mfs_solve_stats));
        if (e != cudaSuccess) {
          rc[b] = MFS_ECUDA;
          msg[b] = cudaGetErrorString(e);
          continue;
        }
        try {   // nothing may escape a worker thread (it would end the process)
          rc[b] = mfs_stokes_solve(probs[b], opts, f[b], g[b], u[b], p[b], &st[b]);
          if (rc[b] != MFS_OK) msg[b] = mfs_last_error();
        } catch (const std::exception& x) {
          rc[b] = MFS_ENOMEM;
          msg[b] = std::string("host exception: ") + x.what();
        } catch (...) {
          rc[b] = MFS_ENOMEM;
          msg[b] = "host exception";
        }
      }
    }
  };
  const int nt = n_threads > 0 && n_threads < ngroups ? n_threads : ngroups;
  std::vector<std::thread> pool;
  try {
    for (int t = 1; t < nt; ++t) pool.emplace_back(worker);
  } catch (const std::system_error&) {
    // fewer threads than asked: the ones running (and this one) take the remaining groups
  }
  worker();
  for (auto& t : pool) t.join();
  if (stats)
    for (int b = 0; b < n; ++b) stats[b] = st[b];
  mfs_status worst = MFS_OK;
  for (int b = 0; b < n; ++b) {
    if (rc[b] == MFS_OK) continue;
    if (rc[b] != MFS_ENOTCONV) {
      set_error("member %d: %s", b, msg[b].c_str());
      return rc[b];
    }
    if (worst == MFS_OK) {
      worst = MFS_ENOTCONV;
      set_error("member %d: %s", b, msg[b].c_str());
    }
  }
  return worst;
}
