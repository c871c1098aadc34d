// Allocation-free variant of the constrained B apply (mfs_apply_B_noalloc).
//
// Why it exists: some callers cannot call cudaMalloc when they apply the operator — for
// example code that runs under an external memory manager that owns all device
// allocations (a framework's caching allocator, an embedded solver inside another
// application's memory budget), or a real-time loop in which a device allocation would
// synchronise the device.  mfs_apply_B keeps its reduction partials in the problem's
// workspace; this variant keeps them in a fixed file-scope device array instead, so the
// call itself touches no allocator.
//
// The scratch array is a static __device__ symbol: every GPU that loads the library holds
// it until the process exits.  In host code the symbol name is only a host-side stand-in,
// so the host looks up its device address once per device with cudaGetSymbolAddress (on
// the first call made on that device, with that device current) and passes the pointer to
// the kernels.  All calls share the array, and it keeps the last call's contents: calls
// that overlap on the GPU (e.g. on two streams) race on it.
#include <mutex>

#include "library.h"

namespace mfs {

// One partial sum per chunk of kChunk pressure entries, at most kMaxPartials chunks.
constexpr int kChunk = 4096;
constexpr int kMaxPartials = 1024;
constexpr int64_t kNoallocMaxP1 = (int64_t)kChunk * kMaxPartials;   // 4,194,304 entries
// partials + one total, for the widest type (double); 8,200 bytes rounded up to 8 KiB + 256
constexpr int kScratchBytes = (kMaxPartials + 32) * 8;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

static std::mutex g_noalloc_mu;
static void* g_noalloc_ptr[256] = {nullptr};

static mfs_status noalloc_scratch(int device, void** out) {
  if (device < 0 || device >= 256) {
    set_error("device ordinal %d outside the no-alloc table", device);
    return MFS_EINVAL;
  }
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_ptr[device]) {
    int cur = -1;
    MFS_CUDA(cudaGetDevice(&cur));
    if (cur != device) MFS_CUDA(cudaSetDevice(device));
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (cur != device) cudaSetDevice(cur);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(no-alloc scratch)");
    g_noalloc_ptr[device] = p;
  }
  *out = g_noalloc_ptr[device];
  return MFS_OK;
}

template <typename T>
__device__ __forceinline__ T na_warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <typename T>
__device__ __forceinline__ T na_block_sum(T v) {
  __shared__ T red[32];
  v = na_warp_sum(v);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  const int nw = (blockDim.x + 31) >> 5;
  v = threadIdx.x < nw ? red[threadIdx.x] : T(0);
  if (w == 0) v = na_warp_sum(v);
  return v;
}

// block b sums entries [b*kChunk, (b+1)*kChunk) into partials[b]
template <typename T>
__global__ void na_chunk_sums(const T* __restrict__ x, int64_t n, T* __restrict__ partials) {
  const int64_t lo = (int64_t)blockIdx.x * kChunk;
  const int64_t hi = lo + kChunk < n ? lo + kChunk : n;
  T acc = T(0);
  for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) acc += x[i];
  acc = na_block_sum(acc);
  if (threadIdx.x == 0) partials[blockIdx.x] = acc;
}

// one block: total of the np partials written by this call, then x -= total / n
template <typename T>
__global__ void na_total(const T* __restrict__ partials, int np, T* __restrict__ total) {
  T acc = T(0);
  for (int i = threadIdx.x; i < np; i += blockDim.x) acc += partials[i];
  acc = na_block_sum(acc);
  if (threadIdx.x == 0) *total = acc;
}

template <typename T>
__global__ void na_sub_mean(T* __restrict__ x, int64_t n, const T* __restrict__ total) {
  const T mean = *total / T(n);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x[i] -= mean;
}

template <typename T>
static mfs_status noalloc_B(mfs_problem* P, int lvl, int constrained, int with_C, const void* u, void* q) {
  mfs_mesh* M = P->mesh;
  cudaStream_t s = M->ctx->stream;
  const int64_t n = M->levels[lvl].nb1.total;
  void* base = nullptr;
  if (constrained) MFS_TRY(noalloc_scratch(M->ctx->device, &base));   // set-up before any launch
  MFS_TRY(launch_apply<T>(P, lvl, OP_B, constrained, with_C, (const T*)u, nullptr, nullptr, (T*)q, nullptr));
  if (!constrained) return MFS_OK;
  T* partials = (T*)base;
  T* total = partials + kMaxPartials;
  const int np = (int)((n + kChunk - 1) / kChunk);
  na_chunk_sums<T><<<np, 256, 0, s>>>((const T*)q, n, partials);
  na_total<T><<<1, 256, 0, s>>>(partials, np, total);
  int blocks = (int)std::min<int64_t>((n + 255) / 256, 4096);
  na_sub_mean<T><<<blocks, 256, 0, s>>>((T*)q, n, total);
  MFS_CUDA(cudaGetLastError());
  return MFS_OK;
}

}  // namespace mfs

using namespace mfs;

mfs_status mfs_apply_B_noalloc(mfs_problem* P, int lvl, mfs_prec prec, mfs_bcmode mode, int with_C, const void* u,
                               void* q) {
  if (!u || !q) {   // the same order of checks as mfs_apply_B: vectors first
    set_error("null vector pointer");
    return MFS_EINVAL;
  }
  if (!P) {
    set_error("null problem");
    return MFS_EINVAL;
  }
  if (lvl < 0 || lvl > P->mesh->l_max) {
    set_error("level %d outside [0, %d]", lvl, P->mesh->l_max);
    return MFS_EINVAL;
  }
  if (!P->has_eta) {
    set_error("viscosity not set (call mfs_set_viscosity first)");
    return MFS_EINVAL;
  }
  const int64_t n = P->mesh->levels[lvl].nb1.total;
  if (n > kNoallocMaxP1) {
    set_error("level %d has %lld pressure entries; mfs_apply_B_noalloc handles at most %lld "
              "(fixed scratch of %d partial sums)", lvl, (long long)n, (long long)kNoallocMaxP1, kMaxPartials);
    return MFS_EINVAL;
  }
  if (prec != MFS_F64 && prec != MFS_F32) {
    set_error("invalid precision %d", (int)prec);
    return MFS_EINVAL;
  }
  const int constrained = mode == MFS_CONSTRAINED;
  if (prec == MFS_F64) return noalloc_B<double>(P, lvl, constrained, with_C ? 1 : 0, u, q);
  return noalloc_B<float>(P, lvl, constrained, with_C ? 1 : 0, u, q);
}
