// C ABI of libmfs (declared in include/mfs.h).
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>

#include "library.h"

namespace mfs {

static thread_local char g_err[512] = "";

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

mfs_status cuda_fail(cudaError_t e, const char* what) {
  set_error("CUDA error %s (%s) in %s", cudaGetErrorName(e), cudaGetErrorString(e), what);
  return e == cudaErrorMemoryAllocation ? MFS_ENOMEM : MFS_ECUDA;
}

template <typename T>
static mfs_status upload(T** dst, const T* src, size_t count, cudaStream_t s) {
  MFS_CUDA(cudaMalloc((void**)dst, sizeof(T) * (count ? count : 1)));
  if (count) MFS_CUDA(cudaMemcpyAsync(*dst, src, sizeof(T) * count, cudaMemcpyHostToDevice, s));
  return MFS_OK;
}

static mfs_status check_level(const mfs_mesh* M, int lvl) {
  if (!M) {
    set_error("null mesh");
    return MFS_EINVAL;
  }
  if (lvl < 0 || lvl > M->l_max) {
    set_error("level %d outside [0, %d]", lvl, M->l_max);
    return MFS_EINVAL;
  }
  return MFS_OK;
}

static mfs_status check_problem(const mfs_problem* P, int lvl, bool need_eta) {
  if (!P) {
    set_error("null problem");
    return MFS_EINVAL;
  }
  MFS_TRY(check_level(P->mesh, lvl));
  if (need_eta && !P->has_eta) {
    set_error("viscosity not set (call mfs_set_viscosity first)");
    return MFS_EINVAL;
  }
  return MFS_OK;
}

template <typename T>
static T* red_of(mfs_problem* P);
template <>
double* red_of<double>(mfs_problem* P) { return P->d_red64; }
template <>
float* red_of<float>(mfs_problem* P) { return P->d_red32; }

std::pair<cudaEvent_t, cudaEvent_t> timing_events(mfs_ctx* ctx) {
  if (!ctx || !ctx->timing) return {nullptr, nullptr};
  cudaEvent_t e[2];
  for (int k = 0; k < 2; ++k) {
    if (!ctx->ev_pool.empty()) {
      e[k] = ctx->ev_pool.back();
      ctx->ev_pool.pop_back();
    } else if (cudaEventCreate(&e[k]) != cudaSuccess) {
      return {nullptr, nullptr};
    }
  }
  ctx->ev_used.push_back({e[0], e[1]});
  return {e[0], e[1]};
}

template <typename T>
mfs_status apply_constrained(mfs_problem* P, int lvl, int op, int constrained, int withc_b, const T* u, const T* p,
                             T* yu, T* yp) {
  mfs_mesh* M = P->mesh;
  cudaStream_t s = M->ctx->stream;
  const LevelData& L = M->levels[lvl];
  T* red = red_of<T>(P);
  const T* psum = nullptr;
  if (constrained && (op & OP_BT)) {   // P_p on the pressure input: the kernel subtracts sum/n
    MFS_TRY(vec_sum<T>(p, L.nb1.total, red, red + kRedBlocks, s));
    psum = red + kRedBlocks;
  }
  MFS_TRY(launch_apply<T>(P, lvl, op, constrained, withc_b, u, p, yu, yp, psum));
  if (constrained && (op & OP_B)) {
    MFS_TRY(vec_sum<T>(yp, L.nb1.total, red, red + kRedBlocks + 2, s));
    MFS_TRY(vec_sub_mean<T>(yp, L.nb1.total, red + kRedBlocks + 2, s));
  }
  return MFS_OK;
}
template mfs_status apply_constrained<float>(mfs_problem*, int, int, int, int, const float*, const float*, float*,
                                             float*);
template mfs_status apply_constrained<double>(mfs_problem*, int, int, int, int, const double*, const double*,
                                              double*, double*);

}  // namespace mfs

using namespace mfs;

// Definitions below inherit C linkage from their declarations in mfs.h.

const char* mfs_last_error(void) { return g_err; }
const char* mfs_version(void) { return "mfs 0.1 (sm_103a)"; }

mfs_status mfs_ctx_create(int device, void* stream, mfs_ctx** out) {
  if (!out) {
    set_error("null output handle");
    return MFS_EINVAL;
  }
  int nd = 0;
  MFS_CUDA(cudaGetDeviceCount(&nd));
  if (device < 0 || device >= nd) {
    set_error("device %d not available (%d devices)", device, nd);
    return MFS_EINVAL;
  }
  MFS_CUDA(cudaSetDevice(device));
  mfs_ctx* c = new (std::nothrow) mfs_ctx;
  if (!c) {
    set_error("host allocation failed");
    return MFS_ENOMEM;
  }
  c->device = device;
  c->stream = (cudaStream_t)stream;
  *out = c;
  return MFS_OK;
}

mfs_status mfs_ctx_set_stream(mfs_ctx* ctx, void* stream) {
  if (!ctx) {
    set_error("null context");
    return MFS_EINVAL;
  }
  ctx->stream = (cudaStream_t)stream;
  return MFS_OK;
}

mfs_status mfs_ctx_destroy(mfs_ctx* ctx) {
  if (!ctx) return MFS_OK;
  for (auto e : ctx->ev_pool) cudaEventDestroy(e);
  for (auto& e : ctx->ev_used) {
    cudaEventDestroy(e.first);
    cudaEventDestroy(e.second);
  }
  delete ctx;
  return MFS_OK;
}

mfs_status mfs_ctx_timing(mfs_ctx* ctx, int enable) {
  if (!ctx) {
    set_error("null context");
    return MFS_EINVAL;
  }
  ctx->timing = enable ? 1 : 0;
  return MFS_OK;
}

mfs_status mfs_ctx_kernel_time(mfs_ctx* ctx, double* total_ms, int64_t* launches) {
  if (!ctx || !total_ms || !launches) {
    set_error("null argument");
    return MFS_EINVAL;
  }
  MFS_CUDA(cudaStreamSynchronize(ctx->stream));
  double tot = 0.0;
  for (auto& e : ctx->ev_used) {
    float ms = 0.f;
    MFS_CUDA(cudaEventElapsedTime(&ms, e.first, e.second));
    tot += ms;
    ctx->ev_pool.push_back(e.first);
    ctx->ev_pool.push_back(e.second);
  }
  *total_ms = tot;
  *launches = (int64_t)ctx->ev_used.size();
  ctx->ev_used.clear();
  return MFS_OK;
}

mfs_status mfs_mesh_shell(mfs_ctx* ctx, double r_cmb, double r_surf, int l_max, int blending, mfs_mesh** out) {
  if (!out) {
    set_error("null output handle");
    return MFS_EINVAL;
  }
  if (!(r_cmb > 0.0) || !(r_surf > r_cmb)) {
    set_error("need 0 < r_cmb < r_surf (got %g, %g)", r_cmb, r_surf);
    return MFS_EINVAL;
  }
  if (l_max < 0 || l_max > 7) {
    set_error("l_max %d outside [0, 7]", l_max);
    return MFS_EINVAL;
  }
  if (ctx) MFS_CUDA(cudaSetDevice(ctx->device));
  mfs_mesh* M = new (std::nothrow) mfs_mesh;
  if (!M) {
    set_error("host allocation failed");
    return MFS_ENOMEM;
  }
  M->ctx = ctx;
  M->l_max = l_max;
  M->host.build(r_cmb, r_surf, blending ? 1 : 0);
  if (!ctx) {  // host-only mesh: numbering, coordinates and classes, no device data
    *out = M;
    return MFS_OK;
  }
  cudaStream_t s = ctx->stream;
  mfs_status st = upload(&M->d_topo, M->host.topo, 60, s);
  MacroGeom<float> g32[60];
  for (int m = 0; m < 60 && st == MFS_OK; ++m) g32[m] = cast_geom<float>(M->host.geom[m]);
  if (st == MFS_OK) st = upload(&M->d_geom64, M->host.geom, 60, s);
  if (st == MFS_OK) st = upload(&M->d_geom32, g32, 60, s);
  for (int l = 0; l <= l_max && st == MFS_OK; ++l) {
    LevelData L;
    L.l = l;
    L.n = 1 << l;
    L.nb2 = make_numbering(2 * L.n);
    L.nb1 = make_numbering(L.n);
    L.n_tets = 60LL << (3 * l);
    L.n_surface = L.n_cmb = 10LL * (1LL << (2 * (l + 1))) + 2;
    HostTiles H = build_tiles(L.n);
    L.n_tiles = (int)H.tiles.size();
    st = upload(&L.d_tiles, H.tiles.data(), H.tiles.size(), s);
    if (st == MFS_OK) st = upload(&L.d_tets, H.tets.data(), H.tets.size(), s);
    if (st == MFS_OK) st = upload(&L.d_classes, H.classes.data(), H.classes.size(), s);
    if (st == MFS_OK) st = build_id_tables(M, L);
    if (st == MFS_OK) MFS_CUDA(cudaStreamSynchronize(s));   // host vectors die here
    M->levels.push_back(L);
    if (st == MFS_OK && l >= 1) st = build_eta_restriction(M, l);
  }
  if (st != MFS_OK) {
    mfs_mesh_destroy(M);
    return st;
  }
  *out = M;
  return MFS_OK;
}

mfs_status mfs_mesh_destroy(mfs_mesh* M) {
  if (!M) return MFS_OK;
  cudaFree(M->d_topo);
  cudaFree(M->d_geom64);
  cudaFree(M->d_geom32);
  for (auto& L : M->levels) {
    cudaFree(L.d_tiles);
    cudaFree(L.d_tets);
    cudaFree(L.d_classes);
    cudaFree(L.d_ids2);
    cudaFree(L.d_ids1);
    cudaFree(L.d_er_rp);
    cudaFree(L.d_er_ci);
    cudaFree(L.d_er_w);
    cudaFree(L.d_vfine);
    cudaFree(L.d_vrad);
    cudaFree(L.d_p2fine);
  }
  delete M;
  return MFS_OK;
}

mfs_status mfs_mesh_info(const mfs_mesh* M, int lvl, mfs_level_info* out) {
  MFS_TRY(check_level(M, lvl));
  if (!out) {
    set_error("null output");
    return MFS_EINVAL;
  }
  out->level = lvl;
  out->n_tets = 60LL << (3 * lvl);
  out->n_p2 = make_numbering(2 << lvl).total;
  out->n_p1 = make_numbering(1 << lvl).total;
  out->n_surface = out->n_cmb = 10LL * (1LL << (2 * (lvl + 1))) + 2;
  return MFS_OK;
}

mfs_status mfs_mesh_coords(const mfs_mesh* M, int lvl, int p2, int blended, double* xyz) {
  MFS_TRY(check_level(M, lvl));
  if (!xyz) {
    set_error("null output buffer");
    return MFS_EINVAL;
  }
  const int N = p2 ? (2 << lvl) : (1 << lvl);
  const int64_t n = make_numbering(N).total;
  for_each_point(M, N, [&](int m, const int* i, int id) {
    double xs[3], x[3];
    M->host.straight_point(m, i, N, xs);
    if (blended) M->host.blend_point(m, xs, x);
    else for (int r = 0; r < 3; ++r) x[r] = xs[r];
    for (int r = 0; r < 3; ++r) xyz[r * n + id] = x[r];
  });
  return MFS_OK;
}

mfs_status mfs_mesh_node_class(const mfs_mesh* M, int lvl, int p2, int8_t* cls) {
  MFS_TRY(check_level(M, lvl));
  if (!cls) {
    set_error("null output buffer");
    return MFS_EINVAL;
  }
  const int N = p2 ? (2 << lvl) : (1 << lvl);
  for_each_point(M, N, [&](int m, const int* i, int id) {
    const int mask = (i[0] > 0) | ((i[1] > 0) << 1) | ((i[2] > 0) << 2) | ((i[3] > 0) << 3);
    const MacroTopo& t = M->host.topo[m];
    int c = 0;
    if ((mask & ~t.topmask & 15) == 0) c = 1;
    else if ((mask & ~t.botmask & 15) == 0) c = 2;
    cls[id] = (int8_t)c;
  });
  return MFS_OK;
}

mfs_status mfs_problem_create(mfs_mesh* M, mfs_bc bc_surface, mfs_bc bc_cmb, mfs_problem** out) {
  if (!M || !out) {
    set_error("null mesh or output handle");
    return MFS_EINVAL;
  }
  if ((bc_surface != MFS_BC_DIRICHLET && bc_surface != MFS_BC_FREESLIP) ||
      (bc_cmb != MFS_BC_DIRICHLET && bc_cmb != MFS_BC_FREESLIP)) {
    set_error("invalid boundary condition type");
    return MFS_EINVAL;
  }
  if (!M->ctx) {
    set_error("mesh was created without a context (host-only)");
    return MFS_EINVAL;
  }
  MFS_CUDA(cudaSetDevice(M->ctx->device));
  mfs_problem* P = new (std::nothrow) mfs_problem;
  if (!P) {
    set_error("host allocation failed");
    return MFS_ENOMEM;
  }
  P->mesh = M;
  P->bc_surface = bc_surface;
  P->bc_cmb = bc_cmb;
  cudaStream_t s = M->ctx->stream;
  const double zero64 = 0.0;
  const float zero32 = 0.0f;
  mfs_status st = upload(&P->d_dlnrho64, &zero64, 1, s);
  if (st == MFS_OK) st = upload(&P->d_dlnrho32, &zero32, 1, s);
  if (st == MFS_OK) {
    cudaError_t e = cudaMalloc((void**)&P->d_red64, sizeof(double) * kRedSlots);
    if (e == cudaSuccess) e = cudaMalloc((void**)&P->d_red32, sizeof(float) * kRedSlots);
    if (e != cudaSuccess) st = cuda_fail(e, "cudaMalloc(reduction workspace)");
  }
  for (int l = 0; l <= M->l_max && st == MFS_OK; ++l) {
    double* e64 = nullptr;
    float* e32 = nullptr;
    const size_t np1 = M->levels[l].nb1.total;
    cudaError_t e = cudaMalloc((void**)&e64, sizeof(double) * np1);
    if (e == cudaSuccess) e = cudaMalloc((void**)&e32, sizeof(float) * np1);
    P->eta64.push_back(e64);
    P->eta32.push_back(e32);
    if (e != cudaSuccess) st = cuda_fail(e, "cudaMalloc(eta)");
  }
  if (st == MFS_OK) {
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) st = cuda_fail(e, "cudaStreamSynchronize");
  }
  if (st != MFS_OK) {
    mfs_problem_destroy(P);
    return st;
  }
  P->n_dlnrho = 1;
  *out = P;
  return MFS_OK;
}

mfs_status mfs_problem_destroy(mfs_problem* P) {
  if (!P) return MFS_OK;
  problem_release_solver(P);
  for (auto p : P->eta64) cudaFree(p);
  for (auto p : P->eta32) cudaFree(p);
  for (auto p : P->temp64) cudaFree(p);
  for (auto p : P->temp32) cudaFree(p);
  cudaFree(P->d_lbase64);
  cudaFree(P->d_lbase32);
  cudaFree(P->d_dlnrho64);
  cudaFree(P->d_dlnrho32);
  cudaFree(P->d_dlnrho_int64);
  cudaFree(P->d_dlnrho_int32);
  cudaFree(P->d_red64);
  cudaFree(P->d_red32);
  delete P;
  return MFS_OK;
}

mfs_status mfs_set_viscosity(mfs_problem* P, const double* eta, int is_log) {
  if (P) P->version++;
  MFS_TRY(check_problem(P, 0, false));
  if (!eta) {
    set_error("null viscosity pointer");
    return MFS_EINVAL;
  }
  mfs_mesh* M = P->mesh;
  cudaStream_t s = M->ctx->stream;
  const int L = M->l_max;
  const size_t np1 = M->levels[L].nb1.total;
  P->l_eta = -1;   // P1 viscosity on every level (a viscosity law set earlier no longer applies)
  MFS_CUDA(cudaMemcpyAsync(P->eta64[L], eta, sizeof(double) * np1, cudaMemcpyDeviceToDevice, s));
  if (is_log) MFS_TRY(exp_inplace(P->eta64[L], (int64_t)np1, s));
  // coarse levels: P1 full weighting of the next finer level (arithmetic average of the
  // coincident vertex and the midpoints of the incident coarse edges)
  for (int l = L; l >= 1; --l) MFS_TRY(restrict_eta(M, l, P->eta64[l], P->eta64[l - 1]));
  for (int l = 0; l <= L; ++l)
    MFS_TRY(convert_f64_f32(P->eta64[l], P->eta32[l], M->levels[l].nb1.total, s));
  P->has_eta = true;
  return MFS_OK;
}


mfs_status mfs_set_viscosity_law(mfs_problem* P, double E_A, double V_A, int n, const double* log10_base, int l_eta) {
  if (P) P->version++;
  MFS_TRY(check_problem(P, 0, false));
  const int L = P->mesh->l_max;
  if (n < 1 || n > 64 || !log10_base || l_eta < -1 || l_eta >= L) {
    set_error("viscosity law: 1 <= n <= 64 table entries and -1 <= l_eta < l_max = %d required", L);
    return MFS_EINVAL;
  }
  cudaStream_t s = P->mesh->ctx->stream;
  MFS_CUDA(cudaStreamSynchronize(s));
  cudaFree(P->d_lbase64);
  cudaFree(P->d_lbase32);
  P->d_lbase64 = nullptr;
  P->d_lbase32 = nullptr;
  P->lbase_host.assign(log10_base, log10_base + n);
  std::vector<float> t32(log10_base, log10_base + n);
  MFS_TRY(upload(&P->d_lbase64, log10_base, (size_t)n, s));
  MFS_TRY(upload(&P->d_lbase32, t32.data(), (size_t)n, s));
  P->E_A = E_A;
  P->V_A = V_A;
  P->l_eta = -1;   // takes effect with mfs_set_temperature
  P->law_l_eta = l_eta;
  MFS_CUDA(cudaStreamSynchronize(s));
  return MFS_OK;
}

// The viscosity law's lookup maps of level l, built on the host: the finest P2 node
// coinciding with each P1 vertex and the vertex's radius (|x| of the blended point), and
// (when p2fine is given) the finest P2 node coinciding with each P2 node of the level.
static mfs_status law_maps_host(const mfs_mesh* M, int l, std::vector<int>* vfine, std::vector<double>* vrad,
                                std::vector<int>* p2fine) {
  const int NF = 2 << M->l_max;   // finest P2 lattice
  const Numbering nbf = make_numbering(NF);
  if (vfine || vrad) {
    const int N1 = 1 << l, sc1 = NF / N1;
    std::vector<int> fine(make_numbering(N1).total, -1);
    std::vector<double> rad(fine.size(), 0.0);
    for_each_point(M, N1, [&](int m, const int* i, int id) {
      double xs[3], x[3];
      M->host.straight_point(m, i, N1, xs);
      if (M->host.blending) M->host.blend_point(m, xs, x);
      else for (int r = 0; r < 3; ++r) x[r] = xs[r];
      fine[id] = lattice_id(M->host.topo[m], nbf, m, i[0] * sc1, i[1] * sc1, i[2] * sc1, i[3] * sc1);
      rad[id] = std::sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
    });
    for (int f : fine)
      if (f < 0 || f >= nbf.total) {
        set_error("internal: vertex without a finest-level node on level %d", l);
        return MFS_EINVAL;
      }
    if (vfine) vfine->swap(fine);
    if (vrad) vrad->swap(rad);
  }
  if (p2fine) {
    const int N2 = 2 << l, sc2 = NF / N2;
    std::vector<int> fine(make_numbering(N2).total, -1);
    for_each_point(M, N2, [&](int m, const int* i, int id) {
      fine[id] = lattice_id(M->host.topo[m], nbf, m, i[0] * sc2, i[1] * sc2, i[2] * sc2, i[3] * sc2);
    });
    for (int f : fine)
      if (f < 0 || f >= nbf.total) {
        set_error("internal: P2 node without a finest-level node on level %d", l);
        return MFS_EINVAL;
      }
    p2fine->swap(fine);
  }
  return MFS_OK;
}

// The maps of law_maps_host on the device, built once per mesh (the P2 map only when p2).
static mfs_status law_maps(mfs_mesh* M, int l, bool p2) {
  LevelData& Lv = M->levels[l];
  cudaStream_t s = M->ctx->stream;
  if (!Lv.d_vfine || !Lv.d_vrad) {
    std::vector<int> fine;
    std::vector<double> rad;
    MFS_TRY(law_maps_host(M, l, &fine, &rad, nullptr));
    cudaFree(Lv.d_vfine);
    cudaFree(Lv.d_vrad);
    Lv.d_vfine = nullptr;
    Lv.d_vrad = nullptr;
    int* dfine = nullptr;
    double* drad = nullptr;
    mfs_status st = upload(&dfine, fine.data(), fine.size(), s);
    if (st == MFS_OK) st = upload(&drad, rad.data(), rad.size(), s);
    cudaError_t e = cudaStreamSynchronize(s);   // the host vectors go out of scope
    if (st == MFS_OK && e != cudaSuccess) st = cuda_fail(e, "law_maps");
    if (st != MFS_OK) {
      cudaFree(dfine);
      cudaFree(drad);
      return st;
    }
    Lv.d_vfine = dfine;
    Lv.d_vrad = drad;
  }
  if (p2 && !Lv.d_p2fine) {
    std::vector<int> fine;
    MFS_TRY(law_maps_host(M, l, nullptr, nullptr, &fine));
    int* dfine = nullptr;
    mfs_status st = upload(&dfine, fine.data(), fine.size(), s);
    cudaError_t e = cudaStreamSynchronize(s);
    if (st == MFS_OK && e != cudaSuccess) st = cuda_fail(e, "law_maps");
    if (st != MFS_OK) {
      cudaFree(dfine);
      return st;
    }
    Lv.d_p2fine = dfine;
  }
  return MFS_OK;
}

mfs_status mfs_mesh_law_maps(const mfs_mesh* M, int lvl, int* vfine, double* vrad, int* p2fine) {
  if (!M || lvl < 0 || lvl > M->l_max) {
    set_error("null mesh or level outside 0..l_max");
    return MFS_EINVAL;
  }
  std::vector<int> f1, f2;
  std::vector<double> rad;
  MFS_TRY(law_maps_host(M, lvl, vfine ? &f1 : nullptr, vrad ? &rad : nullptr, p2fine ? &f2 : nullptr));
  if (vfine) std::memcpy(vfine, f1.data(), sizeof(int) * f1.size());
  if (vrad) std::memcpy(vrad, rad.data(), sizeof(double) * rad.size());
  if (p2fine) std::memcpy(p2fine, f2.data(), sizeof(int) * f2.size());
  return MFS_OK;
}

mfs_status mfs_set_temperature(mfs_problem* P, const double* T_p2) {
  if (P) P->version++;
  MFS_TRY(check_problem(P, 0, false));
  if (!T_p2 || P->lbase_host.empty() || !P->d_lbase64) {
    set_error(T_p2 ? "no viscosity law (call mfs_set_viscosity_law first)" : "null temperature");
    return MFS_EINVAL;
  }
  mfs_mesh* M = P->mesh;
  cudaStream_t s = M->ctx->stream;
  const int L = M->l_max;
  const int l_eta = P->law_l_eta;
  if ((int)P->temp64.size() < L + 1) {
    P->temp64.resize(L + 1, nullptr);
    P->temp32.resize(L + 1, nullptr);
  }
  const int nt = (int)P->lbase_host.size();
  for (int l = 0; l <= L; ++l) {
    // Eq. (ViscosityDef) at every vertex of the level, with the temperature of the finest
    // P2 node at the same point
    MFS_TRY(law_maps(M, l, l <= l_eta));
    const LevelData& Lv = M->levels[l];
    MFS_TRY(law_eta(Lv.nb1.total, Lv.d_vfine, Lv.d_vrad, T_p2, P->d_lbase64, nt, P->E_A, P->V_A, M->host.r_cmb,
                    M->host.r_surf, P->eta64[l], s));
    MFS_TRY(convert_f64_f32(P->eta64[l], P->eta32[l], Lv.nb1.total, s));
    if (l <= l_eta) {   // P2 temperature of the level for the quadrature-point viscosity
      const int64_t n2 = Lv.nb2.total;
      if (!P->temp64[l]) {
        MFS_CUDA(cudaMalloc((void**)&P->temp64[l], sizeof(double) * n2));
        MFS_CUDA(cudaMalloc((void**)&P->temp32[l], sizeof(float) * n2));
      }
      MFS_TRY(gather_f64(n2, Lv.d_p2fine, T_p2, P->temp64[l], s));
      MFS_TRY(convert_f64_f32(P->temp64[l], P->temp32[l], n2, s));
    }
  }
  MFS_CUDA(cudaStreamSynchronize(s));
  P->l_eta = l_eta;
  P->has_eta = true;
  return MFS_OK;
}

mfs_status mfs_set_density(mfs_problem* P, int n, const double* tab) {
  if (P) P->version++;
  MFS_TRY(check_problem(P, 0, false));
  if (n < 1 || !tab) {
    set_error("density table needs n >= 1 entries");
    return MFS_EINVAL;
  }
  cudaStream_t s = P->mesh->ctx->stream;
  MFS_CUDA(cudaStreamSynchronize(s));
  cudaFree(P->d_dlnrho64);
  cudaFree(P->d_dlnrho32);
  P->d_dlnrho64 = nullptr;
  P->d_dlnrho32 = nullptr;
  // a table of equal entries is the constant d ln rho / dr: stored as one entry, so that the
  // sweeps take the constant directly instead of interpolating at every quadrature point
  bool constant = true;
  for (int k = 1; k < n; ++k) constant = constant && tab[k] == tab[0];
  if (constant) n = 1;
  std::vector<float> t32(tab, tab + n);
  // integral of the piecewise-linear table from r_cmb to each node (trapezoids are exact)
  std::vector<double> gi(n, 0.0);
  const double hcell = n > 1 ? (P->mesh->host.r_surf - P->mesh->host.r_cmb) / (n - 1) : 0.0;
  for (int k = 1; k < n; ++k) gi[k] = gi[k - 1] + 0.5 * (tab[k - 1] + tab[k]) * hcell;
  std::vector<float> gi32(gi.begin(), gi.end());
  cudaFree(P->d_dlnrho_int64);
  cudaFree(P->d_dlnrho_int32);
  P->d_dlnrho_int64 = nullptr;
  P->d_dlnrho_int32 = nullptr;
  MFS_TRY(upload(&P->d_dlnrho_int64, gi.data(), (size_t)n, s));
  MFS_TRY(upload(&P->d_dlnrho_int32, gi32.data(), (size_t)n, s));
  MFS_TRY(upload(&P->d_dlnrho64, tab, (size_t)n, s));
  MFS_TRY(upload(&P->d_dlnrho32, t32.data(), (size_t)n, s));
  MFS_CUDA(cudaStreamSynchronize(s));
  P->n_dlnrho = n;
  return MFS_OK;
}


template <typename T>
static mfs_status apply_typed(mfs_problem* P, int lvl, int op, int constrained, int withc_b, const void* u,
                              const void* p, void* yu, void* yp) {
  return apply_constrained<T>(P, lvl, op, constrained, withc_b, (const T*)u, (const T*)p, (T*)yu, (T*)yp);
}

static mfs_status check_vecs(const void* a, const void* b) {
  if (!a || !b) {
    set_error("null vector pointer");
    return MFS_EINVAL;
  }
  return MFS_OK;
}

static mfs_status dispatch(mfs_problem* P, int lvl, mfs_prec prec, int op, int constrained, int withc_b,
                           const void* u, const void* p, void* yu, void* yp) {
  MFS_TRY(check_problem(P, lvl, true));
  if (prec != MFS_F64 && prec != MFS_F32) {
    set_error("invalid precision %d", (int)prec);
    return MFS_EINVAL;
  }
  if (prec == MFS_F64) return apply_typed<double>(P, lvl, op, constrained, withc_b, u, p, yu, yp);
  return apply_typed<float>(P, lvl, op, constrained, withc_b, u, p, yu, yp);
}

mfs_status mfs_set_constraint_form(mfs_problem* P, int rho_weighted) {
  if (!P || (rho_weighted != 0 && rho_weighted != 1)) {
    set_error("null problem or rho_weighted outside {0, 1}");
    return MFS_EINVAL;
  }
  P->rho_weighted = rho_weighted;
  P->version++;
  return MFS_OK;
}

mfs_status mfs_apply_part(mfs_problem* P, int lvl, mfs_prec prec, int fused, int m0, int m1, const void* u,
                          const void* p, void* yu, void* yp) {
  if (!u || !yu || (fused && (!p || !yp))) {
    set_error("null vector pointer");
    return MFS_EINVAL;
  }
  if (m0 < 0 || m1 > kMacroCells || m0 >= m1) {
    set_error("macro range [%d, %d) outside [0, %d) or empty", m0, m1, kMacroCells);
    return MFS_EINVAL;
  }
  MFS_TRY(check_problem(P, lvl, true));
  if (prec != MFS_F64 && prec != MFS_F32) {
    set_error("invalid precision %d", (int)prec);
    return MFS_EINVAL;
  }
  const int op = fused ? (OP_A | OP_BT | OP_B) : OP_A;
  // constrained element arithmetic (P0 on the inputs, P_v on the outputs, identity rows at
  // the Dirichlet nodes the range touches); p used as given, no mean removal of yp
  if (prec == MFS_F64)
    return launch_apply<double>(P, lvl, op, 1, fused, (const double*)u, (const double*)p, (double*)yu,
                                (double*)yp, nullptr, 1, m0, m1);
  return launch_apply<float>(P, lvl, op, 1, fused, (const float*)u, (const float*)p, (float*)yu, (float*)yp,
                             nullptr, 1, m0, m1);
}

mfs_status mfs_mesh_macro_topology(const mfs_mesh* M, int* cells, int* edges, int* faces) {
  if (!M || !cells || !edges || !faces) {
    set_error("null mesh or output");
    return MFS_EINVAL;
  }
  for (int m = 0; m < kMacroCells; ++m) {
    const MacroTopo& t = M->host.topo[m];
    for (int k = 0; k < 4; ++k) cells[4 * m + k] = t.vid[k];
    for (int k = 0; k < 6; ++k) edges[6 * m + k] = t.eid[k];
    for (int k = 0; k < 4; ++k) faces[4 * m + k] = t.fid[k];
  }
  return MFS_OK;
}

mfs_status mfs_apply_A(mfs_problem* P, int lvl, mfs_prec prec, mfs_bcmode mode, const void* u, void* y) {
  MFS_TRY(check_vecs(u, y));
  return dispatch(P, lvl, prec, OP_A, mode == MFS_CONSTRAINED, 0, u, nullptr, y, nullptr);
}

mfs_status mfs_apply_B(mfs_problem* P, int lvl, mfs_prec prec, mfs_bcmode mode, int with_C, const void* u,
                       void* q) {
  MFS_TRY(check_vecs(u, q));
  return dispatch(P, lvl, prec, OP_B, mode == MFS_CONSTRAINED, with_C ? 1 : 0, u, nullptr, nullptr, q);
}

mfs_status mfs_apply_BT(mfs_problem* P, int lvl, mfs_prec prec, mfs_bcmode mode, int with_C, const void* p,
                        void* y) {
  MFS_TRY(check_vecs(p, y));
  const int op = with_C ? (OP_BT | OP_CT) : OP_BT;
  return dispatch(P, lvl, prec, op, mode == MFS_CONSTRAINED, 0, nullptr, p, y, nullptr);
}

mfs_status mfs_apply_stokes(mfs_problem* P, int lvl, mfs_prec prec, int transpose, const void* u, const void* p,
                            void* yu, void* yp) {
  MFS_TRY(check_vecs(u, p));
  MFS_TRY(check_vecs(yu, yp));
  if (transpose) return dispatch(P, lvl, prec, OP_A | OP_BT | OP_CT | OP_B, 1, 0, u, p, yu, yp);
  return dispatch(P, lvl, prec, OP_A | OP_BT | OP_B, 1, 1, u, p, yu, yp);
}

