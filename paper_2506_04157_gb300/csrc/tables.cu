// Per-level tables of the sweep: the global id of every slot of every tile's node blocks
// (P2 slots carry the node's geometric class: 0 inner, 1 surface, 2 CMB, in bits 29-30).
#include "apply.cuh"
#include "library.h"

namespace mfs {

__global__ void id_tables_kernel(const MacroTopo* __restrict__ topo, const Tile* __restrict__ tiles, int n_tiles,
                                 Numbering nb2, Numbering nb1, int* __restrict__ ids2, int* __restrict__ ids1) {
  const int m = blockIdx.y, tidx = blockIdx.x;
  const MacroTopo t = topo[m];
  const Tile tile = tiles[tidx];
  const size_t lin = (size_t)m * n_tiles + tidx;
  const int a0 = tile.ta * TT, b0 = tile.tb * TT, c0 = tile.tc * TT;
  const int N = nb2.N, n = nb1.N;
  for (int s = threadIdx.x; s < NSLOT2; s += blockDim.x) {
    int dA, dB, dC, code = -1;
    if (slot_coords(s, dA, dB, dC)) {
      const int A = 2 * a0 + dA, B = 2 * b0 + dB, C = 2 * c0 + dC;
      if (A <= N && A >= B && B >= C) {
        const int i0 = N - A, i1 = A - B, i2 = B - C, i3 = C;
        const int id = lattice_id(t, nb2, m, i0, i1, i2, i3);
        const int mask = (i0 > 0) | ((i1 > 0) << 1) | ((i2 > 0) << 2) | ((i3 > 0) << 3);
        int gc = 0;
        if ((mask & ~t.topmask & 15) == 0) gc = 1;
        else if ((mask & ~t.botmask & 15) == 0) gc = 2;
        code = slot_code(id, gc);
      }
    }
    ids2[lin * NSLOT2 + s] = code;
  }
  for (int s = threadIdx.x; s < NSLOT1; s += blockDim.x) {
    const int a = a0 + s % NB1, b = b0 + (s / NB1) % NB1, c = c0 + s / (NB1 * NB1);
    int id = -1;
    if (a <= n && a >= b && b >= c) id = lattice_id(t, nb1, m, n - a, a - b, b - c, c);
    ids1[lin * NSLOT1 + s] = id;
  }
}

mfs_status build_id_tables(const mfs_mesh* M, LevelData& L) {
  if (L.nb2.total > kSlotIdMask) {
    set_error("level %d too large for 29-bit node ids", L.l);
    return MFS_EINVAL;
  }
  const size_t nt = (size_t)L.n_tiles * kMacroCells;
  MFS_CUDA(cudaMalloc((void**)&L.d_ids2, sizeof(int) * nt * NSLOT2));
  MFS_CUDA(cudaMalloc((void**)&L.d_ids1, sizeof(int) * nt * NSLOT1));
  dim3 grid(L.n_tiles, kMacroCells);
  id_tables_kernel<<<grid, 256, 0, M->ctx->stream>>>(M->d_topo, L.d_tiles, L.n_tiles, L.nb2, L.nb1, L.d_ids2,
                                                      L.d_ids1);
  MFS_CUDA(cudaGetLastError());
  return MFS_OK;
}

}  // namespace mfs
