// Internal structures of the mfs library (host + device).  Not part of the C ABI.
//
// Geometry (Sec. 4.1 of arxiv 2506.04157, Fig. BlendingTransformation): a micro-tet of
// refinement level l is the image of the reference tet under zeta -> x~ = v0 + Jm (q + T_pi
// zeta)/n (straight macro map Jm in Kuhn coordinates, cube corner q, Freudenthal type pi)
// followed by the blending map B(x~) = (x~.nh/delta) x~/|x~|.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace mfs {

constexpr int kMacroVerts = 24;
constexpr int kMacroEdges = 102;
constexpr int kMacroFaces = 140;
constexpr int kMacroCells = 60;

// Tile of TT^3 lattice cubes handled by one CTA: its P2 node block has (2TT+1)^3 points,
// stored as 8 parity classes of (TT+1)^3 slots; its P1 vertex block has (TT+1)^3 points.
constexpr int TT = 4;
constexpr int NB1 = TT + 1;            // P1 block edge
constexpr int NSLOT1 = NB1 * NB1 * NB1;
constexpr int NSLOT2 = 8 * NSLOT1;

// P2 slot-table entries: the global node id in bits 0-28 and its geometric class (0 interior,
// 1 outer surface, 2 core-mantle boundary) in bits 29-30; -1 marks a slot outside the macro
constexpr int kSlotClassShift = 29;
constexpr int kSlotIdMask = (1 << kSlotClassShift) - 1;
__host__ __device__ __forceinline__ int slot_code(int id, int cls) { return id | (cls << kSlotClassShift); }
__host__ __device__ __forceinline__ int slot_node(int code) { return code & kSlotIdMask; }
__host__ __device__ __forceinline__ int slot_class(int code) { return code >> kSlotClassShift; }

// Numbering of the lattice points of one level (N intervals per macro edge): macro
// vertices, then macro-edge interiors, macro-face interiors, macro-cell interiors.
struct Numbering {
  int N;
  int nE1, nF1, nC1;
  int offE, offF, offC, total;
};

inline Numbering make_numbering(int N) {
  Numbering nb;
  nb.N = N;
  nb.nE1 = N > 1 ? N - 1 : 0;
  nb.nF1 = N > 2 ? (N - 1) * (N - 2) / 2 : 0;
  nb.nC1 = N > 3 ? (N - 3) * (N - 2) * (N - 1) / 6 : 0;
  nb.offE = kMacroVerts;
  nb.offF = nb.offE + kMacroEdges * nb.nE1;
  nb.offC = nb.offF + kMacroFaces * nb.nF1;
  nb.total = nb.offC + kMacroCells * nb.nC1;
  return nb;
}

// Topology of one macro-cell: its vertices in increasing global order (local 0..3),
// the ids of its 6 edges (local pairs 01,02,03,12,13,23), of its 4 faces (face z is
// opposite local vertex z), and which local vertices lie on the surface sphere.
struct MacroTopo {
  int vid[4];
  int eid[6];
  int fid[4];
  int topmask;     // bit k set: local vertex k on r = r_surf
  int botmask;     // bit k set: local vertex k on r = r_cmb
};

// Geometry of one macro-cell in precision T.
template <typename T>
struct MacroGeom {
  T v0[3];      // straight position of local vertex 0
  T Jm[9];      // row-major, columns v1-v0, v2-v1, v3-v2 (Kuhn coordinates)
  T Jinv[9];    // row-major inverse of Jm
  T absdet;     // |det Jm|
  T nh[3];      // unit normal of the icosahedral face of the prism
  T delta;      // nh . (unit vertex direction): offset of the face plane
};

// One tile of a macro: cube range [ta*TT, ta*TT+TT) x ... and its tet-list class.
struct Tile {
  int16_t ta, tb, tc;
  int16_t cls;
};

// Operator sets of the fused micro-tet sweep; OP_CT: the B^T part is (B + C)^T;
// OP_BC: the B part is (B + C).
// OP_ETAQ (with OP_A alone): the viscosity at the quadrature points from the level's P2
// temperature and the viscosity law (levels up to l_eta) instead of the P1 nodal values.
// OP_RHO (with OP_BC / OP_CT): the constraint is the density-weighted -int q div(rho u)
// (mfs_set_constraint_form) — the B + C integrand weighted by rho(r) at the quadrature point.
enum { OP_A = 1, OP_BT = 2, OP_B = 4, OP_CT = 8, OP_BC = 16, OP_ETAQ = 32, OP_RHO = 64 };

// Boundary condition types (match include/mfs.h).
enum { BC_DIRICHLET = 0, BC_FREESLIP = 1 };
// node classes used inside kernels after mapping through the boundary conditions
enum { NODE_FREE = 0, NODE_DIRICHLET = 1, NODE_FREESLIP = 2 };

#if defined(__CUDACC__)
#define MFS_HD __host__ __device__ __forceinline__
#else
#define MFS_HD inline
#endif

MFS_HD int tetnum(int m) { return m > 0 ? m * (m + 1) * (m + 2) / 6 : 0; }

MFS_HD int face_interior_index(int i1, int i2, int N) {
  return (i2 - 1) * (N - 1) - (i2 - 1) * i2 / 2 + (i1 - 1);
}

MFS_HD int cell_interior_index(int i1, int i2, int i3, int N) {
  const int K = N - 2;
  const int before = tetnum(K - 1) - tetnum(K - i3);
  const int M = N - 1 - i3;
  return before + (i2 - 1) * M - (i2 - 1) * i2 / 2 + (i1 - 1);
}

MFS_HD int sel4(int i0, int i1, int i2, int i3, int k) {
  return k == 0 ? i0 : (k == 1 ? i1 : (k == 2 ? i2 : i3));
}

MFS_HD int highest_bit(int m) { return m & 8 ? 3 : (m & 4 ? 2 : (m & 2 ? 1 : 0)); }
MFS_HD int lowest_bit(int m) { return m & 1 ? 0 : (m & 2 ? 1 : (m & 4 ? 2 : 3)); }

// Global id of the lattice point with integer barycentrics (i0..i3), sum N, in macro m.
MFS_HD int lattice_id(const MacroTopo& t, const Numbering& nb, int m, int i0, int i1, int i2,
                      int i3) {
  const int mask = (i0 > 0) | ((i1 > 0) << 1) | ((i2 > 0) << 2) | ((i3 > 0) << 3);
  if (mask == 15) return nb.offC + m * nb.nC1 + cell_interior_index(i1, i2, i3, nb.N);
  const int hi = highest_bit(mask);
  const int lo = lowest_bit(mask);
  const int rest = mask & ~(1 << hi) & ~(1 << lo);
  if (rest) {  // three nonzero: face opposite the zero position; (i1,i2) = (mid, hi)
    const int z = lowest_bit(~mask & 15);
    const int mid = lowest_bit(rest);
    return nb.offF + t.fid[z] * nb.nF1 +
           face_interior_index(sel4(i0, i1, i2, i3, mid), sel4(i0, i1, i2, i3, hi), nb.N);
  }
  if (hi != lo) {  // two nonzero: macro edge (lo, hi), position = weight of hi
    const int e = lo == 0 ? hi - 1 : (lo == 1 ? hi + 1 : 5);
    return nb.offE + t.eid[e] * nb.nE1 + sel4(i0, i1, i2, i3, hi) - 1;
  }
  return t.vid[hi];
}

// Class (NODE_*) of a lattice point from the zero pattern of its barycentrics.
MFS_HD int node_class(const MacroTopo& t, int mask, int bc_surface, int bc_cmb) {
  if ((mask & ~t.topmask & 15) == 0) return bc_surface == BC_DIRICHLET ? NODE_DIRICHLET : NODE_FREESLIP;
  if ((mask & ~t.botmask & 15) == 0) return bc_cmb == BC_DIRICHLET ? NODE_DIRICHLET : NODE_FREESLIP;
  return NODE_FREE;
}

}  // namespace mfs
