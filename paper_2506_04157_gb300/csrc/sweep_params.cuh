// Parameters of the auxiliary micro-tet sweeps (diagonals, mass and Poisson operators,
// gradient, buoyancy) on one level: geometry, tiles and slot tables, the level's nodal
// viscosity, and on the levels up to l_eta the viscosity law's fields.
#pragma once

#include "apply.cuh"
#include "library.h"
#include "solver.h"

namespace mfs {

template <typename T>
inline ApplyParams<T> sweep_params(mfs_problem* P, int lvl) {
  mfs_mesh* M = P->mesh;
  const LevelData& L = M->levels[lvl];
  ApplyParams<T> prm{};
  prm.eta = lvl_eta<T>(P, lvl);
  prm.geom = lvl_geom<T>(M);
  prm.tiles = L.d_tiles;
  prm.tets = L.d_tets;
  prm.classes = L.d_classes;
  prm.ids2 = L.d_ids2;
  prm.ids1 = L.d_ids1;
  prm.n_p2 = L.nb2.total;
  prm.n_p1 = L.nb1.total;
  prm.n = L.n;
  prm.r_cmb = (T)M->host.r_cmb;
  if (lvl <= P->l_eta) {
    prm.temp = lvl_temp<T>(P, lvl);
    prm.lbase = lvl_lbase<T>(P);
    prm.n_lbase = (int)P->lbase_host.size();
    prm.E_A = (T)P->E_A;
    prm.V_A = (T)P->V_A;
    prm.r_surf = (T)M->host.r_surf;
  }
  return prm;
}

}  // namespace mfs
