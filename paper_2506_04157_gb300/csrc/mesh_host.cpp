// Host-side construction of the icosahedral shell macro mesh and of the per-level tile
// tables (arxiv 2506.04157, Sec. 4.1: unstructured coarse mesh of truncated pyramids
// cut into tetrahedra, uniformly refined; blending map onto the shell).
#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <map>
#include <set>

#include "library.h"

namespace mfs {

static void inv3(const double* A, double* Ai, double* det_out) {
  const double a = A[0], b = A[1], c = A[2], d = A[3], e = A[4], f = A[5], g = A[6], h = A[7], i = A[8];
  const double det = a * (e * i - f * h) - b * (d * i - f * g) + c * (d * h - e * g);
  Ai[0] = (e * i - f * h) / det;
  Ai[1] = (c * h - b * i) / det;
  Ai[2] = (b * f - c * e) / det;
  Ai[3] = (f * g - d * i) / det;
  Ai[4] = (a * i - c * g) / det;
  Ai[5] = (c * d - a * f) / det;
  Ai[6] = (d * h - e * g) / det;
  Ai[7] = (b * g - a * h) / det;
  Ai[8] = (a * e - b * d) / det;
  *det_out = det;
}

void HostMacroMesh::build(double rc, double rs, int blend) {
  r_cmb = rc;
  r_surf = rs;
  blending = blend;
  const double phi = (1.0 + std::sqrt(5.0)) / 2.0;
  // 12 icosahedron directions: position p of the cyclic rotation, sign pattern q
  for (int p = 0; p < 3; ++p)
    for (int q = 0; q < 4; ++q) {
      const double s1 = (q >> 1) ? 1.0 : -1.0, s2 = (q & 1) ? 1.0 : -1.0;
      const double base[3] = {0.0, s1, s2 * phi};
      double* v = unit[4 * p + q];
      for (int r = 0; r < 3; ++r) v[r] = base[((r - p) % 3 + 3) % 3];
      const double nrm = std::sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
      for (int r = 0; r < 3; ++r) v[r] /= nrm;
    }
  for (int k = 0; k < 12; ++k)
    for (int r = 0; r < 3; ++r) {
      unit[12 + k][r] = unit[k][r];
      verts[k][r] = rc * unit[k][r];
      verts[12 + k][r] = rs * unit[k][r];
    }
  for (int k = 0; k < 24; ++k) layer[k] = k < 12 ? 0 : 1;
  // icosahedron faces: triples at mutual edge distance, lexicographic
  const double elen = 2.0 / std::sqrt(1.0 + phi * phi);
  auto dist = [&](int i, int j) {
    double s = 0;
    for (int r = 0; r < 3; ++r) s += (unit[i][r] - unit[j][r]) * (unit[i][r] - unit[j][r]);
    return std::sqrt(s);
  };
  std::vector<std::array<int, 3>> ico;
  for (int i = 0; i < 12; ++i)
    for (int j = i + 1; j < 12; ++j) {
      if (std::fabs(dist(i, j) - elen) > 1e-9) continue;
      for (int k = j + 1; k < 12; ++k)
        if (std::fabs(dist(i, k) - elen) < 1e-9 && std::fabs(dist(j, k) - elen) < 1e-9)
          ico.push_back({i, j, k});
    }
  // prisms -> 3 tets each: quad diagonals through the lowest vertex
  int mc = 0;
  for (int f = 0; f < 20; ++f) {
    const int a = ico[f][0], b = ico[f][1], c = ico[f][2];
    const int A = a + 12, B = b + 12, C = c + 12;
    const int tets[3][4] = {{a, b, c, C}, {a, b, C, B}, {a, B, C, A}};
    for (auto& t : tets) {
      int s[4] = {t[0], t[1], t[2], t[3]};
      std::sort(s, s + 4);
      std::memcpy(cells[mc], s, sizeof(s));
      cell_prism[mc] = f;
      ++mc;
    }
    // prism plane normal (outward) and offset
    double u1[3], u2[3], nn[3];
    for (int r = 0; r < 3; ++r) {
      u1[r] = unit[b][r] - unit[a][r];
      u2[r] = unit[c][r] - unit[a][r];
    }
    nn[0] = u1[1] * u2[2] - u1[2] * u2[1];
    nn[1] = u1[2] * u2[0] - u1[0] * u2[2];
    nn[2] = u1[0] * u2[1] - u1[1] * u2[0];
    double l = std::sqrt(nn[0] * nn[0] + nn[1] * nn[1] + nn[2] * nn[2]);
    double d = (nn[0] * unit[a][0] + nn[1] * unit[a][1] + nn[2] * unit[a][2]) / l;
    const double sg = d < 0 ? -1.0 : 1.0;
    for (int r = 0; r < 3; ++r) prism_nh[f][r] = sg * nn[r] / l;
    prism_delta[f] = sg * d;
  }
  // macro edges and faces: unique increasing tuples in lexicographic order
  static const int LE[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}};
  std::set<std::array<int, 2>> es;
  std::set<std::array<int, 3>> fs;
  for (int m = 0; m < 60; ++m) {
    for (auto& e : LE) es.insert({cells[m][e[0]], cells[m][e[1]]});
    for (int z = 0; z < 4; ++z) {
      std::array<int, 3> t;
      int k = 0;
      for (int q = 0; q < 4; ++q)
        if (q != z) t[k++] = cells[m][q];
      fs.insert(t);
    }
  }
  std::map<std::array<int, 2>, int> eidx;
  std::map<std::array<int, 3>, int> fidx;
  int k = 0;
  for (auto& e : es) {
    edges[k][0] = e[0];
    edges[k][1] = e[1];
    eidx[e] = k++;
  }
  k = 0;
  for (auto& f : fs) {
    for (int r = 0; r < 3; ++r) faces[k][r] = f[r];
    fidx[f] = k++;
  }
  for (int m = 0; m < 60; ++m) {
    MacroTopo& t = topo[m];
    t.topmask = t.botmask = 0;
    for (int q = 0; q < 4; ++q) {
      t.vid[q] = cells[m][q];
      if (layer[cells[m][q]] == 1) t.topmask |= 1 << q;
      else t.botmask |= 1 << q;
    }
    for (int e = 0; e < 6; ++e) t.eid[e] = eidx[{cells[m][LE[e][0]], cells[m][LE[e][1]]}];
    for (int z = 0; z < 4; ++z) {
      std::array<int, 3> tt;
      int kk = 0;
      for (int q = 0; q < 4; ++q)
        if (q != z) tt[kk++] = cells[m][q];
      t.fid[z] = fidx[tt];
    }
    MacroGeom<double>& g = geom[m];
    const double* v[4] = {verts[cells[m][0]], verts[cells[m][1]], verts[cells[m][2]], verts[cells[m][3]]};
    for (int r = 0; r < 3; ++r) {
      g.v0[r] = v[0][r];
      g.Jm[3 * r + 0] = v[1][r] - v[0][r];
      g.Jm[3 * r + 1] = v[2][r] - v[1][r];
      g.Jm[3 * r + 2] = v[3][r] - v[2][r];
    }
    double det;
    inv3(g.Jm, g.Jinv, &det);
    g.absdet = std::fabs(det);
    const int f = cell_prism[m];
    for (int r = 0; r < 3; ++r) g.nh[r] = prism_nh[f][r];
    g.delta = prism_delta[f];
  }
}

void HostMacroMesh::straight_point(int m, const int i[4], int N, double x[3]) const {
  for (int r = 0; r < 3; ++r) {
    double s = 0;
    for (int q = 0; q < 4; ++q) s += double(i[q]) * verts[cells[m][q]][r];
    x[r] = s / double(N);
  }
}

void HostMacroMesh::blend_point(int m, const double xs[3], double x[3]) const {
  if (!blending) {
    for (int r = 0; r < 3; ++r) x[r] = xs[r];
    return;
  }
  const int f = cell_prism[m];
  const double h = xs[0] * prism_nh[f][0] + xs[1] * prism_nh[f][1] + xs[2] * prism_nh[f][2];
  const double rho = std::sqrt(xs[0] * xs[0] + xs[1] * xs[1] + xs[2] * xs[2]);
  const double sc = h / prism_delta[f] / rho;
  for (int r = 0; r < 3; ++r) x[r] = sc * xs[r];
}

HostTiles build_tiles(int n) {
  // Freudenthal cubes (a,b,c), n > a >= b >= c >= 0; permutation pi gives the tet
  // q, q+e_pi0, q+e_pi0+e_pi1, q+(1,1,1).  A tet lies in the Kuhn simplex iff its four
  // vertices satisfy x1 >= x2 >= x3 (the bound x1 <= n holds for a < n).
  static const int PERM[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
  HostTiles H;
  const int nt = (n + TT - 1) / TT;
  std::map<std::vector<uint16_t>, int> cls_of;
  std::vector<std::vector<uint16_t>> lists;
  for (int tc = 0; tc < nt; ++tc)
    for (int tb = tc; tb < nt; ++tb)
      for (int ta = tb; ta < nt; ++ta) {
        std::vector<uint16_t> lst;
        for (int pm = 0; pm < 6; ++pm)
          for (int k = 0; k < TT; ++k)
            for (int j = 0; j < TT; ++j)
              for (int i = 0; i < TT; ++i) {
                const int a = ta * TT + i, b = tb * TT + j, c = tc * TT + k;
                if (a >= n || b > a || c > b) continue;
                int v[3] = {a, b, c};
                bool ok = v[0] >= v[1] && v[1] >= v[2];
                for (int s = 0; s < 3 && ok; ++s) {
                  v[PERM[pm][s]] += 1;
                  ok = v[0] >= v[1] && v[1] >= v[2];
                }
                if (ok) lst.push_back(uint16_t((pm << 12) | (k << 8) | (j << 4) | i));
              }
        if (lst.empty()) continue;
        auto it = cls_of.find(lst);
        int cl;
        if (it == cls_of.end()) {
          cl = (int)lists.size();
          cls_of[lst] = cl;
          lists.push_back(lst);
        } else {
          cl = it->second;
        }
        Tile t;
        t.ta = (int16_t)ta;
        t.tb = (int16_t)tb;
        t.tc = (int16_t)tc;
        t.cls = (int16_t)cl;
        H.tiles.push_back(t);
      }
  for (auto& l : lists) {
    int2 c;
    c.x = (int)H.tets.size();
    c.y = (int)l.size();
    H.classes.push_back(c);
    H.tets.insert(H.tets.end(), l.begin(), l.end());
  }
  return H;
}

template <typename T>
MacroGeom<T> cast_geom(const MacroGeom<double>& g) {
  MacroGeom<T> o;
  for (int r = 0; r < 3; ++r) {
    o.v0[r] = (T)g.v0[r];
    o.nh[r] = (T)g.nh[r];
  }
  for (int r = 0; r < 9; ++r) {
    o.Jm[r] = (T)g.Jm[r];
    o.Jinv[r] = (T)g.Jinv[r];
  }
  o.absdet = (T)g.absdet;
  o.delta = (T)g.delta;
  return o;
}
template MacroGeom<float> cast_geom<float>(const MacroGeom<double>&);
template MacroGeom<double> cast_geom<double>(const MacroGeom<double>&);

}  // namespace mfs
