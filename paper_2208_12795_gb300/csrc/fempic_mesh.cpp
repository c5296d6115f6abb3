// Host-side derivation of the mesh tables the particle kernels read.
//
// Numbering (the ABI convention): tet nodes sorted by global id; edges and
// faces numbered lexicographically by their sorted node tuples; local edge e
// joins sorted local nodes kLocalEdge[e]; local face k is opposite node k.
// Geometry (FP64, fixed operation order, compiled without FMA contraction so
// that location is reproducible): e_k = x_k - x_0; c1 = e2 x e3, c2 = e3 x e1,
// c3 = e1 x e2; det = (e1x c1x + e1y c1y) + e1z c1z; grad l_k = c_k / det.
// These gradients are the rows of the inverse of [e1 e2 e3], so
// l_k(r) = grad l_k . (r - x_0) for k = 1..3 and l_0 = 1 - l_1 - l_2 - l_3.
#include <algorithm>
#include <array>
#include <cmath>
#include <numeric>

#include "fempic_internal.h"

namespace fempic {

namespace {

struct Tri {
  int32_t v[3];
  bool operator<(const Tri& o) const {
    if (v[0] != o.v[0]) return v[0] < o.v[0];
    if (v[1] != o.v[1]) return v[1] < o.v[1];
    return v[2] < o.v[2];
  }
  bool operator==(const Tri& o) const { return v[0] == o.v[0] && v[1] == o.v[1] && v[2] == o.v[2]; }
};

void cross(const double* a, const double* b, double* o) {
  o[0] = a[1] * b[2] - a[2] * b[1];
  o[1] = a[2] * b[0] - a[0] * b[2];
  o[2] = a[0] * b[1] - a[1] * b[0];
}

}  // namespace

int build_host_mesh(const fempic_mesh_desc& d, HostMesh* m, std::string* err) {
  if (d.n_nodes <= 0 || d.n_tets <= 0 || !d.nodes_xyz || !d.tet_nodes) {
    *err = "mesh: empty or NULL node/tet arrays";
    return FEMPIC_EINVAL;
  }
  if (d.n_nodes >= (int64_t(1) << 31) || d.n_tets >= (int64_t(1) << 28)) {
    *err = "mesh: too many nodes or tets for 32-bit ids";
    return FEMPIC_EINVAL;
  }
  const int64_t nn = d.n_nodes, nt = d.n_tets;
  m->nn = nn;
  m->nt = nt;
  for (int a = 0; a < 3; a++) {
    m->lo[a] = d.bbox_lo[a];
    m->hi[a] = d.bbox_hi[a];
    if (!(m->hi[a] > m->lo[a])) {
      *err = "mesh: empty bounding box";
      return FEMPIC_EINVAL;
    }
  }
  m->xyz.assign(d.nodes_xyz, d.nodes_xyz + 3 * nn);
  m->tn.resize(4 * nt);
  for (int64_t t = 0; t < nt; t++) {
    std::array<int32_t, 4> v;
    for (int i = 0; i < 4; i++) {
      v[i] = d.tet_nodes[4 * t + i];
      if (v[i] < 0 || v[i] >= nn) {
        *err = "mesh: tet references a node id out of range";
        return FEMPIC_EINVAL;
      }
    }
    std::sort(v.begin(), v.end());
    if (v[0] == v[1] || v[1] == v[2] || v[2] == v[3]) {
      *err = "mesh: tet with a repeated node";
      return FEMPIC_EMESH;
    }
    std::copy(v.begin(), v.end(), m->tn.begin() + 4 * t);
  }

  // Edges: unique sorted (lo, hi) pairs as 64-bit keys.
  std::vector<uint64_t> ekey(6 * nt);
  for (int64_t t = 0; t < nt; t++)
    for (int e = 0; e < 6; e++)
      ekey[6 * t + e] = uint64_t(m->tn[4 * t + kLocalEdge[e][0]]) * uint64_t(nn) +
                        uint64_t(m->tn[4 * t + kLocalEdge[e][1]]);
  std::vector<uint64_t> eu(ekey);
  std::sort(eu.begin(), eu.end());
  eu.erase(std::unique(eu.begin(), eu.end()), eu.end());
  m->ne = int64_t(eu.size());
  m->en.resize(2 * m->ne);
  for (int64_t e = 0; e < m->ne; e++) {
    m->en[2 * e] = int32_t(eu[e] / uint64_t(nn));
    m->en[2 * e + 1] = int32_t(eu[e] % uint64_t(nn));
  }
  m->te.resize(6 * nt);
  for (int64_t i = 0; i < 6 * nt; i++)
    m->te[i] = int32_t(std::lower_bound(eu.begin(), eu.end(), ekey[i]) - eu.begin());

  // Faces: unique sorted node triples.
  std::vector<Tri> fkey(4 * nt);
  for (int64_t t = 0; t < nt; t++)
    for (int f = 0; f < 4; f++)
      for (int i = 0; i < 3; i++) fkey[4 * t + f].v[i] = m->tn[4 * t + kLocalFace[f][i]];
  std::vector<Tri> fu(fkey);
  std::sort(fu.begin(), fu.end());
  fu.erase(std::unique(fu.begin(), fu.end()), fu.end());
  m->nf = int64_t(fu.size());
  m->fn.resize(3 * m->nf);
  for (int64_t f = 0; f < m->nf; f++)
    for (int i = 0; i < 3; i++) m->fn[3 * f + i] = fu[f].v[i];
  m->tf.resize(4 * nt);
  for (int64_t i = 0; i < 4 * nt; i++)
    m->tf[i] = int32_t(std::lower_bound(fu.begin(), fu.end(), fkey[i]) - fu.begin());

  // Neighbours: each face is shared by at most two tets.
  std::vector<int32_t> owner(2 * m->nf, -1);
  for (int64_t t = 0; t < nt; t++)
    for (int k = 0; k < 4; k++) {
      int64_t f = m->tf[4 * t + k];
      if (owner[2 * f] < 0) {
        owner[2 * f] = int32_t(t);
      } else if (owner[2 * f + 1] < 0) {
        owner[2 * f + 1] = int32_t(t);
      } else {
        *err = "mesh: non-conforming (a face belongs to more than two tets)";
        return FEMPIC_EMESH;
      }
    }
  m->nb.resize(4 * nt);
  for (int64_t t = 0; t < nt; t++)
    for (int k = 0; k < 4; k++) {
      int64_t f = m->tf[4 * t + k];
      int32_t other = owner[2 * f] == int32_t(t) ? owner[2 * f + 1] : owner[2 * f];
      if (other >= 0) {
        m->nb[4 * t + k] = other;
        continue;
      }
      int32_t code = kWallOther;
      for (int a = 0; a < 3 && code == kWallOther; a++)
        for (int s = 0; s < 2 && code == kWallOther; s++) {
          const double plane = s ? m->hi[a] : m->lo[a];
          bool on = true;
          for (int i = 0; i < 3; i++) on = on && m->xyz[3 * int64_t(m->fn[3 * f + i]) + a] == plane;
          if (on) code = -1 - (2 * a + s);
        }
      m->nb[4 * t + k] = code;
    }

  // FP64 barycentric geometry.
  m->geom.resize(12 * nt);
  for (int64_t t = 0; t < nt; t++) {
    const double* x0 = &m->xyz[3 * int64_t(m->tn[4 * t])];
    double e[3][3], c[3][3];
    for (int k = 0; k < 3; k++) {
      const double* xk = &m->xyz[3 * int64_t(m->tn[4 * t + k + 1])];
      for (int a = 0; a < 3; a++) e[k][a] = xk[a] - x0[a];
    }
    cross(e[1], e[2], c[0]);
    cross(e[2], e[0], c[1]);
    cross(e[0], e[1], c[2]);
    const double det = (e[0][0] * c[0][0] + e[0][1] * c[0][1]) + e[0][2] * c[0][2];
    if (!(det != 0.0) || !std::isfinite(det)) {
      *err = "mesh: degenerate (zero-volume) tet";
      return FEMPIC_EMESH;
    }
    double* g = &m->geom[12 * t];
    for (int a = 0; a < 3; a++) g[a] = x0[a];
    for (int k = 0; k < 3; k++)
      for (int a = 0; a < 3; a++) g[3 + 3 * k + a] = c[k][a] / det;
  }

  // Location grid: about 6 tets per cell, at most 256 cells per axis.
  int gd = int(std::cbrt(double(nt) / 6.0) + 0.5);
  gd = std::max(1, std::min(gd, 256));
  for (int a = 0; a < 3; a++) {
    m->gd[a] = gd;
    m->ginv[a] = double(gd) / (m->hi[a] - m->lo[a]);
  }
  const int64_t ncell = int64_t(gd) * gd * gd;
  std::vector<int64_t> cnt(ncell + 1, 0);
  auto tet_cells = [&](int64_t t, int* c0, int* c1) {
    for (int a = 0; a < 3; a++) {
      double mn = INFINITY, mx = -INFINITY;
      for (int v = 0; v < 4; v++) {
        double x = m->xyz[3 * int64_t(m->tn[4 * t + v]) + a];
        mn = std::min(mn, x);
        mx = std::max(mx, x);
      }
      c0[a] = grid_cell(mn, m->lo[a], m->ginv[a], gd);
      c1[a] = grid_cell(mx, m->lo[a], m->ginv[a], gd);
    }
  };
  for (int64_t t = 0; t < nt; t++) {
    int c0[3], c1[3];
    tet_cells(t, c0, c1);
    for (int k = c0[2]; k <= c1[2]; k++)
      for (int j = c0[1]; j <= c1[1]; j++)
        for (int i = c0[0]; i <= c1[0]; i++) cnt[1 + i + int64_t(gd) * (j + int64_t(gd) * k)]++;
  }
  std::partial_sum(cnt.begin(), cnt.end(), cnt.begin());
  m->gstart = cnt;
  m->gtet.resize(cnt[ncell]);
  for (int64_t t = 0; t < nt; t++) {  // ascending t keeps each cell's list sorted
    int c0[3], c1[3];
    tet_cells(t, c0, c1);
    for (int k = c0[2]; k <= c1[2]; k++)
      for (int j = c0[1]; j <= c1[1]; j++)
        for (int i = c0[0]; i <= c1[0]; i++) m->gtet[cnt[i + int64_t(gd) * (j + int64_t(gd) * k)]++] = int32_t(t);
  }
  return FEMPIC_OK;
}

}  // namespace fempic
