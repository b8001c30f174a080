// Host-side mesh topology for RWG functions and the quasi-Helmholtz transforms.
//
// Sec. 2, Eq. RWGdef: edge n carries the RWG function supported on its two
// cells c_n^+ and c_n^- with free vertices r_n^+ and r_n^-.
// Sec. 2, Eq. qHofj: Sigma (N x N_C) and Lambda (N x N_V) with entries +-1,
// Lambda^T Sigma = 0.  Sec. 2 (graph Laplacians): Sigma^T Sigma is the cell
// graph Laplacian, the number of RWG edges of a cell on the diagonal and -1 for
// each pair of cells sharing an edge.  Open surfaces (Sec. 2: inner vertices only):
// an edge of one cell is a boundary edge without an RWG function, and the loop
// functions belong to the interior vertices.  Numbering and sign conventions:
// include/rfcmp.h.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <unordered_set>

#include "rfcmp_internal.h"

namespace rfcmp {

namespace {

struct HalfEdge {
  int32_t lo, hi;   // sorted vertex pair
  int32_t cell;     // owning cell
  int32_t local;    // local index of the opposite vertex
  int32_t a, b;     // the cell traverses a -> b
};

uint64_t mix64(uint64_t z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

}  // namespace

int build_topology(const int32_t* tris, int64_t nc, int64_t nv, Topology& T, std::string& err) {
  if (nc <= 0 || nv <= 0 || nc > (int64_t)1 << 28 || nv > (int64_t)1 << 28) {
    err = "mesh sizes out of range";
    return RFCMP_ERR_INVALID_ARG;
  }
  T = Topology();
  T.nc = nc;
  T.nv_mesh = nv;
  T.tris.assign(tris, tris + 3 * nc);
  std::vector<HalfEdge> he;
  he.reserve(3 * nc);
  for (int64_t c = 0; c < nc; ++c) {
    for (int i = 0; i < 3; ++i) {
      int32_t a = tris[3 * c + (i + 1) % 3], b = tris[3 * c + (i + 2) % 3];
      if (a < 0 || a >= nv || b < 0 || b >= nv) {
        err = "vertex index out of range in cell " + std::to_string(c);
        return RFCMP_ERR_MESH_NOT_MANIFOLD;
      }
      if (a == b) {
        err = "degenerate cell " + std::to_string(c);
        return RFCMP_ERR_MESH_NOT_MANIFOLD;
      }
      he.push_back({std::min(a, b), std::max(a, b), (int32_t)c, i, a, b});
    }
  }
  std::sort(he.begin(), he.end(), [](const HalfEdge& x, const HalfEdge& y) {
    if (x.lo != y.lo) return x.lo < y.lo;
    if (x.hi != y.hi) return x.hi < y.hi;
    return x.cell < y.cell;
  });
  // groups of equal vertex pairs: two half-edges make an RWG edge, one a boundary edge
  std::vector<size_t> inner;  // index of the first half-edge of each RWG edge
  std::vector<std::pair<int32_t, int32_t>> bnd;
  for (size_t q = 0; q < he.size();) {
    size_t r = q + 1;
    while (r < he.size() && he[r].lo == he[q].lo && he[r].hi == he[q].hi) ++r;
    if (r - q > 2) {
      err = "edge (" + std::to_string(he[q].lo) + "," + std::to_string(he[q].hi) + ") is shared by " +
            std::to_string(r - q) + " cells (a junction: not a 2-manifold)";
      return RFCMP_ERR_MESH_NOT_MANIFOLD;
    }
    if (r - q == 2) inner.push_back(q);
    else bnd.push_back({he[q].lo, he[q].hi});
    q = r;
  }
  const int64_t ne = (int64_t)inner.size();
  if (ne == 0) {
    err = "the mesh has no edge shared by two cells";
    return RFCMP_ERR_MESH_NOT_MANIFOLD;
  }
  T.ne = ne;
  T.edge_verts.resize(2 * ne);
  T.edge_cells.resize(2 * ne);
  T.edge_free.resize(2 * ne);
  T.cell_edges.assign(3 * nc, -1);
  T.cell_sign.assign(3 * nc, 0);
  for (int64_t n = 0; n < ne; ++n) {
    const HalfEdge& p = he[inner[n]];
    const HalfEdge& m = he[inner[n] + 1];
    if (!(p.a == m.b && p.b == m.a)) {
      err = "cells " + std::to_string(p.cell) + " and " + std::to_string(m.cell) +
            " are not consistently oriented";
      return RFCMP_ERR_MESH_ORIENTATION;
    }
    T.edge_cells[2 * n] = p.cell;
    T.edge_cells[2 * n + 1] = m.cell;
    T.edge_verts[2 * n] = p.a;
    T.edge_verts[2 * n + 1] = p.b;
    T.edge_free[2 * n] = tris[3 * p.cell + p.local];
    T.edge_free[2 * n + 1] = tris[3 * m.cell + m.local];
    T.cell_edges[3 * p.cell + p.local] = (int32_t)n;
    T.cell_sign[3 * p.cell + p.local] = 1;
    T.cell_edges[3 * m.cell + m.local] = (int32_t)n;
    T.cell_sign[3 * m.cell + m.local] = -1;
  }
  // every vertex must be used
  std::vector<int32_t> deg(nv, 0);
  for (int64_t i = 0; i < 3 * nc; ++i) deg[tris[i]]++;
  for (int64_t v = 0; v < nv; ++v)
    if (deg[v] == 0) {
      err = "vertex " + std::to_string(v) + " is not used by any cell";
      return RFCMP_ERR_MESH_NOT_MANIFOLD;
    }
  // boundary curves: each boundary vertex has exactly two boundary edges; the curves are the
  // components of the boundary edges (union-find over their vertices)
  std::vector<int32_t> bdeg(nv, 0), parent(nv);
  for (int64_t v = 0; v < nv; ++v) parent[v] = (int32_t)v;
  auto root = [&](int32_t v) {
    while (parent[v] != v) v = parent[v] = parent[parent[v]];
    return v;
  };
  for (auto& e : bnd) {
    bdeg[e.first]++;
    bdeg[e.second]++;
    parent[root(e.first)] = root(e.second);
  }
  int64_t curves = 0;
  for (int64_t v = 0; v < nv; ++v) {
    if (bdeg[v] != 0 && bdeg[v] != 2) {
      err = "vertex " + std::to_string(v) + " has " + std::to_string(bdeg[v]) +
            " boundary edges (not a 2-manifold)";
      return RFCMP_ERR_MESH_NOT_MANIFOLD;
    }
    if (bdeg[v] == 2 && root((int32_t)v) == v) ++curves;
  }
  // Euler characteristic of an orientable surface of genus g with b boundary curves: 2 - 2g - b
  const int64_t chi = nv - (ne + (int64_t)bnd.size()) + nc;
  if (2 - chi - curves < 0 || (2 - chi - curves) % 2 != 0) {
    err = "Euler characteristic " + std::to_string(chi) + " with " + std::to_string(curves) +
          " boundary curves is not that of an orientable surface";
    return RFCMP_ERR_MESH_NOT_MANIFOLD;
  }
  T.genus = (int)((2 - chi - curves) / 2);
  T.boundaries = (int)curves;
  // loop functions: the interior vertices (all vertices of a closed surface)
  T.loop_of.assign(nv, -1);
  T.loop_verts.clear();
  for (int64_t v = 0; v < nv; ++v)
    if (bdeg[v] == 0) {
      T.loop_of[v] = (int32_t)T.loop_verts.size();
      T.loop_verts.push_back((int32_t)v);
    }
  const int64_t nl = (int64_t)T.loop_verts.size();
  T.nv = nl;
  T.edge_loops.resize(2 * ne);
  for (int64_t i = 0; i < 2 * ne; ++i) T.edge_loops[i] = T.loop_of[T.edge_verts[i]];

  // Lambda^T gather lists over the loop vertices
  T.vtx_ptr.assign(nl + 1, 0);
  for (int64_t i = 0; i < 2 * ne; ++i)
    if (T.edge_loops[i] >= 0) T.vtx_ptr[T.edge_loops[i] + 1]++;
  for (int64_t v = 0; v < nl; ++v) T.vtx_ptr[v + 1] += T.vtx_ptr[v];
  T.vtx_edge.resize(T.vtx_ptr[nl]);
  T.vtx_sign.resize(T.vtx_ptr[nl]);
  {
    std::vector<int32_t> fill(T.vtx_ptr.begin(), T.vtx_ptr.end() - 1);
    for (int64_t n = 0; n < ne; ++n) {
      const int32_t l1 = T.edge_loops[2 * n], l2 = T.edge_loops[2 * n + 1];
      if (l1 >= 0) {
        T.vtx_edge[fill[l1]] = (int32_t)n;
        T.vtx_sign[fill[l1]++] = 1;
      }
      if (l2 >= 0) {
        T.vtx_edge[fill[l2]] = (int32_t)n;
        T.vtx_sign[fill[l2]++] = -1;
      }
    }
  }
  // Sigma^T Sigma (duplicates merged: two cells sharing two edges get -2)
  T.lap_ptr.assign(nc + 1, 0);
  T.lap_col.clear();
  T.lap_val.clear();
  for (int64_t c = 0; c < nc; ++c) {
    int32_t nb[3];
    int ndeg = 0;
    for (int i = 0; i < 3; ++i) {
      int32_t n = T.cell_edges[3 * c + i];
      nb[i] = n < 0 ? -1 : (T.edge_cells[2 * n] == c ? T.edge_cells[2 * n + 1] : T.edge_cells[2 * n]);
      ndeg += n >= 0;
    }
    std::vector<std::pair<int32_t, double>> row = {{(int32_t)c, (double)ndeg}};
    for (int i = 0; i < 3; ++i) {
      if (nb[i] < 0) continue;  // a boundary edge: no RWG function
      bool merged = false;
      for (auto& e : row)
        if (e.first == nb[i]) {
          e.second -= 1.0;
          merged = true;
        }
      if (!merged) row.push_back({nb[i], -1.0});
    }
    std::sort(row.begin(), row.end());
    for (auto& e : row) {
      T.lap_col.push_back(e.first);
      T.lap_val.push_back(e.second);
    }
    T.lap_ptr[c + 1] = (int32_t)T.lap_col.size();
  }
  // near pairs: cells sharing a vertex
  std::vector<int32_t> vc_ptr(nv + 1, 0), vc_cell(3 * nc);
  for (int64_t i = 0; i < 3 * nc; ++i) vc_ptr[tris[i] + 1]++;
  for (int64_t v = 0; v < nv; ++v) vc_ptr[v + 1] += vc_ptr[v];
  {
    std::vector<int32_t> fill(vc_ptr.begin(), vc_ptr.end() - 1);
    for (int64_t c = 0; c < nc; ++c)
      for (int i = 0; i < 3; ++i) vc_cell[fill[tris[3 * c + i]]++] = (int32_t)c;
  }
  T.near_pairs.clear();
  for (int64_t s = 0; s < nc; ++s) {
    std::vector<int32_t> nbrs;
    for (int i = 0; i < 3; ++i) {
      int32_t v = tris[3 * s + i];
      for (int32_t q = vc_ptr[v]; q < vc_ptr[v + 1]; ++q)
        if (vc_cell[q] >= s) nbrs.push_back(vc_cell[q]);
    }
    std::sort(nbrs.begin(), nbrs.end());
    nbrs.erase(std::unique(nbrs.begin(), nbrs.end()), nbrs.end());
    for (int32_t t : nbrs) {
      T.near_pairs.push_back((int32_t)s);
      T.near_pairs.push_back(t);
    }
  }
  uint64_t h = mix64((uint64_t)nv) ^ mix64((uint64_t)nc << 1);
  for (int64_t i = 0; i < 3 * nc; ++i) h = mix64(h ^ (uint64_t)(uint32_t)tris[i]);
  T.hash = h;
  return RFCMP_OK;
}

void mass_matrix_csr(const Topology& T, const double* verts, std::vector<int32_t>& ptr, std::vector<int32_t>& col,
                     std::vector<double>& val) {
  // over the loop vertices: the P1 mass matrix restricted to the interior vertices
  const int64_t nv = T.nv, nc = T.nc;
  std::vector<std::vector<std::pair<int32_t, double>>> rows(nv);
  for (int64_t c = 0; c < nc; ++c) {
    const int32_t* t = &T.tris[3 * c];
    const double* p0 = verts + 3 * t[0];
    const double* p1 = verts + 3 * t[1];
    const double* p2 = verts + 3 * t[2];
    double u[3] = {p1[0] - p0[0], p1[1] - p0[1], p1[2] - p0[2]};
    double w[3] = {p2[0] - p0[0], p2[1] - p0[1], p2[2] - p0[2]};
    double cr[3] = {u[1] * w[2] - u[2] * w[1], u[2] * w[0] - u[0] * w[2], u[0] * w[1] - u[1] * w[0]};
    double area = 0.5 * std::sqrt(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]);
    for (int i = 0; i < 3; ++i) {
      const int32_t li = T.loop_of[t[i]];
      if (li < 0) continue;
      for (int j = 0; j < 3; ++j) {
        const int32_t lj = T.loop_of[t[j]];
        if (lj >= 0) rows[li].push_back({lj, area * (i == j ? 2.0 : 1.0) / 12.0});
      }
    }
  }
  ptr.assign(nv + 1, 0);
  col.clear();
  val.clear();
  for (int64_t v = 0; v < nv; ++v) {
    auto& r = rows[v];
    std::sort(r.begin(), r.end());
    for (size_t q = 0; q < r.size();) {
      int32_t cidx = r[q].first;
      double s = 0.0;
      while (q < r.size() && r[q].first == cidx) s += r[q++].second;
      col.push_back(cidx);
      val.push_back(s);
    }
    ptr[v + 1] = (int32_t)col.size();
  }
}

void gtp_matrix_csr(const Topology& T, std::vector<int32_t>& ptr, std::vector<int32_t>& col,
                    std::vector<double>& val) {
  // (lambda~_m, p_n) by the case formula of Sec. 3:
  //   m = n:                      2/18 (9/2 + sum over the vertices v of m of 1/NoC(v))
  //   cells sharing edge (a, b):  2/18 (1/2 + 1/NoC(a) + 1/NoC(b))
  //   sharing only vertex v:      2/18 (1/NoC(v))
  // with NoC(v) the number of cells around vertex v.  (Closed surfaces: the dual functions.)
  const int64_t nv = T.nv_mesh, nc = T.nc;
  std::vector<int32_t> noc(nv, 0);
  for (int64_t i = 0; i < 3 * nc; ++i) noc[T.tris[i]]++;
  std::vector<std::vector<int32_t>> v2c(nv);
  for (int64_t c = 0; c < nc; ++c)
    for (int i = 0; i < 3; ++i) v2c[T.tris[3 * c + i]].push_back((int32_t)c);
  ptr.assign(nc + 1, 0);
  col.clear();
  val.clear();
  std::vector<int32_t> nb;
  for (int64_t m = 0; m < nc; ++m) {
    const int32_t* tm = &T.tris[3 * m];
    nb.clear();
    for (int i = 0; i < 3; ++i) nb.insert(nb.end(), v2c[tm[i]].begin(), v2c[tm[i]].end());
    std::sort(nb.begin(), nb.end());
    nb.erase(std::unique(nb.begin(), nb.end()), nb.end());
    for (int32_t n : nb) {
      const int32_t* tn = &T.tris[3 * n];
      double s = 0.0;
      int shared = 0;
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
          if (tm[i] == tn[j]) {
            ++shared;
            s += 1.0 / noc[tm[i]];
          }
      double v = 0.0;
      if (n == m) v = 2.0 / 18.0 * (4.5 + s);
      else if (shared == 2) v = 2.0 / 18.0 * (0.5 + s);
      else v = 2.0 / 18.0 * s;
      col.push_back(n);
      val.push_back(v);
    }
    ptr[m + 1] = (int32_t)col.size();
  }
}

}  // namespace rfcmp
