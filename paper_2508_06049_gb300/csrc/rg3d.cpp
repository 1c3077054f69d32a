// Host-side 3D red-green refinement of the macro mesh (Alg. 3, Sec. 3) for the kl-refinement loop
// in 3D.  Red: Bey's eight children.  Closure: every face with two split edges gets its third edge
// split; every tet with more than three split edges, a split edge whose half is split again, or a
// fully split face with a split midline is red-refined; repeat.  Green: the three irregular types
// that remain (one split edge, two opposite split edges, the three edges of one face), reverted
// before the next step.  Sequential by design, like the 2D version (the macro mesh is small).
#include <algorithm>
#include <cstring>
#include <map>
#include <new>
#include <utility>
#include <vector>

#include "../../include/hhg.h"

namespace hhg {
void set_error(const char* fmt, ...);
}

struct hhg_rg3d_s {
  struct Tet {
    int v[4];
    int parent[4];  // the green family's parent (valid when child >= 0)
    int child;      // -1: not green; else index inside its green family
    int nkids;      // size of the green family (2 or 4)
  };
  std::vector<double> xyz;                 // 3 per vertex
  std::vector<Tet> tets;
  std::map<std::pair<int, int>, int> mid;  // edge (min,max) -> midpoint vertex
};

namespace {

// slot pairs of the six edges and slot triples of the four faces (orders fix the numbering)
const int kEdge[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}};
const int kFace[4][3] = {{0, 1, 2}, {0, 1, 3}, {0, 2, 3}, {1, 2, 3}};

typedef hhg_rg3d_s::Tet Tet;

int find_mid(const hhg_rg3d_s* rg, int a, int b) {
  auto it = rg->mid.find({std::min(a, b), std::max(a, b)});
  return it == rg->mid.end() ? -1 : it->second;
}

int make_mid(hhg_rg3d_s* rg, int a, int b) {
  int m = find_mid(rg, a, b);
  if (m >= 0) return m;
  double p[3];
  for (int d = 0; d < 3; ++d) p[d] = (rg->xyz[3 * (size_t)a + d] + rg->xyz[3 * (size_t)b + d]) * 0.5;
  m = (int)(rg->xyz.size() / 3);
  rg->xyz.insert(rg->xyz.end(), p, p + 3);
  rg->mid[{std::min(a, b), std::max(a, b)}] = m;
  return m;
}

Tet plain(int a, int b, int c, int d) {
  Tet t;
  t.v[0] = a; t.v[1] = b; t.v[2] = c; t.v[3] = d;
  t.parent[0] = t.parent[1] = t.parent[2] = t.parent[3] = -1;
  t.child = -1;
  t.nkids = 0;
  return t;
}

// indices (into kEdge) of the split edges of t, in edge order
int split_edges(const hhg_rg3d_s* rg, const Tet& t, int* which) {
  int n = 0;
  for (int e = 0; e < 6; ++e)
    if (find_mid(rg, t.v[kEdge[e][0]], t.v[kEdge[e][1]]) >= 0) which[n++] = e;
  return n;
}

// nested refinement on the boundary of t: a split edge whose half is split, or a fully split face
// one of whose midlines (edges between its edge midpoints) is split
bool over_refined(const hhg_rg3d_s* rg, const Tet& t) {
  for (int e = 0; e < 6; ++e) {
    int a = t.v[kEdge[e][0]], b = t.v[kEdge[e][1]];
    int m = find_mid(rg, a, b);
    if (m >= 0 && (find_mid(rg, a, m) >= 0 || find_mid(rg, m, b) >= 0)) return true;
  }
  for (int f = 0; f < 4; ++f) {
    int a = t.v[kFace[f][0]], b = t.v[kFace[f][1]], c = t.v[kFace[f][2]];
    int ms[3] = {find_mid(rg, a, b), find_mid(rg, b, c), find_mid(rg, c, a)};
    if (ms[0] < 0 || ms[1] < 0 || ms[2] < 0) continue;
    for (int i = 0; i < 3; ++i)
      if (find_mid(rg, ms[i], ms[(i + 1) % 3]) >= 0) return true;
  }
  return false;
}

// split the third edge of every face with exactly two split edges, until none is left
void close_faces(hhg_rg3d_s* rg, const std::vector<Tet>& R) {
  bool changed = true;
  while (changed) {
    changed = false;
    for (const Tet& t : R)
      for (int f = 0; f < 4; ++f) {
        int a = t.v[kFace[f][0]], b = t.v[kFace[f][1]], c = t.v[kFace[f][2]];
        const int e[3][2] = {{a, b}, {b, c}, {a, c}};
        int have = 0, missing = -1;
        for (int q = 0; q < 3; ++q) {
          if (find_mid(rg, e[q][0], e[q][1]) >= 0) ++have;
          else missing = q;
        }
        if (have == 2) {
          make_mid(rg, e[missing][0], e[missing][1]);
          changed = true;
        }
      }
  }
}

void red_children(hhg_rg3d_s* rg, const Tet& t, std::vector<Tet>& out) {
  int x[4] = {t.v[0], t.v[1], t.v[2], t.v[3]};
  int m[6];
  for (int e = 0; e < 6; ++e) m[e] = make_mid(rg, x[kEdge[e][0]], x[kEdge[e][1]]);
  const int x01 = m[0], x02 = m[1], x03 = m[2], x12 = m[3], x13 = m[4], x23 = m[5];
  // Bey's rule; the sixth and eighth child with two slots exchanged so that all eight keep the
  // parent's orientation
  out.push_back(plain(x[0], x01, x02, x03));
  out.push_back(plain(x01, x[1], x12, x13));
  out.push_back(plain(x02, x12, x[2], x23));
  out.push_back(plain(x03, x13, x23, x[3]));
  out.push_back(plain(x01, x02, x03, x13));
  out.push_back(plain(x02, x01, x12, x13));
  out.push_back(plain(x02, x03, x13, x23));
  out.push_back(plain(x12, x02, x13, x23));
}

Tet with_slot(Tet t, int slot, int v) {
  t.v[slot] = v;
  return t;
}

// green family of t with cnt split edges (which[]); false if the pattern is not a green type
bool green_children(const hhg_rg3d_s* rg, const Tet& t, const int* which, int cnt, std::vector<Tet>& kids) {
  kids.clear();
  if (cnt == 1) {
    int i = kEdge[which[0]][0], j = kEdge[which[0]][1];
    int m = find_mid(rg, t.v[i], t.v[j]);
    kids.push_back(with_slot(t, j, m));
    kids.push_back(with_slot(t, i, m));
    return true;
  }
  if (cnt == 2) {
    int i = kEdge[which[0]][0], j = kEdge[which[0]][1];
    int k = kEdge[which[1]][0], l = kEdge[which[1]][1];
    if (i == k || i == l || j == k || j == l) return false;  // not opposite edges
    int m1 = find_mid(rg, t.v[i], t.v[j]);
    int m2 = find_mid(rg, t.v[k], t.v[l]);
    const Tet halves[2] = {with_slot(t, j, m1), with_slot(t, i, m1)};
    for (const Tet& h : halves) {
      kids.push_back(with_slot(h, l, m2));
      kids.push_back(with_slot(h, k, m2));
    }
    return true;
  }
  if (cnt == 3) {
    for (int f = 0; f < 4; ++f) {
      int a = kFace[f][0], b = kFace[f][1], c = kFace[f][2];
      // the face's edges as indices into kEdge (a < b < c)
      int eab = -1, ebc = -1, eac = -1;
      for (int e = 0; e < 6; ++e) {
        if (kEdge[e][0] == a && kEdge[e][1] == b) eab = e;
        if (kEdge[e][0] == b && kEdge[e][1] == c) ebc = e;
        if (kEdge[e][0] == a && kEdge[e][1] == c) eac = e;
      }
      int s[3] = {eab, ebc, eac};
      std::sort(s, s + 3);
      if (s[0] != which[0] || s[1] != which[1] || s[2] != which[2]) continue;
      int mab = find_mid(rg, t.v[a], t.v[b]);
      int mbc = find_mid(rg, t.v[b], t.v[c]);
      int mca = find_mid(rg, t.v[c], t.v[a]);
      kids.push_back(with_slot(with_slot(t, b, mab), c, mca));
      kids.push_back(with_slot(with_slot(t, a, mab), c, mbc));
      kids.push_back(with_slot(with_slot(t, a, mca), b, mbc));
      kids.push_back(with_slot(with_slot(with_slot(t, a, mbc), b, mca), c, mab));
      return true;
    }
  }
  return false;
}

}  // namespace

extern "C" {

hhg_status hhg_rg3d_create(int n_verts, const double* coords, int n_cells, const int* cells, hhg_rg3d* out) {
  if (!out || !coords || !cells || n_verts < 4 || n_cells < 1) {
    hhg::set_error("hhg_rg3d_create: invalid arguments");
    return HHG_ERR_ARG;
  }
  *out = nullptr;
  hhg_rg3d_s* rg = new (std::nothrow) hhg_rg3d_s();
  if (!rg) {
    hhg::set_error("host allocation failed");
    return HHG_ERR_OOM;
  }
  rg->xyz.assign(coords, coords + 3 * (size_t)n_verts);
  rg->tets.reserve(n_cells);
  for (int c = 0; c < n_cells; ++c) {
    int v[4];
    for (int a = 0; a < 4; ++a) {
      v[a] = cells[4 * (size_t)c + a];
      if (v[a] < 0 || v[a] >= n_verts) {
        delete rg;
        hhg::set_error("hhg_rg3d_create: cell %d references vertex %d", c, v[a]);
        return HHG_ERR_ARG;
      }
    }
    // a cell must span a tetrahedron: four distinct vertices, nonzero volume
    const double* p0 = &coords[3 * (size_t)v[0]];
    double e[3][3];
    for (int a = 0; a < 3; ++a)
      for (int r = 0; r < 3; ++r) e[a][r] = coords[3 * (size_t)v[a + 1] + r] - p0[r];
    const double det = e[0][0] * (e[1][1] * e[2][2] - e[1][2] * e[2][1]) -
                       e[0][1] * (e[1][0] * e[2][2] - e[1][2] * e[2][0]) +
                       e[0][2] * (e[1][0] * e[2][1] - e[1][1] * e[2][0]);
    bool repeated = false;
    for (int a = 0; a < 4; ++a)
      for (int b = a + 1; b < 4; ++b) repeated |= v[a] == v[b];
    if (repeated || det == 0.0) {
      delete rg;
      hhg::set_error("hhg_rg3d_create: cell %d is degenerate", c);
      return HHG_ERR_MESH;
    }
    rg->tets.push_back(plain(v[0], v[1], v[2], v[3]));
  }
  *out = rg;
  return HHG_OK;
}

hhg_status hhg_rg3d_destroy(hhg_rg3d rg) {
  delete rg;
  return HHG_OK;
}

hhg_status hhg_rg3d_mesh(hhg_rg3d rg, int* n_verts, double* coords, int* n_cells, int* cells) {
  if (!rg || !n_verts || !n_cells) {
    hhg::set_error("hhg_rg3d_mesh: invalid arguments");
    return HHG_ERR_ARG;
  }
  *n_verts = (int)(rg->xyz.size() / 3);
  *n_cells = (int)rg->tets.size();
  if (coords) memcpy(coords, rg->xyz.data(), rg->xyz.size() * sizeof(double));
  if (cells)
    for (size_t c = 0; c < rg->tets.size(); ++c)
      for (int a = 0; a < 4; ++a) cells[4 * c + a] = rg->tets[c].v[a];
  return HHG_OK;
}

hhg_status hhg_rg3d_refine(hhg_rg3d rg, const unsigned char* marked) {
  if (!rg || !marked) {
    hhg::set_error("hhg_rg3d_refine: invalid arguments");
    return HHG_ERR_ARG;
  }
  // 1. revert green families to their parents; a marked green child marks the parent
  std::vector<Tet> R;
  std::vector<char> flag;
  for (size_t i = 0; i < rg->tets.size();) {
    const Tet& t = rg->tets[i];
    if (t.child >= 0) {
      const size_t n = (size_t)t.nkids;
      bool ok = t.child == 0 && n >= 2 && i + n <= rg->tets.size();
      for (size_t q = 0; ok && q < n; ++q) {
        const Tet& k = rg->tets[i + q];
        ok = k.child == (int)q && k.nkids == t.nkids && memcmp(k.parent, t.parent, sizeof(t.parent)) == 0;
      }
      if (!ok) {
        hhg::set_error("hhg_rg3d_refine: corrupt green family at cell %zu", i);
        return HHG_ERR_STATE;
      }
      bool any = false;
      for (size_t q = 0; q < n; ++q) any |= marked[i + q] != 0;
      R.push_back(plain(t.parent[0], t.parent[1], t.parent[2], t.parent[3]));
      flag.push_back(any ? 1 : 0);
      i += n;
    } else {
      R.push_back(t);
      flag.push_back(marked[i] ? 1 : 0);
      i += 1;
    }
  }
  // 2. red refinement and closure
  for (;;) {
    std::vector<Tet> next;
    next.reserve(R.size() * 2);
    for (size_t q = 0; q < R.size(); ++q) {
      if (flag[q]) red_children(rg, R[q], next);
      else next.push_back(R[q]);
    }
    R.swap(next);
    close_faces(rg, R);
    bool any = false;
    flag.assign(R.size(), 0);
    for (size_t q = 0; q < R.size(); ++q) {
      int which[6];
      int cnt = split_edges(rg, R[q], which);
      flag[q] = (cnt > 3 || over_refined(rg, R[q])) ? 1 : 0;
      any |= flag[q] != 0;
    }
    if (!any) break;
  }
  // 3. green closure
  std::vector<Tet> out, kids;
  out.reserve(R.size() * 2);
  for (const Tet& t : R) {
    int which[6];
    int cnt = split_edges(rg, t, which);
    if (cnt == 0) {
      out.push_back(t);
      continue;
    }
    if (!green_children(rg, t, which, cnt, kids)) {
      hhg::set_error("hhg_rg3d_refine: split pattern of a tet is not a green type (internal)");
      return HHG_ERR_STATE;
    }
    for (size_t q = 0; q < kids.size(); ++q) {
      Tet k = kids[q];
      memcpy(k.parent, t.v, sizeof(t.v));
      k.child = (int)q;
      k.nkids = (int)kids.size();
      out.push_back(k);
    }
  }
  rg->tets.swap(out);
  return HHG_OK;
}

hhg_status hhg_rg3d_mark_refine(hhg_rg3d rg, const double* eta_T, double fraction, unsigned char* marked) {
  if (!rg || !eta_T) {
    hhg::set_error("hhg_rg3d_mark_refine: invalid arguments");
    return HHG_ERR_ARG;
  }
  int n = (int)rg->tets.size();
  std::vector<unsigned char> mk(n);
  hhg_status st = hhg_mark(n, eta_T, fraction, mk.data(), nullptr);
  if (st != HHG_OK) return st;
  if (marked) memcpy(marked, mk.data(), n);
  return hhg_rg3d_refine(rg, mk.data());
}

}  // extern "C"
