// Host-side kl-refinement helpers: top-fraction marking (Sec. 5.1) and 2D red-green refinement of
// the macro mesh with green closures reverted before each step (Sec. 3).  Sequential by design:
// the macro mesh is small (Sec. 3 argues the refinement need not be parallel).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <new>
#include <numeric>
#include <utility>
#include <vector>

#include "../../include/hhg.h"

namespace hhg {
void set_error(const char* fmt, ...);
}

struct hhg_rg2d_s {
  struct Tri {
    int v[3];
    int parent[3];
    int child;  // -1: not a green child; 0/1: first/second child of a green bisection
  };
  std::vector<double> xy;                 // 2 per vertex
  std::vector<Tri> tris;
  std::map<std::pair<int, int>, int> mid;  // edge (min,max) -> midpoint vertex
};

namespace {

int find_mid(hhg_rg2d_s* rg, int a, int b) {
  auto it = rg->mid.find({std::min(a, b), std::max(a, b)});
  return it == rg->mid.end() ? -1 : it->second;
}

int make_mid(hhg_rg2d_s* rg, int a, int b) {
  int m = find_mid(rg, a, b);
  if (m >= 0) return m;
  double x = (rg->xy[2 * a] + rg->xy[2 * b]) * 0.5;
  double y = (rg->xy[2 * a + 1] + rg->xy[2 * b + 1]) * 0.5;
  m = (int)(rg->xy.size() / 2);
  rg->xy.push_back(x);
  rg->xy.push_back(y);
  rg->mid[{std::min(a, b), std::max(a, b)}] = m;
  return m;
}

// split edges of a triangle (edge e = (v[e], v[e+1])); `over` = a split edge whose half is split
int split_edges(hhg_rg2d_s* rg, const int v[3], int* which, bool* over) {
  int cnt = 0;
  *over = false;
  for (int e = 0; e < 3; ++e) {
    int a = v[e], b = v[(e + 1) % 3];
    int m = find_mid(rg, a, b);
    if (m < 0) continue;
    which[cnt++] = e;
    if (find_mid(rg, a, m) >= 0 || find_mid(rg, m, b) >= 0) *over = true;
  }
  return cnt;
}

}  // namespace

extern "C" {

hhg_status hhg_mark(int n, const double* eta, double fraction, unsigned char* marked, int* n_marked) {
  if (n < 0 || (n > 0 && (!eta || !marked))) {
    hhg::set_error("hhg_mark: invalid arguments");
    return HHG_ERR_ARG;
  }
  if (!(fraction > 0.0 && fraction <= 1.0)) {
    hhg::set_error("hhg_mark: fraction must be in (0, 1]");
    return HHG_ERR_ARG;
  }
  for (int i = 0; i < n; ++i)
    if (!std::isfinite(eta[i])) {
      hhg::set_error("hhg_mark: eta[%d] is not finite", i);
      return HHG_ERR_ARG;
    }
  if (n_marked) *n_marked = 0;
  if (n == 0) return HHG_OK;
  long cnt = (long)std::ceil(fraction * n - 1e-9);
  cnt = std::max(1L, std::min((long)n, cnt));
  std::vector<int> order(n);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return eta[a] > eta[b]; });
  double star = eta[order[cnt - 1]];
  int tot = 0;
  for (int i = 0; i < n; ++i) {
    marked[i] = eta[i] >= (1.0 - 1e-8) * star ? 1 : 0;
    tot += marked[i];
  }
  if (n_marked) *n_marked = tot;
  return HHG_OK;
}

hhg_status hhg_rg2d_create(int n_verts, const double* coords, int n_cells, const int* cells, hhg_rg2d* out) {
  if (!out || !coords || !cells || n_verts < 3 || n_cells < 1) {
    hhg::set_error("hhg_rg2d_create: invalid arguments");
    return HHG_ERR_ARG;
  }
  *out = nullptr;
  hhg_rg2d_s* rg = new (std::nothrow) hhg_rg2d_s();
  if (!rg) {
    hhg::set_error("host allocation failed");
    return HHG_ERR_OOM;
  }
  rg->xy.assign(coords, coords + 2 * (size_t)n_verts);
  rg->tris.resize(n_cells);
  for (int c = 0; c < n_cells; ++c) {
    for (int a = 0; a < 3; ++a) {
      int v = cells[3 * c + a];
      if (v < 0 || v >= n_verts) {
        delete rg;
        hhg::set_error("hhg_rg2d_create: cell %d references vertex %d", c, v);
        return HHG_ERR_ARG;
      }
      rg->tris[c].v[a] = v;
      rg->tris[c].parent[a] = -1;
    }
    rg->tris[c].child = -1;
    // a cell must span a triangle: three distinct vertices, nonzero area
    const int* v = rg->tris[c].v;
    const double* p0 = &coords[2 * (size_t)v[0]];
    const double* p1 = &coords[2 * (size_t)v[1]];
    const double* p2 = &coords[2 * (size_t)v[2]];
    const double det = (p1[0] - p0[0]) * (p2[1] - p0[1]) - (p1[1] - p0[1]) * (p2[0] - p0[0]);
    if (v[0] == v[1] || v[0] == v[2] || v[1] == v[2] || det == 0.0) {
      delete rg;
      hhg::set_error("hhg_rg2d_create: cell %d is degenerate", c);
      return HHG_ERR_MESH;
    }
  }
  *out = rg;
  return HHG_OK;
}

hhg_status hhg_rg2d_destroy(hhg_rg2d rg) {
  delete rg;
  return HHG_OK;
}

hhg_status hhg_rg2d_mesh(hhg_rg2d rg, int* n_verts, double* coords, int* n_cells, int* cells) {
  if (!rg || !n_verts || !n_cells) {
    hhg::set_error("hhg_rg2d_mesh: invalid arguments");
    return HHG_ERR_ARG;
  }
  *n_verts = (int)(rg->xy.size() / 2);
  *n_cells = (int)rg->tris.size();
  if (coords) memcpy(coords, rg->xy.data(), rg->xy.size() * sizeof(double));
  if (cells)
    for (size_t c = 0; c < rg->tris.size(); ++c)
      for (int a = 0; a < 3; ++a) cells[3 * c + a] = rg->tris[c].v[a];
  return HHG_OK;
}

hhg_status hhg_rg2d_refine(hhg_rg2d rg, const unsigned char* marked) {
  if (!rg || !marked) {
    hhg::set_error("hhg_rg2d_refine: invalid arguments");
    return HHG_ERR_ARG;
  }
  typedef hhg_rg2d_s::Tri Tri;
  // 1. revert green pairs to their parents; a marked green child marks the parent
  std::vector<Tri> R;
  std::vector<char> flag;
  for (size_t i = 0; i < rg->tris.size();) {
    const Tri& t = rg->tris[i];
    if (t.child >= 0) {
      if (t.child != 0 || i + 1 >= rg->tris.size() || rg->tris[i + 1].child != 1 ||
          memcmp(rg->tris[i + 1].parent, t.parent, sizeof(t.parent)) != 0) {
        hhg::set_error("hhg_rg2d_refine: corrupt green pair at cell %zu", i);
        return HHG_ERR_STATE;
      }
      Tri p;
      memcpy(p.v, t.parent, sizeof(p.v));
      p.parent[0] = p.parent[1] = p.parent[2] = -1;
      p.child = -1;
      R.push_back(p);
      flag.push_back(marked[i] || marked[i + 1]);
      i += 2;
    } else {
      R.push_back(t);
      flag.push_back(marked[i] ? 1 : 0);
      i += 1;
    }
  }
  // 2. red refinement of the flagged triangles, then closure until no triangle has two or more
  //    split edges or a split edge whose half is split again
  for (;;) {
    bool any = false;
    for (char f : flag) any |= (f != 0);
    if (!any) break;
    std::vector<Tri> next;
    next.reserve(R.size() + 3 * R.size() / 4);
    for (size_t q = 0; q < R.size(); ++q) {
      if (!flag[q]) {
        next.push_back(R[q]);
        continue;
      }
      int v0 = R[q].v[0], v1 = R[q].v[1], v2 = R[q].v[2];
      int m01 = make_mid(rg, v0, v1);
      int m12 = make_mid(rg, v1, v2);
      int m20 = make_mid(rg, v2, v0);
      const int kids[4][3] = {{v0, m01, m20}, {m01, v1, m12}, {m20, m12, v2}, {m12, m20, m01}};
      for (auto& k : kids) {
        Tri c;
        memcpy(c.v, k, sizeof(c.v));
        c.parent[0] = c.parent[1] = c.parent[2] = -1;
        c.child = -1;
        next.push_back(c);
      }
    }
    R.swap(next);
    flag.assign(R.size(), 0);
    for (size_t q = 0; q < R.size(); ++q) {
      int which[3];
      bool over;
      int cnt = split_edges(rg, R[q].v, which, &over);
      flag[q] = (cnt >= 2 || over) ? 1 : 0;
    }
  }
  // 3. green closure: bisect triangles with one split edge from the opposite vertex
  std::vector<Tri> out;
  out.reserve(R.size() + R.size() / 4);
  for (const Tri& t : R) {
    int which[3];
    bool over;
    int cnt = split_edges(rg, t.v, which, &over);
    if (cnt == 1) {
      int e = which[0];
      int a = t.v[(e + 2) % 3], b = t.v[e], c = t.v[(e + 1) % 3];
      int m = find_mid(rg, b, c);
      Tri g0, g1;
      g0.v[0] = a; g0.v[1] = b; g0.v[2] = m;
      g1.v[0] = a; g1.v[1] = m; g1.v[2] = c;
      memcpy(g0.parent, t.v, sizeof(t.v));
      memcpy(g1.parent, t.v, sizeof(t.v));
      g0.child = 0;
      g1.child = 1;
      out.push_back(g0);
      out.push_back(g1);
    } else {
      out.push_back(t);
    }
  }
  rg->tris.swap(out);
  return HHG_OK;
}

hhg_status hhg_mark_refine(hhg_rg2d rg, const double* eta_T, double fraction, unsigned char* marked) {
  if (!rg || !eta_T) {
    hhg::set_error("hhg_mark_refine: invalid arguments");
    return HHG_ERR_ARG;
  }
  int n = (int)rg->tris.size();
  std::vector<unsigned char> mk(n);
  hhg_status st = hhg_mark(n, eta_T, fraction, mk.data(), nullptr);
  if (st != HHG_OK) return st;
  if (marked) memcpy(marked, mk.data(), n);
  return hhg_rg2d_refine(rg, mk.data());
}

}  // extern "C"
