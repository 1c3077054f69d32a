// Host-side construction of an HHG mesh object: coarse topology (the macro primitives of Sec. 2),
// per-cell partial stencils of the P1 discretisation of Eq. 5.1 (the constant stencils of one
// uniformly refined macro element, Sec. 2), interface descriptors, interior colourings (the
// Gauss-Seidel stages of Alg. 4), the direct coarse solve of Alg. 4 and the level tables.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <array>
#include <map>

#include "internal.h"

namespace hhg {

static thread_local char g_err[1024] = "";

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

const char* last_error() { return g_err; }

hhg_status cuda_fail(cudaError_t e, const char* what) {
  set_error("CUDA error in %s: %s", what, cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? HHG_ERR_OOM : HHG_ERR_CUDA;
}

#define CK(call)                                              \
  do {                                                        \
    cudaError_t e_ = (call);                                  \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call);       \
  } while (0)

template <typename T>
static hhg_status dalloc(hhg_mesh_s* m, T** p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  cudaError_t e = cudaMalloc((void**)p, count * sizeof(T));
  if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc");
  // every device buffer starts initialised (zero), so no kernel ever reads untouched memory
  e = cudaMemset(*p, 0, count * sizeof(T));
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemset");
  m->bytes += (long long)(count * sizeof(T));
  return HHG_OK;
}

template <typename T>
static hhg_status upload(hhg_mesh_s* m, T** p, const std::vector<T>& v) {
  hhg_status st = dalloc(m, p, v.size());
  if (st != HHG_OK) return st;
  if (!v.empty()) CK(cudaMemcpy(*p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
  return HHG_OK;
}

// ---------------------------------------------------------------- micro elements
// Micro elements of the (infinite) lattice that contain lattice point p, as integer vertex lists.
// 2D: in y = (i, i+j) every unit square splits along (1,1); 3D: Kuhn tets of the y-cube lattice,
// y = (i, i+j, i+j+k).  Both equal red refinement / Bey's rule of the macro element.
static void elements_at(int dim, const int p[3], std::vector<std::array<std::array<int, 3>, 4>>& out) {
  out.clear();
  int y[3] = {p[0], p[0] + p[1], dim == 3 ? p[0] + p[1] + p[2] : 0};
  auto to_e = [&](const int yy[3], std::array<int, 3>& e) {
    e[0] = yy[0];
    e[1] = yy[1] - yy[0];
    e[2] = dim == 3 ? yy[2] - yy[1] : 0;
  };
  if (dim == 2) {
    for (int c0 = y[0] - 1; c0 <= y[0]; ++c0)
      for (int c1 = y[1] - 1; c1 <= y[1]; ++c1)
        for (int tri = 0; tri < 2; ++tri) {
          int v[3][3] = {{c0, c1, 0}, {c0 + (tri == 0), c1 + (tri == 1), 0}, {c0 + 1, c1 + 1, 0}};
          bool has = false;
          for (int a = 0; a < 3; ++a) has |= (v[a][0] == y[0] && v[a][1] == y[1]);
          if (!has) continue;
          std::array<std::array<int, 3>, 4> el{};
          for (int a = 0; a < 3; ++a) to_e(v[a], el[a]);
          out.push_back(el);
        }
    return;
  }
  static const int perms[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
  for (int c0 = y[0] - 1; c0 <= y[0]; ++c0)
    for (int c1 = y[1] - 1; c1 <= y[1]; ++c1)
      for (int c2 = y[2] - 1; c2 <= y[2]; ++c2)
        for (int s = 0; s < 6; ++s) {
          int v[4][3];
          int cur[3] = {c0, c1, c2};
          for (int a = 0; a < 3; ++a) v[0][a] = cur[a];
          for (int q = 0; q < 3; ++q) {
            cur[perms[s][q]] += 1;
            for (int a = 0; a < 3; ++a) v[q + 1][a] = cur[a];
          }
          bool has = false;
          for (int a = 0; a < 4; ++a) has |= (v[a][0] == y[0] && v[a][1] == y[1] && v[a][2] == y[2]);
          if (!has) continue;
          std::array<std::array<int, 3>, 4> el{};
          for (int a = 0; a < 4; ++a) to_e(v[a], el[a]);
          out.push_back(el);
        }
}

static int slot_of(int dim, int di, int dj, int dk) {
  int nd = dim == 2 ? 7 : 15;
  for (int s = 0; s < nd; ++s) {
    int a, b, c;
    dir_vec(dim, s, a, b, c);
    if (a == di && b == dj && c == dk) return s;
  }
  return -1;
}

// P1 element matrices of a simplex with vertices X[a] (dim coordinates each).
static bool element_matrices(int dim, const double X[4][3], double K[4][4], double M[4][4]) {
  int d = dim;
  double J[3][3] = {{0}};
  for (int r = 0; r < d; ++r)
    for (int c = 0; c < d; ++c) J[r][c] = X[c + 1][r] - X[0][r];
  double det, inv[3][3];
  if (d == 2) {
    det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
    if (det == 0) return false;
    inv[0][0] = J[1][1] / det; inv[0][1] = -J[0][1] / det;
    inv[1][0] = -J[1][0] / det; inv[1][1] = J[0][0] / det;
  } else {
    det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) - J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
          J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
    if (det == 0) return false;
    inv[0][0] = (J[1][1] * J[2][2] - J[1][2] * J[2][1]) / det;
    inv[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / det;
    inv[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / det;
    inv[1][0] = (J[1][2] * J[2][0] - J[1][0] * J[2][2]) / det;
    inv[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / det;
    inv[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / det;
    inv[2][0] = (J[1][0] * J[2][1] - J[1][1] * J[2][0]) / det;
    inv[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / det;
    inv[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / det;
  }
  double vol = std::fabs(det) / (d == 2 ? 2.0 : 6.0);
  // gradients of the barycentric coordinates: rows of inv for a = 1..d, grad_0 = -sum
  double G[4][3] = {{0}};
  for (int a = 1; a <= d; ++a)
    for (int c = 0; c < d; ++c) G[a][c] = inv[a - 1][c];
  for (int c = 0; c < d; ++c) G[0][c] = -(G[1][c] + G[2][c] + (d == 3 ? G[3][c] : 0.0));
  for (int a = 0; a <= d; ++a)
    for (int b = 0; b <= d; ++b) {
      double s = 0;
      for (int c = 0; c < d; ++c) s += G[a][c] * G[b][c];
      K[a][b] = vol * s;
      M[a][b] = vol * (a == b ? 2.0 : 1.0) / ((d + 1) * (d + 2));
    }
  return true;
}

// Partial stencils of one macro cell for every boundary type: sum of the element matrices of the
// micro elements inside the cell that contain the node, at unit level scale (level 0 lattice).
static bool cell_stencils(int dim, const double* x0, const double J[3][3], double* S, double* Mst) {
  const int nrep = 6;
  std::fill(S, S + kMaxTypes * kMaxDirs, 0.0);
  std::fill(Mst, Mst + kMaxTypes * kMaxDirs, 0.0);
  std::vector<std::array<std::array<int, 3>, 4>> els;
  // representative lattice points: scan a side-6 lattice, first point of each type
  std::vector<bool> seen(kMaxTypes, false);
  for (int k = 0; k <= (dim == 3 ? nrep : 0); ++k)
    for (int j = 0; j <= nrep - k; ++j)
      for (int i = 0; i <= nrep - k - j; ++i) {
        int t = boundary_type(dim, nrep, i, j, k);
        if (seen[t]) continue;
        // prefer points away from other facets: require one step of slack to the facets not in t
        bool ok = true;
        if (!(t & 1) && i < 1) ok = false;
        if (!(t & 2) && j < 1) ok = false;
        if (dim == 2) {
          if (!(t & 4) && i + j > nrep - 1) ok = false;
        } else {
          if (!(t & 4) && k < 1) ok = false;
          if (!(t & 8) && i + j + k > nrep - 1) ok = false;
        }
        if (!ok) continue;
        seen[t] = true;
        int p[3] = {i, j, k};
        elements_at(dim, p, els);
        for (auto& el : els) {
          bool inside = true;
          for (int a = 0; a <= dim; ++a) {
            int s = el[a][0] + el[a][1] + el[a][2];
            if (el[a][0] < 0 || el[a][1] < 0 || el[a][2] < 0 || s > nrep) inside = false;
          }
          if (!inside) continue;
          double X[4][3] = {{0}};
          for (int a = 0; a <= dim; ++a)
            for (int r = 0; r < dim; ++r) {
              double v = 0;
              for (int c = 0; c < dim; ++c) v += J[r][c] * el[a][c];
              X[a][r] = v;  // translation by x0 does not change the element matrices
            }
          double K[4][4], Mm[4][4];
          if (!element_matrices(dim, X, K, Mm)) return false;
          int alpha = -1;
          for (int a = 0; a <= dim; ++a)
            if (el[a][0] == i && el[a][1] == j && el[a][2] == k) alpha = a;
          for (int b = 0; b <= dim; ++b) {
            int s = slot_of(dim, el[b][0] - i, el[b][1] - j, el[b][2] - k);
            if (s < 0) return false;
            S[t * kMaxDirs + s] += K[alpha][b];
            Mst[t * kMaxDirs + s] += Mm[alpha][b];
          }
        }
      }
  (void)x0;
  return true;
}

// ---------------------------------------------------------------- coarse dense Cholesky
static bool cholesky_inverse(int n, std::vector<double>& A) {
  // A (n x n, row-major, SPD) -> A^{-1} via L L^T
  std::vector<double> Lm(A);
  for (int j = 0; j < n; ++j) {
    double s = Lm[(size_t)j * n + j];
    for (int k = 0; k < j; ++k) s -= Lm[(size_t)j * n + k] * Lm[(size_t)j * n + k];
    if (!(s > 0)) return false;
    double d = std::sqrt(s);
    Lm[(size_t)j * n + j] = d;
    for (int i = j + 1; i < n; ++i) {
      double t = Lm[(size_t)i * n + j];
      for (int k = 0; k < j; ++k) t -= Lm[(size_t)i * n + k] * Lm[(size_t)j * n + k];
      Lm[(size_t)i * n + j] = t / d;
    }
  }
  // inverse column by column: solve L y = e_c, L^T x = y
  std::vector<double> y(n), x(n);
  for (int c = 0; c < n; ++c) {
    for (int i = 0; i < n; ++i) {
      double t = (i == c) ? 1.0 : 0.0;
      for (int k = 0; k < i; ++k) t -= Lm[(size_t)i * n + k] * y[k];
      y[i] = t / Lm[(size_t)i * n + i];
    }
    for (int i = n - 1; i >= 0; --i) {
      double t = y[i];
      for (int k = i + 1; k < n; ++k) t -= Lm[(size_t)k * n + i] * x[k];
      x[i] = t / Lm[(size_t)i * n + i];
    }
    for (int i = 0; i < n; ++i) A[(size_t)i * n + c] = x[i];
  }
  return true;
}

// local vertex sets of the boundary types: type -> (number of vertices, local vertex ids)
static void type_primitive(int dim, int t, int& nv, int a[3]) {
  nv = 0;
  for (int v = 0; v <= dim; ++v) {
    // vertex v lies on facet bit b unless the facet is opposite to it
    // 2D facets: bit0 i==0 (opposite v1), bit1 j==0 (opposite v2), bit2 i+j==n (opposite v0)
    // 3D facets: bit0 i==0 (opp v1), bit1 j==0 (opp v2), bit2 k==0 (opp v3), bit3 sum==n (opp v0)
    bool on_all = true;
    for (int b = 0; b <= dim; ++b) {
      if (!(t >> b & 1)) continue;
      int opp = (b == dim) ? 0 : b + 1;
      if (v == opp) on_all = false;
    }
    if (on_all) a[nv++] = v;
  }
}

// Boundary type, in its cell, of the interior nodes of a primitive with nverts local vertices packed
// in loc (a0 | a1 << 2 | a2 << 4): the node n E_a0 + s (E_a1 - E_a0) + t (E_a2 - E_a0) with n = 4,
// s = t = 1 (s = t = 0 for a vertex) lies inside the primitive.
static int prim_interior_type(int dim, int nverts, int loc) {
  const int n = 4;
  int a[3] = {loc & 3, (loc >> 2) & 3, (loc >> 4) & 3};
  int e[3][3];
  for (int q = 0; q < 3; ++q) {
    e[q][0] = a[q] == 1;
    e[q][1] = a[q] == 2;
    e[q][2] = a[q] == 3;
  }
  int x[3];
  for (int c = 0; c < 3; ++c) {
    x[c] = n * e[0][c];
    if (nverts >= 2) x[c] += e[1][c] - e[0][c];
    if (nverts >= 3) x[c] += e[2][c] - e[0][c];
  }
  return boundary_type(dim, n, x[0], x[1], x[2]);
}

hhg_status upload_coefficient(hhg_mesh_s* m) {
  const int NS = kMaxTypes * kMaxDirs;
  std::vector<double> S((size_t)m->nc * NS);
  std::vector<float> S32((size_t)m->nc * NS), M32((size_t)m->nc * NS);
  for (int c = 0; c < m->nc; ++c)
    for (int q = 0; q < NS; ++q) {
      S[(size_t)c * NS + q] = m->k[c] * m->hS1[(size_t)c * NS + q];
      M32[(size_t)c * NS + q] = (float)m->hM[(size_t)c * NS + q];
    }
  // Couplings below 1e-12 of the largest off-diagonal entry of a partial stencil are rounding
  // residue of exact zeros (the same threshold decides the interior zero pattern and colouring):
  // they are set to zero, and the kernels skip the zero slots (nzs mask, centre always kept).
  std::vector<uint16_t> nzs((size_t)m->nc * kMaxTypes, 0);
  for (int c = 0; c < m->nc; ++c)
    for (int t = 0; t < kMaxTypes; ++t) {
      double* st = &S[(size_t)c * NS + t * kMaxDirs];
      double vmax = 0;
      for (int q = 1; q < kMaxDirs; ++q) vmax = std::max(vmax, std::fabs(st[q]));
      uint16_t mk = 1;
      for (int q = 1; q < kMaxDirs; ++q) {
        if (std::fabs(st[q]) <= 1e-12 * vmax) st[q] = 0.0;
        if (st[q] != 0.0) mk |= (uint16_t)(1u << q);
      }
      nzs[(size_t)c * kMaxTypes + t] = mk;
    }
  for (size_t q = 0; q < S.size(); ++q) S32[q] = (float)S[q];
  CK(cudaMemcpy(m->d_nzs, nzs.data(), nzs.size() * sizeof(uint16_t), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(m->dS, S.data(), S.size() * sizeof(double), cudaMemcpyHostToDevice));
  {
    std::vector<double> inv(m->nc), tn((size_t)m->nc * 16, 0.0);
    std::vector<float> invf(m->nc), tnf((size_t)m->nc * 16, 0.0f);
    for (int c = 0; c < m->nc; ++c) {
      const double* s0 = &S[(size_t)c * NS];  // interior type 0
      inv[c] = 1.0 / s0[0];
      invf[c] = (float)inv[c];
      for (int d = 0; d < kMaxDirs; ++d) {
        tn[(size_t)c * 16 + d] = s0[d] / s0[0];
        tnf[(size_t)c * 16 + d] = (float)tn[(size_t)c * 16 + d];
      }
    }
    CK(cudaMemcpy(m->d_inv0, inv.data(), inv.size() * sizeof(double), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(m->d_inv0f, invf.data(), invf.size() * sizeof(float), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(m->d_tnorm, tn.data(), tn.size() * sizeof(double), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(m->d_tnormf, tnf.data(), tnf.size() * sizeof(float), cudaMemcpyHostToDevice));
    // per level: 1 / (sscale_l * a_ii) = inv0 / sscale_l (power-of-two scale: exact)
    for (auto& Lv : m->lv) {
      double isc = m->dim == 2 ? 1.0 : (double)Lv.n;
      std::vector<double> il(m->nc);
      std::vector<float> ilf(m->nc);
      for (int c = 0; c < m->nc; ++c) {
        il[c] = inv[c] * isc;
        ilf[c] = (float)il[c];
      }
      CK(cudaMemcpy(Lv.d_invl, il.data(), il.size() * sizeof(double), cudaMemcpyHostToDevice));
      CK(cudaMemcpy(Lv.d_invlf, ilf.data(), ilf.size() * sizeof(float), cudaMemcpyHostToDevice));
    }
  }
  CK(cudaMemcpy(m->dS32, S32.data(), S32.size() * sizeof(float), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(m->dM32, M32.data(), M32.size() * sizeof(float), cudaMemcpyHostToDevice));
  {
    // hi = the binary32 rounding of the entry, lo = the binary32 rounding of the rest
    std::vector<float2> Sp(S.size());
    for (size_t q = 0; q < S.size(); ++q) {
      const float h = (float)S[q];
      Sp[q] = make_float2(h, (float)(S[q] - (double)h));
    }
    CK(cudaMemcpy(m->dSp, Sp.data(), Sp.size() * sizeof(float2), cudaMemcpyHostToDevice));
  }
  // inverse assembled diagonal of each primitive's interior nodes: the sum over its cell copies of
  // the centre entry of the copy's partial stencil (the copy's boundary type is the same for all
  // interior nodes of the primitive)
  for (int kind = 0; kind < 3; ++kind) {
    Prims& P = kind == 0 ? m->verts : (kind == 1 ? m->edges : m->faces);
    if (P.count == 0) continue;
    std::vector<double> pv(P.count, 0.0);
    std::vector<float> pf(P.count, 0.0f);
    for (int e = 0; e < P.count; ++e) {
      if (P.dir[e]) continue;
      double dsum = 0;
      for (int c = P.ptr[e]; c < P.ptr[e + 1]; ++c) {
        int t = prim_interior_type(m->dim, kind + 1, P.loc[c]);
        dsum += S[(size_t)P.cell[c] * NS + t * kMaxDirs];
      }
      pv[e] = 1.0 / dsum;
      pf[e] = (float)pv[e];
    }
    CK(cudaMemcpy(P.d_pinv, pv.data(), pv.size() * sizeof(double), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(P.d_pinvf, pf.data(), pf.size() * sizeof(float), cudaMemcpyHostToDevice));
  }
  // in-plane couplings of each macro face (face block of the smoother): for the six face-lattice
  // directions (+a, -a, +b, -b, +a-b, -a+b) the stencil entries of the matching cell directions,
  // summed over the face's copies (unit level scale)
  if (m->dim == 3 && m->faces.count) {
    Prims& P = m->faces;
    std::vector<double> fw((size_t)P.count * 8, 0.0);
    std::vector<float> fwf((size_t)P.count * 8, 0.0f);
    static const int fda[6] = {1, -1, 0, 0, 1, -1}, fdb[6] = {0, 0, 1, -1, -1, 1};
    for (int e = 0; e < P.count; ++e) {
      if (P.dir[e]) continue;
      for (int c = P.ptr[e]; c < P.ptr[e + 1]; ++c) {
        int loc = P.loc[c];
        int t = prim_interior_type(3, 3, loc);
        int v[3][3];
        for (int q = 0; q < 3; ++q) {
          int a = (loc >> (2 * q)) & 3;
          v[q][0] = a == 1;
          v[q][1] = a == 2;
          v[q][2] = a == 3;
        }
        for (int q = 0; q < 6; ++q) {
          int dv[3];
          for (int x = 0; x < 3; ++x) dv[x] = fda[q] * (v[1][x] - v[0][x]) + fdb[q] * (v[2][x] - v[0][x]);
          int sl = slot_of(3, dv[0], dv[1], dv[2]);
          if (sl <= 0) {
            set_error("face direction is not a lattice direction (internal)");
            return HHG_ERR_MESH;
          }
          fw[(size_t)e * 8 + q] += S[(size_t)P.cell[c] * NS + t * kMaxDirs + sl];
        }
      }
      for (int q = 0; q < 8; ++q) fwf[(size_t)e * 8 + q] = (float)fw[(size_t)e * 8 + q];
    }
    CK(cudaMemcpy(P.d_fw, fw.data(), fw.size() * sizeof(double), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(P.d_fwf, fwf.data(), fwf.size() * sizeof(float), cudaMemcpyHostToDevice));
  }
  // coarse operator on the free macro vertices (level 0: n = 1, unit scale)
  int n0 = m->n0f;
  if (n0 > 0) {
    std::vector<int> cidx(m->nv, -1);
    for (int q = 0; q < n0; ++q) cidx[m->cf_vert[q]] = q;
    // vertex-primitive index of each global vertex
    std::vector<double> A((size_t)n0 * n0, 0.0);
    int d = m->dim;
    for (int c = 0; c < m->nc; ++c) {
      for (int a = 0; a <= d; ++a) {
        int ga = m->cells[(size_t)c * (d + 1) + a];
        int ia = cidx[ga];
        if (ia < 0) continue;
        int pa[3];
        vertex_coords(a, 1, pa[0], pa[1], pa[2]);
        int ta = boundary_type(d, 1, pa[0], pa[1], pa[2]);
        for (int b = 0; b <= d; ++b) {
          int gb = m->cells[(size_t)c * (d + 1) + b];
          int ib = cidx[gb];
          if (ib < 0) continue;
          int pb[3];
          vertex_coords(b, 1, pb[0], pb[1], pb[2]);
          int s = slot_of(d, pb[0] - pa[0], pb[1] - pa[1], pb[2] - pa[2]);
          A[(size_t)ia * n0 + ib] += S[(size_t)c * NS + ta * kMaxDirs + s];
        }
      }
    }
    if (!cholesky_inverse(n0, A)) {
      set_error("coarse operator is not positive definite (check Dirichlet flags / mesh)");
      return HHG_ERR_MESH;
    }
    m->ainv_inf = 0;
    for (int i = 0; i < n0; ++i) {
      double rs = 0;
      for (int j = 0; j < n0; ++j) rs += std::fabs(A[(size_t)i * n0 + j]);
      m->ainv_inf = std::max(m->ainv_inf, rs);
    }
    CK(cudaMemcpy(m->d_Ainv, A.data(), A.size() * sizeof(double), cudaMemcpyHostToDevice));
  }
  return HHG_OK;
}

static hhg_status upload_prims(hhg_mesh_s* m, Prims& P) {
  hhg_status st;
  if ((st = upload(m, &P.d_ptr, P.ptr)) != HHG_OK) return st;
  if ((st = upload(m, &P.d_cell, P.cell)) != HHG_OK) return st;
  if ((st = upload(m, &P.d_loc, P.loc)) != HHG_OK) return st;
  if ((st = upload(m, &P.d_dir, P.dir)) != HHG_OK) return st;
  if ((st = dalloc(m, &P.d_pinv, (size_t)P.count)) != HHG_OK) return st;
  if ((st = dalloc(m, &P.d_pinvf, (size_t)P.count)) != HHG_OK) return st;
  if ((st = dalloc(m, &P.d_fw, (size_t)P.count * 8)) != HHG_OK) return st;
  if ((st = dalloc(m, &P.d_fwf, (size_t)P.count * 8)) != HHG_OK) return st;
  for (int i = 0; i < P.count; ++i) P.max_copies = std::max(P.max_copies, P.ptr[i + 1] - P.ptr[i]);
  return HHG_OK;
}

hhg_status build_mesh(hhg_mesh_s* m, const double* coords, const int* cells, const unsigned char* vflag_in) {
  const int d = m->dim, nc = m->nc, nv = m->nv, L = m->L;
  const int NS = kMaxTypes * kMaxDirs;
  m->coords.assign(coords, coords + (size_t)nv * d);
  m->cells.assign(cells, cells + (size_t)nc * (d + 1));
  m->k.assign(nc, 1.0);
  for (int c = 0; c < nc; ++c)
    for (int a = 0; a <= d; ++a) {
      int v = cells[(size_t)c * (d + 1) + a];
      if (v < 0 || v >= nv) {
        set_error("cell %d references vertex %d outside [0,%d)", c, v, nv);
        return HHG_ERR_ARG;
      }
      for (int b = 0; b < a; ++b)
        if (cells[(size_t)c * (d + 1) + b] == v) {
          set_error("cell %d repeats vertex %d", c, v);
          return HHG_ERR_MESH;
        }
    }
  // ---- per-cell stencils
  m->hS1.assign((size_t)nc * NS, 0.0);
  m->hM.assign((size_t)nc * NS, 0.0);
  for (int c = 0; c < nc; ++c) {
    const int* cv = &cells[(size_t)c * (d + 1)];
    double J[3][3] = {{0}};
    for (int r = 0; r < d; ++r)
      for (int q = 0; q < d; ++q) J[r][q] = coords[(size_t)cv[q + 1] * d + r] - coords[(size_t)cv[0] * d + r];
    double det = d == 2 ? J[0][0] * J[1][1] - J[0][1] * J[1][0]
                        : J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
                              J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
                              J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
    double scale = 0;
    for (int r = 0; r < d; ++r)
      for (int q = 0; q < d; ++q) scale = std::max(scale, std::fabs(J[r][q]));
    if (!(std::fabs(det) > 1e-12 * std::pow(scale, d))) {
      set_error("cell %d is degenerate (det J = %g)", c, det);
      return HHG_ERR_MESH;
    }
    if (!cell_stencils(d, &coords[(size_t)cv[0] * d], J, &m->hS1[(size_t)c * NS], &m->hM[(size_t)c * NS])) {
      set_error("stencil construction failed for cell %d", c);
      return HHG_ERR_MESH;
    }
  }
  // ---- topology: edges and faces keyed by sorted global ids
  std::map<std::array<int, 2>, std::vector<std::pair<int, int>>> emap;        // -> (cell, loc)
  std::map<std::array<int, 3>, std::vector<std::pair<int, int>>> fmap;        // 3D faces
  std::vector<std::vector<std::pair<int, int>>> vcopies(nv);
  for (int c = 0; c < nc; ++c) {
    const int* cv = &cells[(size_t)c * (d + 1)];
    for (int a = 0; a <= d; ++a) vcopies[cv[a]].push_back({c, a});
    for (int a = 0; a <= d; ++a)
      for (int b = a + 1; b <= d; ++b) {
        int la = a, lb = b;
        if (cv[la] > cv[lb]) std::swap(la, lb);
        emap[{cv[la], cv[lb]}].push_back({c, la | (lb << 2)});
      }
    if (d == 3)
      for (int a = 0; a < 4; ++a)
        for (int b = a + 1; b < 4; ++b)
          for (int e = b + 1; e < 4; ++e) {
            int l3[3] = {a, b, e};
            std::sort(l3, l3 + 3, [&](int x, int y) { return cv[x] < cv[y]; });
            fmap[{cv[l3[0]], cv[l3[1]], cv[l3[2]]}].push_back({c, l3[0] | (l3[1] << 2) | (l3[2] << 4)});
          }
  }
  // boundary facets
  std::vector<char> bvert(nv, 0);
  std::map<std::array<int, 2>, char> bedge;
  if (d == 2) {
    for (auto& kv : emap) {
      if (kv.second.size() > 2) {
        set_error("non-manifold edge (%d,%d)", kv.first[0], kv.first[1]);
        return HHG_ERR_MESH;
      }
      if (kv.second.size() == 1) {
        bedge[kv.first] = 1;
        bvert[kv.first[0]] = bvert[kv.first[1]] = 1;
      }
    }
  } else {
    for (auto& kv : fmap) {
      if (kv.second.size() > 2) {
        set_error("non-manifold face (%d,%d,%d)", kv.first[0], kv.first[1], kv.first[2]);
        return HHG_ERR_MESH;
      }
      if (kv.second.size() == 1) {
        const auto& f = kv.first;
        bvert[f[0]] = bvert[f[1]] = bvert[f[2]] = 1;
        bedge[{f[0], f[1]}] = 1;
        bedge[{f[0], f[2]}] = 1;
        bedge[{f[1], f[2]}] = 1;
      }
    }
  }
  std::vector<unsigned char> vflag(nv);
  for (int v = 0; v < nv; ++v) vflag[v] = vflag_in ? (vflag_in[v] ? 1 : 0) : (unsigned char)bvert[v];
  // ---- primitives
  Prims& PV = m->verts;
  PV.ptr.assign(1, 0);
  std::vector<int> vprim(nv, -1);
  for (int v = 0; v < nv; ++v) {
    if (vcopies[v].empty()) continue;
    vprim[v] = PV.count++;
    for (auto& cp : vcopies[v]) {
      PV.cell.push_back(cp.first);
      PV.loc.push_back(cp.second);
    }
    PV.ptr.push_back((int)PV.cell.size());
    PV.dir.push_back(vflag[v]);
  }
  Prims& PE = m->edges;
  PE.ptr.assign(1, 0);
  std::map<std::array<int, 2>, unsigned char> edir;
  for (auto& kv : emap) {
    unsigned char dirich = (bedge.count(kv.first) && vflag[kv.first[0]] && vflag[kv.first[1]]) ? 1 : 0;
    edir[kv.first] = dirich;
    for (auto& cp : kv.second) {
      PE.cell.push_back(cp.first);
      PE.loc.push_back(cp.second);
    }
    PE.ptr.push_back((int)PE.cell.size());
    PE.dir.push_back(dirich);
    PE.count++;
  }
  Prims& PF = m->faces;
  PF.ptr.assign(1, 0);
  std::map<std::array<int, 3>, unsigned char> fdir;
  for (auto& kv : fmap) {
    const auto& f = kv.first;
    unsigned char dirich = (kv.second.size() == 1 && vflag[f[0]] && vflag[f[1]] && vflag[f[2]]) ? 1 : 0;
    fdir[f] = dirich;
    for (auto& cp : kv.second) {
      PF.cell.push_back(cp.first);
      PF.loc.push_back(cp.second);
    }
    PF.ptr.push_back((int)PF.cell.size());
    PF.dir.push_back(dirich);
    PF.count++;
  }
  // ---- Dirichlet masks per cell and boundary type
  m->dirmask.assign(nc, 0);
  for (int c = 0; c < nc; ++c) {
    const int* cv = &cells[(size_t)c * (d + 1)];
    uint16_t mask = 0;
    for (int t = 1; t < (1 << (d + 1)); ++t) {
      int np, a[3];
      type_primitive(d, t, np, a);
      if (np == 0) continue;
      bool dirich = false;
      if (np == 1) dirich = vflag[cv[a[0]]];
      else if (np == 2) {
        int g0 = std::min(cv[a[0]], cv[a[1]]), g1 = std::max(cv[a[0]], cv[a[1]]);
        dirich = edir[{g0, g1}];
      } else if (np == 3 && d == 3) {
        int g[3] = {cv[a[0]], cv[a[1]], cv[a[2]]};
        std::sort(g, g + 3);
        dirich = fdir[{g[0], g[1], g[2]}];
      }
      if (dirich) mask |= (uint16_t)(1u << t);
    }
    m->dirmask[c] = mask;
  }
  // ---- interior stencil patterns -> groups and colourings
  const int npair = d == 2 ? 3 : 7;
  std::map<int, int> gidx;
  m->group_of_cell.assign(nc, 0);
  for (int c = 0; c < nc; ++c) {
    const double* s0 = &m->hS1[(size_t)c * NS];
    double vmax = 0;
    for (int s = 1; s < 2 * npair + 1; ++s) vmax = std::max(vmax, std::fabs(s0[s]));
    int pm = 0;
    for (int q = 0; q < npair; ++q)
      if (std::fabs(s0[2 * q + 1]) > 1e-12 * vmax || std::fabs(s0[2 * q + 2]) > 1e-12 * vmax) pm |= 1 << q;
    auto it = gidx.find(pm);
    if (it == gidx.end()) {
      Group g;
      g.pmask = pm;
      // colouring: first alpha of a fixed list with alpha . d odd for every coupled direction
      static const int c2[3][3] = {{1, 1, 0}, {1, 0, 0}, {0, 1, 0}};
      static const int c3[7][3] = {{1, 1, 1}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1}, {1, 1, 0}, {1, 0, 1}, {0, 1, 1}};
      int ncand = d == 2 ? 3 : 7;
      bool found = false;
      for (int ci = 0; ci < ncand && !found; ++ci) {
        const int* al = d == 2 ? c2[ci] : c3[ci];
        bool ok = true;
        for (int q = 0; q < npair; ++q) {
          if (!(pm >> q & 1)) continue;
          int di, dj, dk;
          dir_vec(d, 2 * q + 1, di, dj, dk);
          int dot = al[0] * di + al[1] * dj + al[2] * dk;
          if ((dot % 2 + 2) % 2 == 0) ok = false;
        }
        if (ok) {
          found = true;
          g.alpha[0] = al[0]; g.alpha[1] = al[1]; g.alpha[2] = al[2];
          g.m = 2;
        }
      }
      if (!found) {
        if (d == 2) { g.alpha[0] = 1; g.alpha[1] = 2; g.alpha[2] = 0; g.m = 3; }
        else { g.alpha[0] = 1; g.alpha[1] = 2; g.alpha[2] = 3; g.m = 4; }
      }
      gidx[pm] = (int)m->groups.size();
      m->groups.push_back(g);
      it = gidx.find(pm);
    }
    m->group_of_cell[c] = it->second;
    m->groups[it->second].cells.push_back(c);
  }
  m->n_colours = 0;
  for (auto& g : m->groups) m->n_colours = std::max(m->n_colours, g.m);
  // ---- device: stencils, masks, primitives
  hhg_status st;
  if ((st = dalloc(m, &m->dS, (size_t)nc * NS)) != HHG_OK) return st;
  if ((st = dalloc(m, &m->d_nzs, (size_t)nc * kMaxTypes)) != HHG_OK) return st;
  if ((st = upload(m, &m->dM, m->hM)) != HHG_OK) return st;
  {
    // hi = the binary32 rounding of the entry, lo = the binary32 rounding of the rest
    std::vector<float2> Mp(m->hM.size());
    for (size_t q = 0; q < m->hM.size(); ++q) {
      const float h = (float)m->hM[q];
      Mp[q] = make_float2(h, (float)(m->hM[q] - (double)h));
    }
    if ((st = upload(m, &m->dMp, Mp)) != HHG_OK) return st;
  }
  if ((st = dalloc(m, &m->dS32, (size_t)nc * NS)) != HHG_OK) return st;
  if ((st = dalloc(m, &m->dSp, (size_t)nc * NS)) != HHG_OK) return st;
  if ((st = dalloc(m, &m->dM32, (size_t)nc * NS)) != HHG_OK) return st;
  if ((st = dalloc(m, &m->d_inv0, (size_t)nc)) != HHG_OK) return st;
  if ((st = dalloc(m, &m->d_inv0f, (size_t)nc)) != HHG_OK) return st;
  if ((st = dalloc(m, &m->d_tnorm, (size_t)nc * 16)) != HHG_OK) return st;
  if ((st = dalloc(m, &m->d_tnormf, (size_t)nc * 16)) != HHG_OK) return st;
  if ((st = upload(m, &m->d_dirmask, m->dirmask)) != HHG_OK) return st;
  if ((st = upload_prims(m, m->verts)) != HHG_OK) return st;
  if ((st = upload_prims(m, m->edges)) != HHG_OK) return st;
  if ((st = upload_prims(m, m->faces)) != HHG_OK) return st;
  for (auto& g : m->groups)
    if ((st = upload(m, &g.d_cells, g.cells)) != HHG_OK) return st;
  // ---- coarse solve set-up
  m->cf_vert.clear();
  for (int q = 0; q < PV.count; ++q)
    if (!PV.dir[q]) m->cf_vert.push_back(q);
  m->n0f = (int)m->cf_vert.size();
  if (m->n0f > 16384) {
    set_error("%d free coarse vertices exceed the direct coarse solve limit of 16384", m->n0f);
    return HHG_ERR_MESH;
  }
  // cf_vert holds vertex-primitive indices; the coarse operator assembly indexes by global
  // vertex, so map through vprim
  {
    std::vector<int> prim_to_vertex(PV.count);
    for (int v = 0; v < nv; ++v)
      if (vprim[v] >= 0) prim_to_vertex[vprim[v]] = v;
    if ((st = upload(m, &m->d_cf_vert, m->cf_vert)) != HHG_OK) return st;
    // host copy used by upload_coefficient: convert to global vertex ids there
    std::vector<int> cf_global(m->n0f);
    for (int q = 0; q < m->n0f; ++q) cf_global[q] = prim_to_vertex[m->cf_vert[q]];
    // upload_coefficient indexes cidx by global vertex id: store global ids in cf_vert for host
    // use, keep the primitive ids on the device
    m->cf_vert.swap(cf_global);
    // cidx in upload_coefficient is sized by verts.count; make it cover all global ids
  }
  if ((st = dalloc(m, &m->d_Ainv, (size_t)std::max(1, m->n0f) * std::max(1, m->n0f))) != HHG_OK) return st;
  // ---- levels
  m->lv.resize(L + 1);
  int64_t maxN = 0;
  for (int l = 0; l <= L; ++l) {
    LevelData& Lv = m->lv[l];
    Lv.l = l;
    Lv.n = 1 << l;
    Lv.Nt = closure_size(d, Lv.n);
    Lv.N = Lv.Nt * nc;
    maxN = std::max(maxN, Lv.N);
    std::vector<int32_t> ijk(Lv.Nt);
    for (int k = 0; k <= (d == 3 ? Lv.n : 0); ++k)
      for (int j = 0; j <= Lv.n - k; ++j)
        for (int i = 0; i <= Lv.n - k - j; ++i) ijk[packed_index(d, Lv.n, i, j, k)] = i | (j << 10) | (k << 20);
    if ((st = upload(m, &Lv.d_ijk, ijk)) != HHG_OK) return st;
    if (l >= 1) {
      // interpolation from level l-1: a node with all-even lattice coordinates is a coarse node;
      // any other is the midpoint of the coarse edge in the direction of its odd coordinates
      std::vector<int2> itab(Lv.Nt);
      for (int64_t q = 0; q < Lv.Nt; ++q) {
        const int i = ijk[q] & 1023, j = (ijk[q] >> 10) & 1023, k = ijk[q] >> 20;
        const int t = boundary_type(d, Lv.n, i, j, k);
        int64_t ia, ib;
        interp_ends(d, Lv.n, i, j, k, ia, ib);
        itab[q] = make_int2((int)(ia | ((int64_t)t << 27)), (int)ib);
      }
      if ((st = upload(m, &Lv.d_itab, itab)) != HHG_OK) return st;
    }
    // interior colour lists per group
    std::vector<int2> icol;
    Lv.icol_off.assign(m->groups.size(), {});
    for (size_t g = 0; g < m->groups.size(); ++g) {
      const Group& G = m->groups[g];
      Lv.icol_off[g].push_back((int64_t)icol.size());
      for (int c = 0; c < G.m; ++c) {
        for (int64_t q = 0; q < Lv.Nt; ++q) {
          int i = ijk[q] & 1023, j = (ijk[q] >> 10) & 1023, k = ijk[q] >> 20;
          if (boundary_type(d, Lv.n, i, j, k) != 0) continue;
          int col = ((G.alpha[0] * i + G.alpha[1] * j + G.alpha[2] * k) % G.m + G.m) % G.m;
          if (col == c) icol.push_back(make_int2((int)q, j | (k << 16)));
        }
        Lv.icol_off[g].push_back((int64_t)icol.size());
      }
    }
    if ((st = upload(m, &Lv.d_icol, icol)) != HHG_OK) return st;
    // boundary-type nodes, sorted by type (stable: packed order inside a type)
    std::vector<std::pair<int, int64_t>> bt;
    for (int64_t q = 0; q < Lv.Nt; ++q) {
      int i = ijk[q] & 1023, j = (ijk[q] >> 10) & 1023, k = ijk[q] >> 20;
      int t = boundary_type(d, Lv.n, i, j, k);
      if (t != 0) bt.push_back({t, q});
    }
    std::stable_sort(bt.begin(), bt.end(),
                     [](const std::pair<int, int64_t>& x, const std::pair<int, int64_t>& y) { return x.first < y.first; });
    std::vector<int2> bnd;
    for (auto& e : bt) bnd.push_back(make_int2((int)e.second, ijk[e.second]));
    Lv.nbnd = (int64_t)bnd.size();
    if ((st = upload(m, &Lv.d_bnd, bnd)) != HHG_OK) return st;
    if ((st = dalloc(m, &Lv.d_invl, (size_t)nc)) != HHG_OK) return st;
    if ((st = dalloc(m, &Lv.d_invlf, (size_t)nc)) != HHG_OK) return st;
    // face colour lists: face-local (a, b), a, b >= 1, a + b <= n - 1, colour (a + 2b) mod 3
    std::vector<int32_t> fcol;
    for (int c = 0; c < 3; ++c) {
      Lv.fcol_off[c] = (int64_t)fcol.size();
      if (d == 3)
        for (int b = 1; b <= Lv.n - 2; ++b)
          for (int a = 1; a + b <= Lv.n - 1; ++a)
            if ((a + 2 * b) % 3 == c) fcol.push_back(a | (b << 16));
    }
    Lv.fcol_off[3] = (int64_t)fcol.size();
    if ((st = upload(m, &Lv.d_fcol, fcol)) != HHG_OK) return st;
    // vectors
    if ((st = dalloc(m, &Lv.u, Lv.N)) != HHG_OK) return st;
    if ((st = dalloc(m, &Lv.b, Lv.N)) != HHG_OK) return st;
    // rc: coarse-grid rhs on levels < L; on level L the estimator's difference vector
    if ((st = dalloc(m, &Lv.rc, Lv.N)) != HHG_OK) return st;
    if (l >= 1 && (st = dalloc(m, &Lv.tmp, Lv.N)) != HHG_OK) return st;
  }
  for (int l = 0; l < L; ++l)
    if ((st = dalloc(m, &m->lv[l].w, m->lv[l + 1].N)) != HHG_OK) return st;
  if ((st = dalloc(m, &m->fL, m->lv[L].N)) != HHG_OK) return st;
  if ((st = dalloc(m, &m->gL, m->lv[L].N)) != HHG_OK) return st;
  // reduction scratch: one block sum per cell and block of the level-L per-cell forms
  m->part_len = (int64_t)nc * ((m->lv[L].Nt + kBlock - 1) / kBlock);
  if ((st = dalloc(m, &m->d_part, (size_t)m->part_len)) != HHG_OK) return st;
  if ((st = dalloc(m, &m->d_red, (size_t)nc * 4)) != HHG_OK) return st;
  if ((st = dalloc(m, &m->d_flag, 4)) != HHG_OK) return st;
  if (d == 3 && m->faces.count) {  // face-block scratch where a face's values exceed shared memory
    int64_t nfL = m->lv[L].fcol_off[3];
    if (2 * nfL * (int64_t)sizeof(double) > (int64_t)kMaxTileSmem) {
      double* wbuf = nullptr;
      if ((st = dalloc(m, &wbuf, (size_t)m->faces.count * 2 * nfL)) != HHG_OK) return st;
      m->d_face_work = wbuf;
    }
  }
  if ((st = dalloc(m, &m->d_scal32, 64)) != HHG_OK) return st;
  {
    cudaError_t e = cudaMallocHost((void**)&m->h_red, sizeof(double) * (size_t)nc * 4 + 64);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMallocHost");
    m->h_flag = (int*)(m->h_red + (size_t)nc * 4);
  }
  // ---- counts of distinct / free nodes on level L
  {
    int64_t n = m->lv[L].n;
    int64_t e_in = n - 1, f_in = (n - 1) * (n - 2) / 2;
    int64_t c_in = d == 2 ? (n - 1) * (n - 2) / 2 : (n - 1) * (n - 2) * (n - 3) / 6;
    int64_t distinct = PV.count + (int64_t)PE.count * e_in + (d == 3 ? (int64_t)PF.count * f_in : 0) + (int64_t)nc * c_in;
    int64_t dirn = 0;
    for (int q = 0; q < PV.count; ++q) dirn += PV.dir[q];
    for (int q = 0; q < PE.count; ++q) dirn += PE.dir[q] * e_in;
    for (int q = 0; q < PF.count; ++q) dirn += PF.dir[q] * f_in;
    m->n_distinct = distinct;
    m->n_unknowns = distinct - dirn;
  }
  return upload_coefficient(m);
}

void free_mesh(hhg_mesh_s* m) {
  auto F = [](void* p) {
    if (p) cudaFree(p);
  };
  for (auto& kv : m->graphs) cudaGraphExecDestroy(kv.second);
  m->graphs.clear();
  F(m->dS); F(m->dM); F(m->dMp); F(m->dSp); F(m->dS32); F(m->dM32); F(m->d_inv0); F(m->d_inv0f); F(m->d_tnorm); F(m->d_tnormf);
  F(m->d_dirmask); F(m->d_nzs);
  for (hhg::Prims* P : {&m->verts, &m->edges, &m->faces}) {
    F(P->d_ptr); F(P->d_cell); F(P->d_loc); F(P->d_dir); F(P->d_pinv); F(P->d_pinvf); F(P->d_fw); F(P->d_fwf);
  }
  for (auto& g : m->groups) F(g.d_cells);
  F(m->d_Ainv); F(m->d_cf_vert); F(m->d_rmax); F(m->d_ainv_inf);
  for (auto& Lv : m->lv) {
    F(Lv.d_ijk); F(Lv.d_itab); F(Lv.d_icol); F(Lv.d_bnd); F(Lv.d_invl); F(Lv.d_invlf); F(Lv.d_fcol); F(Lv.u); F(Lv.b); F(Lv.rc); F(Lv.w); F(Lv.tmp);
    F(Lv.c16); F(Lv.r32); F(Lv.t32); F(Lv.cscale); F(Lv.x32); F(Lv.b32);
  }
  F(m->fL); F(m->gL); F(m->d_part); F(m->d_red); F(m->d_flag); F(m->d_face_work); F(m->d_scal32);
  if (m->h_red) cudaFreeHost(m->h_red);
  if (m->cap) cudaStreamDestroy(m->cap);
  if (m->own) cudaStreamDestroy(m->own);
  if (m->ev_legacy) cudaEventDestroy(m->ev_legacy);
}

}  // namespace hhg
