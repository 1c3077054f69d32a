// Structured lattice of one macro element refined uniformly l times (HHG, Sec. 2 of the paper).
//
// A macro triangle (2D) or tetrahedron (3D) with vertices x_0..x_d is refined into the
// lattice x = x_0 + J p / n, n = 2^l, p = (i, j[, k]) integer with p >= 0, sum(p) <= n
// (J = [x_1 - x_0, ..., x_d - x_0]).  Red refinement in 2D and Bey's rule in 3D give exactly
// this lattice; in 3D the micro tets are the Freudenthal/Kuhn simplices of the cube lattice in
// y = (i, i+j, i+j+k), where the macro becomes the Kuhn simplex 0 <= y1 <= y2 <= y3 <= n.
//
// Nodes of the closure of one macro are stored packed: 3D planes k = 0..n (plane k is a
// triangle of side m = n-k), rows j = 0..m inside a plane, i fastest.  2D is one plane.
//
// Lattice edge directions (the P1 stencil has one coupling per direction and sign):
//   2D: e1, e2, e1-e2                      -> 7-point stencil
//   3D: e1, e2, e3, e1-e2, e1-e3, e2-e3, e1-e2+e3 -> 15-point stencil
// Direction slot 0 is the centre, slot 2q+1 is +dir_q, slot 2q+2 is -dir_q.
//
// Boundary type of a closure node: bit mask of the macro faces (facets) it lies on.
//   2D bits: 0: i==0, 1: j==0, 2: i+j==n.        3D bits: 0: i==0, 1: j==0, 2: k==0, 3: i+j+k==n.
// A node with mask 0 is interior; one bit = facet interior; two bits = edge (3D);
// d bits = macro vertex.
#pragma once

#include <stdint.h>

#if defined(__CUDACC__)
#define HHG_HD __host__ __device__ __forceinline__
#else
#define HHG_HD inline
#endif

namespace hhg {

constexpr int kMaxDirs = 15;   // 3D stencil size (2D uses the first 7 slots)
constexpr int kMaxTypes = 16;  // boundary-type masks

// lattice direction vectors, slot order as documented above
HHG_HD void dir_vec(int dim, int slot, int& di, int& dj, int& dk) {
  // pairs: q -> vector
  int q = (slot - 1) >> 1;
  int s = (slot & 1) ? 1 : -1;
  di = dj = dk = 0;
  if (slot == 0) return;
  if (dim == 2) {
    if (q == 0) { di = 1; }
    else if (q == 1) { dj = 1; }
    else { di = 1; dj = -1; }
  } else {
    switch (q) {
      case 0: di = 1; break;
      case 1: dj = 1; break;
      case 2: dk = 1; break;
      case 3: di = 1; dj = -1; break;
      case 4: di = 1; dk = -1; break;
      case 5: dj = 1; dk = -1; break;
      default: di = 1; dj = -1; dk = 1; break;
    }
  }
  di *= s; dj *= s; dk *= s;
}

HHG_HD int64_t tri_size(int64_t m) { return (m + 1) * (m + 2) / 2; }            // nodes of a side-m triangle
HHG_HD int64_t tet_size(int64_t m) { return (m + 1) * (m + 2) * (m + 3) / 6; }  // nodes of a side-m tet
HHG_HD int64_t closure_size(int dim, int64_t n) { return dim == 2 ? tri_size(n) : tet_size(n); }

// packed index of lattice point (i, j, k) in the closure of side n (32-bit arithmetic: exact for
// n <= 1000, where every intermediate product stays below 2^31)
HHG_HD int64_t packed_index(int dim, int64_t n, int64_t i, int64_t j, int64_t k) {
  const int nn = (int)n, ii = (int)i, jj = (int)j, kk = (int)k;
  if (dim == 2) return (int64_t)(jj * (nn + 1) - jj * (jj - 1) / 2 + ii);
  const int m = nn - kk;
  const int tn = (nn + 1) * (nn + 2) * (nn + 3) / 6, tm = (m + 1) * (m + 2) * (m + 3) / 6;
  return (int64_t)((tn - tm) + jj * (m + 1) - jj * (jj - 1) / 2 + ii);
}

HHG_HD int boundary_type(int dim, int n, int i, int j, int k) {
  if (dim == 2) return (i == 0 ? 1 : 0) | (j == 0 ? 2 : 0) | (i + j == n ? 4 : 0);
  return (i == 0 ? 1 : 0) | (j == 0 ? 2 : 0) | (k == 0 ? 4 : 0) | (i + j + k == n ? 8 : 0);
}

// Bit mask of direction slots whose neighbour stays inside the closure, for a node of
// boundary type t (depends on t only: a node not on a facet is at least one step inside it).
HHG_HD uint32_t valid_dirs(int dim, int t) {
  uint32_t m = 0;
  int nd = dim == 2 ? 7 : 15;
  for (int s = 0; s < nd; ++s) {
    int di, dj, dk;
    dir_vec(dim, s, di, dj, dk);
    bool ok = true;
    if ((t & 1) && di < 0) ok = false;
    if ((t & 2) && dj < 0) ok = false;
    if (dim == 2) {
      if ((t & 4) && di + dj > 0) ok = false;
    } else {
      if ((t & 4) && dk < 0) ok = false;
      if ((t & 8) && di + dj + dk > 0) ok = false;
    }
    if (ok) m |= 1u << s;
  }
  return m;
}

// valid_dirs() tabulated (checked against the loop by hhg_lattice_selfcheck)
HHG_HD uint32_t valid_dirs_tab(int dim, int t) {
  constexpr uint32_t k2[16] = {0x7f, 0x3b, 0x4f, 0xb, 0x75, 0x31, 0x45, 0x1, 0x7f, 0x3b, 0x4f, 0xb, 0x75, 0x31, 0x45, 0x1};
  constexpr uint32_t k3[16] = {0x7fff, 0x3afb, 0x4f6f, 0xa6b, 0x35bf, 0x30bb, 0x52f, 0x2b, 0x5fd5, 0x1ad1, 0x4f45, 0xa41, 0x1595, 0x1091, 0x505, 0x1};
  return dim == 2 ? k2[t & 15] : k3[t & 15];
}

// Packed-index offsets of all direction slots from the node at (j, k) (independent of i).
// off[0] = 0.  Offsets of directions leaving the closure are meaningless and must be masked.
HHG_HD void neighbour_offsets(int dim, int64_t n64, int64_t j64, int64_t k64, int64_t* off) {
  // 32-bit arithmetic (exact for n <= 1000)
  const int n = (int)n64, j = (int)j64, k = (int)k64;
  off[0] = 0;
  if (dim == 2) {
    int rl = n + 1 - j;  // length of row j
    off[1] = 1;
    off[2] = -1;
    off[3] = rl;                 // +e2
    off[4] = -(rl + 1);          // -e2
    off[5] = 1 - (rl + 1);       // +e1-e2
    off[6] = -1 + rl;            // -e1+e2
    return;
  }
  const int m = n - k;
  const int Tm = (m + 1) * (m + 2) / 2, Tm1 = (m + 2) * (m + 3) / 2;
  off[1] = 1;
  off[2] = -1;
  off[3] = m + 1 - j;            // +e2
  off[4] = -(m + 2 - j);         // -e2
  off[5] = Tm - j;               // +e3
  off[6] = -Tm1 + j;             // -e3
  off[7] = -(m + 1 - j);         // +e1-e2
  off[8] = m - j;                // -e1+e2
  off[9] = 1 - Tm1 + j;          // +e1-e3
  off[10] = -1 + Tm - j;         // -e1+e3
  off[11] = -Tm1 + m + 2;        // +e2-e3
  off[12] = Tm - m - 1;          // -e2+e3
  off[13] = Tm - m;              // +e1-e2+e3
  off[14] = -Tm1 + m + 1;        // -e1+e2-e3
}

// The same offsets one slot at a time, for loops over a bit mask of slots: every offset is
// c0 + cm m + cj j + cT T(m) + cT1 T(m+1) with m the side of the node's plane (n in 2D).
HHG_HD int64_t dir_offset(int dim, int slot, int64_t m, int64_t j, int64_t Tm, int64_t Tm1) {
  if (dim == 2) {
    switch (slot) {
      case 1: return 1;
      case 2: return -1;
      case 3: return m + 1 - j;
      case 4: return -(m + 2 - j);
      case 5: return -(m + 1 - j);
      case 6: return m - j;
      default: return 0;
    }
  }
  switch (slot) {
    case 1: return 1;
    case 2: return -1;
    case 3: return m + 1 - j;
    case 4: return -(m + 2 - j);
    case 5: return Tm - j;
    case 6: return -Tm1 + j;
    case 7: return -(m + 1 - j);
    case 8: return m - j;
    case 9: return 1 - Tm1 + j;
    case 10: return -1 + Tm - j;
    case 11: return -Tm1 + m + 2;
    case 12: return Tm - m - 1;
    case 13: return Tm - m;
    case 14: return -Tm1 + m + 1;
    default: return 0;
  }
}

// plane side m and triangle sizes T(m), T(m+1) of a node at (j, k) for dir_offset()
struct PlaneBasis {
  int64_t m, Tm, Tm1;
};
HHG_HD PlaneBasis plane_basis(int dim, int64_t n, int64_t k) {
  int64_t m = dim == 2 ? n : n - k;
  return PlaneBasis{m, tri_size(m), tri_size(m + 1)};
}

// Replace the offsets of directions that leave the closure by 0 (the node itself), so that no
// address outside the cell's closure is ever formed; the stencil entries of those directions are 0.
HHG_HD void mask_offsets(int dim, uint32_t vm, int64_t* off) {
  int nd = dim == 2 ? 7 : 15;
  for (int d = 0; d < nd; ++d)
    if (!(vm >> d & 1)) off[d] = 0;
}

// Local vertex a of a macro in lattice coordinates (n * E_a, E_0 = 0, E_a = unit vector a).
HHG_HD void vertex_coords(int a, int n, int& i, int& j, int& k) {
  i = (a == 1) ? n : 0;
  j = (a == 2) ? n : 0;
  k = (a == 3) ? n : 0;
}

// Direction slot that maps a fine node of parity (pi, pj, pk) to its coarse edge (prolongation):
// the fine node p is the midpoint of the coarse nodes (p - d)/2 and (p + d)/2.
HHG_HD int parity_dir_slot(int dim, int pi, int pj, int pk) {
  if (dim == 2) {
    if (pi && pj) return 5;  // e1-e2
    if (pi) return 1;
    return 3;
  }
  int code = pi | (pj << 1) | (pk << 2);
  switch (code) {
    case 1: return 1;    // e1
    case 2: return 3;    // e2
    case 4: return 5;    // e3
    case 3: return 7;    // e1-e2
    case 5: return 9;    // e1-e3
    case 6: return 11;   // e2-e3
    default: return 13;  // e1-e2+e3
  }
}

// Interpolation from the lattice of side n / 2 (n even) to the lattice of side n: the coarse packed
// indices of the two end points of fine node (i, j, k).  A node with all-even coordinates is the
// coarse node (i, j, k) / 2 (ia = ib); any other is the midpoint of the coarse edge along the
// direction of its odd coordinates (checked against brute force by hhg_lattice_selfcheck).
HHG_HD void interp_ends(int dim, int n, int i, int j, int k, int64_t& ia, int64_t& ib) {
  const int nc = n / 2;
  if (!((i | j | k) & 1)) {
    ia = ib = packed_index(dim, nc, i >> 1, j >> 1, k >> 1);
    return;
  }
  int di, dj, dk;
  dir_vec(dim, parity_dir_slot(dim, i & 1, j & 1, k & 1), di, dj, dk);
  ia = packed_index(dim, nc, (i - di) >> 1, (j - dj) >> 1, (k - dk) >> 1);
  ib = packed_index(dim, nc, (i + di) >> 1, (j + dj) >> 1, (k + dk) >> 1);
}

}  // namespace hhg
