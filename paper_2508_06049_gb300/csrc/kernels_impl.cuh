// Templated device code of the HHG kernels (shared by the binary64 and the mixed-precision
// translation units).  One macro cell's lattice is addressed through the packed layout of
// lattice.h; vectors are consistent (equal values in all interface copies) except right-hand sides
// and residuals, which are partial: each copy holds its cell's contribution, and the value of an
// interface row is the sum over copies (the additive interface collection of Sec. 4.4).
#pragma once

#include "device_common.cuh"

namespace hhg {


constexpr int kBlock = 256;

inline double stiff_scale(int d, int n) { return d == 2 ? 1.0 : 1.0 / (double)n; }
inline double mass_scale(int d, int n) {
  double s = 1.0 / ((double)n * (double)n);
  return d == 3 ? s / (double)n : s;
}
inline unsigned blocks_for(int64_t n, int b = kBlock) { return (unsigned)((n + b - 1) / b); }

__device__ __forceinline__ void local_vertex_vec(int a, int& x, int& y, int& z) {
  x = (a == 1);
  y = (a == 2);
  z = (a == 3);
}

// lattice position inside a cell of a node of a primitive: n E_a0 + s (E_a1 - E_a0) + t (E_a2 - E_a0)
__device__ __forceinline__ void prim_position(int loc, int nverts, int n, int s, int t, int& i, int& j, int& k) {
  int a0 = loc & 3, a1 = (loc >> 2) & 3, a2 = (loc >> 4) & 3;
  int x0, y0, z0;
  local_vertex_vec(a0, x0, y0, z0);
  i = n * x0; j = n * y0; k = n * z0;
  if (nverts >= 2) {
    int x1, y1, z1;
    local_vertex_vec(a1, x1, y1, z1);
    i += s * (x1 - x0); j += s * (y1 - y0); k += s * (z1 - z0);
  }
  if (nverts >= 3) {
    int x2, y2, z2;
    local_vertex_vec(a2, x2, y2, z2);
    i += t * (x2 - x0); j += t * (y2 - y0); k += t * (z2 - z0);
  }
}

// partial residual of one cell copy at node (i,j,k): rhs - scale * sum_d S[t][d] u[g + off[d]]
template <int DIM, typename R, typename U, typename B>
__device__ __forceinline__ R partial_residual(const R* __restrict__ S, int T, int n, int64_t Nt, int i, int j, int k,
                                              R sscale, const CVec<R, U>& u, const CVec<R, B>& rhs, R& diag,
                                              int64_t& g) {
  int t = boundary_type(DIM, n, i, j, k);
  int64_t p = packed_index(DIM, n, i, j, k);
  g = (int64_t)T * Nt + p;
  diag = (R)1;
  if (HHG_OOB(p, Nt, 31)) return (R)0;
  int64_t off[15];
  neighbour_offsets(DIM, n, j, k, off);
  uint32_t vm = valid_dirs_tab(DIM, t);
  mask_offsets(DIM, vm, off);
  const R* s = S + (size_t)T * kStencilStride + t * kMaxDirs;
  R acc = 0;
#pragma unroll
  for (int d = 0; d < ndirs<DIM>(); ++d)
    if ((vm >> d & 1) && !HHG_OOB(p + off[d], Nt, 32)) acc += s[d] * u.get(g + off[d]);
  diag = sscale * s[0];
  return rhs.get(g) - sscale * acc;
}

// ---------------------------------------------------------------- right-hand sides (row 2)

// b_l = M_l f_l (partial per cell), f_l injected from the level-L data; zero on Dirichlet rows
template <int DIM>
__global__ void k_build_rhs(LevelCtx lc, int nL, int64_t NtL, int shift, const double* __restrict__ fL,
                            const double* __restrict__ Mst, double mscale, const uint16_t* __restrict__ dirmask,
                            double* __restrict__ b) {
  int64_t loc = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (loc >= lc.Nt) return;
  int T = blockIdx.y;
  int i, j, k;
  decode(lc.ijk[loc], i, j, k);
  int t = boundary_type(DIM, lc.n, i, j, k);
  int64_t g = (int64_t)T * lc.Nt + loc;
  if (dirmask[T] >> t & 1) {
    b[g] = 0.0;
    return;
  }
  uint32_t vm = valid_dirs_tab(DIM, t);
  const double* s = Mst + (size_t)T * kStencilStride + t * kMaxDirs;
  double acc = 0;
  for (int d = 0; d < ndirs<DIM>(); ++d) {
    if (!(vm >> d & 1)) continue;
    int di, dj, dk;
    dir_vec(DIM, d, di, dj, dk);
    int64_t q = packed_index(DIM, nL, (int64_t)(i + di) << shift, (int64_t)(j + dj) << shift,
                             (int64_t)(k + dk) << shift);
    if (HHG_OOB(q, NtL, 71)) continue;
    acc += s[d] * fL[(int64_t)T * NtL + q];
  }
  b[g] = mscale * acc;
}

// u_0 = g on Dirichlet nodes, 0 elsewhere
template <int DIM>
__global__ void k_init_coarse(LevelCtx lc, int nL, int64_t NtL, int shift, const double* __restrict__ gL,
                              const uint16_t* __restrict__ dirmask, double* __restrict__ u) {
  int64_t loc = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (loc >= lc.Nt) return;
  int T = blockIdx.y;
  int i, j, k;
  decode(lc.ijk[loc], i, j, k);
  int t = boundary_type(DIM, lc.n, i, j, k);
  double v = 0.0;
  if ((dirmask[T] >> t & 1) && gL) {
    int64_t q = packed_index(DIM, nL, (int64_t)i << shift, (int64_t)j << shift, (int64_t)k << shift);
    if (HHG_OOB(q, NtL, 82)) return;
    v = gL[(int64_t)T * NtL + q];
  }
  u[(int64_t)T * lc.Nt + loc] = v;
}

// ---------------------------------------------------------------- smoother stages (row 3)

// macro-cell interior nodes of one colour: race free (no coupling inside a colour)
template <int DIM, int PM, typename R, typename U, typename B>
__global__ void __launch_bounds__(kBlock) k_smooth_interior(const int* __restrict__ gcells, const int32_t* __restrict__ list,
                                                            int64_t len, LevelCtx lc, const R* __restrict__ S, R sscale,
                                                            const R* __restrict__ inv0, R isscale, Vec<R, U> u,
                                                            CVec<R, B> rhs) {
  int64_t pos = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (pos >= len) return;
  int T = gcells[blockIdx.y];
  int32_t loc = list[pos];
  if (HHG_OOB(loc, lc.Nt, 41)) return;
  int i, j, k;
  decode(lc.ijk[loc], i, j, k);
  int64_t off[15];
  neighbour_offsets(DIM, lc.n, j, k, off);
#ifdef HHG_CHECK
  for (int d = 1; d < ndirs<DIM>(); ++d)
    if (HHG_OOB(loc + off[d], lc.Nt, 42)) return;
#endif
  const R* s = S + (size_t)T * kStencilStride;
  int64_t g = (int64_t)T * lc.Nt + loc;
  R uc = u.get(g);
  R acc = s[0] * uc;
#pragma unroll
  for (int q = 0; q < npairs<DIM>(); ++q) {
    if (PM >> q & 1) {
      acc += s[2 * q + 1] * u.get(g + off[2 * q + 1]);
      acc += s[2 * q + 2] * u.get(g + off[2 * q + 2]);
    }
  }
  // residual and update; 1/(sscale * a_ii) = inv0[T] * (1/sscale) exactly (power-of-two scale)
  R r = rhs.get(g) - sscale * acc;
  u.set(g, uc + r * (inv0[T] * isscale));
}

// macro vertices: never coupled to each other on levels >= 1, so one pass.  One warp per vertex,
// lanes over the vertex's cell copies (scattered loads in parallel), fixed-order shuffle sums.
template <int DIM, typename R, typename U, typename B>
__global__ void k_smooth_vertex(int nprim, const int* __restrict__ ptr, const int* __restrict__ cell,
                                const int* __restrict__ locv, const unsigned char* __restrict__ dir, LevelCtx lc,
                                const R* __restrict__ S, R sscale, Vec<R, U> u, CVec<R, B> rhs) {
  int v = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  int lane = threadIdx.x & 31;
  if (v >= nprim || dir[v]) return;  // uniform across the warp
  CVec<R, U> uc{u.p, u.scale};
  R res = 0, diag = 0;
  int c0 = ptr[v], c1 = ptr[v + 1];
  int i0, j0, k0;
  prim_position(locv[c0], 1, lc.n, 0, 0, i0, j0, k0);
  R uold = u.get((int64_t)cell[c0] * lc.Nt + packed_index(DIM, lc.n, i0, j0, k0));
  for (int c = c0 + lane; c < c1; c += 32) {
    int i, j, k;
    prim_position(locv[c], 1, lc.n, 0, 0, i, j, k);
    R dg;
    int64_t g;
    res += partial_residual<DIM>(S, cell[c], lc.n, lc.Nt, i, j, k, sscale, uc, rhs, dg, g);
    diag += dg;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    res += __shfl_xor_sync(0xffffffffu, res, o);
    diag += __shfl_xor_sync(0xffffffffu, diag, o);
  }
  R unew = uold + res / diag;
  for (int c = c0 + lane; c < c1; c += 32) {
    int i, j, k;
    prim_position(locv[c], 1, lc.n, 0, 0, i, j, k);
    int64_t p = packed_index(DIM, lc.n, i, j, k);
    if (HHG_OOB(p, lc.Nt, 92)) continue;
    u.set((int64_t)cell[c] * lc.Nt + p, unew);
  }
}

// Edge (parity) and face (colour) stages.  Every node of a stage is updated from the values at the
// start of the stage.  Nodes of one stage can couple only next to a shared macro vertex (odd edge
// nodes t = 1, n-1) or a shared macro edge (face nodes with a = 1, b = 1 or a + b = n-1): these "rim"
// nodes are computed into du and applied by a second kernel.  All other ("inner") nodes of the stage
// have no neighbour in the stage, so one pass updates them in place.
//
// Position of entry q of a stage: edges: rim q -> t in {1, n-1} (odd stage only), inner q ->
// t = 2q+3 (odd) or 2q+2 (even); faces: (a, b) from the stage's rim or inner list.
__device__ __forceinline__ void stage_position(int nverts, int parity, bool rim, int n, int q,
                                               const int32_t* __restrict__ list, int& s, int& t) {
  if (nverts == 2) {
    t = 0;
    if (rim) s = (q == 0) ? 1 : n - 1;
    else s = parity ? 2 * q + 3 : 2 * q + 2;
  } else {
    int32_t ab = list[q];
    s = ab & 0xffff;
    t = ab >> 16;
  }
}

template <int DIM, typename R, typename U, typename B>
__global__ void k_iface_stage(int nprim, int nverts, int parity, int cnt_rim, int cnt_inner,
                              const int32_t* __restrict__ rim_list, const int32_t* __restrict__ inner_list,
                              const int* __restrict__ ptr, const int* __restrict__ cell, const int* __restrict__ locv,
                              const unsigned char* __restrict__ dir, LevelCtx lc, const R* __restrict__ S, R sscale,
                              Vec<R, U> u, CVec<R, B> rhs, R* __restrict__ du) {
  int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t n_rim = (int64_t)nprim * cnt_rim;
  bool rim = tid < n_rim;
  int64_t lt = rim ? tid : tid - n_rim;
  int cnt = rim ? cnt_rim : cnt_inner;
  if (!rim && lt >= (int64_t)nprim * cnt_inner) return;
  int e = (int)(lt / cnt), q = (int)(lt % cnt);
  if (dir[e]) {
    if (rim) du[tid] = 0;
    return;
  }
  int s, t;
  stage_position(nverts, parity, rim, lc.n, q, rim ? rim_list : inner_list, s, t);
  CVec<R, U> uc{u.p, u.scale};
  R res = 0, diag = 0;
  int64_t g0 = -1;
  for (int c = ptr[e]; c < ptr[e + 1]; ++c) {
    int i, j, k;
    prim_position(locv[c], nverts, lc.n, s, t, i, j, k);
    R dg;
    int64_t g;
    res += partial_residual<DIM>(S, cell[c], lc.n, lc.Nt, i, j, k, sscale, uc, rhs, dg, g);
    diag += dg;
    if (g0 < 0) g0 = g;
  }
  if (rim) {
    du[tid] = res / diag;
    return;
  }
  R unew = u.get(g0) + res / diag;
  for (int c = ptr[e]; c < ptr[e + 1]; ++c) {
    int i, j, k;
    prim_position(locv[c], nverts, lc.n, s, t, i, j, k);
    int64_t p = packed_index(DIM, lc.n, i, j, k);
    if (HHG_OOB(p, lc.Nt, 91)) continue;
    u.set((int64_t)cell[c] * lc.Nt + p, unew);
  }
}

template <int DIM, typename R, typename U>
__global__ void k_iface_apply(int nprim, int nverts, int parity, int cnt_rim, const int32_t* __restrict__ rim_list,
                              const int* __restrict__ ptr, const int* __restrict__ cell, const int* __restrict__ locv,
                              const unsigned char* __restrict__ dir, LevelCtx lc, Vec<R, U> u, const R* __restrict__ du) {
  int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= (int64_t)nprim * cnt_rim) return;
  int e = (int)(tid / cnt_rim), q = (int)(tid % cnt_rim);
  if (dir[e]) return;
  int s, t;
  stage_position(nverts, parity, true, lc.n, q, rim_list, s, t);
  R d = du[tid];
  for (int c = ptr[e]; c < ptr[e + 1]; ++c) {
    int i, j, k;
    prim_position(locv[c], nverts, lc.n, s, t, i, j, k);
    int64_t p = packed_index(DIM, lc.n, i, j, k);
    if (HHG_OOB(p, lc.Nt, 91)) continue;
    int64_t g = (int64_t)cell[c] * lc.Nt + p;
    u.set(g, u.get(g) + d);
  }
}

// ---------------------------------------------------------------- residual, restriction (row 4)

template <int DIM, int PM, typename R, typename U, typename B, typename O>
__global__ void __launch_bounds__(kBlock) k_residual(const int* __restrict__ gcells, LevelCtx lc, const R* __restrict__ S,
                                                     const uint16_t* __restrict__ dirmask, R sscale, CVec<R, U> u,
                                                     CVec<R, B> rhs, O* __restrict__ out) {
  int64_t loc = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (loc >= lc.Nt) return;
  int T = gcells[blockIdx.y];
  int i, j, k;
  decode(lc.ijk[loc], i, j, k);
  int t = boundary_type(DIM, lc.n, i, j, k);
  int64_t g = (int64_t)T * lc.Nt + loc;
  if (dirmask[T] >> t & 1) {
    out[g] = (O)0;
    return;
  }
  int64_t off[15];
  neighbour_offsets(DIM, lc.n, j, k, off);
  const R* s = S + (size_t)T * kStencilStride + t * kMaxDirs;
  R acc = s[0] * u.get(g);
  if (t == 0) {
#pragma unroll
    for (int q = 0; q < npairs<DIM>(); ++q) {
      if (PM >> q & 1) {
        acc += s[2 * q + 1] * u.get(g + off[2 * q + 1]);
        acc += s[2 * q + 2] * u.get(g + off[2 * q + 2]);
      }
    }
  } else {
    uint32_t vm = valid_dirs_tab(DIM, t);
    mask_offsets(DIM, vm, off);
#pragma unroll
    for (int d = 1; d < ndirs<DIM>(); ++d)
      if ((vm >> d & 1) && !HHG_OOB(loc + off[d], lc.Nt, 51)) acc += s[d] * u.get(g + off[d]);
  }
  out[g] = (O)(rhs.get(g) - sscale * acc);
}

// coarse partial rhs = P^T (fine partial residual), per cell: r_c(q) = r_f(2q) + 1/2 sum_d r_f(2q+d)
template <int DIM, typename R, typename I, typename O>
__global__ void k_restrict(LevelCtx fc, LevelCtx cc, const uint16_t* __restrict__ dirmask, const I* __restrict__ rf,
                           O* __restrict__ rcv) {
  int64_t loc = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (loc >= cc.Nt) return;
  int T = blockIdx.y;
  int i, j, k;
  decode(cc.ijk[loc], i, j, k);
  int t = boundary_type(DIM, cc.n, i, j, k);
  if (dirmask[T] >> t & 1) {  // Dirichlet rows of a correction's rhs are zero
    rcv[(int64_t)T * cc.Nt + loc] = (O)0;
    return;
  }
  int64_t pf = packed_index(DIM, fc.n, 2 * i, 2 * j, 2 * k);
  if (HHG_OOB(pf, fc.Nt, 61)) return;
  int64_t gf = (int64_t)T * fc.Nt + pf;
  int64_t off[15];
  neighbour_offsets(DIM, fc.n, 2 * j, 2 * k, off);
  uint32_t vm = valid_dirs_tab(DIM, t);
  mask_offsets(DIM, vm, off);
  R acc = 0;
#pragma unroll
  for (int d = 1; d < ndirs<DIM>(); ++d)
    if ((vm >> d & 1) && !HHG_OOB(pf + off[d], fc.Nt, 62)) acc += (R)rf[gf + off[d]];
  rcv[(int64_t)T * cc.Nt + loc] = (O)((R)rf[gf] + (R)0.5 * acc);
}

// ---------------------------------------------------------------- prolongation (rows 6, 7)

template <int DIM, typename R, typename C>
__device__ __forceinline__ R interp(LevelCtx cc, int T, int i, int j, int k, const C& uc) {
  int pi = i & 1, pj = j & 1, pk = k & 1;
  if (!(pi | pj | pk)) return uc.get((int64_t)T * cc.Nt + packed_index(DIM, cc.n, i >> 1, j >> 1, k >> 1));
  int di, dj, dk;
  dir_vec(DIM, parity_dir_slot(DIM, pi, pj, pk), di, dj, dk);
  int64_t ia = packed_index(DIM, cc.n, (i - di) >> 1, (j - dj) >> 1, (k - dk) >> 1);
  int64_t ib = packed_index(DIM, cc.n, (i + di) >> 1, (j + dj) >> 1, (k + dk) >> 1);
  if (HHG_OOB(ia, cc.Nt, 21) || HHG_OOB(ib, cc.Nt, 22)) return (R)0;
  R a = uc.get((int64_t)T * cc.Nt + ia);
  R b = uc.get((int64_t)T * cc.Nt + ib);
  return (R)0.5 * (a + b);
}

// u_f += I u_c on free nodes
template <int DIM, typename R, typename UC, typename UF>
__global__ void k_prolong_add(LevelCtx fc, LevelCtx cc, const uint16_t* __restrict__ dirmask, CVec<R, UC> uc,
                              Vec<R, UF> uf) {
  int64_t loc = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (loc >= fc.Nt) return;
  int T = blockIdx.y;
  int i, j, k;
  decode(fc.ijk[loc], i, j, k);
  int t = boundary_type(DIM, fc.n, i, j, k);
  if (dirmask[T] >> t & 1) return;
  int64_t g = (int64_t)T * fc.Nt + loc;
  uf.set(g, uf.get(g) + interp<DIM, R>(cc, T, i, j, k, uc));
}

// FMG transition: u_{l+1} = I u_l (Dirichlet nodes from g_L, or 0 if gL is null), w_l = u_{l+1}
template <int DIM>
__global__ void k_fmg_prolong(LevelCtx fc, LevelCtx cc, int nL, int64_t NtL, int shift, const double* __restrict__ gL,
                              const uint16_t* __restrict__ dirmask, const double* __restrict__ uc,
                              double* __restrict__ uf, double* __restrict__ w) {
  int64_t loc = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (loc >= fc.Nt) return;
  int T = blockIdx.y;
  int i, j, k;
  decode(fc.ijk[loc], i, j, k);
  int t = boundary_type(DIM, fc.n, i, j, k);
  double v;
  if (dirmask[T] >> t & 1) {
    int64_t q = packed_index(DIM, nL, (int64_t)i << shift, (int64_t)j << shift, (int64_t)k << shift);
    if (HHG_OOB(q, NtL, 81)) return;
    v = gL ? gL[(int64_t)T * NtL + q] : 0.0;
  }
  else
    v = interp<DIM, double>(cc, T, i, j, k, CVec<double, double>{uc, nullptr});
  int64_t g = (int64_t)T * fc.Nt + loc;
  uf[g] = v;
  if (w) w[g] = v;
}

// plain interpolation v_f = I v_c (all nodes)
template <int DIM>
__global__ void k_prolong(LevelCtx fc, LevelCtx cc, const double* __restrict__ vc, double* __restrict__ vf) {
  int64_t loc = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (loc >= fc.Nt) return;
  int T = blockIdx.y;
  int i, j, k;
  decode(fc.ijk[loc], i, j, k);
  vf[(int64_t)T * fc.Nt + loc] = interp<DIM, double>(cc, T, i, j, k, CVec<double, double>{vc, nullptr});
}

// ---------------------------------------------------------------- direct coarse solve (row 5)

// One CTA: residual of the free macro vertices (summed over cell copies), c = A_ff^{-1} r, update
// every copy.  n0f <= 16384 (checked at set-up); the residual vector lives in shared memory.
template <int DIM>
__global__ void __launch_bounds__(1024) k_coarse(int n0f, const int* __restrict__ cf, const int* __restrict__ ptr,
                                                 const int* __restrict__ cell, const int* __restrict__ locv,
                                                 LevelCtx lc, const double* __restrict__ S,
                                                 const double* __restrict__ rhs, double* __restrict__ u,
                                                 const double* __restrict__ Ainv) {
  extern __shared__ double r[];
  CVec<double, double> uc{u, nullptr};
  CVec<double, double> rc{rhs, nullptr};
  {
    // residual of each free coarse vertex: one warp per vertex, lanes over its cell copies
    int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int q = warp; q < n0f; q += nw) {
      int v = cf[q];
      double res = 0, dg;
      for (int c = ptr[v] + lane; c < ptr[v + 1]; c += 32) {
        int i, j, k;
        prim_position(locv[c], 1, lc.n, 0, 0, i, j, k);
        int64_t g;
        res += partial_residual<DIM>(S, cell[c], lc.n, lc.Nt, i, j, k, 1.0, uc, rc, dg, g);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) res += __shfl_xor_sync(0xffffffffu, res, o);
      if (lane == 0) r[q] = res;
    }
  }
  __syncthreads();
  int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int row = warp; row < n0f; row += nw) {
    const double* a = Ainv + (size_t)row * n0f;
    double acc = 0;
    for (int c = lane; c < n0f; c += 32) acc += a[c] * r[c];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) {
      int v = cf[row];
      for (int c = ptr[v]; c < ptr[v + 1]; ++c) {
        int i, j, k;
        prim_position(locv[c], 1, lc.n, 0, 0, i, j, k);
        int64_t p = packed_index(DIM, lc.n, i, j, k);
        if (HHG_OOB(p, lc.Nt, 93)) continue;
        u[(int64_t)cell[c] * lc.Nt + p] += acc;
      }
    }
  }
}

// ---------------------------------------------------------------- reductions (row 8, row 11)

// Per node p of a cell's closure, the symmetric-form contribution
//   c_p = S[t][0] x_p y_p + sum_{d positive, valid} S[t][d] (x_p y_{p+d} + x_{p+d} y_p),
// with x = y = a - b (b may be null) for the mass form, or x = a, y = b for a bilinear form.  Summed
// over the closure this is x^T S_T y, because the partial stencil of a cell is symmetric (the entry
// p->p+d seen from p equals the entry p+d->p seen from p+d: both sum the cell's elements on that
// edge), so each lattice edge is visited once.  Written to a level-L scratch vector; k_cell_sum adds
// each cell's contributions in a fixed order.
template <int DIM, bool DIFF>
__global__ void k_node_form(LevelCtx lc, const double* __restrict__ tab, const double* __restrict__ a,
                            const double* __restrict__ b, double* __restrict__ contrib) {
  int64_t loc = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (loc >= lc.Nt) return;
  int T = blockIdx.y;
  int i, j, k;
  decode(lc.ijk[loc], i, j, k);
  int t = boundary_type(DIM, lc.n, i, j, k);
  if (HHG_OOB(t, kMaxTypes, 12)) return;
  int64_t g = (int64_t)T * lc.Nt + loc;
  int64_t off[15];
  neighbour_offsets(DIM, lc.n, j, k, off);
  uint32_t vm = valid_dirs_tab(DIM, t);
  mask_offsets(DIM, vm, off);
  const double* s = tab + (size_t)T * kStencilStride + t * kMaxDirs;
  double xp, yp;
  if (DIFF) {
    xp = a[g];
    if (b) xp -= b[g];
    yp = xp;
  } else {
    xp = a[g];
    yp = b[g];
  }
  double sum = s[0] * xp * yp;
#pragma unroll
  for (int q = 0; q < npairs<DIM>(); ++q) {
    int d = 2 * q + 1;
    if (!(vm >> d & 1)) continue;
    if (HHG_OOB(loc + off[d], lc.Nt, 13)) continue;
    double xq, yq;
    if (DIFF) {
      xq = a[g + off[d]];
      if (b) xq -= b[g + off[d]];
      yq = xq;
    } else {
      xq = a[g + off[d]];
      yq = b[g + off[d]];
    }
    sum += s[d] * (xp * yq + xq * yp);
  }
  contrib[g] = sum;
}

// ---------------------------------------------------------------- operators for testing / adjoint

// out = scale * Stab_T in (partial rows) on all closure nodes; with inS: zero for cells not in S,
// factor `fac`, zero Dirichlet rows
template <int DIM>
__global__ void k_apply_partial(LevelCtx lc, const double* __restrict__ tab, double scale,
                                const double* __restrict__ in, double* __restrict__ out,
                                const unsigned char* __restrict__ inS, const uint16_t* __restrict__ dirmask) {
  int64_t loc = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (loc >= lc.Nt) return;
  int T = blockIdx.y;
  int i, j, k;
  decode(lc.ijk[loc], i, j, k);
  int t = boundary_type(DIM, lc.n, i, j, k);
  int64_t g = (int64_t)T * lc.Nt + loc;
  if (inS && (!inS[T] || (dirmask[T] >> t & 1))) {
    out[g] = 0.0;
    return;
  }
  int64_t off[15];
  neighbour_offsets(DIM, lc.n, j, k, off);
  uint32_t vm = valid_dirs_tab(DIM, t);
  mask_offsets(DIM, vm, off);
  const double* s = tab + (size_t)T * kStencilStride + t * kMaxDirs;
  double acc = 0;
  for (int d = 0; d < ndirs<DIM>(); ++d)
    if (vm >> d & 1) acc += s[d] * in[g + off[d]];
  out[g] = scale * acc;
}

// sum partial interface values over the copies of each primitive node and store the sum in all
template <int DIM>
__global__ void k_sum_prims(int nprim, int nverts, int cnt, const int32_t* __restrict__ flist, const int* __restrict__ ptr,
                            const int* __restrict__ cell, const int* __restrict__ locv, LevelCtx lc,
                            double* __restrict__ v) {
  int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= (int64_t)nprim * cnt) return;
  int e = (int)(tid / cnt), q = (int)(tid % cnt);
  int s = 0, t = 0;
  if (nverts == 2) s = q + 1;
  else if (nverts == 3) {
    s = flist[q] & 0xffff;
    t = flist[q] >> 16;
  }
  double sum = 0;
  for (int c = ptr[e]; c < ptr[e + 1]; ++c) {
    int i, j, k;
    prim_position(locv[c], nverts, lc.n, s, t, i, j, k);
    sum += v[(int64_t)cell[c] * lc.Nt + packed_index(DIM, lc.n, i, j, k)];
  }
  for (int c = ptr[e]; c < ptr[e + 1]; ++c) {
    int i, j, k;
    prim_position(locv[c], nverts, lc.n, s, t, i, j, k);
    v[(int64_t)cell[c] * lc.Nt + packed_index(DIM, lc.n, i, j, k)] = sum;
  }
}



// Collect partial interface values: the sum over a primitive node's copies goes to its first copy,
// the other copies get 0 (still a partial split of the same row).  Used before narrowing a binary64
// residual, whose partials cancel, to binary32.
template <int DIM>
__global__ void k_owner_collect(int nprim, int nverts, int cnt, const int32_t* __restrict__ flist,
                                const int* __restrict__ ptr, const int* __restrict__ cell, const int* __restrict__ locv,
                                LevelCtx lc, double* __restrict__ v) {
  int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= (int64_t)nprim * cnt) return;
  int e = (int)(tid / cnt), q = (int)(tid % cnt);
  int s = 0, t = 0;
  if (nverts == 2) s = q + 1;
  else if (nverts == 3) {
    s = flist[q] & 0xffff;
    t = flist[q] >> 16;
  }
  double sum = 0;
  for (int c = ptr[e]; c < ptr[e + 1]; ++c) {
    int i, j, k;
    prim_position(locv[c], nverts, lc.n, s, t, i, j, k);
    sum += v[(int64_t)cell[c] * lc.Nt + packed_index(DIM, lc.n, i, j, k)];
  }
  for (int c = ptr[e]; c < ptr[e + 1]; ++c) {
    int i, j, k;
    prim_position(locv[c], nverts, lc.n, s, t, i, j, k);
    v[(int64_t)cell[c] * lc.Nt + packed_index(DIM, lc.n, i, j, k)] = (c == ptr[e]) ? sum : 0.0;
  }
}

}  // namespace hhg
