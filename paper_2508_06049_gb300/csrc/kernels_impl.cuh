// Templated device code of the HHG kernels (shared by the binary64 and the mixed-precision
// translation units).  One macro cell's lattice is addressed through the packed layout of
// lattice.h; vectors are consistent (equal values in all interface copies) except right-hand sides
// and residuals, which are partial: each copy holds its cell's contribution, and the value of an
// interface row is the sum over copies (the additive interface collection of Sec. 4.4).
#pragma once

#include <utility>

#include "device_common.cuh"
#include "dfloat.cuh"

namespace hhg {



inline double stiff_scale(int d, int n) { return d == 2 ? 1.0 : 1.0 / (double)n; }
inline double mass_scale(int d, int n) {
  double s = 1.0 / ((double)n * (double)n);
  return d == 3 ? s / (double)n : s;
}
inline unsigned blocks_for(int64_t n, int b = kBlock) { return (unsigned)((n + b - 1) / b); }

// Launch on stream s with programmatic stream serialisation allowed (see grid_dependency_sync).
// Launch errors surface through cudaGetLastError / the stream, as with <<< >>>.
template <typename... KArgs, typename... Args>
inline void hhg_launch(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                       Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

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

// Stencil terms of one cell copy of an interface node (i,j,k): acc += sum_d S[t][d] u[g + off_d] over
// the slots whose neighbour lies in the closure and whose entry is nonzero (all slots unrolled,
// loads issued together), bsum += rhs[g]; returns g.
template <int DIM, typename R, typename U, typename B>
__device__ __forceinline__ int64_t copy_terms(const R* __restrict__ S, const uint16_t* __restrict__ nzs, int T, int n,
                                              int64_t Nt, int i, int j, int k, const CVec<R, U>& u,
                                              const CVec<R, B>& rhs, R& acc, R& bsum) {
  int t = boundary_type(DIM, n, i, j, k);
  int64_t p = packed_index(DIM, n, i, j, k);
  int64_t g = (int64_t)T * Nt + p;
  if (HHG_OOB(p, Nt, 31)) return g;
  uint32_t vm = valid_dirs_tab(DIM, t) & nzs[T * kMaxTypes + t];
  const R* s = S + (size_t)T * kStencilStride + t * kMaxDirs;
  R a = s[0] * u.get(g);
  int64_t off[15];
  neighbour_offsets(DIM, n, j, k, off);
  mask_offsets(DIM, vm, off);
#pragma unroll
  for (int d = 1; d < ndirs<DIM>(); ++d)
    if ((vm >> d & 1) && !HHG_OOB(p + off[d], Nt, 32)) a += s[d] * u.get(g + off[d]);
  acc += a;
  bsum += rhs.get(g);
  return g;
}

// ---------------------------------------------------------------- right-hand sides b_l = M_l f_l (Eq. 4.15, Sec. 4.4)

// b_l = M_l f_l (partial per cell), f_l injected from the level-L data; zero on Dirichlet rows.
// R: the arithmetic and mass-stencil type (binary64, or binary32 for the coarse right-hand sides of
// the mixed path's binary32 FMG), O: the stored type.
template <int DIM, typename R, typename O>
__global__ void k_build_rhs(LevelCtx lc, int nL, int64_t NtL, int shift, const double* __restrict__ fL,
                            const R* __restrict__ Mst, R mscale, const uint16_t* __restrict__ dirmask,
                            O* __restrict__ b) {
  grid_dependency_sync();
  int64_t loc = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (loc >= lc.Nt) return;
  int T = blockIdx.y;
  int i, j, k;
  decode(lc.ijk[loc], i, j, k);
  int t = boundary_type(DIM, lc.n, i, j, k);
  int64_t g = (int64_t)T * lc.Nt + loc;
  if (dirmask[T] >> t & 1) {
    b[g] = (O)0;
    return;
  }
  uint32_t vm = valid_dirs_tab(DIM, t);
  const R* s = Mst + (size_t)T * kStencilStride + t * kMaxDirs;
  const double* f = fL + (int64_t)T * NtL;
  R acc = 0;
  if (shift == 0) {  // level L itself: the level's own neighbour offsets
    int64_t off[15];
    neighbour_offsets(DIM, lc.n, j, k, off);
    mask_offsets(DIM, vm, off);
#pragma unroll
    for (int d = 0; d < ndirs<DIM>(); ++d)
      if ((vm >> d & 1) && !HHG_OOB(loc + off[d], NtL, 71)) acc += s[d] * (R)f[loc + off[d]];
  } else {
#pragma unroll
    for (int d = 0; d < ndirs<DIM>(); ++d) {
      if (!(vm >> d & 1)) continue;
      int di, dj, dk;
      dir_vec(DIM, d, di, dj, dk);
      int64_t q = packed_index(DIM, nL, (int64_t)(i + di) << shift, (int64_t)(j + dj) << shift,
                               (int64_t)(k + dk) << shift);
      if (HHG_OOB(q, NtL, 71)) continue;
      acc += s[d] * (R)f[q];
    }
  }
  b[g] = (O)(mscale * acc);
}

// u_0 = g on Dirichlet nodes, 0 elsewhere
template <int DIM>
__global__ void k_init_coarse(LevelCtx lc, int nL, int64_t NtL, int shift, const double* __restrict__ gL,
                              const uint16_t* __restrict__ dirmask, double* __restrict__ u) {
  grid_dependency_sync();
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

// ---------------------------------------------------------------- smoother stages (Gauss-Seidel of Alg. 4)

// Macro-cell interior nodes of one colour: race free (no coupling inside a colour).  The update
// u_i <- u_i + (b_i - (A u)_i) / a_ii is evaluated in the equivalent form
// u_i <- b_i / a_ii - sum_d (a_id / a_ii) u_{i+d}: with the normalised stencil t = a / a_ii of the cell
// and inv = 1 / a_ii of the level, one multiply and one FMA per coupled neighbour.  The list entries
// carry (packed index, j | k << 16), so the neighbour offsets need no further lookup.
template <int DIM, int PM, typename R, typename U, typename B>
__global__ void __launch_bounds__(kBlock) k_smooth_interior(const int* __restrict__ gcells, const int2* __restrict__ list,
                                                            int64_t len, LevelCtx lc, const R* __restrict__ tnorm,
                                                            const R* __restrict__ invl, Vec<R, U> u, CVec<R, B> rhs) {
  grid_dependency_sync();
  int64_t pos = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (pos >= len) return;
  int T = gcells[blockIdx.y];
  int2 e = list[pos];
  int loc = e.x;
  if (HHG_OOB(loc, lc.Nt, 41)) return;
  int j = e.y & 0xffff, k = e.y >> 16;
  int64_t off[15];
  neighbour_offsets(DIM, lc.n, j, k, off);
#ifdef HHG_CHECK
  for (int d = 1; d < ndirs<DIM>(); ++d)
    if (HHG_OOB(loc + off[d], lc.Nt, 42)) return;
#endif
  const R* t = tnorm + (size_t)T * 16;
  int64_t g = (int64_t)T * lc.Nt + loc;
  R acc = rhs.get(g) * invl[T];
#pragma unroll
  for (int q = 0; q < npairs<DIM>(); ++q) {
    if (PM >> q & 1) {
      acc -= t[2 * q + 1] * u.get(g + off[2 * q + 1]);
      acc -= t[2 * q + 2] * u.get(g + off[2 * q + 2]);
    }
  }
  u.set(g, acc);
}

// The same stage with CPB cells per thread (grid.y = groups of CPB cells): the list entry and its
// neighbour offsets serve all of them, and their loads are in flight together.
template <int DIM, int PM, int CPB, typename R, typename U, typename B>
__global__ void __launch_bounds__(kBlock) k_smooth_interior_multi(const int* __restrict__ gcells, int ncells,
                                                                  const int2* __restrict__ list, int64_t len,
                                                                  LevelCtx lc, const R* __restrict__ tnorm,
                                                                  const R* __restrict__ invl, Vec<R, U> u,
                                                                  CVec<R, B> rhs) {
  grid_dependency_sync();
  int64_t pos = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (pos >= len) return;
  const int c0 = CPB * blockIdx.y;
  int2 e = list[pos];
  int loc = e.x;
  if (HHG_OOB(loc, lc.Nt, 41)) return;
  int j = e.y & 0xffff, k = e.y >> 16;
  int64_t off[15];
  neighbour_offsets(DIM, lc.n, j, k, off);
#ifdef HHG_CHECK
  for (int d = 1; d < ndirs<DIM>(); ++d)
    if (HHG_OOB(loc + off[d], lc.Nt, 42)) return;
#endif
  int64_t g[CPB];
  const R* t[CPB];
  R acc[CPB];
#pragma unroll
  for (int c = 0; c < CPB; ++c) {
    const int T = gcells[min(c0 + c, ncells - 1)];  // a short last group repeats its last cell
    g[c] = (int64_t)T * lc.Nt + loc;
    t[c] = tnorm + (size_t)T * 16;
    acc[c] = rhs.get(g[c]) * invl[T];
  }
#pragma unroll
  for (int q = 0; q < npairs<DIM>(); ++q) {
    if (PM >> q & 1) {
#pragma unroll
      for (int c = 0; c < CPB; ++c) acc[c] -= t[c][2 * q + 1] * u.get(g[c] + off[2 * q + 1]);
#pragma unroll
      for (int c = 0; c < CPB; ++c) acc[c] -= t[c][2 * q + 2] * u.get(g[c] + off[2 * q + 2]);
    }
  }
#pragma unroll
  for (int c = 0; c < CPB; ++c)
    if (c0 + c < ncells) u.set(g[c], acc[c]);
}

// Colour offsets of one group's interior lists on one level (m <= 4 colours).
struct ColourOffsets {
  int64_t off[5];
  int m;
};

// Every interior colour of a small cell in one launch: one CTA per cell of the group runs the colours
// in order, each as the list stage above, with a block barrier between colours.  The interior nodes
// of a cell couple only with nodes of the same cell, and the barrier makes a colour's writes visible
// to the CTA before the next colour reads them, so this equals the colour stages one by one.  For
// levels whose per-cell colour lists are short (a few entries per thread).
template <int DIM, int PM, typename R, typename U, typename B>
__global__ void __launch_bounds__(kBlock) k_smooth_interior_cell(const int* __restrict__ gcells,
                                                                 const int2* __restrict__ list, ColourOffsets co,
                                                                 LevelCtx lc, const R* __restrict__ tnorm,
                                                                 const R* __restrict__ invl, Vec<R, U> u,
                                                                 CVec<R, B> rhs) {
  grid_dependency_sync();
  const int T = gcells[blockIdx.x];
  const R* t = tnorm + (size_t)T * 16;
  const R inv = invl[T];
  const int64_t base = (int64_t)T * lc.Nt;
  for (int c = 0; c < co.m; ++c) {
    for (int64_t pos = co.off[c] + threadIdx.x; pos < co.off[c + 1]; pos += blockDim.x) {
      const int2 e = list[pos];
      if (HHG_OOB(e.x, lc.Nt, 43)) continue;
      const int j = e.y & 0xffff, k = e.y >> 16;
      int64_t off[15];
      neighbour_offsets(DIM, lc.n, j, k, off);
      const int64_t g = base + e.x;
      R acc = rhs.get(g) * inv;
#pragma unroll
      for (int q = 0; q < npairs<DIM>(); ++q) {
        if (PM >> q & 1) {
          acc -= t[2 * q + 1] * u.get(g + off[2 * q + 1]);
          acc -= t[2 * q + 2] * u.get(g + off[2 * q + 2]);
        }
      }
      u.set(g, acc);
    }
    __syncthreads();
  }
}

// the per-cell launch pays off while every colour list of every group has at most this many entries
constexpr int64_t kCellInteriorMax = 2 * kBlock;

inline bool interior_per_cell(const LevelData& Lv, const std::vector<Group>& groups) {
  for (size_t gi = 0; gi < groups.size(); ++gi)
    for (int c = 0; c < groups[gi].m; ++c)
      if (Lv.icol_off[gi][c + 1] - Lv.icol_off[gi][c] > kCellInteriorMax) return false;
  return true;
}

inline ColourOffsets colour_offsets(const LevelData& Lv, int gi, int m) {
  ColourOffsets co{};
  co.m = m;
  for (int c = 0; c <= m && c < 5; ++c) co.off[c] = Lv.icol_off[gi][c] - Lv.icol_off[gi][0];
  return co;
}

// macro vertices: never coupled to each other on levels >= 1, so one pass.  One warp per vertex,
// lanes over the vertex's cell copies (scattered loads in parallel), fixed-order shuffle sums.
template <int DIM, typename R, typename U, typename B>
__device__ __forceinline__ void vertex_update(int v, int lane, int nprim, const int* __restrict__ ptr,
                                              const int* __restrict__ cell, const int* __restrict__ locv,
                                              const unsigned char* __restrict__ dir, const LevelCtx& lc,
                                              const R* __restrict__ S, R sscale, const R* __restrict__ pinv,
                                              R isscale, Vec<R, U> u, CVec<R, B> rhs) {
  if (v >= nprim || dir[v]) return;  // uniform across the warp
  CVec<R, U> uc{u.p, u.scale};
  R acc = 0, bs = 0;
  int c0 = ptr[v], c1 = ptr[v + 1];
  int i0, j0, k0;
  prim_position(locv[c0], 1, lc.n, 0, 0, i0, j0, k0);
  R uold = u.get((int64_t)cell[c0] * lc.Nt + packed_index(DIM, lc.n, i0, j0, k0));
  for (int c = c0 + lane; c < c1; c += 32) {
    int i, j, k;
    prim_position(locv[c], 1, lc.n, 0, 0, i, j, k);
    copy_terms<DIM>(S, lc.nzs, cell[c], lc.n, lc.Nt, i, j, k, uc, rhs, acc, bs);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    acc += __shfl_xor_sync(0xffffffffu, acc, o);
    bs += __shfl_xor_sync(0xffffffffu, bs, o);
  }
  // u += (b - A u) / a_ii with 1 / a_ii = pinv (unit level scale) / sscale
  R unew = uold + (bs - sscale * acc) * (pinv[v] * isscale);
  for (int c = c0 + lane; c < c1; c += 32) {
    int i, j, k;
    prim_position(locv[c], 1, lc.n, 0, 0, i, j, k);
    int64_t p = packed_index(DIM, lc.n, i, j, k);
    if (HHG_OOB(p, lc.Nt, 92)) continue;
    u.set((int64_t)cell[c] * lc.Nt + p, unew);
  }
}

template <int DIM, typename R, typename U, typename B>
__global__ void k_smooth_vertex(int nprim, const int* __restrict__ ptr, const int* __restrict__ cell,
                                const int* __restrict__ locv, const unsigned char* __restrict__ dir, LevelCtx lc,
                                const R* __restrict__ S, R sscale, const R* __restrict__ pinv, R isscale, Vec<R, U> u,
                                CVec<R, B> rhs) {
  grid_dependency_sync();
  int v = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  vertex_update<DIM>(v, threadIdx.x & 31, nprim, ptr, cell, locv, dir, lc, S, sscale, pinv, isscale, u, rhs);
}

// Edge stages (even, then odd edge-local index).  Every node of a stage is updated from the values
// at the start of the stage.  Nodes of one stage can couple only next to a shared macro vertex (odd
// edge nodes t = 1, n-1): these "rim" nodes are computed into du and applied by a second kernel.
// All other ("inner") nodes of the stage have no neighbour in the stage, so one pass updates them
// in place.  (The face stages are the face block further down.)
//
// Position of entry q of a stage: rim q -> t in {1, n-1} (odd stage only), inner q -> t = 2q+3
// (odd) or 2q+2 (even); for a primitive with three vertices (a, b) from the given list.
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

// One interface stage (edge parity) on the nodes of nprim primitives.  G lanes
// (a power of two dividing 32) serve one node: lane r takes the copies ptr[e] + r, + r + G, ...,
// and the partial residuals and diagonals are summed over the lanes by an xor butterfly, so every
// lane holds the same sum.  Rim nodes (those that can neighbour another node of the same stage in
// some cell) store their correction in du for k_iface_apply; inner nodes are updated in place.
template <int DIM, int G, typename R, typename U, typename B>
__device__ __forceinline__ void iface_update(int64_t gid, int nprim, int nverts, int parity, int cnt_rim, int cnt_inner,
                                             const int32_t* __restrict__ rim_list,
                                             const int32_t* __restrict__ inner_list, const int* __restrict__ ptr,
                                             const int* __restrict__ cell, const int* __restrict__ locv,
                                             const unsigned char* __restrict__ dir, const LevelCtx& lc,
                                             const R* __restrict__ S, R sscale, const R* __restrict__ pinv,
                                             R isscale, Vec<R, U> u, CVec<R, B> rhs, R* __restrict__ du) {
  int lane = (int)(gid & (G - 1));
  int64_t tid = gid / G;
  int64_t n_rim = (int64_t)nprim * cnt_rim;
  bool rim = tid < n_rim;
  int64_t lt = rim ? tid : tid - n_rim;
  int cnt = rim ? cnt_rim : cnt_inner;
  bool active = rim || lt < (int64_t)nprim * cnt_inner;
  int e = 0, q = 0;
  if (active) {
    e = (int)(lt / cnt);
    q = (int)(lt % cnt);
    if (dir[e]) {
      if (rim && lane == 0) du[tid] = 0;
      active = false;
    }
  }
  int s = 0, t = 0;
  R acc = 0, bs = 0;
  int64_t g0 = -1;
  CVec<R, U> uc{u.p, u.scale};
  if (active) {
    stage_position(nverts, parity, rim, lc.n, q, rim ? rim_list : inner_list, s, t);
    for (int c = ptr[e] + lane; c < ptr[e + 1]; c += G) {
      int i, j, k;
      prim_position(locv[c], nverts, lc.n, s, t, i, j, k);
      int64_t g = copy_terms<DIM>(S, lc.nzs, cell[c], lc.n, lc.Nt, i, j, k, uc, rhs, acc, bs);
      if (g0 < 0) g0 = g;
    }
  }
#pragma unroll
  for (int w = 1; w < G; w <<= 1) {
    acc += __shfl_xor_sync(0xffffffffu, acc, w);
    bs += __shfl_xor_sync(0xffffffffu, bs, w);
  }
  // correction (b - A u) / a_ii with 1 / a_ii = pinv (unit level scale) / sscale; the new value is
  // taken from the first copy (lane 0) and broadcast to the group
  R corr = 0, unew = 0;
  if (active && lane == 0) {
    corr = (bs - sscale * acc) * (pinv[e] * isscale);
    if (!rim) unew = u.get(g0) + corr;
  }
  if (G > 1) unew = __shfl_sync(0xffffffffu, unew, 0, G);
  if (!active) return;
  if (rim) {
    if (lane == 0) du[tid] = corr;
    return;
  }
  for (int c = ptr[e] + lane; c < ptr[e + 1]; c += G) {
    int i, j, k;
    prim_position(locv[c], nverts, lc.n, s, t, i, j, k);
    int64_t p = packed_index(DIM, lc.n, i, j, k);
    if (HHG_OOB(p, lc.Nt, 91)) continue;
    u.set((int64_t)cell[c] * lc.Nt + p, unew);
  }
}

template <int DIM, int G, typename R, typename U, typename B>
__global__ void k_iface_stage(int nprim, int nverts, int parity, int cnt_rim, int cnt_inner,
                              const int32_t* __restrict__ rim_list, const int32_t* __restrict__ inner_list,
                              const int* __restrict__ ptr, const int* __restrict__ cell, const int* __restrict__ locv,
                              const unsigned char* __restrict__ dir, LevelCtx lc, const R* __restrict__ S, R sscale,
                              const R* __restrict__ pinv, R isscale, Vec<R, U> u, CVec<R, B> rhs,
                              R* __restrict__ du) {
  grid_dependency_sync();
  iface_update<DIM, G>((int64_t)blockIdx.x * blockDim.x + threadIdx.x, nprim, nverts, parity, cnt_rim, cnt_inner,
                       rim_list, inner_list, ptr, cell, locv, dir, lc, S, sscale, pinv, isscale, u, rhs, du);
}

// The vertex stage and the even edge stage in one launch: no vertex neighbours an even edge node
// (which sits at least two lattice steps from every macro vertex), so running them together gives
// the results of the two stages in sequence.  Blocks [0, nbv) take the vertices (a warp each), the
// others the even edge nodes (G lanes each, no rim nodes in the even stage).
template <int DIM, int G, typename R, typename U, typename B>
__global__ void k_vertex_edge_even(int nbv, int nv, const int* __restrict__ vptr, const int* __restrict__ vcell,
                                   const int* __restrict__ vloc, const unsigned char* __restrict__ vdir,
                                   const R* __restrict__ vpinv, int ne, int cnt_inner, const int* __restrict__ eptr,
                                   const int* __restrict__ ecell, const int* __restrict__ eloc,
                                   const unsigned char* __restrict__ edir, const R* __restrict__ epinv, LevelCtx lc,
                                   const R* __restrict__ S, R sscale, R isscale, Vec<R, U> u, CVec<R, B> rhs) {
  grid_dependency_sync();
  if ((int)blockIdx.x < nbv) {
    int v = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    vertex_update<DIM>(v, threadIdx.x & 31, nv, vptr, vcell, vloc, vdir, lc, S, sscale, vpinv, isscale, u, rhs);
  } else {
    iface_update<DIM, G>((int64_t)(blockIdx.x - nbv) * blockDim.x + threadIdx.x, ne, 2, 0, 0, cnt_inner, nullptr,
                         nullptr, eptr, ecell, eloc, edir, lc, S, sscale, epinv, isscale, u, rhs, (R*)nullptr);
  }
}

// second phase of a stage for its rim nodes: u += du on every copy (G lanes per node, as above)
template <int DIM, int G, typename R, typename U>
__global__ void k_iface_apply(int nprim, int nverts, int parity, int cnt_rim, const int32_t* __restrict__ rim_list,
                              const int* __restrict__ ptr, const int* __restrict__ cell, const int* __restrict__ locv,
                              const unsigned char* __restrict__ dir, LevelCtx lc, Vec<R, U> u, const R* __restrict__ du) {
  grid_dependency_sync();
  int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int lane = (int)(gid & (G - 1));
  int64_t tid = gid / G;
  if (tid >= (int64_t)nprim * cnt_rim) return;
  int e = (int)(tid / cnt_rim), q = (int)(tid % cnt_rim);
  if (dir[e]) return;
  int s, t;
  stage_position(nverts, parity, true, lc.n, q, rim_list, s, t);
  R d = du[tid];
  for (int c = ptr[e] + lane; c < ptr[e + 1]; c += G) {
    int i, j, k;
    prim_position(locv[c], nverts, lc.n, s, t, i, j, k);
    int64_t p = packed_index(DIM, lc.n, i, j, k);
    if (HHG_OOB(p, lc.Nt, 91)) continue;
    int64_t g = (int64_t)cell[c] * lc.Nt + p;
    u.set(g, u.get(g) + d);
  }
}

// binary64 face blocks with at least this many face nodes visit only the nonzero outside couplings
// (a loop over set bits: fewer DFMA instructions, one memory round trip per term); smaller ones
// unroll all slots (the 384-tet cube has 1.7e6 face nodes at level 6, 4.0e5 at 5, 9.1e4 at 4)
constexpr int64_t kSparseFaceNodes = 100000;

// lanes per interface node: the copy count rounded up to a power of two, at most a warp
inline int iface_lanes(int max_copies) {
  int g = 1;
  while (g < max_copies && g < 32) g <<= 1;
  return g;
}

// launch one interface stage over the primitives of P, then (if it has rim nodes) its apply phase
template <int DIM, int G, typename R, typename U, typename B>
void launch_iface_g(int nprim, const int* ptr, const int* cell, const int* locv, const unsigned char* dir,
                    int nverts, int parity, int cnt_rim, int cnt_inner, const int32_t* rim_list,
                    const int32_t* inner_list, LevelCtx lc, const R* S, R ss, const R* pinv, Vec<R, U> u,
                    CVec<R, B> rhs, R* du, cudaStream_t s) {
  int64_t nodes = (int64_t)nprim * (cnt_rim + cnt_inner);
  hhg_launch(k_iface_stage<DIM, G, R, U, B>, blocks_for(nodes * G), kBlock, 0, s, 
      nprim, nverts, parity, cnt_rim, cnt_inner, rim_list, inner_list, ptr, cell, locv, dir, lc, S, ss, pinv,
      (R)1 / ss, u, rhs, du);
  if (cnt_rim > 0)
    hhg_launch(k_iface_apply<DIM, G, R, U>, blocks_for((int64_t)nprim * cnt_rim * G), kBlock, 0, s, 
        nprim, nverts, parity, cnt_rim, rim_list, ptr, cell, locv, dir, lc, u, du);
}

template <int DIM, typename R, typename U, typename B>
void launch_iface(int lanes, int nprim, const int* ptr, const int* cell, const int* locv, const unsigned char* dir,
                  int nverts, int parity, int cnt_rim, int cnt_inner, const int32_t* rim_list,
                  const int32_t* inner_list, LevelCtx lc, const R* S, R ss, const R* pinv, Vec<R, U> u,
                  CVec<R, B> rhs, R* du, cudaStream_t s) {
#define HHG_IFACE_G(GL)                                                                                          \
  launch_iface_g<DIM, GL, R, U, B>(nprim, ptr, cell, locv, dir, nverts, parity, cnt_rim, cnt_inner, rim_list, \
                                   inner_list, lc, S, ss, pinv, u, rhs, du, s)
  switch (lanes) {
    case 1: HHG_IFACE_G(1); break;
    case 2: HHG_IFACE_G(2); break;
    case 4: HHG_IFACE_G(4); break;
    case 8: HHG_IFACE_G(8); break;
    case 16: HHG_IFACE_G(16); break;
    default: HHG_IFACE_G(32); break;
  }
#undef HHG_IFACE_G
}

// ---------------------------------------------------------------- face block (3D; Gauss-Seidel of Alg. 4)
//
// The three face colours form one block: every macro face is smoothed on its own, Gauss-Seidel over
// its interior nodes in colour order (a + 2b) mod 3, with every node outside the face (edges,
// vertices, cell interiors, the nodes of other faces) at its value from the start of the block.
// Two kernels: k_face_ext sums, per face node, b - A u over the couplings that leave the face
// (over both cell copies), from the values at the start of the block; k_face_gs then runs the
// colour sweeps of one face in one CTA on the face's own values held in shared memory, using the
// face's in-plane couplings (summed over its copies), and writes the result to every copy.
// Face-interior nodes (a, b >= 1, a + b <= n - 1) are indexed (a, b) -> face_pos in the
// per-face vectors.

__device__ __forceinline__ int face_pos(int n, int a, int b) {
  return (b - 1) * (n - 2) - (b - 1) * (b - 2) / 2 + (a - 1);
}

__device__ __forceinline__ bool face_interior(int n, int a, int b) { return a >= 1 && b >= 1 && a + b <= n - 1; }

// in-plane directions of a face in its local (a, b) coordinates
__device__ __forceinline__ void face_dir(int q, int& da, int& db) {
  da = (q == 0 || q == 4) ? 1 : ((q == 1 || q == 5) ? -1 : 0);
  db = (q == 2 || q == 5) ? 1 : ((q == 3 || q == 4) ? -1 : 0);
}

// stencil slot of lattice vector v (0 if v is not a lattice direction)
__device__ __forceinline__ int slot_of_vec(int di, int dj, int dk) {
#pragma unroll
  for (int s = 1; s < 15; ++s) {
    int a, b, c;
    dir_vec(3, s, a, b, c);
    if (a == di && b == dj && c == dk) return s;
  }
  return 0;
}

// cell-local slot of face direction q for the copy whose local face vertices are packed in loc
__device__ __forceinline__ int face_dir_slot(int loc, int q) {
  int a0 = loc & 3, a1 = (loc >> 2) & 3, a2 = (loc >> 4) & 3;
  int x0, y0, z0, x1, y1, z1, x2, y2, z2;
  local_vertex_vec(a0, x0, y0, z0);
  local_vertex_vec(a1, x1, y1, z1);
  local_vertex_vec(a2, x2, y2, z2);
  int da, db;
  face_dir(q, da, db);
  return slot_of_vec(da * (x1 - x0) + db * (x2 - x0), da * (y1 - y0) + db * (y2 - y0), da * (z1 - z0) + db * (z2 - z0));
}

template <int G, bool SPARSE, typename R, typename U, typename B>
__global__ void k_face_ext(int nprim, int nf, const int32_t* __restrict__ fnodes, const int* __restrict__ ptr,
                           const int* __restrict__ cell, const int* __restrict__ locv,
                           const unsigned char* __restrict__ dir, LevelCtx lc, const R* __restrict__ S, R sscale,
                           CVec<R, U> u, CVec<R, B> rhs, R* __restrict__ E) {
  grid_dependency_sync();
  int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int lane = (int)(gid & (G - 1));
  int64_t tid = gid / G;
  bool active = tid < (int64_t)nprim * nf;
  int e = 0, a = 0, b = 0;
  if (active) {
    e = (int)(tid / nf);
    int32_t ab = fnodes[tid % nf];
    a = ab & 0xffff;
    b = ab >> 16;
    if (dir[e]) active = false;
  }
  R acc = 0, bs = 0;
  if (active) {
    const int n = lc.n;
    for (int c = ptr[e] + lane; c < ptr[e + 1]; c += G) {
      int loc = locv[c];
      int i, j, k;
      prim_position(loc, 3, n, a, b, i, j, k);
      // leave out the node itself and its in-plane neighbours that are face-interior nodes
      uint32_t excl = 1u;
#pragma unroll
      for (int q = 0; q < 6; ++q) {
        int da, db;
        face_dir(q, da, db);
        if (face_interior(n, a + da, b + db)) excl |= 1u << face_dir_slot(loc, q);
      }
      const int T = cell[c];
      int t = boundary_type(3, n, i, j, k);
      int64_t p = packed_index(3, n, i, j, k);
      if (HHG_OOB(p, lc.Nt, 33)) continue;
      int64_t g = (int64_t)T * lc.Nt + p;
      uint32_t vm = valid_dirs_tab(3, t) & lc.nzs[T * kMaxTypes + t] & ~excl;
      const R* s = S + (size_t)T * kStencilStride + t * kMaxDirs;
      R x = 0;
      if (SPARSE) {
        PlaneBasis pb = plane_basis(3, n, k);
        for (uint32_t mm = vm; mm; mm &= mm - 1) {
          int d = __ffs(mm) - 1;
          int64_t o = dir_offset(3, d, pb.m, j, pb.Tm, pb.Tm1);
          if (HHG_OOB(p + o, lc.Nt, 34)) continue;
          x += s[d] * u.get(g + o);
        }
      } else {
        int64_t off[15];
        neighbour_offsets(3, n, j, k, off);
        mask_offsets(3, vm, off);
#pragma unroll
        for (int d = 1; d < 15; ++d)
          if ((vm >> d & 1) && !HHG_OOB(p + off[d], lc.Nt, 34)) x += s[d] * u.get(g + off[d]);
      }
      acc += x;
      bs += rhs.get(g);
    }
  }
#pragma unroll
  for (int w = 1; w < G; w <<= 1) {
    acc += __shfl_xor_sync(0xffffffffu, acc, w);
    bs += __shfl_xor_sync(0xffffffffu, bs, w);
  }
  if (active && lane == 0) E[(int64_t)e * nf + face_pos(lc.n, a, b)] = bs - sscale * acc;
}

// FPC faces per CTA (FPC = 1: the CTA's kBlock threads sweep one face, synchronised by block
// barriers; FPC = 8: one warp per face, warp barriers, for levels whose faces have few nodes).
// fcol: colour offsets of fnodes (colour c entries [fcol.c, fcol.c+1)); W: the face's six in-plane
// couplings (unit level scale, summed over copies); pinv: 1 / diagonal (unit scale); isscale = 1 /
// level scale.  work: 2 nf values of scratch per face when they do not fit in shared memory
// (nullptr: shared memory, 2 nf values per face of the CTA).
template <int FPC, typename R, typename U>
__global__ void __launch_bounds__(kBlock) k_face_gs(int nprim, int nf, int4 fcol, const int32_t* __restrict__ fnodes,
                                                    const int* __restrict__ ptr, const int* __restrict__ cell,
                                                    const int* __restrict__ locv, const unsigned char* __restrict__ dir,
                                                    LevelCtx lc, const R* __restrict__ W, const R* __restrict__ pinv,
                                                    R isscale, Vec<R, U> u, const R* __restrict__ E, R* work) {
  grid_dependency_sync();
  static_assert(FPC == 1 || kBlock / FPC == 32, "one CTA or one warp per face");
  constexpr int TPF = kBlock / FPC;  // threads per face
  extern __shared__ __align__(16) unsigned char smem[];
  const int grp = (int)threadIdx.x / TPF, t = (int)threadIdx.x % TPF;
  const int e = (int)blockIdx.x * FPC + grp;
  if (e >= nprim || dir[e]) return;  // uniform across the face's threads (the CTA or the warp)
  auto sync = [] {
    if (FPC == 1) __syncthreads();
    else __syncwarp();
  };
  const int n = lc.n;
  R* uf = work ? work + (int64_t)e * 2 * nf : (R*)smem + (size_t)grp * 2 * nf;
  R* ef = uf + nf;
  const int c0 = ptr[e];
  const int loc0 = locv[c0];
  const int64_t base0 = (int64_t)cell[c0] * lc.Nt;
  // gather the face's values (copy 0) and outside sums, four per thread in flight
  constexpr int kUnroll = 4;
  for (int q0 = t; q0 < nf; q0 += kUnroll * TPF) {
    R uv[kUnroll], ev[kUnroll];
    int ps[kUnroll];
#pragma unroll
    for (int r = 0; r < kUnroll; ++r) {
      int q = q0 + r * TPF;
      ps[r] = -1;
      if (q < nf) {
        int32_t ab = fnodes[q];
        int a = ab & 0xffff, b = ab >> 16;
        int i, j, k;
        prim_position(loc0, 3, n, a, b, i, j, k);
        int pos = face_pos(n, a, b);
        int64_t p = packed_index(3, n, i, j, k);
        ps[r] = pos;
        uv[r] = HHG_OOB(p, lc.Nt, 35) ? (R)0 : u.get(base0 + p);
        ev[r] = E[(int64_t)e * nf + pos];
      }
    }
#pragma unroll
    for (int r = 0; r < kUnroll; ++r)
      if (ps[r] >= 0) {
        uf[ps[r]] = uv[r];
        ef[ps[r]] = ev[r] * isscale;
      }
  }
  R w[6];
#pragma unroll
  for (int q = 0; q < 6; ++q) w[q] = W[(int64_t)e * 8 + q];
  const R pv = pinv[e];
  sync();
  const int cb[4] = {fcol.x, fcol.y, fcol.z, fcol.w};
  for (int col = 0; col < 3; ++col) {
    for (int q = cb[col] + t; q < cb[col + 1]; q += TPF) {
      int32_t ab = fnodes[q];
      int a = ab & 0xffff, b = ab >> 16;
      int pos = face_pos(n, a, b);
      R v = ef[pos];
#pragma unroll
      for (int d = 0; d < 6; ++d) {
        int da, db;
        face_dir(d, da, db);
        if (face_interior(n, a + da, b + db)) v -= w[d] * uf[face_pos(n, a + da, b + db)];
      }
      uf[pos] = v * pv;
    }
    sync();
  }
  for (int c = c0; c < ptr[e + 1]; ++c) {
    const int loc = locv[c];
    const int64_t base = (int64_t)cell[c] * lc.Nt;
    for (int q = t; q < nf; q += TPF) {
      int32_t ab = fnodes[q];
      int a = ab & 0xffff, b = ab >> 16;
      int i, j, k;
      prim_position(loc, 3, n, a, b, i, j, k);
      int64_t p = packed_index(3, n, i, j, k);
      if (HHG_OOB(p, lc.Nt, 36)) continue;
      u.set(base + p, uf[face_pos(n, a, b)]);
    }
  }
}

// Launch the vertex stage and the even edge stage together (k_vertex_edge_even).
template <int DIM, typename R, typename U, typename B>
void launch_vertex_edge_even(const Prims& V, const Prims& Ed, int n, LevelCtx lc, const R* S, R ss, const R* vpinv,
                             const R* epinv, Vec<R, U> u, CVec<R, B> rhs, cudaStream_t s) {
  const int cnt_inner = n / 2 - 1;  // even edge-local indices 2, 4, .., n-2
  const unsigned nbv = blocks_for((int64_t)V.count * 32);
  const int ne = cnt_inner > 0 ? Ed.count : 0;
  const int G = iface_lanes(Ed.max_copies);
  const unsigned nbe = blocks_for((int64_t)ne * (cnt_inner > 0 ? cnt_inner : 0) * G);
  if (nbv + nbe == 0) return;
#define HHG_VE(GL)                                                                                                    \
  hhg_launch(k_vertex_edge_even<DIM, GL, R, U, B>, nbv + nbe, kBlock, 0, s, (int)nbv, V.count, V.d_ptr, V.d_cell,   \
             V.d_loc, V.d_dir, vpinv, ne, cnt_inner, Ed.d_ptr, Ed.d_cell, Ed.d_loc, Ed.d_dir, epinv, lc, S, ss,     \
             (R)1 / ss, u, rhs)
  switch (G) {
    case 1: HHG_VE(1); break;
    case 2: HHG_VE(2); break;
    case 4: HHG_VE(4); break;
    case 8: HHG_VE(8); break;
    case 16: HHG_VE(16); break;
    default: HHG_VE(32); break;
  }
#undef HHG_VE
}

inline int4 fcol4(const LevelData& Lv) {
  return make_int4((int)Lv.fcol_off[0], (int)Lv.fcol_off[1], (int)Lv.fcol_off[2], (int)Lv.fcol_off[3]);
}

// Launch the face block on one level: E in `E` (P.count x nf values), the per-face sweeps in shared
// memory when 2 nf values fit (else in `work`, P.count x 2 nf values).
template <typename R, typename U, typename B>
void launch_face_block(const Prims& P, const LevelData& Lv, LevelCtx lc, const R* S, R ss, const R* W,
                       const R* pinv, Vec<R, U> u, CVec<R, B> rhs, R* E, R* work, bool sparse, cudaStream_t s) {
  const int nf = (int)Lv.fcol_off[3];
  if (P.count == 0 || nf == 0) return;
  const int64_t nodes = (int64_t)P.count * nf;
  CVec<R, U> uc{u.p, u.scale};
  const int G = iface_lanes(P.max_copies);
#define HHG_FACE_EXT(GL, SP)                                                                                       \
  hhg_launch(k_face_ext<GL, SP, R, U, B>, blocks_for(nodes * GL), kBlock, 0, s, P.count, nf, Lv.d_fcol, P.d_ptr, \
             P.d_cell, P.d_loc, P.d_dir, lc, S, ss, uc, rhs, E)
  if (G == 1) {
    if (sparse) HHG_FACE_EXT(1, true);
    else HHG_FACE_EXT(1, false);
  } else {
    if (sparse) HHG_FACE_EXT(2, true);
    else HHG_FACE_EXT(2, false);
  }
#undef HHG_FACE_EXT
  // faces with few nodes: one warp per face, eight faces per CTA
  constexpr int kFacesPerWarpCta = kBlock / 32;
  if (nf <= 64) {
    const size_t smem8 = (size_t)kFacesPerWarpCta * 2 * nf * sizeof(R);
    hhg_launch(k_face_gs<kFacesPerWarpCta, R, U>, (unsigned)((P.count + kFacesPerWarpCta - 1) / kFacesPerWarpCta),
               kBlock, smem8, s, P.count, nf, fcol4(Lv), Lv.d_fcol, P.d_ptr, P.d_cell, P.d_loc, P.d_dir, lc, W, pinv,
               (R)1 / ss, u, (const R*)E, (R*)nullptr);
    return;
  }
  const size_t smem = 2 * (size_t)nf * sizeof(R);
  const bool fits = smem <= kMaxTileSmem;
  if (fits && smem > 48 * 1024)
    cudaFuncSetAttribute(k_face_gs<1, R, U>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMaxTileSmem);
  hhg_launch(k_face_gs<1, R, U>, (unsigned)P.count, kBlock, fits ? smem : 0, s, P.count, nf, fcol4(Lv), Lv.d_fcol,
             P.d_ptr, P.d_cell, P.d_loc, P.d_dir, lc, W, pinv, (R)1 / ss, u, (const R*)E, fits ? (R*)nullptr : work);
}

// ---------------------------------------------------------------- residual, restriction (V-cycle of Alg. 4; transfers of Sec. 4.4)

// list segments of k_residual_list for one group on one level: directly after a sweep the last
// interior colour's entries are zeroed instead of computed
struct ResidualSegments {
  const int2* ilist;
  int64_t ncomp, nzero;
  unsigned bcomp, bzero;
};
inline ResidualSegments residual_segments(const LevelData& Lv, const Group& G, int gi, bool after_sweep) {
  const std::vector<int64_t>& off = Lv.icol_off[gi];
  int64_t a = off[0], z = off[G.m - 1], b = off[G.m];
  ResidualSegments r;
  r.ilist = Lv.d_icol + a;
  r.ncomp = after_sweep ? z - a : b - a;
  r.nzero = after_sweep ? b - z : 0;
  r.bcomp = blocks_for(r.ncomp);
  r.bzero = blocks_for(r.nzero);
  return r;
}

// Partial residual r = b - A u on every closure node of the group's cells (grid.y), zero on
// Dirichlet rows, from node lists in three block-uniform segments: blocks [0, bcomp) take interior list entries [0, ncomp) with the compile-time stencil
// pattern PM; blocks [bcomp, bcomp + bzero) write 0 at entries [ncomp, ncomp + nzero) (the interior
// colour updated last, directly after a sweep); the remaining blocks take the boundary-type nodes
// (list sorted by type, so a warp mostly shares one slot mask), zero on Dirichlet types.
template <int DIM, int PM, int CPB, bool SPARSE, typename R, typename U, typename B, typename O>
__global__ void __launch_bounds__(kBlock) k_residual_list(const int* __restrict__ gcells, int ncells, LevelCtx lc,
                                                          const R* __restrict__ S, const uint16_t* __restrict__ dirmask,
                                                          R sscale, CVec<R, U> u, CVec<R, B> rhs, O* __restrict__ out,
                                                          const int2* __restrict__ ilist, int64_t ncomp, int64_t nzero,
                                                          const int2* __restrict__ blist, int64_t nbnd, unsigned bcomp,
                                                          unsigned bzero) {
  grid_dependency_sync();
  const int c0 = CPB * blockIdx.y;
  int Ts[CPB];
#pragma unroll
  for (int c = 0; c < CPB; ++c) Ts[c] = gcells[min(c0 + c, ncells - 1)];  // a short last group repeats
  unsigned bx = blockIdx.x;
  if (bx < bcomp) {
    int64_t pos = (int64_t)bx * blockDim.x + threadIdx.x;
    if (pos >= ncomp) return;
    int2 e = ilist[pos];
    if (HHG_OOB(e.x, lc.Nt, 52)) return;
    int j = e.y & 0xffff, k = e.y >> 16;
    int64_t off[15];
    neighbour_offsets(DIM, lc.n, j, k, off);
    int64_t g[CPB];
    const R* st[CPB];
    R acc[CPB];
#pragma unroll
    for (int c = 0; c < CPB; ++c) {
      g[c] = (int64_t)Ts[c] * lc.Nt + e.x;
      st[c] = S + (size_t)Ts[c] * kStencilStride;  // interior type 0
      acc[c] = st[c][0] * u.get(g[c]);
    }
#pragma unroll
    for (int q = 0; q < npairs<DIM>(); ++q) {
      if (PM >> q & 1) {
#pragma unroll
        for (int c = 0; c < CPB; ++c) acc[c] += st[c][2 * q + 1] * u.get(g[c] + off[2 * q + 1]);
#pragma unroll
        for (int c = 0; c < CPB; ++c) acc[c] += st[c][2 * q + 2] * u.get(g[c] + off[2 * q + 2]);
      }
    }
#pragma unroll
    for (int c = 0; c < CPB; ++c)
      if (c0 + c < ncells) out[g[c]] = (dirmask[Ts[c]] & 1) ? (O)0 : (O)(rhs.get(g[c]) - sscale * acc[c]);
  } else if (bx < bcomp + bzero) {
    int64_t pos = (int64_t)(bx - bcomp) * blockDim.x + threadIdx.x;
    if (pos >= nzero) return;
    int loc = ilist[ncomp + pos].x;
    if (HHG_OOB(loc, lc.Nt, 53)) return;
#pragma unroll
    for (int c = 0; c < CPB; ++c)
      if (c0 + c < ncells) out[(int64_t)Ts[c] * lc.Nt + loc] = (O)0;
  } else {
    int64_t pos = (int64_t)(bx - bcomp - bzero) * blockDim.x + threadIdx.x;
    if (pos >= nbnd) return;
    int2 e = blist[pos];
    if (HHG_OOB(e.x, lc.Nt, 54)) return;
    int i, j, k;
    decode(e.y, i, j, k);
    const int t = boundary_type(DIM, lc.n, i, j, k);
#pragma unroll
    for (int c = 0; c < CPB; ++c) {
      if (c0 + c >= ncells) continue;
      const int T = Ts[c];
      const int64_t g = (int64_t)T * lc.Nt + e.x;
      if (dirmask[T] >> t & 1) {
        out[g] = (O)0;
        continue;
      }
      uint32_t vm = valid_dirs_tab(DIM, t) & lc.nzs[T * kMaxTypes + t];
      const R* s = S + (size_t)T * kStencilStride + t * kMaxDirs;
      R acc = s[0] * u.get(g);
      if (SPARSE) {  // binary64: only the nonzero terms (DFMA-bound)
        PlaneBasis pb = plane_basis(DIM, lc.n, k);
        for (uint32_t mm = vm & ~1u; mm; mm &= mm - 1) {
          int d = __ffs(mm) - 1;
          int64_t o = dir_offset(DIM, d, pb.m, j, pb.Tm, pb.Tm1);
          if (HHG_OOB(e.x + o, lc.Nt, 55)) continue;
          acc += s[d] * u.get(g + o);
        }
      } else {  // binary32: every slot unrolled, the loads issued together
        int64_t off[15];
        neighbour_offsets(DIM, lc.n, j, k, off);
        mask_offsets(DIM, vm, off);
#pragma unroll
        for (int d = 1; d < ndirs<DIM>(); ++d)
          if ((vm >> d & 1) && !HHG_OOB(e.x + off[d], lc.Nt, 55)) acc += s[d] * u.get(g + off[d]);
      }
      out[g] = (O)(rhs.get(g) - sscale * acc);
    }
  }
}

// coarse partial rhs = P^T (fine partial residual), per cell: r_c(q) = r_f(2q) + 1/2 sum_d r_f(2q+d).
// zero (may be null): a coarse-level vector set to 0 at every node on the way (the coarse
// correction's starting value, which would otherwise take a memset of its own).
template <int DIM, typename R, typename I, typename O, typename Z = O>
__global__ void k_restrict(LevelCtx fc, LevelCtx cc, const uint16_t* __restrict__ dirmask, const I* __restrict__ rf,
                           O* __restrict__ rcv, Z* __restrict__ zero = nullptr) {
  grid_dependency_sync();
  int64_t loc = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (loc >= cc.Nt) return;
  int T = blockIdx.y;
  if (zero) zero[(int64_t)T * cc.Nt + loc] = Z(0.0f);
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

// ---------------------------------------------------------------- prolongation, FMG transition (Alg. 4; interpolation of Sec. 4.4)


// I u_c at fine node loc of cell T from the level's interpolation table (fc.itab), and the node's
// boundary type: (u_c[a] + u_c[b]) / 2, with a = b at a coarse node (exact: (x + x) / 2 = x)
template <typename R, typename C>
__device__ __forceinline__ R interp_tab(const LevelCtx& fc, const LevelCtx& cc, int T, int64_t loc, const C& uc,
                                        int& t) {
  const int2 e = fc.itab[loc];
  t = e.x >> 27;
  const int ia = e.x & 0x7ffffff, ib = e.y;
  if (HHG_OOB(ia, cc.Nt, 23) || HHG_OOB(ib, cc.Nt, 24)) return (R)0;
  const int64_t gc = (int64_t)T * cc.Nt;
  return (R)0.5 * (uc.get(gc + ia) + uc.get(gc + ib));
}

// u_f += I u_c on free nodes.  The end points and the boundary type come from the level's
// interpolation table (the index arithmetic per node kept the kernel issue-bound): I u_c at a node
// is (u_c[a] + u_c[b]) / 2, with a = b at a coarse node (exact: (x + x) / 2 = x).
template <int DIM, typename R, typename UC, typename UF>
__global__ void k_prolong_add(LevelCtx fc, LevelCtx cc, const uint16_t* __restrict__ dirmask, CVec<R, UC> uc,
                              Vec<R, UF> uf) {
  grid_dependency_sync();
  int64_t loc = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (loc >= fc.Nt) return;
  int T = blockIdx.y;
  int t;
  const R v = interp_tab<R>(fc, cc, T, loc, uc, t);
  if (dirmask[T] >> t & 1) return;
  const int64_t g = (int64_t)T * fc.Nt + loc;
  uf.set(g, uf.get(g) + v);
}

// FMG transition: u_{l+1} = I u_l (Dirichlet nodes from g_L, or 0 if gL is null), w_l = u_{l+1}
template <int DIM>
__global__ void k_fmg_prolong(LevelCtx fc, LevelCtx cc, int nL, int64_t NtL, int shift, const double* __restrict__ gL,
                              const uint16_t* __restrict__ dirmask, const double* __restrict__ uc,
                              double* __restrict__ uf, double* __restrict__ w) {
  grid_dependency_sync();
  int64_t loc = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (loc >= fc.Nt) return;
  int T = blockIdx.y;
  int t;
  double v = interp_tab<double>(fc, cc, T, loc, CVec<double, double>{uc, nullptr}, t);
  if (dirmask[T] >> t & 1) {
    int i, j, k;
    decode(fc.ijk[loc], i, j, k);
    int64_t q = packed_index(DIM, nL, (int64_t)i << shift, (int64_t)j << shift, (int64_t)k << shift);
    if (HHG_OOB(q, NtL, 81)) return;
    v = gL ? gL[(int64_t)T * NtL + q] : 0.0;
  }
  int64_t g = (int64_t)T * fc.Nt + loc;
  uf[g] = v;
  if (w) w[g] = v;
}

// the estimator's difference u_L - I w_c in binary64, stored as its binary32 hi/lo pair (df_split)
// for k_node_form_pair
template <int DIM>
__global__ void k_prolong_diff_pair(LevelCtx fc, LevelCtx cc, const double* __restrict__ vc,
                                    const double* __restrict__ minuend, float2* __restrict__ xf) {
  grid_dependency_sync();
  int64_t loc = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (loc >= fc.Nt) return;
  int T = blockIdx.y;
  int t;
  int64_t g = (int64_t)T * fc.Nt + loc;
  double v = interp_tab<double>(fc, cc, T, loc, CVec<double, double>{vc, nullptr}, t);
  xf[g] = df_split(minuend[g] - v);
}

// plain interpolation v_f = I v_c (all nodes)
template <int DIM>
// vf = I vc, or vf = minuend - I vc when minuend is given (the estimator's difference u_L - I w)
__global__ void k_prolong(LevelCtx fc, LevelCtx cc, const double* __restrict__ vc, double* __restrict__ vf,
                          const double* __restrict__ minuend) {
  grid_dependency_sync();
  int64_t loc = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (loc >= fc.Nt) return;
  int T = blockIdx.y;
  int t;
  int64_t g = (int64_t)T * fc.Nt + loc;
  double v = interp_tab<double>(fc, cc, T, loc, CVec<double, double>{vc, nullptr}, t);
  vf[g] = minuend ? minuend[g] - v : v;
}

// ---------------------------------------------------------------- direct coarse solve (Alg. 4; the converged limit of Sec. 5.4's CG)

// One CTA: residual of the free macro vertices (summed over cell copies), c = A_ff^{-1} r, update
// every copy.  n0f <= 16384 (checked at set-up); the residual vector lives in shared memory.
template <int DIM>
__global__ void __launch_bounds__(1024) k_coarse(int n0f, const int* __restrict__ cf, const int* __restrict__ ptr,
                                                 const int* __restrict__ cell, const int* __restrict__ locv,
                                                 LevelCtx lc, const double* __restrict__ S,
                                                 const double* __restrict__ rhs, double* __restrict__ u,
                                                 const double* __restrict__ Ainv) {
  grid_dependency_sync();
  extern __shared__ double r[];
  CVec<double, double> uc{u, nullptr};
  CVec<double, double> rc{rhs, nullptr};
  {
    // residual of each free coarse vertex: one warp per vertex, lanes over its cell copies
    int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int q = warp; q < n0f; q += nw) {
      int v = cf[q];
      double acc = 0, bs = 0;
      for (int c = ptr[v] + lane; c < ptr[v + 1]; c += 32) {
        int i, j, k;
        prim_position(locv[c], 1, lc.n, 0, 0, i, j, k);
        copy_terms<DIM>(S, lc.nzs, cell[c], lc.n, lc.Nt, i, j, k, uc, rc, acc, bs);
      }
      double res = bs - acc;  // level 0: unit stiffness scale
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
    // every lane holds the sum: the lanes update the vertex's copies
    int v = cf[row];
    for (int c = ptr[v] + lane; c < ptr[v + 1]; c += 32) {
      int i, j, k;
      prim_position(locv[c], 1, lc.n, 0, 0, i, j, k);
      int64_t p = packed_index(DIM, lc.n, i, j, k);
      if (HHG_OOB(p, lc.Nt, 93)) continue;
      u[(int64_t)cell[c] * lc.Nt + p] += acc;
    }
  }
}

// ---------------------------------------------------------------- reductions (ErrorEstimate of Alg. 4, Eqs. 4.5 and 4.14; adjoint gradients)

// Fixed-order sum of one value per thread over a block of kBlock threads: xor butterflies inside each
// warp, then the warp sums combined by the first warp with butterflies over kBlock / 32 lanes.  Every
// thread of the block must call it (no thread may have returned); thread 0 gets the sum.  The order
// of the additions depends on the thread index only, so the result is the same on every run.
__device__ __forceinline__ double block_sum_fixed(double v, double* wsum) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0;
  if (threadIdx.x < 32) {
    t = threadIdx.x < kBlock / 32 ? wsum[threadIdx.x] : 0.0;
#pragma unroll
    for (int o = kBlock / 64; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  }
  return t;
}

// Per node p of a cell's closure (one node per thread, one grid row per cell), the symmetric-form
// contribution
//   c_p = S[t][0] x_p y_p + sum_{d positive, valid} S[t][d] (x_p y_{p+d} + x_{p+d} y_p),
// with x = y = a - b (b may be null) for the mass form, or x = a, y = b for a bilinear form.  Summed
// over the closure this is x^T S_T y, because the partial stencil of a cell is symmetric (the entry
// p->p+d seen from p equals the entry p+d->p seen from p+d: both sum the cell's elements on that
// edge), so each lattice edge is visited once.  Each thread adds the contributions of kFormNodes
// nodes (block stride apart), each block sums its threads' values in a fixed order
// (block_sum_fixed) into part[cell][block], and k_cell_sum adds a cell's block sums.
constexpr int kFormNodes = 8;

template <int DIM, bool DIFF>
__global__ void __launch_bounds__(kBlock) k_node_form(LevelCtx lc, const double* __restrict__ tab,
                                                      const double* __restrict__ a, const double* __restrict__ b,
                                                      double* __restrict__ part) {
  grid_dependency_sync();
  __shared__ double wsum[kBlock / 32];
  int T = blockIdx.y;
  double tsum = 0;
  for (int r = 0; r < kFormNodes; ++r) {
    const int64_t loc = ((int64_t)blockIdx.x * kFormNodes + r) * kBlock + threadIdx.x;
    double sum = 0;
    if (loc < lc.Nt) {
      int i, j, k;
      decode(lc.ijk[loc], i, j, k);
      int t = boundary_type(DIM, lc.n, i, j, k);
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
      // x_p (M y)_p restricted to the half stencil: s0 x_p y_p + sum_{+d} s_d (x_p y_q + x_q y_p),
      // grouped as x_p (s0 y_p + sum s_d y_q) + y_p sum s_d x_q (one accumulator when x = y)
      double ay = 0, ax = 0;
#pragma unroll
      for (int q = 0; q < npairs<DIM>(); ++q) {
        int d = 2 * q + 1;
        if (!(vm >> d & 1)) continue;
        if (HHG_OOB(loc + off[d], lc.Nt, 13)) continue;
        if (DIFF) {
          double xq = a[g + off[d]];
          if (b) xq -= b[g + off[d]];
          ay += s[d] * xq;
        } else {
          ay += s[d] * b[g + off[d]];
          ax += s[d] * a[g + off[d]];
        }
      }
      sum = DIFF ? xp * (s[0] * xp + 2.0 * ay) : xp * (s[0] * yp + ay) + yp * ax;
    }
    tsum += sum;
  }
  const double tot = block_sum_fixed(tsum, wsum);
  if (threadIdx.x == 0) part[(int64_t)T * gridDim.x + blockIdx.x] = tot;
}

// The estimator's squared mass norm of a difference vector x per cell, in binary32 pairs: x is read
// as the hi/lo pairs written by k_sub_pair / k_prolong_diff_pair, the mass stencil as hi/lo pairs
// of its binary64 values, and x_p (s0 x_p + 2 sum s_d x_q) over the half stencil is accumulated with
// exact products and sums (dfloat.cuh), about 2^-44 relative per node.  Same blocking and block
// sums as k_node_form (one binary64 value per block, fixed order).
template <int DIM>
__global__ void __launch_bounds__(kBlock) k_node_form_pair(LevelCtx lc, const float2* __restrict__ tab,
                                                           const float2* __restrict__ x, double* __restrict__ part) {
  grid_dependency_sync();
  __shared__ double wsum[kBlock / 32];
  const int T = blockIdx.y;
  DfAcc tsum;
  for (int r = 0; r < kFormNodes; ++r) {
    const int64_t loc = ((int64_t)blockIdx.x * kFormNodes + r) * kBlock + threadIdx.x;
    if (loc < lc.Nt) {
      int i, j, k;
      decode(lc.ijk[loc], i, j, k);
      const int t = boundary_type(DIM, lc.n, i, j, k);
      const int64_t g = (int64_t)T * lc.Nt + loc;
      int64_t off[15];
      neighbour_offsets(DIM, lc.n, j, k, off);
      const uint32_t vm = valid_dirs_tab(DIM, t);
      mask_offsets(DIM, vm, off);
      const float2* s = tab + (size_t)T * kStencilStride + t * kMaxDirs;
      const float2 xp = x[g];
      float2 xq[npairs<DIM>()];
#pragma unroll
      for (int q = 0; q < npairs<DIM>(); ++q) {
        const int d = 2 * q + 1;
        const bool ok = (vm >> d & 1) && !HHG_OOB(loc + off[d], lc.Nt, 13);
        xq[q] = ok ? x[g + off[d]] : make_float2(0.f, 0.f);
      }
      DfAcc ay;
#pragma unroll
      for (int q = 0; q < npairs<DIM>(); ++q) ay.add_prod(s[2 * q + 1], xq[q]);
      ay.hi = __fmul_rn(ay.hi, 2.f);  // exact
      ay.lo = __fmul_rn(ay.lo, 2.f);
      ay.add_prod(s[0], xp);
      tsum.add_prod(xp, ay.value());
    }
  }
  // warp butterflies on pairs (binary32 pipe), one binary64 value per warp, then as block_sum_fixed
  float2 v = tsum.value();
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    DfAcc a;
    a.hi = v.x;
    a.lo = v.y;
    a.add(make_float2(__shfl_xor_sync(0xffffffffu, v.x, o), __shfl_xor_sync(0xffffffffu, v.y, o)));
    v = a.value();
  }
  if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = df_to_double(v);
  __syncthreads();
  if (threadIdx.x < 32) {
    double t = threadIdx.x < kBlock / 32 ? wsum[threadIdx.x] : 0.0;
#pragma unroll
    for (int o = kBlock / 64; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (threadIdx.x == 0) part[(int64_t)T * gridDim.x + blockIdx.x] = t;
  }
}

// ---------------------------------------------------------------- operators for testing / adjoint

// out = scale * Stab_T in (partial rows) on all closure nodes; with inS: zero for cells not in S,
// factor `fac`, zero Dirichlet rows
template <int DIM>
__global__ void k_apply_partial(LevelCtx lc, const double* __restrict__ tab, double scale,
                                const double* __restrict__ in, double* __restrict__ out,
                                const unsigned char* __restrict__ inS, const uint16_t* __restrict__ dirmask) {
  grid_dependency_sync();
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
  grid_dependency_sync();
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
  grid_dependency_sync();
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
