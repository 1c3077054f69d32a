// Binary64 launchers of the HHG FMG (Alg. 4): right-hand sides, stage-ordered Gauss-Seidel,
// residual + restriction, prolongation, the direct coarse solve and the per-cell reductions of
// the error estimator.  The kernel templates live in kernels_impl.cuh.
#include <cstdio>

#include "internal.h"
#include "kernels_impl.cuh"

namespace hhg {

// One block per cell: the cell's np block sums (from k_node_form) added in a fixed order (strided
// per-thread sums, then block_sum_fixed).
__global__ void __launch_bounds__(kBlock) k_cell_sum(int64_t np, double scale, const double* __restrict__ part,
                                                     double* __restrict__ out) {
  grid_dependency_sync();
  __shared__ double wsum[kBlock / 32];
  int T = blockIdx.x;
  const double* c = part + (int64_t)T * np;
  double acc = 0;
  for (int64_t q = threadIdx.x; q < np; q += kBlock) acc += c[q];
  const double tot = block_sum_fixed(acc, wsum);
  if (threadIdx.x == 0) out[T] = scale * tot;
}

// x = a - b elementwise (level vectors, 256-byte aligned: two values per 16-byte access, the odd
// tail by thread 0 of block 0)
__global__ void k_sub(const double* __restrict__ a, const double* __restrict__ b, double* __restrict__ x,
                      int64_t n) {
  grid_dependency_sync();
  const int64_t n2 = n / 2;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n2; i += (int64_t)gridDim.x * blockDim.x) {
    const double2 p = reinterpret_cast<const double2*>(a)[i], q = reinterpret_cast<const double2*>(b)[i];
    reinterpret_cast<double2*>(x)[i] = make_double2(p.x - q.x, p.y - q.y);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0 && (n & 1)) x[n - 1] = a[n - 1] - b[n - 1];
}

// x = a - b (b may be null: x = a) in binary64, stored as its binary32 hi/lo pair (df_split) in the
// same 8 bytes per value: the estimator's difference vector for k_node_form_pair
__global__ void k_sub_pair(const double* __restrict__ a, const double* __restrict__ b, float2* __restrict__ x,
                           int64_t n) {
  grid_dependency_sync();
  const int64_t n2 = n / 2;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n2; i += (int64_t)gridDim.x * blockDim.x) {
    double2 p = reinterpret_cast<const double2*>(a)[i];
    if (b) {
      const double2 q = reinterpret_cast<const double2*>(b)[i];
      p.x -= q.x;
      p.y -= q.y;
    }
    const float2 h0 = df_split(p.x), h1 = df_split(p.y);
    reinterpret_cast<float4*>(x)[i] = make_float4(h0.x, h0.y, h1.x, h1.y);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0 && (n & 1)) x[n - 1] = df_split(b ? a[n - 1] - b[n - 1] : a[n - 1]);
}

// Level-l node coordinates x = x_0 + J p / n of every cell's closure lattice (hhg_level_coords into
// device memory).  geom: per cell x_0 (3) and J row-major (3 x 3).  The products and sums are
// rounded separately, in the host path's order, so both paths give the same bits.
__global__ void k_level_coords(int dim, int n, int64_t Nt, int64_t N, const int32_t* __restrict__ ijk,
                               const double* __restrict__ geom, double* __restrict__ xyz) {
  grid_dependency_sync();
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < N; idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = idx / Nt;
    const int32_t e = ijk[idx - c * Nt];
    const double p[3] = {(double)(e & 1023), (double)((e >> 10) & 1023), (double)(e >> 20)};
    const double* G = geom + c * 12;
    for (int r = 0; r < dim; ++r) {
      double v = 0;
      for (int a = 0; a < dim; ++a) v = __dadd_rn(v, __dmul_rn(G[3 + 3 * r + a], p[a]));
      xyz[idx * dim + r] = __dadd_rn(G[r], v / (double)n);
    }
  }
}

__global__ void k_finite(const double* __restrict__ v, int64_t n, int* __restrict__ flag) {
  grid_dependency_sync();
  int bad = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    if (!isfinite(v[i])) bad = 1;
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(flag, 1);
}

// ================================================================= host launchers

static LevelCtx ctx(const hhg_mesh_s* m, int l) {
  const LevelData& Lv = m->lv[l];
  return LevelCtx{Lv.n, Lv.Nt, Lv.d_ijk, m->d_nzs, Lv.d_itab};
}

#define DISPATCH_DIM(m, KER, ...)                 \
  do {                                            \
    if ((m)->dim == 2) hhg_launch(KER<2>, __VA_ARGS__); \
    else hhg_launch(KER<3>, __VA_ARGS__);               \
  } while (0)

void launch_build_rhs(hhg_mesh_s* m, int l, cudaStream_t s) {
  const LevelData& Lv = m->lv[l];
  dim3 grid(blocks_for(Lv.Nt), m->nc);
  double ms = mass_scale(m->dim, Lv.n);
  const LevelData& LL = m->lv[m->L];
  if (m->dim == 2)
    hhg_launch(k_build_rhs<2, double, double>, grid, kBlock, 0, s, ctx(m, l), LL.n, LL.Nt, m->L - l, m->fL,
               (const double*)m->dM, ms, (const uint16_t*)m->d_dirmask, Lv.b);
  else
    hhg_launch(k_build_rhs<3, double, double>, grid, kBlock, 0, s, ctx(m, l), LL.n, LL.Nt, m->L - l, m->fL,
               (const double*)m->dM, ms, (const uint16_t*)m->d_dirmask, Lv.b);
}

// the same in binary32 (binary32 mass stencils and arithmetic) into the level's binary32 rhs b32
void launch_build_rhs32(hhg_mesh_s* m, int l, cudaStream_t s) {
  const LevelData& Lv = m->lv[l];
  dim3 grid(blocks_for(Lv.Nt), m->nc);
  float ms = (float)mass_scale(m->dim, Lv.n);
  const LevelData& LL = m->lv[m->L];
  if (m->dim == 2)
    hhg_launch(k_build_rhs<2, float, float>, grid, kBlock, 0, s, ctx(m, l), LL.n, LL.Nt, m->L - l, m->fL,
               (const float*)m->dM32, ms, (const uint16_t*)m->d_dirmask, Lv.b32);
  else
    hhg_launch(k_build_rhs<3, float, float>, grid, kBlock, 0, s, ctx(m, l), LL.n, LL.Nt, m->L - l, m->fL,
               (const float*)m->dM32, ms, (const uint16_t*)m->d_dirmask, Lv.b32);
}

void launch_build_rhs_restricted(hhg_mesh_s* m, cudaStream_t s);

void launch_init_coarse_g(hhg_mesh_s* m, const double* g, cudaStream_t s) {
  const LevelData& Lv = m->lv[0];
  const LevelData& LL = m->lv[m->L];
  dim3 grid(blocks_for(Lv.Nt), m->nc);
  DISPATCH_DIM(m, k_init_coarse, grid, kBlock, 0, s, ctx(m, 0), LL.n, LL.Nt, m->L, g, m->d_dirmask, Lv.u);
}

void launch_init_coarse(hhg_mesh_s* m, cudaStream_t s) { launch_init_coarse_g(m, m->gL, s); }

template <int DIM, int PM>
static void interior_stage(hhg_mesh_s* m, int l, int gi, int colour, double* u, const double* rhs, cudaStream_t s) {
  const LevelData& Lv = m->lv[l];
  const Group& G = m->groups[gi];
  int64_t a = Lv.icol_off[gi][colour], b = Lv.icol_off[gi][colour + 1];
  if (b <= a || G.cells.empty()) return;
  dim3 grid(blocks_for(b - a), (unsigned)G.cells.size());
  hhg_launch(k_smooth_interior<DIM, PM, double, double, double>, grid, kBlock, 0, s, 
      G.d_cells, Lv.d_icol + a, b - a, ctx(m, l), m->d_tnorm, Lv.d_invl, Vec<double, double>{u, nullptr},
      CVec<double, double>{rhs, nullptr});
}

// all interior colours of a group at once, one CTA per cell (levels with short colour lists)
template <int DIM, int PM>
static void interior_cells(hhg_mesh_s* m, int l, int gi, double* u, const double* rhs, cudaStream_t s) {
  const LevelData& Lv = m->lv[l];
  const Group& G = m->groups[gi];
  if (G.cells.empty() || Lv.icol_off[gi][G.m] <= Lv.icol_off[gi][0]) return;
  hhg_launch(k_smooth_interior_cell<DIM, PM, double, double, double>, (unsigned)G.cells.size(), kBlock, 0, s,
             G.d_cells, Lv.d_icol + Lv.icol_off[gi][0], colour_offsets(Lv, gi, G.m), ctx(m, l), m->d_tnorm, Lv.d_invl,
             Vec<double, double>{u, nullptr}, CVec<double, double>{rhs, nullptr});
}

template <int DIM>
static void interior_cells_dispatch(hhg_mesh_s* m, int l, int gi, double* u, const double* rhs, cudaStream_t s) {
  int pm = m->groups[gi].pmask;
  if (DIM == 2) {
    switch (pm) {
      case 0x3: interior_cells<DIM, 0x3>(m, l, gi, u, rhs, s); return;
      case 0x5: interior_cells<DIM, 0x5>(m, l, gi, u, rhs, s); return;
      case 0x6: interior_cells<DIM, 0x6>(m, l, gi, u, rhs, s); return;
      default: interior_cells<DIM, 0x7>(m, l, gi, u, rhs, s); return;
    }
  } else {
    if (pm == 0x29) interior_cells<DIM, 0x29>(m, l, gi, u, rhs, s);
    else interior_cells<DIM, 0x7f>(m, l, gi, u, rhs, s);
  }
}

// compile-time stencil patterns: the full stencil and the Kuhn / right-isosceles patterns
template <int DIM>
static void interior_stage_dispatch(hhg_mesh_s* m, int l, int gi, int colour, double* u, const double* rhs,
                                    cudaStream_t s) {
  int pm = m->groups[gi].pmask;
  if (DIM == 2) {
    switch (pm) {
      case 0x3: interior_stage<DIM, 0x3>(m, l, gi, colour, u, rhs, s); return;
      case 0x5: interior_stage<DIM, 0x5>(m, l, gi, colour, u, rhs, s); return;
      case 0x6: interior_stage<DIM, 0x6>(m, l, gi, colour, u, rhs, s); return;
      default: interior_stage<DIM, 0x7>(m, l, gi, colour, u, rhs, s); return;
    }
  } else {
    switch (pm) {
      case 0x29: interior_stage<DIM, 0x29>(m, l, gi, colour, u, rhs, s); return;  // e1, e1-e2, e2-e3
      default: interior_stage<DIM, 0x7f>(m, l, gi, colour, u, rhs, s); return;
    }
  }
}

template <int DIM>
static void iface_stage(hhg_mesh_s* m, int l, const Prims& P, int nverts, int parity, int cnt_rim, int cnt_inner,
                        const int32_t* rim_list, const int32_t* inner_list, double* u, const double* rhs,
                        cudaStream_t s) {
  if (P.count == 0 || (cnt_rim <= 0 && cnt_inner <= 0)) return;
  const LevelData& Lv = m->lv[l];
  double* du = Lv.tmp;  // residual scratch is free during a sweep (sized N_l >= the rim nodes)
  double ss = stiff_scale(DIM, Lv.n);
  // copies spread over lanes (the edge stages are latency-bound)
  launch_iface<DIM, double, double, double>(iface_lanes(P.max_copies), P.count, P.d_ptr, P.d_cell, P.d_loc, P.d_dir, nverts, parity,
                                            cnt_rim, cnt_inner, rim_list, inner_list, ctx(m, l), m->dS, ss, P.d_pinv,
                                            Vec<double, double>{u, nullptr}, CVec<double, double>{rhs, nullptr}, du,
                                            s);
}

template <int DIM>
static void sweep_impl(hhg_mesh_s* m, int l, const double* rhs, cudaStream_t s) {
  LevelData& Lv = m->lv[l];
  double* u = Lv.u;
  int n = Lv.n;
  double ss = stiff_scale(DIM, n);
  // stage list: vertex, edge even, edge odd, [face block], interior colours
  const int nst = 3 + (DIM == 3 ? 1 : 0) + m->n_colours;
  for (int st = 0; st < nst; ++st) {
    if (st == 0) {
      // stages 0 and 1 (vertices, even edge nodes) do not couple: one launch
      launch_vertex_edge_even<DIM, double, double, double>(m->verts, m->edges, n, ctx(m, l), m->dS, ss,
                                                           m->verts.d_pinv, m->edges.d_pinv,
                                                           Vec<double, double>{u, nullptr},
                                                           CVec<double, double>{rhs, nullptr}, s);
    } else if (st == 1) {
      continue;
    } else if (st == 2) {
      // odd edge nodes: t = 1 and n-1 are rim
      int cnt_rim = n == 2 ? 1 : 2;
      int cnt_inner = n == 2 ? 0 : n / 2 - 2;
      iface_stage<DIM>(m, l, m->edges, 2, 1, cnt_rim, cnt_inner, nullptr, nullptr, u, rhs, s);
    } else if (DIM == 3 && st == 3) {
      // binary64 face-node pass over the outside couplings: sparse slot loop where DFMA-bound
      bool sparse = (int64_t)m->faces.count * Lv.fcol_off[3] >= kSparseFaceNodes;
      launch_face_block<double, double, double>(m->faces, Lv, ctx(m, l), m->dS, ss, m->faces.d_fw, m->faces.d_pinv,
                                                Vec<double, double>{u, nullptr}, CVec<double, double>{rhs, nullptr},
                                                Lv.tmp, (double*)m->d_face_work, sparse, s);
    } else {
      int c = st - (DIM == 3 ? 4 : 3);
      if (interior_per_cell(Lv, m->groups)) {  // short lists: every colour in one launch per group
        if (c == 0)
          for (size_t gi = 0; gi < m->groups.size(); ++gi) interior_cells_dispatch<DIM>(m, l, (int)gi, u, rhs, s);
        continue;
      }
      for (size_t gi = 0; gi < m->groups.size(); ++gi)
        if (c < m->groups[gi].m) interior_stage_dispatch<DIM>(m, l, (int)gi, c, u, rhs, s);
    }
  }
}

void launch_sweep(hhg_mesh_s* m, int l, const double* rhs, cudaStream_t s) {
  if (m->dim == 2) sweep_impl<2>(m, l, rhs, s);
  else sweep_impl<3>(m, l, rhs, s);
}

template <int DIM, int PM>
static void residual_group(hhg_mesh_s* m, int l, int gi, const double* rhs, cudaStream_t s, bool after_sweep) {
  const LevelData& Lv = m->lv[l];
  const Group& G = m->groups[gi];
  ResidualSegments rs = residual_segments(Lv, G, gi, after_sweep);
  dim3 grid(rs.bcomp + rs.bzero + blocks_for(Lv.nbnd), (unsigned)G.cells.size());
  hhg_launch(k_residual_list<DIM, PM, 1, true, double, double, double, double>, grid, kBlock, 0, s, G.d_cells,
             (int)G.cells.size(), ctx(m, l), m->dS, m->d_dirmask, stiff_scale(DIM, Lv.n),
             CVec<double, double>{Lv.u, nullptr}, CVec<double, double>{rhs, nullptr}, Lv.tmp, rs.ilist, rs.ncomp,
             rs.nzero, Lv.d_bnd, Lv.nbnd, rs.bcomp, rs.bzero);
}

void launch_residual_after(hhg_mesh_s* m, int l, const double* rhs, cudaStream_t s, bool after_sweep);

void launch_residual(hhg_mesh_s* m, int l, const double* rhs, cudaStream_t s) {
  launch_residual_after(m, l, rhs, s, false);
}

void launch_residual_after(hhg_mesh_s* m, int l, const double* rhs, cudaStream_t s, bool after_sweep) {
  for (size_t gi = 0; gi < m->groups.size(); ++gi) {
    int pm = m->groups[gi].pmask;
    if (m->dim == 2) {
      switch (pm) {
        case 0x3: residual_group<2, 0x3>(m, l, (int)gi, rhs, s, after_sweep); break;
        case 0x5: residual_group<2, 0x5>(m, l, (int)gi, rhs, s, after_sweep); break;
        case 0x6: residual_group<2, 0x6>(m, l, (int)gi, rhs, s, after_sweep); break;
        default: residual_group<2, 0x7>(m, l, (int)gi, rhs, s, after_sweep); break;
      }
    } else {
      if (pm == 0x29) residual_group<3, 0x29>(m, l, (int)gi, rhs, s, after_sweep);
      else residual_group<3, 0x7f>(m, l, (int)gi, rhs, s, after_sweep);
    }
  }
}

void launch_restrict(hhg_mesh_s* m, int l, const double* fine, double* coarse, cudaStream_t s, double* zero) {
  const LevelData& C = m->lv[l - 1];
  dim3 grid(blocks_for(C.Nt), m->nc);
  if (m->dim == 2)
    hhg_launch(k_restrict<2, double, double, double>, grid, kBlock, 0, s, ctx(m, l), ctx(m, l - 1), m->d_dirmask, fine,
               coarse, zero);
  else
    hhg_launch(k_restrict<3, double, double, double>, grid, kBlock, 0, s, ctx(m, l), ctx(m, l - 1), m->d_dirmask, fine,
               coarse, zero);
}

void launch_prolong_add(hhg_mesh_s* m, int l, cudaStream_t s) {
  const LevelData& F = m->lv[l];
  dim3 grid(blocks_for(F.Nt), m->nc);
  CVec<double, double> uc{m->lv[l - 1].u, nullptr};
  Vec<double, double> uf{F.u, nullptr};
  if (m->dim == 2)
    hhg_launch(k_prolong_add<2, double, double, double>, grid, kBlock, 0, s, ctx(m, l), ctx(m, l - 1), m->d_dirmask, uc, uf);
  else
    hhg_launch(k_prolong_add<3, double, double, double>, grid, kBlock, 0, s, ctx(m, l), ctx(m, l - 1), m->d_dirmask, uc, uf);
}

void launch_fmg_prolong_g(hhg_mesh_s* m, int l, const double* g, double* w, cudaStream_t s) {
  const LevelData& F = m->lv[l + 1];
  const LevelData& LL = m->lv[m->L];
  dim3 grid(blocks_for(F.Nt), m->nc);
  DISPATCH_DIM(m, k_fmg_prolong, grid, kBlock, 0, s, ctx(m, l + 1), ctx(m, l), LL.n, LL.Nt, m->L - l - 1, g,
                                                         m->d_dirmask, m->lv[l].u, F.u, w);
}

void launch_fmg_prolong(hhg_mesh_s* m, int l, cudaStream_t s) { launch_fmg_prolong_g(m, l, m->gL, m->lv[l].w, s); }

void launch_prolong(hhg_mesh_s* m, int l, const double* coarse, double* fine, cudaStream_t s, const double* minuend) {
  const LevelData& F = m->lv[l];
  dim3 grid(blocks_for(F.Nt), m->nc);
  DISPATCH_DIM(m, k_prolong, grid, kBlock, 0, s, ctx(m, l), ctx(m, l - 1), coarse, fine, minuend);
}

void launch_sub(hhg_mesh_s* m, const double* a, const double* b, double* x, int64_t n, cudaStream_t s) {
  hhg_launch(k_sub, 16 * m->sm_count, kBlock, 0, s, a, b, x, n);
}

void launch_level_coords(hhg_mesh_s* m, int l, const double* geom, double* xyz, cudaStream_t s) {
  const LevelData& Lv = m->lv[l];
  hhg_launch(k_level_coords, 8 * m->sm_count, kBlock, 0, s, m->dim, Lv.n, Lv.Nt, Lv.N, Lv.d_ijk, geom, xyz);
}

void launch_coarse_solve(hhg_mesh_s* m, const double* rhs, cudaStream_t s) {
  if (m->n0f == 0) return;
  size_t smem = (size_t)m->n0f * sizeof(double);
  // the attribute belongs to the current device, so it is set on every call that needs it
  if (smem > 48 * 1024) {
    if (m->dim == 2) cudaFuncSetAttribute(k_coarse<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    else cudaFuncSetAttribute(k_coarse<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  }
  const Prims& P = m->verts;
  DISPATCH_DIM(m, k_coarse, 1, 1024, smem, s, m->n0f, m->d_cf_vert, P.d_ptr, P.d_cell, P.d_loc, ctx(m, 0), m->dS,
                                                  rhs, m->lv[0].u, m->d_Ainv);
}

void launch_finite_check(hhg_mesh_s* m, const double* v, int64_t n, cudaStream_t s) {
  hhg_launch(k_finite, 2 * m->sm_count, kBlock, 0, s, v, n, m->d_flag);
}

static void cell_form(hhg_mesh_s* m, bool diff, const double* tab, double scale, const double* a, const double* b,
                      double* out, cudaStream_t s) {
  const LevelData& Lv = m->lv[m->L];
  double* contrib = m->d_part;  // one block sum per cell and block of k_node_form
  dim3 grid(blocks_for(Lv.Nt, kBlock * kFormNodes), m->nc);
  if (diff) {
    if (m->dim == 2) hhg_launch(k_node_form<2, true>, grid, kBlock, 0, s, ctx(m, m->L), tab, a, b, contrib);
    else hhg_launch(k_node_form<3, true>, grid, kBlock, 0, s, ctx(m, m->L), tab, a, b, contrib);
  } else {
    if (m->dim == 2) hhg_launch(k_node_form<2, false>, grid, kBlock, 0, s, ctx(m, m->L), tab, a, b, contrib);
    else hhg_launch(k_node_form<3, false>, grid, kBlock, 0, s, ctx(m, m->L), tab, a, b, contrib);
  }
  hhg_launch(k_cell_sum, m->nc, kBlock, 0, s, (int64_t)grid.x, scale, contrib, out);
}

// Per-cell squared mass norm of a difference vector held as binary32 hi/lo pairs on level L.
void launch_mass_norm_sq_pair(hhg_mesh_s* m, const float2* x, double* out, cudaStream_t s) {
  const LevelData& Lv = m->lv[m->L];
  dim3 grid(blocks_for(Lv.Nt, kBlock * kFormNodes), m->nc);
  if (m->dim == 2) hhg_launch(k_node_form_pair<2>, grid, kBlock, 0, s, ctx(m, m->L), (const float2*)m->dMp, x, m->d_part);
  else hhg_launch(k_node_form_pair<3>, grid, kBlock, 0, s, ctx(m, m->L), (const float2*)m->dMp, x, m->d_part);
  hhg_launch(k_cell_sum, m->nc, kBlock, 0, s, (int64_t)grid.x, mass_scale(m->dim, Lv.n), m->d_part, out);
}

void launch_sub_pair(hhg_mesh_s* m, const double* a, const double* b, float2* x, int64_t n, cudaStream_t s) {
  hhg_launch(k_sub_pair, 16 * m->sm_count, kBlock, 0, s, a, b, x, n);
}

// x_L = minuend - I v on level L (v on level L-1) as binary32 hi/lo pairs
void launch_prolong_diff_pair(hhg_mesh_s* m, const double* coarse, const double* minuend, float2* x, cudaStream_t s) {
  const int l = m->L;
  const LevelData& F = m->lv[l];
  dim3 grid(blocks_for(F.Nt), m->nc);
  DISPATCH_DIM(m, k_prolong_diff_pair, grid, kBlock, 0, s, ctx(m, l), ctx(m, l - 1), coarse, minuend, x);
}

void launch_mass_norm_sq(hhg_mesh_s* m, const double* a, const double* b, double* out, cudaStream_t s) {
  cell_form(m, true, m->dM, mass_scale(m->dim, m->lv[m->L].n), a, b, out, s);
}

void launch_energy_norm_sq(hhg_mesh_s* m, const double* a, const double* b, double* out, cudaStream_t s) {
  cell_form(m, true, m->dS, stiff_scale(m->dim, m->lv[m->L].n), a, b, out, s);
}

void launch_stiff_bilinear(hhg_mesh_s* m, const double* x, const double* y, double* out, cudaStream_t s) {
  cell_form(m, false, m->dS, stiff_scale(m->dim, m->lv[m->L].n), x, y, out, s);
}

void launch_sum_interfaces(hhg_mesh_s* m, int l, double* v, cudaStream_t s) {
  const LevelData& Lv = m->lv[l];
  int n = Lv.n;
  const Prims& PV = m->verts;
  if (PV.count)
    DISPATCH_DIM(m, k_sum_prims, blocks_for(PV.count), kBlock, 0, s, PV.count, 1, 1, nullptr, PV.d_ptr, PV.d_cell,
                                                                          PV.d_loc, ctx(m, l), v);
  const Prims& PE = m->edges;
  if (PE.count && n >= 2)
    DISPATCH_DIM(m, k_sum_prims, blocks_for((int64_t)PE.count * (n - 1)), kBlock, 0, s, 
                                     PE.count, 2, n - 1, nullptr, PE.d_ptr, PE.d_cell, PE.d_loc, ctx(m, l), v);
  const Prims& PF = m->faces;
  int64_t nf = Lv.fcol_off[3];
  if (m->dim == 3 && PF.count && nf > 0)
    hhg_launch(k_sum_prims<3>, blocks_for((int64_t)PF.count * nf), kBlock, 0, s, PF.count, 3, (int)nf, Lv.d_fcol, PF.d_ptr,
                                                                         PF.d_cell, PF.d_loc, ctx(m, l), v);
}

void launch_apply_op(hhg_mesh_s* m, int l, int op, const double* in, double* out, cudaStream_t s) {
  const LevelData& Lv = m->lv[l];
  dim3 grid(blocks_for(Lv.Nt), m->nc);
  const double* tab = op == 0 ? m->dS : m->dM;
  double sc = op == 0 ? stiff_scale(m->dim, Lv.n) : mass_scale(m->dim, Lv.n);
  DISPATCH_DIM(m, k_apply_partial, grid, kBlock, 0, s, ctx(m, l), tab, sc, in, out, nullptr, m->d_dirmask);
}

void launch_adjoint_rhs(hhg_mesh_s* m, const unsigned char* d_inS, const double* u, double* out, cudaStream_t s) {
  const LevelData& Lv = m->lv[m->L];
  dim3 grid(blocks_for(Lv.Nt), m->nc);
  DISPATCH_DIM(m, k_apply_partial, grid, kBlock, 0, s, ctx(m, m->L), m->dM, 2.0 * mass_scale(m->dim, Lv.n), u,
                                                           out, d_inS, m->d_dirmask);
}

// adjoint FMG right-hand sides on the coarser levels: b_{l-1} = P^T b_l
void launch_restrict_rhs_chain(hhg_mesh_s* m, cudaStream_t s) {
  for (int l = m->L; l >= 1; --l) launch_restrict(m, l, m->lv[l].b, m->lv[l - 1].b, s);
}

// Algorithmic model of one interior-colour launch on level L (group 0, colour 0): every closure
// value u of the group's cells is read once (the neighbours are the other colours), b is read and u
// written for the updated nodes; flops = 4 p + 1 per updated node (p coupled direction pairs: one FMA
// per neighbour, FMA = 2 flops, plus b_i / a_ii).
// kernel 1: the level-L face stage of colour 0 (3D), timed only.
void launch_profile_face(hhg_mesh_s* m, int reps, cudaStream_t s, long long* units) {
  const int L = m->L;
  LevelData& Lv = m->lv[L];
  *units = (long long)m->faces.count * Lv.fcol_off[3];
  if (m->dim != 3) return;
  bool sparse = (int64_t)m->faces.count * Lv.fcol_off[3] >= kSparseFaceNodes;
  for (int r = 0; r < reps; ++r)
    launch_face_block<double, double, double>(m->faces, Lv, ctx(m, L), m->dS, stiff_scale(3, Lv.n), m->faces.d_fw,
                                              m->faces.d_pinv, Vec<double, double>{Lv.u, nullptr},
                                              CVec<double, double>{Lv.b, nullptr}, Lv.tmp, (double*)m->d_face_work,
                                              sparse, s);
}

static int ndirs_of(int dim) { return dim == 2 ? 7 : 15; }

// binary64 level-L probes: 2 prolongation-add, 3 residual (all nodes computed), 4 estimator mass form
// of a difference vector (node form + per-cell sum)
void launch_profile_level(hhg_mesh_s* m, int kernel, int reps, cudaStream_t s, long long* units, double* bytes,
                          double* flops) {
  const int L = m->L;
  LevelData& Lv = m->lv[L];
  const double N = (double)Lv.N, Nc = (double)m->lv[L - 1].N;
  *units = (long long)Lv.N;
  if (kernel == 2) {
    *bytes = 8.0 * (2.0 * N + Nc);
    *flops = 3.0 * N;
  } else if (kernel == 3) {
    *bytes = 8.0 * 3.0 * N;
    *flops = (2.0 * (1 + 2 * __builtin_popcount(m->groups[0].pmask)) + 2.0) * N;
  } else {
    // the pair form reads x once (8 bytes per node); flops: the form's binary64-equivalent count
    *bytes = 8.0 * N;
    *flops = 2.0 * (ndirs_of(m->dim) + 1) / 2 * N + 2.0 * N;
    launch_sub_pair(m, Lv.u, nullptr, (float2*)Lv.tmp, Lv.N, s);
  }
  for (int r = 0; r < reps; ++r) {
    if (kernel == 2) launch_prolong_add(m, L, s);
    else if (kernel == 3) launch_residual(m, L, Lv.b, s);
    else launch_mass_norm_sq_pair(m, (const float2*)Lv.tmp, m->d_red, s);
  }
}

void launch_profile_interior(hhg_mesh_s* m, int precision, int reps, cudaStream_t s, long long* units,
                             double* bytes, double* flops) {
  const int L = m->L;
  const LevelData& Lv = m->lv[L];
  const Group& G = m->groups[0];
  int64_t len = Lv.icol_off[0][1] - Lv.icol_off[0][0];
  long long nodes = (long long)len * (long long)G.cells.size();
  int p = __builtin_popcount(G.pmask);
  double sval = precision == 0 ? 8.0 : 4.0;
  *units = nodes;
  *bytes = sval * ((double)Lv.Nt * G.cells.size() + 2.0 * nodes);
  *flops = (4.0 * p + 1.0) * nodes;
  if (precision != 0) return;  // the binary32 variant is launched by the mixed-path module
  for (int r = 0; r < reps; ++r) {
    if (m->dim == 2) interior_stage_dispatch<2>(m, L, 0, 0, Lv.u, Lv.b, s);
    else interior_stage_dispatch<3>(m, L, 0, 0, Lv.u, Lv.b, s);
  }
}

// Load every kernel of this module up front (module loading is otherwise deferred to first launch).
hhg_status preload_kernels() {
  cudaFuncAttributes fa;
  const void* fns[] = {
      (const void*)k_build_rhs<2, double, double>, (const void*)k_build_rhs<3, double, double>, (const void*)k_init_coarse<2>,
      (const void*)k_init_coarse<3>, (const void*)k_fmg_prolong<2>, (const void*)k_fmg_prolong<3>,
      (const void*)k_prolong<2>, (const void*)k_prolong<3>, (const void*)k_coarse<2>, (const void*)k_coarse<3>,
      (const void*)k_node_form<2, true>, (const void*)k_node_form<3, true>, (const void*)k_node_form<2, false>,
      (const void*)k_node_form<3, false>, (const void*)k_cell_sum, (const void*)k_apply_partial<2>,
      (const void*)k_apply_partial<3>, (const void*)k_sum_prims<2>, (const void*)k_sum_prims<3>,
      (const void*)k_finite, (const void*)k_sub, (const void*)k_sub_pair, (const void*)k_node_form_pair<2>,
      (const void*)k_node_form_pair<3>, (const void*)k_prolong_diff_pair<2>, (const void*)k_prolong_diff_pair<3>};
  for (const void* f : fns) {
    cudaError_t e = cudaFuncGetAttributes(&fa, f);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncGetAttributes");
  }
  return HHG_OK;
}

// debug build: read and clear the first recorded bounds failure (zeros otherwise)
hhg_status read_check(long long* out) {
  for (int q = 0; q < 8; ++q) out[q] = 0;
#ifdef HHG_CHECK
  cudaError_t e = cudaMemcpyFromSymbol(out, g_hhg_check, 8 * sizeof(long long));
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyFromSymbol");
  long long z[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  cudaMemcpyToSymbol(g_hhg_check, z, sizeof(z));
  out[7] = 1;  // marks a checking build
#endif
  return HHG_OK;
}

}  // namespace hhg
