// Mixed-precision iterative refinement (no counterpart in the paper).
//
// Step 1: FMG (Alg. 4 structure, same stage-ordered smoother) computed in binary32 on the original
//         problem: the iterate of the current FMG top level is a binary32 vector, the coarse-grid
//         corrections below it are stored as binary32, bfloat16 or binary16 and accumulated in
//         binary32.  The prolongated iterates w_l are written in binary64 for the estimator.
//         binary16 has five exponent bits, so each level's correction is stored times a power of two
//         chosen, after the restriction, from max |r| of its right-hand side and a bound of
//         |A_l^{-1}|_inf (k_set_scale16).
// Steps 2..: r = b_L - A_L u_L and u_L += c in binary64 on level L; the correction c solves
//         A_L c = r with V-cycles computed in binary32 (same storage rule for the coarse levels).
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <type_traits>

#include "internal.h"
#include "kernels_impl.cuh"

namespace hhg {

// ---------------------------------------------------------------- elementwise kernels

__global__ void k_to_f32(const double* __restrict__ a, float* __restrict__ b, int64_t n) {
  grid_dependency_sync();
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = (float)a[i];
}

__global__ void k_to_f64(const float* __restrict__ a, double* __restrict__ b, int64_t n) {
  grid_dependency_sync();
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = (double)a[i];
}

// level-L binary64 iterate from the binary32 FMG result; Dirichlet nodes take the exact binary64 g
// (the binary32 copy of g would perturb the boundary data the refinement converges to)
template <int DIM>
__global__ void k_to_f64_level(LevelCtx lc, const uint16_t* __restrict__ dirmask, const double* __restrict__ gL,
                               const float* __restrict__ x, double* __restrict__ u) {
  grid_dependency_sync();
  int64_t loc = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (loc >= lc.Nt) return;
  int T = blockIdx.y;
  int i, j, k;
  decode(lc.ijk[loc], i, j, k);
  int t = boundary_type(DIM, lc.n, i, j, k);
  int64_t g = (int64_t)T * lc.Nt + loc;
  u[g] = (dirmask[T] >> t & 1) ? gL[g] : (double)x[g];
}

// u += c (binary64 accumulate of a binary32 correction; c is zero on Dirichlet nodes)
__global__ void k_add_f32(const float* __restrict__ c, double* __restrict__ u, int64_t n) {
  grid_dependency_sync();
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) u[i] += (double)c[i];
}

// ---- binary16 correction storage: per-level power-of-two scale ----
// The correction c_l of a coarse level solves A_l c_l = r_l, so |c_l|_inf <= |A_l^{-1}|_inf |r_l|_inf.
// For nested P1 meshes |A_l^{-1}|_inf grows like 2^{l d} |A_0^{-1}|_inf (the discrete Green's function
// of a level-l lattice), and |A_0^{-1}|_inf is known exactly from the direct coarse solve.  The stored
// right-hand sides are partial at interface nodes (a node's value is the sum over its copies), so the
// assembled |r_l|_inf is bounded by the largest copy count times the largest stored |r|.  The scale
// 2^e puts that bound at or below kScale16Target, far enough under binary16's largest finite value
// (65504) to absorb an underestimate of |A_l^{-1}|_inf (coefficient jumps make the level-0 estimate
// low by a small factor) and Gauss-Seidel iterates overshooting the solution.
constexpr double kScale16Target = 1024.0;

// max |r| over a vector, as the bit pattern of a non-negative binary32 (ordered like unsigned
// integers; NaN orders above infinity), combined per warp and then by atomicMax into *out
__global__ void k_absmax_bits(const float* __restrict__ r, int64_t n, unsigned* __restrict__ out) {
  grid_dependency_sync();
  unsigned v = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    v = max(v, __float_as_uint(fabsf(r[i])));
  v = __reduce_max_sync(0xffffffffu, v);
  if ((threadIdx.x & 31) == 0) atomicMax(out, v);
}

// scale = the largest 2^e (|e| <= 120) with 2^e * bound * max|r| <= kScale16Target, where
// bound = level_factor * |A_0^{-1}|_inf; 1 when max|r| is zero or not finite (the solve's finite
// check then reports the divergence)
__global__ void k_set_scale16(const unsigned* __restrict__ rmax_bits, const double* __restrict__ ainv_inf,
                              double level_factor, float* __restrict__ scale) {
  grid_dependency_sync();
  if (threadIdx.x != 0) return;
  const float rmax = __uint_as_float(*rmax_bits);
  const double bound = level_factor * *ainv_inf;
  float sc = 1.0f;
  if (rmax > 0.0f && isfinite(rmax) && bound > 0.0) {
    int e = ilogb(kScale16Target / (bound * (double)rmax));
    e = max(-120, min(120, e));
    sc = ldexpf(1.0f, e);
  }
  *scale = sc;
}

// binary32 FMG start: x_0 = g on Dirichlet nodes, 0 elsewhere
template <int DIM>
__global__ void k_init_coarse32(LevelCtx lc, int nL, int64_t NtL, int shift, const double* __restrict__ gL,
                                const uint16_t* __restrict__ dirmask, float* __restrict__ u) {
  grid_dependency_sync();
  int64_t loc = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (loc >= lc.Nt) return;
  int T = blockIdx.y;
  int i, j, k;
  decode(lc.ijk[loc], i, j, k);
  int t = boundary_type(DIM, lc.n, i, j, k);
  float v = 0.0f;
  if (dirmask[T] >> t & 1) {
    int64_t q = packed_index(DIM, nL, (int64_t)i << shift, (int64_t)j << shift, (int64_t)k << shift);
    if (HHG_OOB(q, NtL, 82)) return;
    v = (float)gL[(int64_t)T * NtL + q];
  }
  u[(int64_t)T * lc.Nt + loc] = v;
}

// binary32 FMG transition: x_{l+1} = I x_l (Dirichlet nodes from g_L), w_l = x_{l+1} in binary64
template <int DIM>
__global__ void k_fmg_prolong32(LevelCtx fc, LevelCtx cc, int nL, int64_t NtL, int shift, const double* __restrict__ gL,
                                const uint16_t* __restrict__ dirmask, const float* __restrict__ xc,
                                float* __restrict__ xf, double* __restrict__ w) {
  grid_dependency_sync();
  int64_t loc = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (loc >= fc.Nt) return;
  int T = blockIdx.y;
  int i, j, k;
  decode(fc.ijk[loc], i, j, k);
  int t = boundary_type(DIM, fc.n, i, j, k);
  int64_t g = (int64_t)T * fc.Nt + loc;
  if (dirmask[T] >> t & 1) {
    int64_t q = packed_index(DIM, nL, (int64_t)i << shift, (int64_t)j << shift, (int64_t)k << shift);
    if (HHG_OOB(q, NtL, 81)) return;
    double gv = gL[(int64_t)T * NtL + q];
    xf[g] = (float)gv;
    w[g] = gv;
    return;
  }
  float v = interp<DIM, float>(cc, T, i, j, k, CVec<float, float>{xc, nullptr});
  xf[g] = v;
  w[g] = (double)v;
}

// Direct coarse solve for the binary32 path: residual and A_ff^{-1} r in binary64, the update is
// stored in the level-0 vector's storage type.
template <int DIM, typename U>
__global__ void __launch_bounds__(1024) k_coarse_mixed(int n0f, const int* __restrict__ cf, const int* __restrict__ ptr,
                                                       const int* __restrict__ cell, const int* __restrict__ locv,
                                                       LevelCtx lc, const double* __restrict__ S,
                                                       const float* __restrict__ rhs, Vec<float, U> u,
                                                       const double* __restrict__ Ainv) {
  grid_dependency_sync();
  extern __shared__ double r[];
  {
    int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int q = warp; q < n0f; q += nw) {
      int v = cf[q];
      double res = 0;
      for (int c = ptr[v] + lane; c < ptr[v + 1]; c += 32) {
        int i, j, k;
        prim_position(locv[c], 1, lc.n, 0, 0, i, j, k);
        int T = cell[c];
        int t = boundary_type(DIM, lc.n, i, j, k);
        int64_t p = packed_index(DIM, lc.n, i, j, k);
        if (HHG_OOB(p, lc.Nt, 94)) continue;
        int64_t g = (int64_t)T * lc.Nt + p;
        int64_t off[15];
        neighbour_offsets(DIM, lc.n, j, k, off);
        uint32_t vm = valid_dirs_tab(DIM, t) & lc.nzs[T * kMaxTypes + t];
        mask_offsets(DIM, vm, off);
        const double* s = S + (size_t)T * kStencilStride + t * kMaxDirs;
        double acc = 0;
        for (int d = 0; d < ndirs<DIM>(); ++d)
          if ((vm >> d & 1) && !HHG_OOB(p + off[d], lc.Nt, 95)) acc += s[d] * (double)u.get(g + off[d]);
        res += (double)rhs[g] - acc;
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
    // every lane holds the sum: the lanes update the vertex's copies
    int v = cf[row];
    for (int c = ptr[v] + lane; c < ptr[v + 1]; c += 32) {
      int i, j, k;
      prim_position(locv[c], 1, lc.n, 0, 0, i, j, k);
      int64_t p = packed_index(DIM, lc.n, i, j, k);
      if (HHG_OOB(p, lc.Nt, 96)) continue;
      int64_t g = (int64_t)cell[c] * lc.Nt + p;
      u.set(g, (float)((double)u.get(g) + acc));
    }
  }
}

// ---------------------------------------------------------------- fused interior sweep (3D)
//
// All interior colour stages of one Gauss-Seidel sweep (the last stages of the smoother of Alg. 4)
// in one pass over each macro cell, one CTA per cell.  A node of plane k couples only with nodes of
// planes k-1 .. k+1 (no lattice direction changes k by more than one) and never with a node of its
// own colour, so the colour stages can be pipelined over the planes: at step p the CTA updates
// colour 0 on plane p, colour 1 on plane p-1, ..., colour M-1 on plane p-M+1.  Every neighbour value
// an update reads is then either still from the start of the sweep (a colour not yet updated there)
// or already final (a colour updated before), exactly as in the stage-by-stage order, and each node
// is computed with the list kernel's arithmetic in the same order, so the results are the same bits.
// u and b are read once and u written once per sweep, instead of once per colour stage.
// The cell's u planes p-M .. p+1 and b planes p-M+1 .. p sit in shared-memory rings (one slot per
// plane, slot = plane index mod ring size).  During step p one thread brings u plane p+2 and b
// plane p+1 in by bulk asynchronous copies (16-byte aligned windows around the planes, completing
// on one of two mbarriers) and prefetches planes kSweepL2Ahead further ahead into L2.  The nodes of
// one colour and plane are a contiguous range of the colour's list (entries: packed index, j | k << 16;
// the ranges are tabulated per plane), one node per thread.  Updated values go to shared memory and
// straight to global memory.  A copy that does not arrive within the bounded wait sets *err; the CTA
// then waits (bounded) for its copies in flight and returns.
constexpr int kSweepThreads = 256;
constexpr int kSweepL2Ahead = 6;

// elements of one ring slot: the largest plane (plane 0, side n) with its 16-byte rounding
inline int sweep_slot_elems(int n, int esize) {
  int64_t bytes = tri_size(n) * esize + 32;
  bytes = (bytes + 15) & ~(int64_t)15;
  return (int)(bytes / esize);
}
// bytes of the per-CTA tables (u and b plane windows: 8-byte start + 4-byte size each, u
// shared-memory deltas with one spare row, colour-list plane ranges)
inline int sweep_table_bytes(int n, int mcol) {
  return (int)((24 * (n + 1) + 8 * (n + 1) + 4 * mcol * (n + 2) + 15) & ~15);
}

// plane k of stencil slot d's neighbour, relative to the node's plane
__device__ constexpr int slot_dk(int d) {
  return (d == 5 || d == 10 || d == 12 || d == 13) ? 1 : ((d == 6 || d == 9 || d == 11 || d == 14) ? -1 : 0);
}

// packed-index offset of 3D stencil slot d from a node in row j of a plane of side m (T(m), T(m+1):
// the sizes of triangles of side m and m+1), in 32-bit arithmetic (dir_offset of the lattice)
__device__ __forceinline__ int slot_offset(int d, int m, int j, int Tm, int Tm1) {
  switch (d) {
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
    default: return -Tm1 + m + 1;
  }
}

// list entries per thread and colour phase kept in registers ahead (a phase with more nodes than
// kSweepThreads * kSweepAhead reads the rest directly)
constexpr int kSweepAhead = 4;

template <int PM, int M, typename U>
__global__ void __launch_bounds__(kSweepThreads) k_sweep_interior_fused(
    const int* __restrict__ gcells, LevelCtx lc, const int2* __restrict__ icol, const int* __restrict__ pcol,
    const float* __restrict__ tnorm, const float* __restrict__ invl, Vec<float, U> u, const float* __restrict__ b,
    int slotU, int tbytes, int* __restrict__ err) {
  grid_dependency_sync();
  constexpr int NU = M + 4, K = kSweepAhead;
  extern __shared__ __align__(16) unsigned char smem[];
  const int n = lc.n;
  const int T = gcells[blockIdx.x];
  U* ug = u.p + (int64_t)T * lc.Nt;
  const float* bg = b + (int64_t)T * lc.Nt;
  // per-CTA tables: u plane windows (16-byte aligned start, bytes), b plane windows (for the L2
  // prefetch), u shared-memory deltas, colour-list plane ranges
  unsigned long long* wua = (unsigned long long*)(smem + 16);
  unsigned long long* wba = wua + (n + 1);
  uint32_t* wub = (uint32_t*)(wba + (n + 1));
  uint32_t* wbb = wub + (n + 1);
  int* sdu = (int*)(wbb + (n + 1));   // u: shared index of packed index p in plane k is p + sdu[k]
  int* spc = sdu + 2 * (n + 1);       // colour-list plane ranges [c][k]
  U* su = (U*)(smem + 16 + tbytes);
  const uint32_t bar0 = smem_addr(smem);
  const int last_u = n - 2, last_b = n - 3;  // planes read: u 0 .. n-2, b (updated planes) 1 .. n-3
  if (threadIdx.x == 0) {
    mbar_init(bar0, 1);
    mbar_init(bar0 + 8, 1);
  }
  const int tn = (int)tet_size(n);
  for (int k = threadIdx.x; k <= n; k += blockDim.x) {
    const int P0 = tn - (n - k + 1) * (n - k + 2) * (n - k + 3) / 6;
    const int P1 = tn - (n - k) * (n - k + 1) * (n - k + 2) / 6;  // start of plane k+1
    const uintptr_t us = (uintptr_t)(ug + P0), ue = ((uintptr_t)(ug + P1) + 15) & ~(uintptr_t)15;
    const uintptr_t bs = (uintptr_t)(bg + P0), be = ((uintptr_t)(bg + P1) + 15) & ~(uintptr_t)15;
    wua[k] = us & ~(uintptr_t)15;
    wub[k] = (uint32_t)(ue - (us & ~(uintptr_t)15));
    wba[k] = bs & ~(uintptr_t)15;
    wbb[k] = (uint32_t)(be - (bs & ~(uintptr_t)15));
    sdu[k] = (k % NU) * slotU + (int)((us & 15) / sizeof(U)) - P0;
  }
  for (int q = threadIdx.x; q < M * (n + 2); q += blockDim.x) spc[q] = pcol[q];
  float sc = 1.0f, isc = 1.0f;
  if constexpr (IsNarrow<U>::value) {
    sc = *u.scale;
    isc = 1.0f / *u.scale;
  }
  float tv[15];
#pragma unroll
  for (int d = 1; d < 15; ++d) tv[d] = ((PM >> ((d - 1) >> 1)) & 1) ? tnorm[(size_t)T * 16 + d] : 0.0f;
  const float il = invl[T];
  __syncthreads();

  // u copies issued at step s (s = 0: the prologue, planes 0..3; s >= 1: plane s+3) complete on
  // barrier s & 1 and are first read at step s+2 (step 1 for the prologue); u and b planes further
  // ahead are prefetched into L2
  auto issue = [&](int s) {
    const uint32_t bar = bar0 + 8u * (uint32_t)(s & 1);
    const int u0 = s == 0 ? 0 : s + 3, u1 = min(s + 3, last_u);
    uint32_t total = 0;
    for (int q = u0; q <= u1; ++q) total += wub[q];
    mbar_arrive_expect_tx(bar, total);
    for (int q = u0; q <= u1; ++q) bulk_g2s(smem_addr(su + (q % NU) * slotU), (const void*)wua[q], wub[q], bar);
    for (int q = (s == 0 ? 4 : s + 3 + kSweepL2Ahead); q <= min(s + 3 + kSweepL2Ahead, last_u); ++q)
      bulk_prefetch_l2((const void*)wua[q], wub[q]);
    for (int q = (s == 0 ? 1 : s + 2 + kSweepL2Ahead); q <= min(s + 2 + kSweepL2Ahead, last_b); ++q)
      bulk_prefetch_l2((const void*)wba[q], wbb[q]);
  };
  // this thread's list entries of the colour phases of step p (colour c on plane p - c), packed as
  // p | j << 16 (-1: none)
  auto load_entries = [&](int p, int (&buf)[M][K]) {
#pragma unroll
    for (int c = 0; c < M; ++c) {
      const int q = p - c;
      const bool on = q >= 1 && q <= n - 3;
      const int lo = on ? spc[c * (n + 2) + q] : 0, hi = on ? spc[c * (n + 2) + q + 1] : 0;
#pragma unroll
      for (int r = 0; r < K; ++r) {
        const int e = lo + (int)threadIdx.x + r * kSweepThreads;
        int v = -1;
        if (e < hi) {
          const int2 en = icol[e];
          v = en.x | ((en.y & 0xffff) << 16);
        }
        buf[c][r] = v;
      }
    }
  };
  // the right-hand side at those entries (from global memory; the planes were prefetched into L2)
  auto load_b = [&](const int (&ent)[M][K], float (&bv)[M][K]) {
#pragma unroll
    for (int c = 0; c < M; ++c)
#pragma unroll
      for (int r = 0; r < K; ++r) bv[c][r] = ent[c][r] >= 0 ? bg[ent[c][r] & 0xffff] : 0.0f;
  };
  // one node: packed index p, row j of plane q (side m = n - q), right-hand side bp
  auto update = [&](int p, int j, float bp, int m, int Tm, int Tm1, int dm, int d0, int dp) {
    float acc = bp * il;
#pragma unroll
    for (int qq = 0; qq < 7; ++qq) {
      if (PM >> qq & 1) {
        const int da = 2 * qq + 1, dbb = 2 * qq + 2;
        const int sa = slot_dk(da) == 0 ? d0 : (slot_dk(da) > 0 ? dp : dm);
        const int sbb = slot_dk(dbb) == 0 ? d0 : (slot_dk(dbb) > 0 ? dp : dm);
        acc -= tv[da] * (Conv<float, U>::ld(su + (p + slot_offset(da, m, j, Tm, Tm1) + sa)) * isc);
        acc -= tv[dbb] * (Conv<float, U>::ld(su + (p + slot_offset(dbb, m, j, Tm, Tm1) + sbb)) * isc);
      }
    }
    U v;
    Conv<float, U>::st(&v, IsNarrow<U>::value ? acc * sc : acc);
    su[p + d0] = v;
    ug[p] = v;
  };

  // entries two steps ahead, right-hand sides one step ahead
  int e0[M][K], e1[M][K], e2[M][K];
  float b0[M][K], b1[M][K];
  if (threadIdx.x == 0) issue(0);
  load_entries(1, e0);
  load_entries(2, e1);
  load_b(e0, b0);
  int ok = __syncthreads_and(mbar_wait_bounded(bar0, 0, kBulkWaitTries));
  const int p_end = n - 3 + M - 1;
  int p = 1;
  for (; ok && p <= p_end; ++p) {
    if (threadIdx.x == 0) issue(p);  // after the last copy (s = n-5) only an arrival: the phase completes
    if (p + 2 <= p_end) load_entries(p + 2, e2);
    if (p + 1 <= p_end) load_b(e1, b1);
#pragma unroll
    for (int c = 0; c < M; ++c) {
      const int q = p - c;
      if (q >= 1 && q <= n - 3) {
        const int dm = sdu[q - 1], d0 = sdu[q], dp = sdu[q + 1];
        const int m = n - q, Tm = (m + 1) * (m + 2) / 2, Tm1 = (m + 2) * (m + 3) / 2;
#pragma unroll
        for (int r = 0; r < K; ++r)
          if (e0[c][r] >= 0) update(e0[c][r] & 0xffff, e0[c][r] >> 16, b0[c][r], m, Tm, Tm1, dm, d0, dp);
        const int hi = spc[c * (n + 2) + q + 1];
        for (int e = spc[c * (n + 2) + q] + (int)threadIdx.x + K * kSweepThreads; e < hi; e += kSweepThreads) {
          const int2 en = icol[e];
          update(en.x, en.y & 0xffff, bg[en.x], m, Tm, Tm1, dm, d0, dp);
        }
      }
      if (c < M - 1) __syncthreads();
    }
#pragma unroll
    for (int c = 0; c < M; ++c)
#pragma unroll
      for (int r = 0; r < K; ++r) {
        e0[c][r] = e1[c][r];
        e1[c][r] = e2[c][r];
        b0[c][r] = b1[c][r];
      }
    // the next step reads the u copies issued in the previous one (issue(0) for steps 1 and 2 was
    // waited on before the loop: its phase has completed, so the wait at p = 1 returns at once)
    const int s = p - 1;
    const bool w = (p == p_end) || mbar_wait_bounded(bar0 + 8u * (uint32_t)(s & 1), (uint32_t)((s >> 1) & 1),
                                                      kBulkWaitTries);
    ok = __syncthreads_and(w);
  }
  if (!ok) {
    if (threadIdx.x == 0) atomicOr(err, 1);
    // copies issued in the last two steps may still be in flight: let them land before exiting
    for (int s = max(0, p - 2); s <= p - 1; ++s)
      mbar_wait_bounded(bar0 + 8u * (uint32_t)(s & 1), (uint32_t)((s >> 1) & 1), kBulkWaitTries);
  }
}

// ---------------------------------------------------------------- launchers

static LevelCtx ctx(const hhg_mesh_s* m, int l) {
  const LevelData& Lv = m->lv[l];
  return LevelCtx{Lv.n, Lv.Nt, Lv.d_ijk, m->d_nzs};
}

template <typename U> static Vec<float, U> vec_of(hhg_mesh_s* m, int l, U* p) {
  return Vec<float, U>{p, m->lv[l].cscale};
}
template <typename U> static CVec<float, U> cvec_of(hhg_mesh_s* m, int l, const U* p) {
  return CVec<float, U>{p, m->lv[l].cscale};
}

template <int DIM, int PM, typename U>
static void interior32(hhg_mesh_s* m, int l, int gi, int colour, U* u, const float* rhs, cudaStream_t s) {
  const LevelData& Lv = m->lv[l];
  const Group& G = m->groups[gi];
  int64_t a = Lv.icol_off[gi][colour], b = Lv.icol_off[gi][colour + 1];
  if (b <= a || G.cells.empty()) return;
  // four cells per thread: the list entry and offsets shared, all cells' loads in flight together
  // (measured at level 6 of the 384-tet cube: 42.5 us with four, 44.6 us with two, 55 us with one)
  constexpr int CPB = 4;
  dim3 grid(blocks_for(b - a), (unsigned)((G.cells.size() + CPB - 1) / CPB));
  hhg_launch(k_smooth_interior_multi<DIM, PM, CPB, float, U, float>, grid, kBlock, 0, s, G.d_cells,
             (int)G.cells.size(), Lv.d_icol + a, b - a, ctx(m, l), m->d_tnormf, Lv.d_invlf, vec_of<U>(m, l, u),
             CVec<float, float>{rhs, nullptr});
}

// the fused interior sweep of group gi on level l (3D): one CTA per cell, all colours in one pass
// shared memory of the fused sweep on a level of side n with m colours and u stored in esize bytes
inline size_t fused_smem(int n, int mcol, int esize) {
  return 16 + (size_t)sweep_table_bytes(n, mcol) + (size_t)(mcol + 4) * sweep_slot_elems(n, esize) * esize;
}

template <int PM, int M, typename U>
static void fused32(hhg_mesh_s* m, int l, int gi, U* u, const float* rhs, cudaStream_t s) {
  const LevelData& Lv = m->lv[l];
  const Group& G = m->groups[gi];
  const int slotU = sweep_slot_elems(Lv.n, (int)sizeof(U));
  const size_t smem = fused_smem(Lv.n, M, (int)sizeof(U));
  if (smem > 48 * 1024)
    cudaFuncSetAttribute(k_sweep_interior_fused<PM, M, U>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  hhg_launch(k_sweep_interior_fused<PM, M, U>, (unsigned)G.cells.size(), kSweepThreads, smem, s, G.d_cells, ctx(m, l),
             (const int2*)(Lv.d_icol + Lv.icol_off[gi][0]), (const int*)(Lv.d_pcol + Lv.pcol_off[gi]), m->d_tnormf,
             Lv.d_invlf, vec_of<U>(m, l, u), rhs, slotU, sweep_table_bytes(Lv.n, M), m->d_err);
}

// The fused sweep is used on 3D levels with kFusedMinN <= n <= kFusedMaxN (its packed indices travel
// in 16 bits) whose rings fit in shared memory; other levels run the colour stages as separate list
// launches.
constexpr int kFusedMinN = 8, kFusedMaxN = 64;
template <typename U>
static bool use_fused(const hhg_mesh_s* m, int l, int gi) {
  const int n = m->lv[l].n;
  return m->dim == 3 && n >= kFusedMinN && n <= kFusedMaxN &&
         fused_smem(n, m->groups[gi].m, (int)sizeof(U)) <= kMaxTileSmem;
}

template <typename U>
static void fused32_dispatch(hhg_mesh_s* m, int l, int gi, U* u, const float* rhs, cudaStream_t s) {
  const Group& G = m->groups[gi];
  if (G.pmask == 0x29 && G.m == 2) fused32<0x29, 2, U>(m, l, gi, u, rhs, s);
  else if (G.m == 2) fused32<0x7f, 2, U>(m, l, gi, u, rhs, s);
  else fused32<0x7f, 4, U>(m, l, gi, u, rhs, s);
}

template <int DIM, typename U>
static void interior32_dispatch(hhg_mesh_s* m, int l, int gi, int colour, U* u, const float* rhs, cudaStream_t s) {
  int pm = m->groups[gi].pmask;
  if (DIM == 2) {
    switch (pm) {
      case 0x3: interior32<DIM, 0x3, U>(m, l, gi, colour, u, rhs, s); return;
      case 0x5: interior32<DIM, 0x5, U>(m, l, gi, colour, u, rhs, s); return;
      case 0x6: interior32<DIM, 0x6, U>(m, l, gi, colour, u, rhs, s); return;
      default: interior32<DIM, 0x7, U>(m, l, gi, colour, u, rhs, s); return;
    }
  } else {
    if (pm == 0x29) interior32<DIM, 0x29, U>(m, l, gi, colour, u, rhs, s);
    else interior32<DIM, 0x7f, U>(m, l, gi, colour, u, rhs, s);
  }
}

template <int DIM, typename U>
static void iface32(hhg_mesh_s* m, int l, const Prims& P, int nverts, int parity, int cnt_rim, int cnt_inner,
                    const int32_t* rim_list, const int32_t* inner_list, U* u, const float* rhs, cudaStream_t s) {
  if (P.count == 0 || (cnt_rim <= 0 && cnt_inner <= 0)) return;
  const LevelData& Lv = m->lv[l];
  float ss = (float)stiff_scale(DIM, Lv.n);
  launch_iface<DIM, float, U, float>(iface_lanes(P.max_copies), P.count, P.d_ptr, P.d_cell, P.d_loc, P.d_dir, nverts,
                                     parity, cnt_rim, cnt_inner, rim_list, inner_list, ctx(m, l), m->dS32, ss,
                                     P.d_pinvf, vec_of<U>(m, l, u), CVec<float, float>{rhs, nullptr}, Lv.t32, s);
}

template <int DIM, typename U>
static void sweep32(hhg_mesh_s* m, int l, U* u, const float* rhs, cudaStream_t s) {
  LevelData& Lv = m->lv[l];
  int n = Lv.n;
  float ss = (float)stiff_scale(DIM, n);
  const int nst = 3 + (DIM == 3 ? 1 : 0) + m->n_colours;
  for (int st = 0; st < nst; ++st) {
    if (st == 0) {
      // stages 0 and 1 (vertices, even edge nodes) do not couple: one launch
      launch_vertex_edge_even<DIM, float, U, float>(m->verts, m->edges, n, ctx(m, l), m->dS32, ss, m->verts.d_pinvf,
                                                    m->edges.d_pinvf, vec_of<U>(m, l, u),
                                                    CVec<float, float>{rhs, nullptr}, s);
    } else if (st == 1) {
      continue;
    } else if (st == 2) {
      int cnt_rim = n == 2 ? 1 : 2;
      int cnt_inner = n == 2 ? 0 : n / 2 - 2;
      iface32<DIM, U>(m, l, m->edges, 2, 1, cnt_rim, cnt_inner, nullptr, nullptr, u, rhs, s);
    } else if (DIM == 3 && st == 3) {
      launch_face_block<float, U, float>(m->faces, Lv, ctx(m, l), m->dS32, ss, m->faces.d_fwf, m->faces.d_pinvf,
                                         vec_of<U>(m, l, u), CVec<float, float>{rhs, nullptr}, Lv.t32,
                                         (float*)m->d_face_work, false, s);
    } else {
      int c = st - (DIM == 3 ? 4 : 3);
      for (size_t gi = 0; gi < m->groups.size(); ++gi) {
        if (use_fused<U>(m, l, (int)gi)) {
          if (c == 0) fused32_dispatch<U>(m, l, (int)gi, u, rhs, s);  // every colour in one launch
        } else if (c < m->groups[gi].m) {
          interior32_dispatch<DIM, U>(m, l, (int)gi, c, u, rhs, s);
        }
      }
    }
  }
}

template <int DIM, int PM, typename R, typename U, typename B>
static void residual_group_t(hhg_mesh_s* m, int l, int gi, CVec<R, U> u, CVec<R, B> rhs, const R* S, float* out,
                             cudaStream_t s, bool after_sweep) {
  const LevelData& Lv = m->lv[l];
  const Group& G = m->groups[gi];
  ResidualSegments rs = residual_segments(Lv, G, gi, after_sweep);
  // binary32: two cells per thread, every boundary slot unrolled (latency, not arithmetic, bounds it)
  constexpr int CPB = 2;
  dim3 grid(rs.bcomp + rs.bzero + blocks_for(Lv.nbnd), (unsigned)((G.cells.size() + CPB - 1) / CPB));
  hhg_launch(k_residual_list<DIM, PM, CPB, false, R, U, B, float>, grid, kBlock, 0, s, G.d_cells,
             (int)G.cells.size(), ctx(m, l), S, m->d_dirmask, (R)stiff_scale(DIM, Lv.n), u, rhs, out, rs.ilist,
             rs.ncomp, rs.nzero, Lv.d_bnd, Lv.nbnd, rs.bcomp, rs.bzero);
}

template <int DIM, typename R, typename U, typename B>
static void residual_t(hhg_mesh_s* m, int l, CVec<R, U> u, CVec<R, B> rhs, const R* S, float* out, cudaStream_t s,
                       bool after_sweep) {
  for (size_t gi = 0; gi < m->groups.size(); ++gi) {
    int pm = m->groups[gi].pmask;
    if (DIM == 2) {
      switch (pm) {
        case 0x3: residual_group_t<DIM, 0x3>(m, l, (int)gi, u, rhs, S, out, s, after_sweep); break;
        case 0x5: residual_group_t<DIM, 0x5>(m, l, (int)gi, u, rhs, S, out, s, after_sweep); break;
        case 0x6: residual_group_t<DIM, 0x6>(m, l, (int)gi, u, rhs, S, out, s, after_sweep); break;
        default: residual_group_t<DIM, 0x7>(m, l, (int)gi, u, rhs, S, out, s, after_sweep); break;
      }
    } else {
      if (pm == 0x29) residual_group_t<DIM, 0x29>(m, l, (int)gi, u, rhs, S, out, s, after_sweep);
      else residual_group_t<DIM, 0x7f>(m, l, (int)gi, u, rhs, S, out, s, after_sweep);
    }
  }
}

template <int DIM, typename U>
static void coarse32(hhg_mesh_s* m, U* u, const float* rhs, cudaStream_t s) {
  if (m->n0f == 0) return;
  size_t smem = (size_t)m->n0f * sizeof(double);
  if (smem > 48 * 1024) cudaFuncSetAttribute(k_coarse_mixed<DIM, U>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  const Prims& P = m->verts;
  hhg_launch(k_coarse_mixed<DIM, U>, 1, 1024, smem, s, m->n0f, m->d_cf_vert, P.d_ptr, P.d_cell, P.d_loc, ctx(m, 0), m->dS, rhs,
                                               vec_of<U>(m, 0, u), m->d_Ainv);
}

// the scale of level l's binary16 correction from its restricted right-hand side r32 (k_set_scale16)
template <int DIM>
static void set_scale16(hhg_mesh_s* m, int l, cudaStream_t s) {
  const LevelData& C = m->lv[l];
  cudaMemsetAsync(m->d_rmax + l, 0, sizeof(unsigned), s);
  unsigned nb = std::min<unsigned>(blocks_for(C.N), (unsigned)(2 * m->sm_count));
  hhg_launch(k_absmax_bits, nb, kBlock, 0, s, (const float*)C.r32, (int64_t)C.N, m->d_rmax + l);
  const int copies = std::max({1, m->verts.max_copies, m->edges.max_copies, m->faces.max_copies});
  const double level_factor = std::ldexp((double)copies, l * DIM);
  hhg_launch(k_set_scale16, 1, 32, 0, s, (const unsigned*)(m->d_rmax + l), (const double*)m->d_ainv_inf,
             level_factor, C.cscale);
}

// V(pre, post)-cycle in binary32 on level l for A x = rhs; x has storage type U (binary32 on the
// top level), the coarse corrections have storage type S.
template <int DIM, typename S, typename U>
static void vcycle32(hhg_mesh_s* m, int l, U* x, const float* rhs, const hhg_solve_params& p, cudaStream_t s) {
  if (l == 0) {
    coarse32<DIM, U>(m, x, rhs, s);
    return;
  }
  LevelData& Lv = m->lv[l];
  LevelData& C = m->lv[l - 1];
  for (int q = 0; q < p.pre; ++q) sweep32<DIM, U>(m, l, x, rhs, s);
  // Every node's residual is computed: the last interior colour's residual after a sweep is zero
  // only up to rounding, and in binary32 that rounding (and the rounding of the normalised stencil
  // the sweep uses) is systematic and not small against the residual the coarse grid has to see.
  residual_t<DIM, float, U, float>(m, l, cvec_of<U>(m, l, x), CVec<float, float>{rhs, nullptr}, m->dS32, Lv.t32, s,
                                   false);
  dim3 gr(blocks_for(C.Nt), m->nc);
  hhg_launch(k_restrict<DIM, float, float, float>, gr, kBlock, 0, s, ctx(m, l), ctx(m, l - 1), m->d_dirmask, Lv.t32, C.r32);
  if constexpr (std::is_same<S, __half>::value) set_scale16<DIM>(m, l - 1, s);
  S* c = (S*)C.c16;
  cudaMemsetAsync(c, 0, sizeof(S) * (size_t)C.N, s);
  vcycle32<DIM, S, S>(m, l - 1, c, C.r32, p, s);
  dim3 gf(blocks_for(Lv.Nt), m->nc);
  hhg_launch(k_prolong_add<DIM, float, S, U>, gf, kBlock, 0, s, ctx(m, l), ctx(m, l - 1), m->d_dirmask,
                                                         cvec_of<S>(m, l - 1, c), vec_of<U>(m, l, x));
  for (int q = 0; q < p.post; ++q) sweep32<DIM, U>(m, l, x, rhs, s);
}

void launch_build_rhs(hhg_mesh_s* m, int l, cudaStream_t s);
void launch_build_rhs32(hhg_mesh_s* m, int l, cudaStream_t s);
void launch_residual(hhg_mesh_s* m, int l, const double* rhs, cudaStream_t s);

void launch_to_f32(const double* a, float* b, int64_t n, cudaStream_t s) {
  hhg_launch(k_to_f32, blocks_for(n), kBlock, 0, s, a, b, n);
}
void launch_to_f64(const float* a, double* b, int64_t n, cudaStream_t s) {
  hhg_launch(k_to_f64, blocks_for(n), kBlock, 0, s, a, b, n);
}

// binary64 level-L residual of the refinement, interface partials collected in binary64, then
// narrowed to binary32 (r32_L)
template <int DIM>
static void ir_residual(hhg_mesh_s* m, cudaStream_t s) {
  const int L = m->L;
  LevelData& LL = m->lv[L];
  launch_residual(m, L, LL.b, s);  // partial binary64 residual of u_L into LL.tmp
  int n = LL.n;
  const Prims& PV = m->verts;
  if (PV.count)
    hhg_launch(k_owner_collect<DIM>, blocks_for(PV.count), kBlock, 0, s, PV.count, 1, 1, nullptr, PV.d_ptr, PV.d_cell,
                                                                 PV.d_loc, ctx(m, L), LL.tmp);
  const Prims& PE = m->edges;
  if (PE.count && n >= 2)
    hhg_launch(k_owner_collect<DIM>, blocks_for((int64_t)PE.count * (n - 1)), kBlock, 0, s, 
        PE.count, 2, n - 1, nullptr, PE.d_ptr, PE.d_cell, PE.d_loc, ctx(m, L), LL.tmp);
  const Prims& PF = m->faces;
  int64_t nf = LL.fcol_off[3];
  if (DIM == 3 && PF.count && nf > 0)
    hhg_launch(k_owner_collect<DIM>, blocks_for((int64_t)PF.count * nf), kBlock, 0, s, 
        PF.count, 3, (int)nf, LL.d_fcol, PF.d_ptr, PF.d_cell, PF.d_loc, ctx(m, L), LL.tmp);
  hhg_launch(k_to_f32, blocks_for(LL.N), kBlock, 0, s, LL.tmp, LL.r32, LL.N);
}
void launch_finite_check(hhg_mesh_s* m, const double* v, int64_t n, cudaStream_t s);

template <int DIM, typename S>
static void mixed_solve_t(hhg_mesh_s* m, const hhg_solve_params& p, cudaStream_t s) {
  const int L = m->L;
  const LevelData& LL = m->lv[L];
  // binary64 b_L (the refinement's residual right-hand side) and its binary32 copy for the binary32
  // FMG's top level; the coarser right-hand sides only serve the binary32 FMG: built in binary32
  launch_build_rhs(m, L, s);
  hhg_launch(k_to_f32, blocks_for(LL.N), kBlock, 0, s, LL.b, LL.b32, LL.N);
  if (p.rhs == 0) {
    for (int l = 0; l < L; ++l) launch_build_rhs32(m, l, s);
  } else {  // b_{l-1} = I^T b_l from the binary32 copy of b_L
    for (int l = L; l >= 1; --l) {
      dim3 gr(blocks_for(m->lv[l - 1].Nt), m->nc);
      hhg_launch(k_restrict<DIM, float, float, float>, gr, kBlock, 0, s, ctx(m, l), ctx(m, l - 1), m->d_dirmask,
                 (const float*)m->lv[l].b32, m->lv[l - 1].b32);
    }
  }
  {
    const LevelData& L0 = m->lv[0];
    dim3 g0(blocks_for(L0.Nt), m->nc);
    hhg_launch(k_init_coarse32<DIM>, g0, kBlock, 0, s, ctx(m, 0), LL.n, LL.Nt, L, m->gL, m->d_dirmask, L0.x32);
  }
  // step 1: binary32 FMG
  for (int l = 0; l <= L; ++l) {
    for (int q = 0; q < p.nu; ++q) vcycle32<DIM, S, float>(m, l, m->lv[l].x32, m->lv[l].b32, p, s);
    if (l < L) {
      const LevelData& F = m->lv[l + 1];
      dim3 gf(blocks_for(F.Nt), m->nc);
      hhg_launch(k_fmg_prolong32<DIM>, gf, kBlock, 0, s, ctx(m, l + 1), ctx(m, l), LL.n, LL.Nt, L - l - 1, m->gL,
                                                 m->d_dirmask, m->lv[l].x32, F.x32, m->lv[l].w);
    }
  }
  {
    dim3 gl(blocks_for(LL.Nt), m->nc);
    hhg_launch(k_to_f64_level<DIM>, gl, kBlock, 0, s, ctx(m, L), m->d_dirmask, m->gL, LL.x32, LL.u);
  }
  // refinement steps: binary64 residual and update, binary32 V-cycles on the correction
  for (int it = 0; it < p.ir_steps; ++it) {
    ir_residual<DIM>(m, s);
    cudaMemsetAsync(LL.x32, 0, sizeof(float) * (size_t)LL.N, s);
    for (int q = 0; q < p.ir_vcycles; ++q) vcycle32<DIM, S, float>(m, L, LL.x32, LL.r32, p, s);
    hhg_launch(k_add_f32, blocks_for(LL.N), kBlock, 0, s, LL.x32, LL.u, LL.N);
  }
  for (int q = 0; q < p.n_extra; ++q) {
    ir_residual<DIM>(m, s);
    cudaMemsetAsync(LL.x32, 0, sizeof(float) * (size_t)LL.N, s);
    vcycle32<DIM, S, float>(m, L, LL.x32, LL.r32, p, s);
    hhg_launch(k_add_f32, blocks_for(LL.N), kBlock, 0, s, LL.x32, LL.u, LL.N);
  }
  cudaMemsetAsync(m->d_flag, 0, sizeof(int), s);
  launch_finite_check(m, LL.u, LL.N, s);
}

// One binary64 refinement step on level L: r = b_L - A_L u_L in binary64 (interface partials
// collected), the correction from nv binary32 V-cycles (coarse corrections stored as S), u_L += c.
template <int DIM, typename S>
static void ir_step(hhg_mesh_s* m, int nv, const hhg_solve_params& p, cudaStream_t s) {
  LevelData& LL = m->lv[m->L];
  ir_residual<DIM>(m, s);
  cudaMemsetAsync(LL.x32, 0, sizeof(float) * (size_t)LL.N, s);
  for (int q = 0; q < nv; ++q) vcycle32<DIM, S, float>(m, m->L, LL.x32, LL.r32, p, s);
  hhg_launch(k_add_f32, blocks_for(LL.N), kBlock, 0, s, LL.x32, LL.u, LL.N);
}

// Mixed-precision adjoint solve A lam = b_L, where b_L holds the adjoint right-hand side and the
// Dirichlet values are zero: binary64 refinement from lam = 0 with the forward solve's storage rule.
// The adjoint right-hand side is given on level L only, so the first step takes ir_vcycles binary32
// V-cycles where the forward solve takes a binary32 FMG; ir_steps steps of ir_vcycles V-cycles and
// n_extra steps of one V-cycle follow, as in the forward solve.
template <int DIM, typename S>
static void mixed_adjoint_t(hhg_mesh_s* m, const hhg_solve_params& p, cudaStream_t s) {
  LevelData& LL = m->lv[m->L];
  cudaMemsetAsync(LL.u, 0, sizeof(double) * (size_t)LL.N, s);
  for (int it = 0; it <= p.ir_steps; ++it) ir_step<DIM, S>(m, p.ir_vcycles, p, s);
  for (int q = 0; q < p.n_extra; ++q) ir_step<DIM, S>(m, 1, p, s);
  cudaMemsetAsync(m->d_flag, 0, sizeof(int), s);
  launch_finite_check(m, LL.u, LL.N, s);
}

// nsweeps binary32 sweeps of the mixed path's smoother on level l, in place on lv[l].x32 with
// right-hand side lv[l].b32 (operator testing, hhg_apply op 4)
void mixed_sweeps(hhg_mesh_s* m, int l, int nsweeps, cudaStream_t s) {
  for (int q = 0; q < nsweeps; ++q) {
    if (m->dim == 2) sweep32<2, float>(m, l, m->lv[l].x32, m->lv[l].b32, s);
    else sweep32<3, float>(m, l, m->lv[l].x32, m->lv[l].b32, s);
  }
}

void mixed_enqueue_adjoint(hhg_mesh_s* m, const hhg_solve_params& p, cudaStream_t s) {
  if (p.storage == 1) {
    if (m->dim == 2) mixed_adjoint_t<2, __nv_bfloat16>(m, p, s);
    else mixed_adjoint_t<3, __nv_bfloat16>(m, p, s);
  } else if (p.storage == 2) {
    if (m->dim == 2) mixed_adjoint_t<2, __half>(m, p, s);
    else mixed_adjoint_t<3, __half>(m, p, s);
  } else {
    if (m->dim == 2) mixed_adjoint_t<2, float>(m, p, s);
    else mixed_adjoint_t<3, float>(m, p, s);
  }
}

void mixed_enqueue_solve(hhg_mesh_s* m, const hhg_solve_params& p, cudaStream_t s) {
  if (p.storage == 1) {
    if (m->dim == 2) mixed_solve_t<2, __nv_bfloat16>(m, p, s);
    else mixed_solve_t<3, __nv_bfloat16>(m, p, s);
  } else if (p.storage == 2) {
    if (m->dim == 2) mixed_solve_t<2, __half>(m, p, s);
    else mixed_solve_t<3, __half>(m, p, s);
  } else {
    if (m->dim == 2) mixed_solve_t<2, float>(m, p, s);
    else mixed_solve_t<3, float>(m, p, s);
  }
}

// binary16 storage: the bound |A_0^{-1}|_inf (changed by hhg_set_coefficient) is copied on the mesh
// stream before every solve, so graphs captured earlier read the current value
static hhg_status upload_ainv_inf(hhg_mesh_s* m) {
  cudaError_t e = cudaMemcpyAsync(m->d_ainv_inf, &m->ainv_inf, sizeof(double), cudaMemcpyHostToDevice, m->stream);
  return e == cudaSuccess ? HHG_OK : cuda_fail(e, "cudaMemcpyAsync");
}

hhg_status mixed_prepare(hhg_mesh_s* m, int storage) {
  if (storage == 2 && m->n0f == 0) {
    set_error("binary16 correction storage needs at least one free macro vertex (the range of the corrections "
              "is bounded through the inverse of the level-0 operator); use storage 0 or 1");
    return HHG_ERR_ARG;
  }
  size_t esz = storage == 0 ? 4 : 2;
  if (m->mixed_alloc && m->last_storage == storage) return storage == 2 ? upload_ainv_inf(m) : HHG_OK;
  if (m->mixed_alloc) {
    // the correction buffers are reallocated below for the new storage type, and the cached
    // mixed-precision graphs (keys "mixed:..." and "mixed-adjoint:...") hold their old addresses:
    // let queued work finish, then drop those graphs (they are captured again on their next use;
    // their launch counts stay valid)
    cudaError_t e = cudaStreamSynchronize(m->stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    for (auto it = m->graphs.begin(); it != m->graphs.end();) {
      if (it->first.compare(0, 5, "mixed") == 0) {
        cudaGraphExecDestroy(it->second);
        it = m->graphs.erase(it);
      } else {
        ++it;
      }
    }
  }
  if (storage == 2 && !m->d_rmax) {
    cudaError_t e;
    if ((e = cudaMalloc(&m->d_rmax, sizeof(unsigned) * (m->L + 1))) != cudaSuccess) return cuda_fail(e, "cudaMalloc");
    if ((e = cudaMemset(m->d_rmax, 0, sizeof(unsigned) * (m->L + 1))) != cudaSuccess) return cuda_fail(e, "cudaMemset");
    if ((e = cudaMalloc(&m->d_ainv_inf, sizeof(double))) != cudaSuccess) return cuda_fail(e, "cudaMalloc");
    m->bytes += (long long)(sizeof(unsigned) * (m->L + 1) + sizeof(double));
  }
  for (auto& Lv : m->lv) {
    if (m->mixed_alloc && m->last_storage == 2) {
      // leaving binary16 storage: the other storage types run with scale 1
      float one = 1.0f;
      cudaError_t e = cudaMemcpy(Lv.cscale, &one, sizeof(float), cudaMemcpyHostToDevice);
      if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy");
    }
    if (!m->mixed_alloc) {
      cudaError_t e;
      // kVecPad spare values: the fused sweep's bulk copies read 16-byte windows that may end past
      // the last node
      const size_t nb = sizeof(float) * (Lv.N + kVecPad);
      if ((e = cudaMalloc(&Lv.x32, nb)) != cudaSuccess) return cuda_fail(e, "cudaMalloc");
      if ((e = cudaMalloc(&Lv.b32, nb)) != cudaSuccess) return cuda_fail(e, "cudaMalloc");
      if ((e = cudaMalloc(&Lv.r32, nb)) != cudaSuccess) return cuda_fail(e, "cudaMalloc");
      if ((e = cudaMalloc(&Lv.t32, nb)) != cudaSuccess) return cuda_fail(e, "cudaMalloc");
      if ((e = cudaMalloc(&Lv.cscale, sizeof(float))) != cudaSuccess) return cuda_fail(e, "cudaMalloc");
      m->bytes += (long long)(4 * nb + 4);
      for (float* q : {Lv.x32, Lv.b32, Lv.r32, Lv.t32})
        if ((e = cudaMemset(q, 0, nb)) != cudaSuccess) return cuda_fail(e, "cudaMemset");
      float one = 1.0f;
      if ((e = cudaMemcpy(Lv.cscale, &one, sizeof(float), cudaMemcpyHostToDevice)) != cudaSuccess)
        return cuda_fail(e, "cudaMemcpy");
    }
    if (Lv.c16) {
      cudaFree(Lv.c16);
      Lv.c16 = nullptr;
    }
    cudaError_t e = cudaMalloc(&Lv.c16, esz * (Lv.N + kVecPad));
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc");
    if ((e = cudaMemset(Lv.c16, 0, esz * (Lv.N + kVecPad))) != cudaSuccess) return cuda_fail(e, "cudaMemset");
  }
  m->mixed_alloc = true;
  m->last_storage = storage;
  return storage == 2 ? upload_ainv_inf(m) : HHG_OK;
}

// Profiling: the level-L interior stage of the first cell group as the solve runs it: the fused sweep
// (all colours; algorithmic bytes = u of every closure node read once, b read and u written at the
// interior nodes) or, where the fused sweep is not used, the colour-0 list stage (u of the group's
// closures read once, b read and u written at the colour's nodes).
hhg_status mixed_profile_interior(hhg_mesh_s* m, int reps, cudaStream_t s, long long* units, double* bytes,
                                  double* flops) {
  const int L = m->L;
  LevelData& Lv = m->lv[L];
  const Group& G = m->groups[0];
  const bool fused = use_fused<float>(m, L, 0);
  int64_t len = fused ? Lv.icol_off[0][G.m] - Lv.icol_off[0][0] : Lv.icol_off[0][1] - Lv.icol_off[0][0];
  long long nodes = (long long)len * (long long)G.cells.size();
  int p = __builtin_popcount(G.pmask);
  *units = nodes;
  *bytes = 4.0 * ((double)Lv.Nt * G.cells.size() + 2.0 * nodes);
  *flops = (4.0 * p + 1.0) * nodes;
  for (int r = 0; r < reps; ++r) {
    if (fused) fused32_dispatch<float>(m, L, 0, Lv.x32, Lv.b32, s);
    else if (m->dim == 2) interior32_dispatch<2, float>(m, L, 0, 0, Lv.x32, Lv.b32, s);
    else interior32_dispatch<3, float>(m, L, 0, 0, Lv.x32, Lv.b32, s);
  }
  return HHG_OK;
}

}  // namespace hhg
