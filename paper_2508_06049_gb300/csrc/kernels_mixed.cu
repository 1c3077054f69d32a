// Mixed-precision iterative refinement (no counterpart in the paper).
//
// Step 1: FMG (Alg. 4 structure, same stage-ordered smoother) computed in binary32 on the original
//         problem: the iterate of the current FMG top level is a binary32 vector, the coarse-grid
//         corrections below it are stored as binary32, bfloat16 or binary16 and accumulated in
//         binary32.  The prolongated iterates w_l are written in binary64 for the estimator.
//         binary16 has five exponent bits, so each level's correction is stored times a power of two
//         chosen, after the restriction, from max |r| of its right-hand side and a bound of
//         |A_l^{-1}|_inf (k_set_scale16).
// Steps 2..: r = b_L - A_L u_L and u_L += c on level L, carried in pairs of binary32 values with
//         exact products and sums (about 2^-46 relative per operation, against binary64's 2^-53;
//         GB300 runs binary32 at 64 times its binary64 rate); the correction c solves A_L c = r with
//         V-cycles computed in binary32 (same storage rule for the coarse levels).  u_L is returned
//         in binary64.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <type_traits>

#include "internal.h"
#include "kernels_impl.cuh"

namespace hhg {

// ---------------------------------------------------------------- elementwise kernels

// Elementwise kernels over whole level vectors (cudaMalloc'd, so 256-byte aligned): four values per
// thread and step through 16-byte vector accesses, grid-stride, the n % 4 tail by thread 0 of block 0.
__global__ void k_to_f32(const double* __restrict__ a, float* __restrict__ b, int64_t n) {
  grid_dependency_sync();
  const int64_t n4 = n / 4;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += (int64_t)gridDim.x * blockDim.x) {
    const double2 x = reinterpret_cast<const double2*>(a)[2 * i], y = reinterpret_cast<const double2*>(a)[2 * i + 1];
    reinterpret_cast<float4*>(b)[i] = make_float4((float)x.x, (float)x.y, (float)y.x, (float)y.y);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0)
    for (int64_t i = 4 * n4; i < n; ++i) b[i] = (float)a[i];
}

__global__ void k_to_f64(const float* __restrict__ a, double* __restrict__ b, int64_t n) {
  grid_dependency_sync();
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = (double)a[i];
}

// grid of the vectorised elementwise kernels: enough blocks to fill the GPU several times over
inline unsigned elementwise_blocks(const hhg_mesh_s* m, int64_t n) {
  return std::max(1u, std::min<unsigned>(blocks_for((n + 3) / 4), (unsigned)(16 * m->sm_count)));
}
// the same for the kernels that take two values per access
inline unsigned pair_blocks(const hhg_mesh_s* m, int64_t n) {
  return std::max(1u, std::min<unsigned>(blocks_for((n + 1) / 2), (unsigned)(16 * m->sm_count)));
}

// ---- refinement on level L in binary32 hi/lo pairs ----
// The level-L iterate u_L, the right-hand side b_L and the residual of the refinement steps need
// more than binary32; GB300 runs binary64 at 2 FMA per SM and clock against 128 for binary32, so
// they are carried as pairs of binary32 values with exact products and sums (dfloat.cuh): u_L as a
// pair per node (in the 8 bytes of its binary64 slot), b_L formed from pairs and stored in binary64,
// the residual as pairs until its interface partials are collected.  At the end u_L is written back
// in binary64.

// b_L = M_L f_L from f_L as pairs (fp, split once by k_sub_pair) and the mass stencils as pairs;
// stored in binary64 (b) and rounded to binary32 (b32); zero on Dirichlet rows.  mscale: the level's
// mass scale, a power of two (exact on pairs).
template <int DIM>
__global__ void k_build_rhs_pair(LevelCtx lc, const float2* __restrict__ fp, const float2* __restrict__ Mp,
                                 float mscale, const uint16_t* __restrict__ dirmask, double* __restrict__ b,
                                 float* __restrict__ b32) {
  grid_dependency_sync();
  int64_t loc = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (loc >= lc.Nt) return;
  int T = blockIdx.y;
  int i, j, k;
  decode(lc.ijk[loc], i, j, k);
  int t = boundary_type(DIM, lc.n, i, j, k);
  int64_t g = (int64_t)T * lc.Nt + loc;
  if (dirmask[T] >> t & 1) {
    b[g] = 0.0;
    b32[g] = 0.f;
    return;
  }
  const uint32_t vm = valid_dirs_tab(DIM, t);
  const float2* sm = Mp + (size_t)T * kStencilStride + t * kMaxDirs;
  int64_t off[15];
  neighbour_offsets(DIM, lc.n, j, k, off);
  mask_offsets(DIM, vm, off);
  float2 f[ndirs<DIM>()];
#pragma unroll
  for (int d = 0; d < ndirs<DIM>(); ++d) {
    const bool ok = (vm >> d & 1) && !HHG_OOB(loc + off[d], lc.Nt, 71);
    f[d] = ok ? fp[g + off[d]] : make_float2(0.f, 0.f);
  }
  DfAcc acc;
#pragma unroll
  for (int d = 0; d < ndirs<DIM>(); ++d) acc.add_prod(sm[d], f[d]);
  float2 v = acc.value();
  v.x = __fmul_rn(v.x, mscale);
  v.y = __fmul_rn(v.y, mscale);
  b[g] = df_to_double(v);
  b32[g] = __fadd_rn(v.x, v.y);
}

// u_L as pairs from the binary32 FMG result; Dirichlet nodes take the binary64 g split into a pair
template <int DIM>
__global__ void k_to_pair_level(LevelCtx lc, const uint16_t* __restrict__ dirmask, const double* __restrict__ gL,
                                const float* __restrict__ x, float2* __restrict__ up) {
  grid_dependency_sync();
  int64_t loc = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (loc >= lc.Nt) return;
  int T = blockIdx.y;
  int i, j, k;
  decode(lc.ijk[loc], i, j, k);
  int t = boundary_type(DIM, lc.n, i, j, k);
  int64_t g = (int64_t)T * lc.Nt + loc;
  up[g] = (dirmask[T] >> t & 1) ? df_split(gL[g]) : make_float2(x[g], 0.f);
}

// r = b - ss A u for one node of one cell copy on pairs: terms (stencil pair, value pair) already
// gathered, b in binary64 split here; ss: the level's stiffness scale, a power of two (exact)
template <int N>
__device__ __forceinline__ float2 pair_residual(const float2 (&s)[N], const float2 (&v)[N], double b, float ss) {
  DfAcc acc;
#pragma unroll
  for (int d = 0; d < N; ++d) acc.add_prod(s[d], v[d]);
  const float2 au = acc.value();
  DfAcc res;
  res.add(df_split(b));
  res.add(make_float2(-__fmul_rn(au.x, ss), -__fmul_rn(au.y, ss)));
  return res.value();
}

// Partial residual r = b - ss A_T u on pairs (u and r as pairs, b in binary64) for every closure node
// of the group's cells, zero on Dirichlet rows, from the node lists of k_residual_list (one cell per
// grid row): BND = false takes the interior list entries [0, ncomp) with the compile-time stencil
// pattern PM, BND = true the boundary-type nodes (every valid slot, the zero ones masked).  Two
// launches, so that the interior one keeps few registers (its occupancy hides the load latency).
template <int DIM, int PM, bool BND>
__global__ void __launch_bounds__(kBlock) k_residual_pair(const int* __restrict__ gcells, int ncells, LevelCtx lc,
                                                          const float2* __restrict__ Sp,
                                                          const uint16_t* __restrict__ dirmask, float ss,
                                                          const double* __restrict__ b, const float2* __restrict__ up,
                                                          float2* __restrict__ r, const int2* __restrict__ ilist,
                                                          int64_t ncomp, const int2* __restrict__ blist, int64_t nbnd,
                                                          unsigned bcomp) {
  grid_dependency_sync();
  constexpr int CPB = 1;
  constexpr int NT = 1 + 2 * __builtin_popcount(PM);  // centre + the coupled directions
  const int c0 = CPB * blockIdx.y;
  int Ts[CPB];
#pragma unroll
  for (int c = 0; c < CPB; ++c) Ts[c] = gcells[min(c0 + c, ncells - 1)];  // a short last group repeats
  const unsigned bx = blockIdx.x;
  if (!BND) {
    const int64_t pos = (int64_t)bx * blockDim.x + threadIdx.x;
    if (pos >= ncomp) return;
    const int2 e = ilist[pos];
    if (HHG_OOB(e.x, lc.Nt, 56)) return;
    const int j = e.y & 0xffff, k = e.y >> 16;
    int64_t off[15];
    neighbour_offsets(DIM, lc.n, j, k, off);
    float2 sv[CPB][NT], uv[CPB][NT];
    int64_t g[CPB];
#pragma unroll
    for (int c = 0; c < CPB; ++c) {
      g[c] = (int64_t)Ts[c] * lc.Nt + e.x;
      const float2* st = Sp + (size_t)Ts[c] * kStencilStride;  // interior type 0
      int n = 0;
      sv[c][n] = st[0];
      uv[c][n++] = up[g[c]];
#pragma unroll
      for (int q = 0; q < npairs<DIM>(); ++q)
        if (PM >> q & 1) {
          sv[c][n] = st[2 * q + 1];
          uv[c][n++] = up[g[c] + off[2 * q + 1]];
          sv[c][n] = st[2 * q + 2];
          uv[c][n++] = up[g[c] + off[2 * q + 2]];
        }
    }
#pragma unroll
    for (int c = 0; c < CPB; ++c)
      if (c0 + c < ncells)
        r[g[c]] = (dirmask[Ts[c]] & 1) ? make_float2(0.f, 0.f) : pair_residual(sv[c], uv[c], b[g[c]], ss);
  } else {
    const int64_t pos = (int64_t)bx * blockDim.x + threadIdx.x;
    if (pos >= nbnd) return;
    const int2 e = blist[pos];
    if (HHG_OOB(e.x, lc.Nt, 57)) return;
    int i, j, k;
    decode(e.y, i, j, k);
    const int t = boundary_type(DIM, lc.n, i, j, k);
    int64_t off[15];
    neighbour_offsets(DIM, lc.n, j, k, off);
    const uint32_t vt = valid_dirs_tab(DIM, t);
#pragma unroll
    for (int c = 0; c < CPB; ++c) {
      if (c0 + c >= ncells) continue;
      const int T = Ts[c];
      const int64_t g = (int64_t)T * lc.Nt + e.x;
      if (dirmask[T] >> t & 1) {
        r[g] = make_float2(0.f, 0.f);
        continue;
      }
      const uint32_t vm = vt & lc.nzs[T * kMaxTypes + t];
      const float2* st = Sp + (size_t)T * kStencilStride + t * kMaxDirs;
      float2 sv[ndirs<DIM>()], uv[ndirs<DIM>()];
#pragma unroll
      for (int d = 0; d < ndirs<DIM>(); ++d) {
        const bool ok = (vm >> d & 1) && !HHG_OOB(e.x + off[d], lc.Nt, 58);
        sv[d] = ok ? st[d] : make_float2(0.f, 0.f);
        uv[d] = ok ? up[g + off[d]] : make_float2(0.f, 0.f);
      }
      r[g] = pair_residual(sv, uv, b[g], ss);
    }
  }
}

// the pair partials of each interface node summed into its first copy, the other copies set to 0
// (k_owner_collect on pairs)
template <int DIM>
__global__ void k_owner_collect_pair(int nprim, int nverts, int cnt, const int32_t* __restrict__ flist,
                                     const int* __restrict__ ptr, const int* __restrict__ cell,
                                     const int* __restrict__ locv, LevelCtx lc, float2* __restrict__ v) {
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
  DfAcc sum;
  for (int c = ptr[e]; c < ptr[e + 1]; ++c) {
    int i, j, k;
    prim_position(locv[c], nverts, lc.n, s, t, i, j, k);
    sum.add(v[(int64_t)cell[c] * lc.Nt + packed_index(DIM, lc.n, i, j, k)]);
  }
  const float2 tot = sum.value();
  for (int c = ptr[e]; c < ptr[e + 1]; ++c) {
    int i, j, k;
    prim_position(locv[c], nverts, lc.n, s, t, i, j, k);
    v[(int64_t)cell[c] * lc.Nt + packed_index(DIM, lc.n, i, j, k)] = (c == ptr[e]) ? tot : make_float2(0.f, 0.f);
  }
}

// r32 = hi + lo rounded to binary32 (two pairs per 16-byte access, grid-stride)
__global__ void k_pair_to_f32(const float2* __restrict__ r, float* __restrict__ r32, int64_t n) {
  grid_dependency_sync();
  const int64_t n2 = n / 2;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n2; i += (int64_t)gridDim.x * blockDim.x) {
    const float4 p = reinterpret_cast<const float4*>(r)[i];
    reinterpret_cast<float2*>(r32)[i] = make_float2(__fadd_rn(p.x, p.y), __fadd_rn(p.z, p.w));
  }
  if (blockIdx.x == 0 && threadIdx.x == 0 && (n & 1)) r32[n - 1] = __fadd_rn(r[n - 1].x, r[n - 1].y);
}

// u + c on pairs (c binary32), renormalised
__device__ __forceinline__ float2 df_add_f(float2 u, float c) {
  const float2 s = df_two_sum(u.x, c);
  return df_fast_two_sum(s.x, __fadd_rn(u.y, s.y));
}

// u += c (c zero on Dirichlet nodes), two values per access, grid-stride
__global__ void k_add_pair(const float* __restrict__ c, float2* __restrict__ u, int64_t n) {
  grid_dependency_sync();
  const int64_t n2 = n / 2;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n2; i += (int64_t)gridDim.x * blockDim.x) {
    const float2 d = reinterpret_cast<const float2*>(c)[i];
    const float4 p = reinterpret_cast<const float4*>(u)[i];
    const float2 a = df_add_f(make_float2(p.x, p.y), d.x), b = df_add_f(make_float2(p.z, p.w), d.y);
    reinterpret_cast<float4*>(u)[i] = make_float4(a.x, a.y, b.x, b.y);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0 && (n & 1)) u[n - 1] = df_add_f(u[n - 1], c[n - 1]);
}

// u_L back to binary64 in place (each thread rewrites the 8 bytes it read)
__global__ void k_pair_to_f64(void* __restrict__ u, int64_t n) {
  grid_dependency_sync();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float2 p = reinterpret_cast<const float2*>(u)[i];
    reinterpret_cast<double*>(u)[i] = df_to_double(p);
  }
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
  int t;
  const float v = interp_tab<float>(fc, cc, T, loc, CVec<float, float>{xc, nullptr}, t);
  int64_t g = (int64_t)T * fc.Nt + loc;
  if (dirmask[T] >> t & 1) {
    int i, j, k;
    decode(fc.ijk[loc], i, j, k);
    int64_t q = packed_index(DIM, nL, (int64_t)i << shift, (int64_t)j << shift, (int64_t)k << shift);
    if (HHG_OOB(q, NtL, 81)) return;
    double gv = gL[(int64_t)T * NtL + q];
    xf[g] = (float)gv;
    w[g] = gv;
    return;
  }
  xf[g] = v;
  w[g] = df_widen(v);  // exact, without the conversion instruction (binary64 pipe)
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

// ---------------------------------------------------------------- launchers

static LevelCtx ctx(const hhg_mesh_s* m, int l) {
  const LevelData& Lv = m->lv[l];
  return LevelCtx{Lv.n, Lv.Nt, Lv.d_ijk, m->d_nzs, Lv.d_itab};
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

// all interior colours of a group at once, one CTA per cell (levels with short colour lists)
template <int DIM, int PM, typename U>
static void interior32_cells(hhg_mesh_s* m, int l, int gi, U* u, const float* rhs, cudaStream_t s) {
  const LevelData& Lv = m->lv[l];
  const Group& G = m->groups[gi];
  if (G.cells.empty() || Lv.icol_off[gi][G.m] <= Lv.icol_off[gi][0]) return;
  hhg_launch(k_smooth_interior_cell<DIM, PM, float, U, float>, (unsigned)G.cells.size(), kBlock, 0, s, G.d_cells,
             Lv.d_icol + Lv.icol_off[gi][0], colour_offsets(Lv, gi, G.m), ctx(m, l), m->d_tnormf, Lv.d_invlf,
             vec_of<U>(m, l, u), CVec<float, float>{rhs, nullptr});
}

template <int DIM, typename U>
static void interior32_cells_dispatch(hhg_mesh_s* m, int l, int gi, U* u, const float* rhs, cudaStream_t s) {
  int pm = m->groups[gi].pmask;
  if (DIM == 2) {
    switch (pm) {
      case 0x3: interior32_cells<DIM, 0x3, U>(m, l, gi, u, rhs, s); return;
      case 0x5: interior32_cells<DIM, 0x5, U>(m, l, gi, u, rhs, s); return;
      case 0x6: interior32_cells<DIM, 0x6, U>(m, l, gi, u, rhs, s); return;
      default: interior32_cells<DIM, 0x7, U>(m, l, gi, u, rhs, s); return;
    }
  } else {
    if (pm == 0x29) interior32_cells<DIM, 0x29, U>(m, l, gi, u, rhs, s);
    else interior32_cells<DIM, 0x7f, U>(m, l, gi, u, rhs, s);
  }
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
      if (interior_per_cell(Lv, m->groups)) {  // short lists: every colour in one launch per group
        if (c == 0)
          for (size_t gi = 0; gi < m->groups.size(); ++gi) interior32_cells_dispatch<DIM, U>(m, l, (int)gi, u, rhs, s);
        continue;
      }
      for (size_t gi = 0; gi < m->groups.size(); ++gi)
        if (c < m->groups[gi].m) interior32_dispatch<DIM, U>(m, l, (int)gi, c, u, rhs, s);
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
  S* c = (S*)C.c16;
  // restriction, and the coarse correction's starting value c = 0 in the same launch
  hhg_launch(k_restrict<DIM, float, float, float, S>, gr, kBlock, 0, s, ctx(m, l), ctx(m, l - 1), m->d_dirmask,
             (const float*)Lv.t32, C.r32, c);
  if constexpr (std::is_same<S, __half>::value) set_scale16<DIM>(m, l - 1, s);
  vcycle32<DIM, S, S>(m, l - 1, c, C.r32, p, s);
  dim3 gf(blocks_for(Lv.Nt), m->nc);
  hhg_launch(k_prolong_add<DIM, float, S, U>, gf, kBlock, 0, s, ctx(m, l), ctx(m, l - 1), m->d_dirmask,
                                                         cvec_of<S>(m, l - 1, c), vec_of<U>(m, l, x));
  for (int q = 0; q < p.post; ++q) sweep32<DIM, U>(m, l, x, rhs, s);
}

void launch_build_rhs(hhg_mesh_s* m, int l, cudaStream_t s);
void launch_build_rhs32(hhg_mesh_s* m, int l, cudaStream_t s);

void launch_to_f32(const double* a, float* b, int64_t n, cudaStream_t s) {
  hhg_launch(k_to_f32, std::max(1u, std::min<unsigned>(blocks_for((n + 3) / 4), 16u * 152u)), kBlock, 0, s, a, b, n);
}
void launch_to_f64(const float* a, double* b, int64_t n, cudaStream_t s) {
  hhg_launch(k_to_f64, blocks_for(n), kBlock, 0, s, a, b, n);
}

// level-L residual of the refinement on pairs (u_L as pairs in LL.u), interface partials collected
// on pairs, then rounded to binary32 (r32_L)
template <int DIM>
static void ir_residual(hhg_mesh_s* m, cudaStream_t s) {
  const int L = m->L;
  LevelData& LL = m->lv[L];
  float2* rp = (float2*)LL.tmp;
  for (size_t gi = 0; gi < m->groups.size(); ++gi) {
    const Group& G = m->groups[gi];
    if (G.cells.empty()) continue;
    ResidualSegments rs = residual_segments(LL, G, (int)gi, false);
    dim3 gi_(rs.bcomp, (unsigned)G.cells.size()), gb_(blocks_for(LL.nbnd), (unsigned)G.cells.size());
    const float ss = (float)stiff_scale(DIM, LL.n);
#define HHG_RP(PM)                                                                                                    \
  do {                                                                                                                \
  if (rs.bcomp)                                                                                                       \
    hhg_launch(k_residual_pair<DIM, PM, false>, gi_, kBlock, 0, s, G.d_cells, (int)G.cells.size(), ctx(m, L),        \
               (const float2*)m->dSp, m->d_dirmask, ss, (const double*)LL.b, (const float2*)LL.u, rp, rs.ilist,       \
               rs.ncomp, LL.d_bnd, LL.nbnd, rs.bcomp);                                                                \
  if (LL.nbnd)                                                                                                        \
    hhg_launch(k_residual_pair<DIM, PM, true>, gb_, kBlock, 0, s, G.d_cells, (int)G.cells.size(), ctx(m, L),         \
               (const float2*)m->dSp, m->d_dirmask, ss, (const double*)LL.b, (const float2*)LL.u, rp, rs.ilist,       \
               rs.ncomp, LL.d_bnd, LL.nbnd, rs.bcomp);                                                                \
  } while (0)
    if constexpr (DIM == 2) {
      switch (G.pmask) {
        case 0x3: HHG_RP(0x3); break;
        case 0x5: HHG_RP(0x5); break;
        case 0x6: HHG_RP(0x6); break;
        default: HHG_RP(0x7); break;
      }
    } else {
      if (G.pmask == 0x29) HHG_RP(0x29);
      else HHG_RP(0x7f);
    }
#undef HHG_RP
  }
  int n = LL.n;
  const Prims& PV = m->verts;
  if (PV.count)
    hhg_launch(k_owner_collect_pair<DIM>, blocks_for(PV.count), kBlock, 0, s, PV.count, 1, 1, nullptr, PV.d_ptr,
               PV.d_cell, PV.d_loc, ctx(m, L), rp);
  const Prims& PE = m->edges;
  if (PE.count && n >= 2)
    hhg_launch(k_owner_collect_pair<DIM>, blocks_for((int64_t)PE.count * (n - 1)), kBlock, 0, s, PE.count, 2, n - 1,
               nullptr, PE.d_ptr, PE.d_cell, PE.d_loc, ctx(m, L), rp);
  const Prims& PF = m->faces;
  int64_t nf = LL.fcol_off[3];
  if (DIM == 3 && PF.count && nf > 0)
    hhg_launch(k_owner_collect_pair<DIM>, blocks_for((int64_t)PF.count * nf), kBlock, 0, s, PF.count, 3, (int)nf,
               LL.d_fcol, PF.d_ptr, PF.d_cell, PF.d_loc, ctx(m, L), rp);
  hhg_launch(k_pair_to_f32, pair_blocks(m, LL.N), kBlock, 0, s, (const float2*)rp, LL.r32, LL.N);
}

// u_L (pairs) += the binary32 correction x32_L
static void ir_update(hhg_mesh_s* m, cudaStream_t s) {
  LevelData& LL = m->lv[m->L];
  hhg_launch(k_add_pair, pair_blocks(m, LL.N), kBlock, 0, s, (const float*)LL.x32, (float2*)LL.u, LL.N);
}

// u_L from pairs back to binary64, in place
static void ir_finish(hhg_mesh_s* m, cudaStream_t s) {
  LevelData& LL = m->lv[m->L];
  hhg_launch(k_pair_to_f64, elementwise_blocks(m, LL.N), kBlock, 0, s, (void*)LL.u, LL.N);
}
void launch_finite_check(hhg_mesh_s* m, const double* v, int64_t n, cudaStream_t s);

template <int DIM, typename S>
static void mixed_solve_t(hhg_mesh_s* m, const hhg_solve_params& p, cudaStream_t s) {
  const int L = m->L;
  const LevelData& LL = m->lv[L];
  // b_L (the refinement's residual right-hand side) from pairs, stored in binary64 and as the binary32
  // FMG's top-level right-hand side; the coarser right-hand sides only serve the binary32 FMG: built
  // in binary32
  launch_sub_pair(m, m->fL, nullptr, (float2*)LL.tmp, LL.N, s);
  {
    dim3 gl(blocks_for(LL.Nt), m->nc);
    hhg_launch(k_build_rhs_pair<DIM>, gl, kBlock, 0, s, ctx(m, L), (const float2*)LL.tmp, (const float2*)m->dMp,
               (float)mass_scale(DIM, LL.n), m->d_dirmask, LL.b, LL.b32);
  }
  if (p.rhs == 0) {
    for (int l = 0; l < L; ++l) launch_build_rhs32(m, l, s);
  } else {  // b_{l-1} = I^T b_l from the binary32 copy of b_L
    for (int l = L; l >= 1; --l) {
      dim3 gr(blocks_for(m->lv[l - 1].Nt), m->nc);
      hhg_launch(k_restrict<DIM, float, float, float>, gr, kBlock, 0, s, ctx(m, l), ctx(m, l - 1), m->d_dirmask,
                 (const float*)m->lv[l].b32, m->lv[l - 1].b32, (float*)nullptr);
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
    hhg_launch(k_to_pair_level<DIM>, gl, kBlock, 0, s, ctx(m, L), m->d_dirmask, m->gL, LL.x32, (float2*)LL.u);
  }
  // refinement steps: residual and update on pairs, binary32 V-cycles on the correction
  for (int it = 0; it < p.ir_steps; ++it) {
    ir_residual<DIM>(m, s);
    cudaMemsetAsync(LL.x32, 0, sizeof(float) * (size_t)LL.N, s);
    for (int q = 0; q < p.ir_vcycles; ++q) vcycle32<DIM, S, float>(m, L, LL.x32, LL.r32, p, s);
    ir_update(m, s);
  }
  for (int q = 0; q < p.n_extra; ++q) {
    ir_residual<DIM>(m, s);
    cudaMemsetAsync(LL.x32, 0, sizeof(float) * (size_t)LL.N, s);
    vcycle32<DIM, S, float>(m, L, LL.x32, LL.r32, p, s);
    ir_update(m, s);
  }
  ir_finish(m, s);
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
  ir_update(m, s);
}

// Mixed-precision adjoint solve A lam = b_L, where b_L holds the adjoint right-hand side and the
// Dirichlet values are zero: binary64 refinement from lam = 0 with the forward solve's storage rule.
// The adjoint right-hand side is given on level L only, so the first step takes ir_vcycles binary32
// V-cycles where the forward solve takes a binary32 FMG; ir_steps steps of ir_vcycles V-cycles and
// n_extra steps of one V-cycle follow, as in the forward solve.
template <int DIM, typename S>
static void mixed_adjoint_t(hhg_mesh_s* m, const hhg_solve_params& p, cudaStream_t s) {
  LevelData& LL = m->lv[m->L];
  cudaMemsetAsync(LL.u, 0, sizeof(double) * (size_t)LL.N, s);  // all-zero bits: the pair (0, 0)
  for (int it = 0; it <= p.ir_steps; ++it) ir_step<DIM, S>(m, p.ir_vcycles, p, s);
  for (int q = 0; q < p.n_extra; ++q) ir_step<DIM, S>(m, 1, p, s);
  ir_finish(m, s);
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
      const size_t nb = sizeof(float) * Lv.N;
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
    cudaError_t e = cudaMalloc(&Lv.c16, esz * Lv.N);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc");
    if ((e = cudaMemset(Lv.c16, 0, esz * Lv.N)) != cudaSuccess) return cuda_fail(e, "cudaMemset");
  }
  m->mixed_alloc = true;
  m->last_storage = storage;
  return storage == 2 ? upload_ainv_inf(m) : HHG_OK;
}

// Profiling: the level-L interior stage of colour 0 for the first cell group, as the solve launches it
// (algorithmic bytes: u of the group's closures read once, b read and u written at the colour's nodes)
hhg_status mixed_profile_interior(hhg_mesh_s* m, int reps, cudaStream_t s, long long* units, double* bytes,
                                  double* flops) {
  const int L = m->L;
  LevelData& Lv = m->lv[L];
  const Group& G = m->groups[0];
  int64_t len = Lv.icol_off[0][1] - Lv.icol_off[0][0];
  long long nodes = (long long)len * (long long)G.cells.size();
  int p = __builtin_popcount(G.pmask);
  *units = nodes;
  *bytes = 4.0 * ((double)Lv.Nt * G.cells.size() + 2.0 * nodes);
  *flops = (4.0 * p + 1.0) * nodes;
  for (int r = 0; r < reps; ++r) {
    if (m->dim == 2) interior32_dispatch<2, float>(m, L, 0, 0, Lv.x32, Lv.b32, s);
    else interior32_dispatch<3, float>(m, L, 0, 0, Lv.x32, Lv.b32, s);
  }
  return HHG_OK;
}

}  // namespace hhg
