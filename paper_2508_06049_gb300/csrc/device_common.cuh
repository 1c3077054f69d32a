// Device-side helpers shared by the HHG kernels: storage conversions and per-level context.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "lattice.h"

namespace hhg {

// ---- storage <-> compute conversions (vectors may be stored narrower than they are computed) ----
template <typename R, typename S> struct Conv;
template <> struct Conv<double, double> {
  static __device__ __forceinline__ double ld(const double* p) { return *p; }
  static __device__ __forceinline__ void st(double* p, double v) { *p = v; }
};
template <> struct Conv<float, float> {
  static __device__ __forceinline__ float ld(const float* p) { return *p; }
  static __device__ __forceinline__ void st(float* p, float v) { *p = v; }
};
template <> struct Conv<float, __nv_bfloat16> {
  static __device__ __forceinline__ float ld(const __nv_bfloat16* p) { return __bfloat162float(*p); }
  static __device__ __forceinline__ void st(__nv_bfloat16* p, float v) { *p = __float2bfloat16_rn(v); }
};
template <> struct Conv<float, __half> {
  static __device__ __forceinline__ float ld(const __half* p) { return __half2float(*p); }
  // saturating store: a magnitude beyond binary16's largest finite value is stored as +-65504 (NaN
  // stays NaN), so a correction that outgrows its scale is clipped, not turned into an infinity
  static __device__ __forceinline__ void st(__half* p, float v) {
    if (fabsf(v) > 65504.0f) v = copysignf(65504.0f, v);
    *p = __float2half_rn(v);
  }
};

template <typename S> struct IsNarrow { static constexpr bool value = false; };
template <> struct IsNarrow<__nv_bfloat16> { static constexpr bool value = true; };
template <> struct IsNarrow<__half> { static constexpr bool value = true; };

// A vector of one level: storage pointer plus (for 16-bit storage) a power-of-two scale held in
// device memory: stored value = true value * scale.
template <typename R, typename S> struct Vec {
  S* p;
  const float* scale;  // device pointer or nullptr (scale 1)
  __device__ __forceinline__ R get(int64_t i) const {
    R v = Conv<R, S>::ld(p + i);
    if constexpr (IsNarrow<S>::value) v = v * (R)(1.0f / *scale);
    return v;
  }
  __device__ __forceinline__ void set(int64_t i, R v) const {
    if constexpr (IsNarrow<S>::value) v = v * (R)(*scale);
    Conv<R, S>::st(p + i, v);
  }
};
template <typename R, typename S> struct CVec {
  const S* p;
  const float* scale;
  __device__ __forceinline__ R get(int64_t i) const {
    R v = Conv<R, S>::ld(p + i);
    if constexpr (IsNarrow<S>::value) v = v * (R)(1.0f / *scale);
    return v;
  }
};

// ---- per-level lattice context ----
// Every kernel is launched with programmatic stream serialisation (hhg_launch): the next kernel in a
// stream or graph may be scheduled while the current one drains.  Each kernel therefore starts by
// waiting (griddepcontrol.wait, a hardware wait, before any global memory access) until the
// preceding grid has completed and its writes are visible, and then allows its own successor to be
// scheduled.  Launched without the attribute, both instructions have no effect.
__device__ __forceinline__ void grid_dependency_sync() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

struct LevelCtx {
  int n;             // 2^l
  int64_t Nt;        // closure nodes per macro cell
  const int32_t* ijk;  // decode table: packed index -> i | j<<10 | k<<20
  const uint16_t* nzs;  // [cell][type]: stiffness slots with a nonzero entry (nullptr: all)
  const int2* itab;     // levels >= 1: interpolation end points and boundary type per node
};

__device__ __forceinline__ void decode(int32_t c, int& i, int& j, int& k) {
  i = c & 1023;
  j = (c >> 10) & 1023;
  k = c >> 20;
}

// ---- debug build (-DHHG_CHECK): bounds checks that record the first failure and skip the access
#ifdef HHG_CHECK
// one copy per translation unit (only kernels.cu launches checked kernels and reads it)
static __device__ long long g_hhg_check[8];
__device__ __forceinline__ bool hhg_bounds_fail(long long idx, long long n, int code) {
  if (idx >= 0 && idx < n) return false;
  if (atomicCAS((unsigned long long*)&g_hhg_check[0], 0ull, (unsigned long long)code) == 0ull) {
    g_hhg_check[1] = blockIdx.x;
    g_hhg_check[2] = blockIdx.y;
    g_hhg_check[3] = threadIdx.x;
    g_hhg_check[4] = idx;
    g_hhg_check[5] = n;
  }
  return true;
}
// true if idx is outside [0, n): the caller skips the access (never returns before a barrier)
#define HHG_OOB(idx, n, code) hhg_bounds_fail((long long)(idx), (long long)(n), (code))
#else
#define HHG_OOB(idx, n, code) false
#endif

// stencil table layout: [cell][kMaxTypes][kMaxDirs]
constexpr int kStencilStride = kMaxTypes * kMaxDirs;

template <int DIM> __host__ __device__ constexpr int ndirs() { return DIM == 2 ? 7 : 15; }
template <int DIM> __host__ __device__ constexpr int npairs() { return DIM == 2 ? 3 : 7; }

}  // namespace hhg
