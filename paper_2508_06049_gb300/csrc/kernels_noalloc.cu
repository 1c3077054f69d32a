// Allocation-free variant of the per-cell mass-norm reduction (the estimator's eta_T^2 kernel).
//
// Some callers cannot allocate device memory at the point where they need the local indicators: a
// caller that is itself recording a CUDA stream capture (cudaMalloc is not allowed inside a capture),
// or a serving process that runs under a fixed, pre-reserved device-memory budget where a fresh
// allocation can fail in the middle of a run.  hhg_cell_mass_norms_noalloc takes its inputs and its
// output from the caller and keeps its only scratch (one partial sum per cell and chunk) in the
// file-scope array below: kNoAllocScratch doubles (8 MiB) on every GPU that loads the library, held
// until the process exits.
#include <cstdio>

#include "internal.h"
#include "kernels_impl.cuh"

namespace hhg {

constexpr int64_t kNoAllocScratch = int64_t(1) << 20;  // doubles (8 MiB)
static __device__ __align__(256) double g_noalloc_part[kNoAllocScratch];

// Host code may not use g_noalloc_part as an address (it is a host-side stand-in): the device address
// is looked up once per device with that device current and cached here.
static constexpr int kMaxDevices = 64;
static double* g_part_addr[kMaxDevices] = {nullptr};

// x^T M_T x with x = a - b over the nodes of one chunk of cell T (symmetric half stencil, as in the
// estimator), block tree sum in shared memory, one partial per (cell, chunk).
template <int DIM>
__global__ void __launch_bounds__(256) k_noalloc_form(LevelCtx lc, int items, int nchunks, const double* __restrict__ tab,
                                                      const double* __restrict__ a, const double* __restrict__ b,
                                                      double* __restrict__ part) {
  grid_dependency_sync();
  __shared__ double sh[256];
  int T = blockIdx.y, chunk = blockIdx.x;
  double acc = 0;
  int64_t base = (int64_t)chunk * items * 256;
  for (int it = 0; it < items; ++it) {
    int64_t loc = base + (int64_t)it * 256 + threadIdx.x;
    if (loc >= lc.Nt) break;
    int i, j, k;
    decode(lc.ijk[loc], i, j, k);
    int t = boundary_type(DIM, lc.n, i, j, k);
    int64_t g = (int64_t)T * lc.Nt + loc;
    int64_t off[15];
    neighbour_offsets(DIM, lc.n, j, k, off);
    uint32_t vm = valid_dirs_tab(DIM, t);
    mask_offsets(DIM, vm, off);
    const double* s = tab + (size_t)T * kStencilStride + t * kMaxDirs;
    double xp = a[g] - (b ? b[g] : 0.0);
    double sum = s[0] * xp * xp;
    for (int q = 0; q < npairs<DIM>(); ++q) {
      int d = 2 * q + 1;
      if (!(vm >> d & 1)) continue;
      double xq = a[g + off[d]] - (b ? b[g + off[d]] : 0.0);
      sum += 2.0 * s[d] * xp * xq;
    }
    acc += sum;
  }
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[(int64_t)T * nchunks + chunk] = sh[0];
}

__global__ void k_noalloc_sum(int nc, int nchunks, double scale, const double* __restrict__ part,
                              double* __restrict__ out) {
  grid_dependency_sync();
  int T = blockIdx.x * blockDim.x + threadIdx.x;
  if (T >= nc) return;
  double s = 0;
  for (int c = 0; c < nchunks; ++c) s += part[(int64_t)T * nchunks + c];
  out[T] = scale * s;
}

}  // namespace hhg

using namespace hhg;

extern "C" hhg_status hhg_cell_mass_norms_noalloc(hhg_mesh m, const double* a, const double* b, double* out) {
  if (!m || !a || !out) {
    set_error("hhg_cell_mass_norms_noalloc: NULL argument");
    return HHG_ERR_ARG;
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev != m->device) {
    set_error("hhg_cell_mass_norms_noalloc: the mesh's device (%d) must be current (is %d)", m->device, dev);
    return HHG_ERR_ARG;
  }
  if (dev < 0 || dev >= kMaxDevices) {
    set_error("hhg_cell_mass_norms_noalloc: device index %d beyond %d", dev, kMaxDevices);
    return HHG_ERR_ARG;
  }
#ifdef HHG_CHECK
  // checked build: every pointer must be device memory of the mesh's device (allocates nothing)
  {
    const void* ptrs[3] = {a, b, out};
    const char* names[3] = {"a", "b", "out"};
    for (int q = 0; q < 3; ++q) {
      if (!ptrs[q]) continue;
      cudaPointerAttributes pa;
      cudaError_t pe = cudaPointerGetAttributes(&pa, ptrs[q]);
      if (pe != cudaSuccess || pa.type != cudaMemoryTypeDevice || pa.device != m->device) {
        cudaGetLastError();
        set_error("hhg_cell_mass_norms_noalloc: %s = %p is not device memory of device %d", names[q], ptrs[q],
                  m->device);
        return HHG_ERR_STATE;
      }
    }
  }
#endif
  const LevelData& Lv = m->lv[m->L];
  // chunks of items * 256 nodes per cell such that all partials fit the static scratch
  int64_t per_cell_max = kNoAllocScratch / m->nc;
  if (per_cell_max < 1 || m->nc > 65535) {
    set_error("hhg_cell_mass_norms_noalloc: %d cells exceed the limit (65535 cells and a static scratch of "
              "%lld partial sums)", m->nc, (long long)kNoAllocScratch);
    return HHG_ERR_ARG;
  }
  int items = 1;
  int64_t nchunks = (Lv.Nt + 255) / 256;
  while (nchunks > per_cell_max || nchunks > 65535) {
    items *= 2;
    nchunks = (Lv.Nt + 256LL * items - 1) / (256LL * items);
  }
  if (!g_part_addr[dev]) {  // first call on this device: look up the array's device address
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_part);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress");
    g_part_addr[dev] = (double*)p;
  }
  double* part = g_part_addr[dev];
  cudaStream_t s = m->stream;
  if (m->own) {  // order after the caller's legacy-stream work, as every entry point does
    if ((e = cudaEventRecord(m->ev_legacy, (cudaStream_t)0)) != cudaSuccess) return cuda_fail(e, "cudaEventRecord");
    if ((e = cudaStreamWaitEvent(s, m->ev_legacy, 0)) != cudaSuccess) return cuda_fail(e, "cudaStreamWaitEvent");
  }
  LevelCtx lc{Lv.n, Lv.Nt, Lv.d_ijk, nullptr};
  dim3 grid((unsigned)nchunks, (unsigned)m->nc);
  if (m->dim == 2) hhg_launch(k_noalloc_form<2>, grid, 256, 0, s, lc, items, (int)nchunks, m->dM, a, b, part);
  else hhg_launch(k_noalloc_form<3>, grid, 256, 0, s, lc, items, (int)nchunks, m->dM, a, b, part);
  double n = (double)Lv.n;
  double scale = m->dim == 2 ? 1.0 / (n * n) : 1.0 / (n * n * n);
  hhg_launch(k_noalloc_sum, (m->nc + 255) / 256, 256, 0, s, m->nc, (int)nchunks, scale, part, out);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "hhg_cell_mass_norms_noalloc launch");
  return HHG_OK;
}
