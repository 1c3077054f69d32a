// Peak probe for the roofline denominators: binary64 and binary32 FMA throughput (8 independent FMA
// chains per thread, 8 CTAs of 256 threads per SM) and a device-to-device copy.  Bounded loops,
// in-bounds accesses only.  Build and run: python -m paper_2508_06049_gb300.peaks
#include <cstdio>
#include <cuda_runtime.h>
template <typename T>
__global__ void fma_loop(T* out, int iters, T a, T b) {
  T x0 = threadIdx.x * (T)1e-3, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3, x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6, x7 = x0 + 7;
  for (int i = 0; i < iters; ++i) {
    x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
    x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}
__global__ void copy_k(const double2* __restrict__ a, double2* __restrict__ b, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) b[i] = a[i];
}
int main() {
  cudaDeviceProp p; cudaGetDeviceProperties(&p, 0);
  printf("name %s sms %d cc %d.%d smem/block optin %zu l2 %d MB\n", p.name, p.multiProcessorCount, p.major, p.minor,
         p.sharedMemPerBlockOptin, p.l2CacheSize >> 20);
  int blocks = p.multiProcessorCount * 8, threads = 256, iters = 20000;
  double* od; float* of; cudaMalloc(&od, blocks * threads * 8); cudaMalloc(&of, blocks * threads * 4);
  cudaEvent_t e0, e1; cudaEventCreate(&e0); cudaEventCreate(&e1); float ms;
  for (int rep = 0; rep < 3; ++rep) {
    cudaEventRecord(e0); fma_loop<double><<<blocks, threads>>>(od, iters, 0.999999, 1e-7); cudaEventRecord(e1);
    cudaEventSynchronize(e1); cudaEventElapsedTime(&ms, e0, e1);
    printf("DFMA: %.3f TFLOP/s (%.3f ms)\n", 2.0 * 8 * iters * (double)blocks * threads / (ms * 1e-3) / 1e12, ms);
    cudaEventRecord(e0); fma_loop<float><<<blocks, threads>>>(of, iters * 4, 0.999999f, 1e-7f); cudaEventRecord(e1);
    cudaEventSynchronize(e1); cudaEventElapsedTime(&ms, e0, e1);
    printf("FFMA: %.3f TFLOP/s (%.3f ms)\n", 2.0 * 8 * iters * 4 * (double)blocks * threads / (ms * 1e-3) / 1e12, ms);
  }
  size_t n = (size_t)1 << 27; // 128 Mi double2 = 4 GiB each
  double2 *a, *b; cudaMalloc(&a, n * 16); cudaMalloc(&b, n * 16); cudaMemset(a, 0, n * 16);
  for (int rep = 0; rep < 4; ++rep) {
    cudaEventRecord(e0); copy_k<<<p.multiProcessorCount * 4, 512>>>(a, b, n); cudaEventRecord(e1);
    cudaEventSynchronize(e1); cudaEventElapsedTime(&ms, e0, e1);
    printf("copy: %.1f GB/s\n", 2.0 * n * 16 / (ms * 1e-3) / 1e9);
  }
  printf("err %s\n", cudaGetErrorString(cudaGetLastError()));
  return 0;
}
