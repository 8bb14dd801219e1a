// Test harness for the integer-pipe FP64 <-> FP32 conversions of device_common.cuh: applies them
// element-wise so the test can compare with CUDA's own conversions (torch's .float()/.double()).
#include <cuda_runtime.h>

#include "device_common.cuh"

__global__ void k_conv(const double* x, float* f, const float* y, double* d, float* dv, int n, float rh, float rl) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  f[i] = cfs::d2f_fast(x[i]);
  d[i] = cfs::f2d_fast(y[i]);
  dv[i] = cfs::dev_fast(x[i], rh, rl);
}

extern "C" int conv_check(const double* x, float* f, const float* y, double* d, float* dv, int n, float rh, float rl) {
  k_conv<<<(n + 255) / 256, 256>>>(x, f, y, d, dv, n, rh, rl);
  return (int)cudaDeviceSynchronize();
}
