// Test harness (not part of the library): applies the library's device conversions between
// binary32 and binary64 (widen_all / narrow_all of lbm_core.cuh, the integer forms with their
// per-warp fallback) to host arrays, so that a test can compare them with IEEE 754 conversions.
#include <cuda_runtime.h>

#include "lbm_core.cuh"

namespace {

__global__ void k_convert(const float* x32, double* y64, const double* x64, float* y32, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float a[1] = {x32[i]};
  double b[1];
  lbm::widen_all<1>(a, b);
  y64[i] = b[0];
  const double c[1] = {x64[i]};
  float d[1];
  lbm::narrow_all<1>(c, d);
  y32[i] = d[0];
}

}  // namespace

// Returns 0 on success, else the CUDA error code.
extern "C" int convert_check(const float* x32, double* y64, const double* x64, float* y32, int n) {
  float *dx32 = nullptr, *dy32 = nullptr;
  double *dx64 = nullptr, *dy64 = nullptr;
  cudaError_t e = cudaSuccess;
  const size_t b4 = sizeof(float) * (size_t)n, b8 = sizeof(double) * (size_t)n;
  if ((e = cudaMalloc(&dx32, b4)) || (e = cudaMalloc(&dy32, b4)) || (e = cudaMalloc(&dx64, b8)) ||
      (e = cudaMalloc(&dy64, b8)) || (e = cudaMemcpy(dx32, x32, b4, cudaMemcpyHostToDevice)) ||
      (e = cudaMemcpy(dx64, x64, b8, cudaMemcpyHostToDevice)))
    goto out;
  k_convert<<<(n + 255) / 256, 256>>>(dx32, dy64, dx64, dy32, n);
  if ((e = cudaGetLastError()) || (e = cudaMemcpy(y64, dy64, b8, cudaMemcpyDeviceToHost)) ||
      (e = cudaMemcpy(y32, dy32, b4, cudaMemcpyDeviceToHost)))
    goto out;
out:
  cudaFree(dx32);
  cudaFree(dy32);
  cudaFree(dx64);
  cudaFree(dy64);
  return (int)e;
}
