// Test probe: applies the library's FP64 reciprocal (rcp64 in csrc/common.cuh) to an
// array, so that a test can compare it with IEEE division element by element.  Built by
// tests/test_gpu_rcp64.py; not part of libband.
#include <cstdint>

#include "common.cuh"

__global__ void k_rcp_probe(const double* in, double* out, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = band::rcp64(in[i]);
}

extern "C" int rcp64_probe(const double* in, double* out, int64_t n) {
  if (n <= 0) return 0;
  k_rcp_probe<<<(unsigned)((n + 255) / 256), 256>>>(in, out, n);
  if (cudaGetLastError() != cudaSuccess) return 1;
  return cudaDeviceSynchronize() == cudaSuccess ? 0 : 1;
}
