// peak.cu -- diagnostic: the FP64 FMA issue rate of this GPU, the roofline that bounds
// the FP64 recurrences (GB300 has far fewer FP64 units than FP32 ones).
#include <cuda_runtime.h>

#include "band.h"

namespace {

// Eight independent FMA chains per thread; every thread does iters * 64 DFMAs.
__global__ void __launch_bounds__(256) k_dfma(double* out, int iters, double y, double z) {
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  double v[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) v[j] = 1.0 + 1e-9 * tid + 0.1 * j;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < 8; ++u) {
#pragma unroll
      for (int j = 0; j < 8; ++j) v[j] = fma(v[j], y, z);
    }
  }
  double s = 0.0;
#pragma unroll
  for (int j = 0; j < 8; ++j) s += v[j];
  out[tid] = s;
}

}  // namespace

extern "C" double band_fp64_fma_rate(void* scratch, size_t scratch_bytes, void* stream) {
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return -1.0;
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return -1.0;
  const int threads = 256, blocks = nsm * 8, iters = 512;
  if (!scratch || scratch_bytes < sizeof(double) * (size_t)threads * blocks) return -1.0;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  double* out = static_cast<double*>(scratch);
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return -1.0;
  if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); return -1.0; }
  k_dfma<<<blocks, threads, 0, st>>>(out, 16, 0.9999999, 1e-7);  // warm-up
  float best = 1e30f;
  for (int rep = 0; rep < 3; ++rep) {
    cudaEventRecord(e0, st);
    k_dfma<<<blocks, threads, 0, st>>>(out, iters, 0.9999999, 1e-7);
    cudaEventRecord(e1, st);
    if (cudaEventSynchronize(e1) != cudaSuccess) { best = -1.0f; break; }
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best) best = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (best <= 0.0f) return -1.0;
  const double fmas = (double)blocks * threads * iters * 64.0;
  return fmas / (best * 1e-3);
}
