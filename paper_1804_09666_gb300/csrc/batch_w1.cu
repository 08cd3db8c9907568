// batch_w1.cu -- k_batch (batch_kernel.cuh) with one warp per block, for the autotuner's
// choice of block size; its own translation unit so that the variants compile in
// parallel.
#include "batch_kernel.cuh"

namespace band {
cudaError_t launch_batch_w1(const BatchTable& t, int64_t warps, cudaStream_t st) {
  return launch_batch_w<1>(t, warps, st);
}
}  // namespace band
