// batch_w4.cu -- k_batch (batch_kernel.cuh) with four warps per block, for the autotuner's
// choice of block size; its own translation unit so that the variants compile in
// parallel.
#include "batch_kernel.cuh"

namespace band {
cudaError_t launch_batch_w4(const BatchTable& t, int64_t warps, cudaStream_t st) {
  return launch_batch_w<4>(t, warps, st);
}
}  // namespace band
