// reduce kernels instantiated for int (one translation unit per element type).
#include "k_reduce.cuh"

namespace dr {
cudaError_t launch_reduce_i32(const ReduceParams& p, int grid, cudaStream_t s) {
  return kreduce::dispatch<int>(p, grid, s);
}
}  // namespace dr
