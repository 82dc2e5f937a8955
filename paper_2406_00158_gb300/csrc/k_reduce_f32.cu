// reduce kernels instantiated for float (one translation unit per element type).
#include "k_reduce.cuh"

namespace dr {
cudaError_t launch_reduce_f32(const ReduceParams& p, int grid, cudaStream_t s) {
  return kreduce::dispatch<float>(p, grid, s);
}
}  // namespace dr
