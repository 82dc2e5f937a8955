// reduce kernels instantiated for long long (one translation unit per element type).
#include "k_reduce.cuh"

namespace dr {
cudaError_t launch_reduce_i64(const ReduceParams& p, int grid, cudaStream_t s) {
  return kreduce::dispatch<long long>(p, grid, s);
}
}  // namespace dr
