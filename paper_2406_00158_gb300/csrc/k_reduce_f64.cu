// reduce kernels instantiated for double (one translation unit per element type).
#include "k_reduce.cuh"

namespace dr {
cudaError_t launch_reduce_f64(const ReduceParams& p, int grid, cudaStream_t s) {
  return kreduce::dispatch<double>(p, grid, s);
}
}  // namespace dr
