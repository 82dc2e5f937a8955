// scan kernels instantiated for int with the piece table in device memory (calls
// of more than 128 pieces; one translation unit per element type).
#include "k_scan.cuh"

namespace dr {
cudaError_t launch_scan_i32_ext(const ScanParams& p, bool reverse, int grid, cudaStream_t s) {
  return kscan::dispatch<int, true>(p, reverse, grid, s);
}
}  // namespace dr
