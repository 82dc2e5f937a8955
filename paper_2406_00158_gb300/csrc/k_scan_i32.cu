// scan kernels instantiated for int (one translation unit per element type).
#include "k_scan.cuh"

namespace dr {
cudaError_t launch_scan_i32(const ScanParams& p, bool reverse, int grid, cudaStream_t s) {
  return kscan::dispatch<int, false>(p, reverse, grid, s);
}
}  // namespace dr
