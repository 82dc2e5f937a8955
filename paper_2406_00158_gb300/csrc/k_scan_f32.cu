// scan kernels instantiated for float (one translation unit per element type).
#include "k_scan.cuh"

namespace dr {
cudaError_t launch_scan_f32(const ScanParams& p, bool reverse, int grid, cudaStream_t s) {
  return kscan::dispatch<float, false>(p, reverse, grid, s);
}
}  // namespace dr
