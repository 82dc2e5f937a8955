// scan kernels instantiated for double (one translation unit per element type).
#include "k_scan.cuh"

namespace dr {
cudaError_t launch_scan_f64(const ScanParams& p, bool reverse, int grid, cudaStream_t s) {
  return kscan::dispatch<double, false>(p, reverse, grid, s);
}
}  // namespace dr
