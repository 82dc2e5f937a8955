// scan kernels instantiated for long long (one translation unit per element type).
#include "k_scan.cuh"

namespace dr {
cudaError_t launch_scan_i64(const ScanParams& p, bool reverse, int grid, cudaStream_t s) {
  return kscan::dispatch<long long, false>(p, reverse, grid, s);
}
}  // namespace dr
