// scan kernels instantiated for float with the piece table in device memory (calls
// of more than 128 pieces; one translation unit per element type).
#include "k_scan.cuh"

namespace dr {
cudaError_t launch_scan_f32_ext(const ScanParams& p, bool reverse, int grid, cudaStream_t s) {
  return kscan::dispatch<float, true>(p, reverse, grid, s);
}
}  // namespace dr
