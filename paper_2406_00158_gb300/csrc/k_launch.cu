// Launch glue: tile geometry, workspace sizes, grid sizes, and the switch from
// a call's element type to the per-type kernel translation unit.
#include "k_reduce.cuh"
#include "k_scan.cuh"

namespace dr {

cudaError_t launch_scan_f32(const ScanParams& p, bool reverse, int grid, cudaStream_t s);
cudaError_t launch_scan_f64(const ScanParams& p, bool reverse, int grid, cudaStream_t s);
cudaError_t launch_scan_i64(const ScanParams& p, bool reverse, int grid, cudaStream_t s);
cudaError_t launch_scan_i32(const ScanParams& p, bool reverse, int grid, cudaStream_t s);
cudaError_t launch_scan_f32_ext(const ScanParams& p, bool reverse, int grid, cudaStream_t s);
cudaError_t launch_scan_f64_ext(const ScanParams& p, bool reverse, int grid, cudaStream_t s);
cudaError_t launch_scan_i64_ext(const ScanParams& p, bool reverse, int grid, cudaStream_t s);
cudaError_t launch_scan_i32_ext(const ScanParams& p, bool reverse, int grid, cudaStream_t s);
cudaError_t launch_reduce_f32(const ReduceParams& p, int grid, cudaStream_t s);
cudaError_t launch_reduce_f64(const ReduceParams& p, int grid, cudaStream_t s);
cudaError_t launch_reduce_i64(const ReduceParams& p, int grid, cudaStream_t s);
cudaError_t launch_reduce_i32(const ReduceParams& p, int grid, cudaStream_t s);

static bool is4(int dtype) { return dtype == DR_F32 || dtype == DR_I32; }

int scan_tile_elems(int dtype, bool view) {
  if (view) return is4(dtype) ? kscan::stile<float, kscan::kViewChunks>() : kscan::stile<double, kscan::kViewChunks>();
  return is4(dtype) ? kscan::stile<float>() : kscan::stile<double>();
}

size_t scan_ws_bytes(int64_t ntiles, int dtype) {
  return sizeof(WsHeader) + (is4(dtype) ? Slots<float>::bytes(ntiles) : Slots<double>::bytes(ntiles));
}

int scan_grid(int, int64_t) { return 0; }  // 0: occupancy-sized persistent grid

cudaError_t launch_scan(const ScanParams& p, bool reverse, int grid, cudaStream_t s) {
  if (p.pc_ext) {  // more pieces than the kernel parameters hold: the device-table kernels
    switch (p.dtype) {
      case DR_F32: return launch_scan_f32_ext(p, reverse, grid, s);
      case DR_F64: return launch_scan_f64_ext(p, reverse, grid, s);
      case DR_I64: return launch_scan_i64_ext(p, reverse, grid, s);
      default: return launch_scan_i32_ext(p, reverse, grid, s);
    }
  }
  switch (p.dtype) {
    case DR_F32: return launch_scan_f32(p, reverse, grid, s);
    case DR_F64: return launch_scan_f64(p, reverse, grid, s);
    case DR_I64: return launch_scan_i64(p, reverse, grid, s);
    default: return launch_scan_i32(p, reverse, grid, s);
  }
}

int reduce_tile_elems(int dtype) {
  return is4(dtype) ? kreduce::rtile<float>() : kreduce::rtile<double>();
}

size_t reduce_ws_bytes(int grid) { return sizeof(WsHeader) + (size_t)grid * 8; }

int reduce_ctas_per_sm() { return kreduce::RCTAS; }

// Fixed grid: RCTAS CTAs per SM of the current device.
int reduce_grid(int) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms * kreduce::RCTAS;
}

cudaError_t launch_reduce(const ReduceParams& p, int grid, cudaStream_t s) {
  switch (p.dtype) {
    case DR_F32: return launch_reduce_f32(p, grid, s);
    case DR_F64: return launch_reduce_f64(p, grid, s);
    case DR_I64: return launch_reduce_i64(p, grid, s);
    default: return launch_reduce_i32(p, grid, s);
  }
}

}  // namespace dr
