// Elementwise kernels over re-segmented pieces: the adjoint of the dot product
// (scale-by-partner: for d = <x, y> and incoming gradient g, x_bar = g*y and
// y_bar = g*x).  Grid-stride over tiles of 256 threads x 4 x float4, 128-bit
// loads and stores on aligned full tiles, scalar otherwise.  16 B / element
// when both gradients are written (8 B read, 8 B written).
#include "dr_device.cuh"

namespace dr {
namespace {

constexpr int ET = 256;
constexpr int ECH = 4;
constexpr int ETILE = ET * ECH * 4;

__device__ __forceinline__ int find_piece4(const ScaleParams& P, int64_t tile) {
  int lo = 0, hi = P.npieces - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (P.pc[mid].tile_begin <= tile) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

__global__ void __launch_bounds__(ET) k_scale(const __grid_constant__ ScaleParams P) {
  const float g = __ldg(P.g);
  const int tid = threadIdx.x;
  for (int64_t tile = blockIdx.x; tile < P.ntiles; tile += gridDim.x) {
    const auto& pc = P.pc[find_piece4(P, tile)];
    const int64_t base = (tile - pc.tile_begin) * ETILE;
    if (pc.vec_ok && pc.len - base >= ETILE) {
      V16<float> xs[ECH], ys[ECH];
#pragma unroll
      for (int c = 0; c < ECH; ++c) {
        const int64_t off = (base + (int64_t)(c * ET + tid) * 4) * 4;
        if (pc.gy) xs[c] = ld16<float>(pc.x + off);
        if (pc.gx) ys[c] = ld16<float>(pc.y + off);
      }
#pragma unroll
      for (int c = 0; c < ECH; ++c) {
        const int64_t off = (base + (int64_t)(c * ET + tid) * 4) * 4;
        if (pc.gx) {
          V16<float> o;
#pragma unroll
          for (int e = 0; e < 4; ++e) o.v[e] = g * ys[c].v[e];
          st16<float>(pc.gx + off, o);
        }
        if (pc.gy) {
          V16<float> o;
#pragma unroll
          for (int e = 0; e < 4; ++e) o.v[e] = g * xs[c].v[e];
          st16<float>(pc.gy + off, o);
        }
      }
    } else {
      for (int64_t i = base + tid; i < min(base + ETILE, pc.len); i += ET) {
        if (pc.gx) reinterpret_cast<float*>(pc.gx)[i] = g * __ldg(reinterpret_cast<const float*>(pc.y) + i);
        if (pc.gy) reinterpret_cast<float*>(pc.gy)[i] = g * __ldg(reinterpret_cast<const float*>(pc.x) + i);
      }
    }
  }
}

}  // namespace

int scale_tile_elems() { return ETILE; }

cudaError_t launch_scale(const ScaleParams& p, int grid, cudaStream_t s) {
  if (p.ntiles <= 0) return cudaSuccess;
  if (grid <= 0) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    grid = sms * 4;
  }
  if (p.ntiles < grid) grid = (int)p.ntiles;
  k_scale<<<grid, ET, 0, s>>>(p);
  return cudaGetLastError();
}

}  // namespace dr
