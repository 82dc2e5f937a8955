// A dot-product entry point that allocates nothing.
//
// dr_transform_reduce keeps its scratch (a counter header and one partial per
// CTA) in a workspace it cudaMalloc's on a view's first use.  Some callers
// cannot allocate device memory at that point: code embedded in a framework that
// owns all device memory through its own pool, or a latency-critical loop that
// cannot pay for cudaMalloc, or for the device-wide synchronization cudaFree
// implies when the workspace is released.  dr_dot_f32_noalloc runs the same
// reduce kernel with its scratch in a fixed, file-scope device array instead.
//
// The array is shared by every call on a device and keeps the last call's
// contents; each call clears the part that must start at zero (the counter
// header) on its own stream before the kernel.  Two calls that can overlap on
// the GPU (unordered streams) race on the array and give wrong results.
#include <cstring>
#include <mutex>

#include "dr_host.h"

namespace {

// Scratch: the reduce kernel's 64-byte header plus one 8-byte partial per CTA,
// for up to kNoAllocMaxCtas CTAs: 64 + 8 * 4096 = 32,832 bytes on every device
// that loads the library (held until the process exits).
constexpr int kNoAllocMaxCtas = 4096;
constexpr size_t kNoAllocBytes = sizeof(dr::WsHeader) + 8 * (size_t)kNoAllocMaxCtas;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// Host code must not use g_noalloc_scratch as an address (in host code it names
// a host-side stand-in): the device address is looked up once per device.
constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
void* g_scratch_dev[kMaxDevices];

}  // namespace

extern "C" int dr_dot_f32_noalloc(int nseg, const int64_t* lens, const float* const* x_segs,
                                  const float* const* y_segs, float init, float* dev_result,
                                  dr_stream_t stream) {
  using namespace dr;
  clear_error();
  const char* who = "dr_dot_f32_noalloc";
  if (nseg < 1 || !lens || !x_segs || !y_segs || !dev_result)
    return fail(DR_E_INVAL, "%s: need nseg >= 1, lens, x_segs, y_segs, dev_result", who);
  if (nseg > kMaxPieces)
    return fail(DR_E_UNSUPPORTED, "%s: %d segments; at most %d per call", who, nseg, kMaxPieces);
  if ((uintptr_t)dev_result % 4) return fail(DR_E_ALIGN, "%s: result pointer misaligned", who);
  for (int k = 0; k < nseg; ++k) {
    if (lens[k] < 0) return fail(DR_E_INVAL, "%s: segment %d has negative length", who, k);
    if (lens[k] > 0 && (!x_segs[k] || !y_segs[k]))
      return fail(DR_E_INVAL, "%s: segment %d pointer is NULL", who, k);
    if ((uintptr_t)x_segs[k] % 4 || (uintptr_t)y_segs[k] % 4)
      return fail(DR_E_ALIGN, "%s: segment %d pointer not 4-byte aligned", who, k);
  }
  const int grid = reduce_grid(DR_F32);
  if (grid > kNoAllocMaxCtas)
    return fail(DR_E_UNSUPPORTED, "%s: the device needs %d CTAs; the fixed scratch holds partials for %d", who,
                grid, kNoAllocMaxCtas);

  // set-up, once per device, with that device current
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) return fail(DR_E_UNSUPPORTED, "%s: device %d out of range", who, dev);
  void* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_setup_mu);
    if (!g_scratch_dev[dev]) {
      e = cudaGetSymbolAddress(&g_scratch_dev[dev], g_noalloc_scratch);
      if (e != cudaSuccess) {
        g_scratch_dev[dev] = nullptr;
        return cuda_fail(e, "cudaGetSymbolAddress(scratch)");
      }
    }
    scratch = g_scratch_dev[dev];
  }
  unsigned* status = status_word();
  if (!status) return fail(DR_E_CUDA, "%s: no device status word", who);

  ReduceParams p;  // on the stack: nothing is allocated
  std::memset(&p, 0, sizeof p);
  p.vc.kind = 1;  // zip(x, y) | multiply
  p.vc.nleaf = 2;
  p.vc.zipop = DR_MUL;
  p.op = DR_PLUS;
  p.dtype = DR_F32;
  p.result = dev_result;
  std::memcpy(&p.init_bits, &init, sizeof init);
  const int tile = reduce_tile_elems(DR_F32);
  int np = 0;
  int64_t tiles = 0;
  for (int k = 0; k < nseg; ++k) {
    if (lens[k] == 0) continue;
    KPiece& q = p.pc[np++];
    q.a = reinterpret_cast<const char*>(x_segs[k]);
    q.b = reinterpret_cast<const char*>(y_segs[k]);
    q.len = lens[k];
    q.tile_begin = tiles;
    q.vec_ok = (uintptr_t)x_segs[k] % 16 == 0 && (uintptr_t)y_segs[k] % 16 == 0;
    tiles += (lens[k] + tile - 1) / tile;
  }
  p.npieces = np;
  p.ntiles = tiles;
  p.ws = static_cast<char*>(scratch);
  p.ws_partials = kNoAllocMaxCtas;
  p.status = status;

  cudaStream_t s = (cudaStream_t)stream;
  e = cudaMemsetAsync(scratch, 0, sizeof(WsHeader), s);  // the counters must start at zero
  if (e != cudaSuccess) return cuda_fail(e, "clearing the scratch header");
  e = launch_reduce(p, grid, s);
  return e == cudaSuccess ? DR_OK : cuda_fail(e, who);
}
