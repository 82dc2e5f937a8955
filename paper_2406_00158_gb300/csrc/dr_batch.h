// Device tables and launch interface of the batched persistent kernel.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "dr.h"
#include "dr_kernels.h"

namespace dr {

struct BPiece {  // host side: one piece of one vector (x, p, y re-segmented together)
  const float* x;
  const float* p;
  float* y;
  int64_t len;
  int32_t vec;
  int32_t vec_ok;
};

// One tile of one vector, flattened on the host so that a tile costs the kernel
// one 48-byte load (three independent 16-byte loads), not a chain of lookups.
struct alignas(16) BDesc {
  const float* x;       // x, p, y at the tile's first element
  const float* p;
  float* y;
  int64_t first_tile;   // the vector's first tile
  int32_t len;          // elements in this tile (<= the tile size; 0 for an empty vector)
  int32_t vec;          // vector index
  int32_t ntiles;       // tiles of the vector
  int32_t full;         // len == tile size and x, p, y 16-byte aligned
};
static_assert(sizeof(BDesc) == 48, "descriptor size");

struct BatchParams {
  const BDesc* desc;    // one per tile, vector after vector
  int64_t ntiles;
  int nvec;
  char* ws;  // WsHeader | per-vector counters | lookback slots | per-tile dot partials
  float* dots;
  unsigned* status;
  int64_t spin_limit;
};

bool batch_shape_supported(int variant, int threads, int items);
size_t batch_ws_bytes(int64_t ntiles, int nvec);
cudaError_t launch_batch(const BatchParams& p, const dr_tune& t, int sms, cudaStream_t s);

}  // namespace dr
