// Device tables and launch interface of the batched persistent kernel.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "dr.h"
#include "dr_kernels.h"

namespace dr {

struct BPiece {  // one piece of one vector: x, p, y re-segmented together
  const float* x;
  const float* p;
  float* y;
  int64_t len;
  int32_t vec;
  int32_t vec_ok;
};

struct BTile {  // a tile covers [off, min(off + TILE, len)) of piece `piece`
  int32_t piece;
  int32_t pad_;
  int64_t off;
};

struct BVec {  // the vector's tiles are [first_tile, first_tile + ntiles)
  int64_t first_tile;
  int32_t ntiles;
  int32_t pad_;
};

struct BatchParams {
  const BPiece* pieces;
  const BTile* tiles;
  const BVec* vecs;
  int64_t ntiles;
  int nvec;
  char* ws;  // WsHeader | lookback slots | per-tile dot partials | per-vector counters
  float* dots;
  unsigned* status;
  int64_t spin_limit;
};

bool batch_shape_supported(int variant, int threads, int items);
size_t batch_ws_bytes(int64_t ntiles, int nvec);
cudaError_t launch_batch(const BatchParams& p, const dr_tune& t, int sms, cudaStream_t s);

}  // namespace dr
