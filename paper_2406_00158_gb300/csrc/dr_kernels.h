// Interface between the host side of the library (dr_api.cu: handles, views,
// re-segmentation, validation) and the kernel translation units.  Kernel
// parameters are plain structs passed by value (__grid_constant__), so a call
// over up to kMaxPieces segments needs no device-side table.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "dr.h"

namespace dr {

constexpr int kMaxChain = 4;     // unary ops per chain in a fused view
// Pieces (segments after re-segmentation) carried inline in a launch's
// parameters; a scan, reduce, transform or for_each call with more pieces keeps
// its whole piece table in device memory instead (pc_ext), the other calls
// reject it.
constexpr int kMaxPieces = 128;
constexpr int kMaxZip = DR_MAX_ZIP;  // operands of a k-ary zip (and of one re-segmentation)

// Fused view: element = post(zipop(pre0(a), pre1(b))) (or post(pre0(a)) for one leaf).
// kind: 0 = one leaf, no ops; 1 = two leaves times each other, no other ops
// (the dot product); 2 = anything else (interpreted per element, uniform branches).
struct KViewCode {
  int kind;
  int nleaf;
  int zipop;
  int npre[2];
  int npost;
  int pre_op[2][kMaxChain];
  int post_op[kMaxChain];
  double pre_arg[2][kMaxChain];
  double post_arg[kMaxChain];
  // the same scalars converted once on the host for fp32 and integer views
  float pre_argf[2][kMaxChain];
  float post_argf[kMaxChain];
  long long pre_argi[2][kMaxChain];
  long long post_argi[kMaxChain];
};

// One piece of a call: `len` elements, operands at a / b, output at o (byte
// pointers at the piece's first element), first tile index of the piece in the
// call's global tile order.  vec_ok: all of a, b, o are 16-byte aligned.
struct KPiece {
  const char* a;
  const char* b;
  char* o;
  int64_t len;
  int64_t tile_begin;
  int32_t vec_ok;
  int32_t pad_;
};

// Self-cleaning workspace header: the last CTA of every launch restores
// ticket = done = 0 and advances epoch, so no memset is needed between launches.
struct WsHeader {
  unsigned long long ticket;
  unsigned done;
  unsigned epoch;
  unsigned long long pad_[6];
};
static_assert(sizeof(WsHeader) == 64, "header size");

struct ReduceParams {
  KViewCode vc;
  int op;
  int dtype;
  int npieces;
  int64_t ntiles;
  char* ws;          // WsHeader + one partial (8 bytes) per CTA
  int ws_partials;   // partial slots in ws (checked builds verify the grid fits)
  unsigned* status;  // per-device status word
  void* result;      // one element of dtype
  unsigned long long init_bits;
  const KPiece* pc_ext;  // the piece table in device memory when npieces > kMaxPieces, else NULL
  KPiece pc[kMaxPieces];
};

struct ScanParams {
  KViewCode vc;
  int op;
  int dtype;
  int npieces;
  int exclusive;
  int64_t ntiles;
  char* ws;  // WsHeader + lookback slots
  unsigned* status;
  int64_t spin_limit;
  int64_t skip_tile;  // test hook: this logical tile never publishes (-1: none)
  unsigned long long init_bits;
  const void* carry;  // device carry-in (one element) or NULL; forward scans only
  const KPiece* pc_ext;  // the piece table in device memory when npieces > kMaxPieces, else NULL
  KPiece pc[kMaxPieces];
};

struct ScaleParams {  // dot adjoint: gx = g*y, gy = g*x
  const float* g;
  int npieces;
  int64_t ntiles;
  struct P4 {
    const char* x;
    const char* y;
    char* gx;
    char* gy;
    int64_t len;
    int64_t tile_begin;
    int32_t vec_ok;
    int32_t pad_;
  } pc[kMaxPieces];
};

// for_each over a k-ary zip: piece i has `len` elements at p[0..k-1] (byte
// pointers at the piece's first element).  vec_ok: every p is 16-byte aligned.
struct FePiece {
  char* p[kMaxZip];
  int64_t len;
  int64_t tile_begin;
  int32_t vec_ok;
  int32_t pad_;
};

struct ForEachParams {
  unsigned* status;  // per-device status word (checked builds)
  int fn;      // enum dr_foreach_fn
  int dtype;   // DR_F32 or DR_F64
  int npieces;
  int64_t ntiles;
  double arg[2];
  const FePiece* pc_ext;  // the piece table in device memory when npieces > kMaxPieces, else NULL
  FePiece pc[kMaxPieces];
};

// transform: out = the fused view, piece by piece (KPiece a, b = leaves, o = out).
struct TransformParams {
  unsigned* status;  // per-device status word (checked builds)
  KViewCode vc;
  int dtype;
  int npieces;
  int64_t ntiles;
  const KPiece* pc_ext;  // the piece table in device memory when npieces > kMaxPieces, else NULL
  KPiece pc[kMaxPieces];
};

// sort: input view pieces (first pass and histogram), output segments (last
// pass), and the scratch of the current pass.
struct SortOut {
  char* p;
  int64_t start;  // global index of the segment's first element
};

struct SortParams {
  KViewCode vc;
  int dtype;
  int npin;
  int npout;
  int pass;            // digit index: bits [8 pass, 8 pass + 8)
  int64_t n;
  int64_t ntiles;      // tiles of this launch
  const char* src;     // key bits of the previous pass (contiguous)
  char* dst;           // key bits of this pass (contiguous; not on the last pass)
  unsigned* counts;    // [256][ntiles] per-tile digit counts, then their exclusive scan
  unsigned* status;
  int64_t spin_limit;
  KPiece in[kMaxPieces];
  SortOut out[kMaxPieces];
};

struct SortLaunch {
  int64_t ntiles0;     // tiles of the first pass (per-piece tiling of the view)
  int64_t ntiles;      // tiles of the other passes (ceil(n / tile))
  char* tmp[2];        // two contiguous scratch buffers of n keys
  char* scan_ws;       // workspace of the counts' scan (self-cleaning; zeroed once)
  ScanParams* scan;    // host scratch for the scan's parameters
};

struct StencilSeg {
  const float* in;   // allocation incl. ghost rows: (rows + 2) * cols
  const float* prev; // weight-gradient step only: the forward state u_{t-1} (same layout)
  float* out;
  float* out_prev;   // output allocation of the block above (NULL for the first)
  float* out_next;   // output allocation of the block below (NULL for the last)
  int64_t rows;
  int64_t prev_rows; // own rows of the block above
  int64_t rb_begin;  // first row-block index of this segment
};

struct StencilParams {
  unsigned* status;  // per-device status word (checked builds)
  int nseg;
  int64_t cols;
  int64_t nrb;       // total row blocks
  int64_t rb_lo;     // first row block of this launch (grid.y row blocks from there)
  int outer_only;    // 1: grid.y = 1 or 2 row blocks, the first and the last
  int ext_top;       // 1: the first block's top ghost row holds real data (a neighbour's row)
  int ext_bot;       // 1: the last block's bottom ghost row holds real data
  float wc, wn;
  int vec_ok;        // cols % 4 == 0 and all pointers 16-byte aligned
  double* acc;       // weight-gradient step only: acc[0] += <in, prev>, acc[1] += <N(in), prev>
  StencilSeg seg[kMaxPieces];
};

struct HaloParams {
  int nbound;  // interior boundaries
  int64_t cols;
  struct B {
    const float* src_last;  // block k's last own row
    float* dst_top_ghost;   // block k+1's row 0
    const float* src_first; // block k+1's first own row
    float* dst_bot_ghost;   // block k's bottom ghost row
  } b[kMaxPieces];
};

// Tile geometry (elements per tile) of each kernel family for a dtype.
int reduce_tile_elems(int dtype);
// view: the scan of a fused view (ops or a zip; its kernels' tiles are shorter)
int scan_tile_elems(int dtype, bool view = false);
int scale_tile_elems();
int foreach_tile_elems(int dtype);  // for_each and transform
int sort_tile_elems(int dtype);
int sort_passes(int dtype);
#ifndef DR_STENCIL_ROWS
#define DR_STENCIL_ROWS 64
#endif
constexpr int kStencilThreads = 128;   // 4 columns per thread -> 512 columns per CTA
constexpr int kStencilRowsPerCta = DR_STENCIL_ROWS;

size_t reduce_ws_bytes(int grid);
size_t scan_ws_bytes(int64_t ntiles, int dtype);

// Launchers (kernel TUs).  Return the launch's cudaError_t.
cudaError_t launch_reduce(const ReduceParams& p, int grid, cudaStream_t s);
cudaError_t launch_scan(const ScanParams& p, bool reverse, int grid, cudaStream_t s);
cudaError_t launch_scale(const ScaleParams& p, int grid, cudaStream_t s);
cudaError_t launch_stencil(const StencilParams& p, int64_t nrb_launch, cudaStream_t s);
cudaError_t launch_halo(const HaloParams& p, cudaStream_t s);
cudaError_t launch_for_each(const ForEachParams& p, cudaStream_t s);
cudaError_t launch_transform(const TransformParams& p, cudaStream_t s);
cudaError_t launch_sort(SortParams& p, const SortLaunch& L, cudaStream_t s);

// Resident-CTA count helpers (host).
int reduce_grid(int dtype);
int reduce_ctas_per_sm();
int scan_grid(int dtype, int64_t ntiles);

}  // namespace dr
