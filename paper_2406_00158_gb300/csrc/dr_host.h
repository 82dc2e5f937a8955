// Host-side objects behind the opaque handles of dr.h, and helpers shared by
// the host translation units.
#pragma once

#include <cstdarg>
#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "dr.h"
#include "dr_kernels.h"

namespace dr {

// Sets this thread's error message and returns `code`.
int fail(int code, const char* fmt, ...);
int cuda_fail(cudaError_t e, const char* what);
void clear_error();

int esize(int dtype);
bool valid_dtype(int dtype);

// Device workspace owned by a handle: allocated (and zeroed) on first use,
// grown when a larger one is needed.  Kernels keep it self-cleaning.  Memory
// comes from a per-device pool of the library in stream order, so allocating
// and releasing never synchronizes the device: mark(s) after the launches that
// use it remembers the stream, and release() frees the memory on that stream,
// after the work queued there (the next allocation on the same stream reuses it
// at once).  A workspace that was never marked is released after a device
// synchronization.
struct Workspace {
  void* ptr = nullptr;
  size_t bytes = 0;
  int device = -1;
  cudaStream_t last = nullptr;  // stream of the latest use (mark)
  bool marked = false;
  // zero: bytes at the start that must read as zero before the first kernel
  // (the self-cleaning counters); the rest is scratch the kernels write first
  int ensure(size_t need, cudaStream_t s, size_t zero = ~size_t(0));
  void mark(cudaStream_t s);
  void release();
  ~Workspace() { release(); }
};

unsigned* status_word();      // device address of the current device's status word
int64_t spin_limit();
int64_t take_skip_publish();  // returns the armed test hook value and disarms it
int sm_count();

// One operand's segment list, trimmed to a window of its container.
struct Seg {
  char* p;
  int64_t len;
  int32_t idx;  // segment index in the container
  int64_t off;  // element offset of p within that segment
};

// A piece of a k-way re-segmentation (k <= kMaxZip).
struct Piece {
  int64_t start, len;
  char* p[kMaxZip];
  int32_t seg[kMaxZip];
  int64_t off[kMaxZip];
};

// Cuts k segment lists at the union of their boundaries (Sec. 4.4 "Zip": take
// the largest run that fits in the current segment of every operand, i.e. the
// minimum remaining distance, then advance).  Stops when any list ends; empty
// segments produce no piece.
std::vector<Piece> resegment(const std::vector<std::vector<Seg>>& ops, int esz);

}  // namespace dr

struct dr_vec {
  int dtype = 0;
  int esz = 4;
  std::vector<char*> ptr;
  std::vector<int64_t> len, start;
  int64_t n = 0;
  // the segments of the window [lo, hi) of the vector's elements
  std::vector<dr::Seg> window(int64_t lo, int64_t hi) const;
};

struct dr_md2 {
  int dtype = 0;
  int64_t rows = 0, cols = 0;
  std::vector<char*> ptr;
  std::vector<int64_t> srows;
  // the array is one rank's share of a taller grid: its outer ghost rows hold
  // the neighbouring shares' boundary rows (filled by the caller) instead of zero
  int ext_top = 0, ext_bot = 0;
};

struct dr_view {
  struct Leaf {
    const dr_vec* vec;
    int64_t lo, hi;  // element window of the vector (take / drop)
  };
  int dtype = 0;
  int arity = 1;  // 1 = single-valued, k >= 2 = raw k-ary zip
  int nleaf = 1;
  Leaf leaf[dr::kMaxZip];
  int npre[2] = {0, 0};
  int pre_op[2][dr::kMaxChain];
  double pre_arg[2][dr::kMaxChain];
  int zipop = -1;
  int npost = 0;
  int post_op[dr::kMaxChain];
  double post_arg[dr::kMaxChain];
  int64_t size = 0;
  std::vector<dr::Piece> pieces;  // re-segmentation of the leaves' windows
  dr::Workspace ws_scan, ws_reduce, ws_sort;
  dr::Workspace ws_table;  // piece table of calls with more pieces than fit in a launch

  void recompute();
  dr::KViewCode code() const;
};
