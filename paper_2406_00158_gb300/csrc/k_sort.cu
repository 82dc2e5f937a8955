// sort (Sec. 4.3 "sort"): the elements of a view in ascending order, written to
// a segmented vector.  Floating-point keys follow the IEEE totalOrder (-NaN <
// -inf < ... < -0 < +0 < ... < +inf < +NaN), so the sorted sequence is unique.
//
// The paper's distributed partition sort cuts the range at sampled splitters so
// that each memory locale sorts one chunk.  With every segment in one HBM the
// partition is a radix pass (the digit values are the splitters, the per-chunk
// counts are the digit counts), so the whole sort is a least-significant-digit
// radix sort over the segment table, one 8-bit digit per pass, each pass three
// launches in the reduce-then-scan form:
//   1. k_sort_count: every tile counts its keys per digit and stores the 256
//      counts digit-major (counts[d * ntiles + t]);
//   2. the library's own exclusive scan over that array, in place: entry
//      (d, t) becomes the global position of tile t's first key with digit d
//      (all keys of smaller digits, then those of digit d in earlier tiles);
//   3. k_sort_scatter: every tile ranks its keys per digit (stable: warp
//      order, item order, lane order) and writes each digit's run through
//      shared memory to its global position.
// No CTA waits on another (a single-pass "onesweep" lookback chains every tile
// to its predecessors; on a GPU this wide the chain, not the memory, set the
// pace).  Keys are carried between passes as order-preserving unsigned bit
// patterns in two contiguous scratch buffers; the first pass reads (and
// evaluates) the view through its pieces, the last writes the output segments.
#include <cstring>

#include "dr_device.cuh"

namespace dr {
namespace {

#ifndef DR_SORT_THREADS
#define DR_SORT_THREADS 256
#endif
#ifndef DR_SORT_ITEMS
#define DR_SORT_ITEMS 16
#endif
#ifndef DR_SORT_MINB
#define DR_SORT_MINB 4  // resident CTAs per SM the scatter is compiled for (0: no bound)
#endif
#if DR_SORT_MINB > 0
#define DR_SORT_SCATTER_BOUNDS __launch_bounds__(ST, DR_SORT_MINB)
#else
#define DR_SORT_SCATTER_BOUNDS __launch_bounds__(ST)
#endif
constexpr int ST = DR_SORT_THREADS;  // threads per CTA (a multiple of 256)
constexpr int SW = ST / 32;
constexpr int RADIX = 256;           // threads < RADIX own one digit in the digit phases
static_assert(ST % RADIX == 0, "one thread per digit");
// keys per thread per tile: DR_SORT_ITEMS for 4-byte keys, half as many for
// 8-byte keys (the tile's keys are staged in shared memory)
template <int KB>
struct Tile {
  static constexpr int IT = KB == 4 ? DR_SORT_ITEMS : DR_SORT_ITEMS / 2;
  static constexpr int N = ST * IT;
  // the scatter kernel's static shared memory: staged keys, per-warp digit counts,
  // per-digit starts / shifts / bases, output starts (must stay within 48 KB)
  static constexpr int kSmem = N * KB + (ST / 32) * 256 * 4 + 256 * (4 + 4 + 8 + 4) + 128 * 8 + 64;
  static_assert(kSmem <= 48 * 1024, "sort tile too large for static shared memory");
};
static_assert(Tile<4>::kSmem > 0 && Tile<8>::kSmem > 0, "tile shapes");

// Order-preserving maps between element values and unsigned keys.
template <typename T>
struct KeyOf;
template <>
struct KeyOf<float> {
  using K = unsigned;
  static __device__ __forceinline__ K to(float v) {
    const unsigned u = __float_as_uint(v);
    return u ^ ((unsigned)(-(int)(u >> 31)) | 0x80000000u);
  }
  static __device__ __forceinline__ float from(K u) { return __uint_as_float(u ^ (((u >> 31) - 1u) | 0x80000000u)); }
};
template <>
struct KeyOf<double> {
  using K = unsigned long long;
  static __device__ __forceinline__ K to(double v) {
    const unsigned long long u = (unsigned long long)__double_as_longlong(v);
    return u ^ ((unsigned long long)(-(long long)(u >> 63)) | 0x8000000000000000ull);
  }
  static __device__ __forceinline__ double from(K u) {
    return __longlong_as_double((long long)(u ^ (((u >> 63) - 1ull) | 0x8000000000000000ull)));
  }
};
template <>
struct KeyOf<int> {
  using K = unsigned;
  static __device__ __forceinline__ K to(int v) { return (unsigned)v ^ 0x80000000u; }
  static __device__ __forceinline__ int from(K u) { return (int)(u ^ 0x80000000u); }
};
template <>
struct KeyOf<long long> {
  using K = unsigned long long;
  static __device__ __forceinline__ K to(long long v) { return (unsigned long long)v ^ 0x8000000000000000ull; }
  static __device__ __forceinline__ long long from(K u) { return (long long)(u ^ 0x8000000000000000ull); }
};

// Exclusive scan of one value per thread over the CTA (ST threads); returns the
// thread's exclusive prefix, *total the sum.  Contains __syncthreads.
__device__ __forceinline__ unsigned cta_excl_scan(unsigned v, unsigned* wsum, unsigned* total) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  unsigned x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wsum[w] = x;
  __syncthreads();
  unsigned base = 0, all = 0;
#pragma unroll
  for (int k = 0; k < SW; ++k) {
    const unsigned s = wsum[k];
    if (k < w) base += s;
    all += s;
  }
  __syncthreads();
  *total = all;
  return base + x - v;
}

__device__ __forceinline__ int find_in_piece(const SortParams& P, int64_t tile) {
  int lo = 0, hi = P.npin - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (P.in[mid].tile_begin <= tile) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// Element j of piece pc, through the view (SRC 0: one plain leaf; 1: the
// interpreted view code).
template <typename T, int SRC>
__device__ __forceinline__ T view_elem(const KPiece& pc, int64_t j, const ViewEval<T>& ve, bool two) {
  const T a = reinterpret_cast<const T*>(pc.a)[j];
  if constexpr (SRC == 0) {
    return a;
  } else {
    const T b = two ? reinterpret_cast<const T*>(pc.b)[j] : T(0);
    return ve(a, b);
  }
}

// The lanes of the warp whose digit equals this lane's: the intersection of one
// ballot per digit bit (NB bits: 8 for a full tile; 9 when lanes without a key
// carry the digit RADIX), or match.any (DR_SORT_MATCH=1).  Measured on GB300,
// 2^28 fp32 keys: ballots 7.5 ms, match.any 9.0 ms (its latency, not the
// issue slots, bounds the ranking).  Shapes: 256 x 16 and 512 x 12 tie; 1024
// threads and 24 items per thread are slower.  The scatter compiled for 4 CTAs per
// SM (64 registers) beats 3 (78 registers) by 2 %; 12 or 8 items per thread at 4 or
// 6 CTAs per SM are slower (6.17, 6.91 ms against 5.98 ms for 2^28 fp32 keys),
// match.any at 4 CTAs per SM takes 7.6 ms, and two interleaved counter chains per
// warp (half the items each, the second half adding the first half's counts)
// 6.21 ms: the rank is bound by instruction issue, not by the chain's latency.
#ifndef DR_SORT_MATCH
#define DR_SORT_MATCH 0
#endif
template <int NB>
__device__ __forceinline__ unsigned same_digit_lanes(int di) {
#if DR_SORT_MATCH
  return __match_any_sync(0xffffffffu, di);
#else
  unsigned peers = 0xffffffffu;
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    const unsigned bal = __ballot_sync(0xffffffffu, (di >> b) & 1);
    peers &= ((di >> b) & 1) ? bal : ~bal;
  }
  return peers;
#endif
}

// Loads the tile's keys: warp w holds tile positions [w*32*SIT, (w+1)*32*SIT),
// item i of lane l at w*32*SIT + i*32 + l, so (warp, item, lane) order is the
// input order.  Returns the tile's key count.
template <typename T, int SRC>
__device__ __forceinline__ int load_tile(const SortParams& P, int64_t tile, typename KeyOf<T>::K* key) {
  using KO = KeyOf<T>;
  using K = typename KO::K;
  constexpr int SIT = Tile<sizeof(K)>::IT, STILE = Tile<sizeof(K)>::N;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int cnt;
  if constexpr (SRC == 2) {
    const int64_t base = tile * STILE;
    cnt = (int)min((int64_t)STILE, P.n - base);
    const K* src = reinterpret_cast<const K*>(P.src) + base;
#pragma unroll
    for (int i = 0; i < SIT; ++i) {
      const int pos = w * 32 * SIT + i * 32 + lane;
      key[i] = pos < cnt ? src[pos] : K(0);
    }
  } else {
    const KPiece& pc = P.in[find_in_piece(P, tile)];
    const int64_t base = (tile - pc.tile_begin) * STILE;
    cnt = (int)min((int64_t)STILE, pc.len - base);
    ViewEval<T> ve;
    ve.init(P.vc);
    const bool two = P.vc.nleaf == 2;
    if (SRC == 1 && cnt == STILE) {
      T xa[SIT], xb[SIT];
#pragma unroll
      for (int i = 0; i < SIT; ++i) {
        const int64_t j = base + w * 32 * SIT + i * 32 + lane;
        xa[i] = reinterpret_cast<const T*>(pc.a)[j];
        xb[i] = two ? reinterpret_cast<const T*>(pc.b)[j] : T(0);
      }
      ve.template eval_all<SIT>(xa, xb);
#pragma unroll
      for (int i = 0; i < SIT; ++i) key[i] = KO::to(xa[i]);
    } else {
#pragma unroll
      for (int i = 0; i < SIT; ++i) {
        const int pos = w * 32 * SIT + i * 32 + lane;
        key[i] = pos < cnt ? KO::to(view_elem<T, SRC>(pc, base + pos, ve, two)) : K(0);
      }
    }
  }
  return cnt;
}

// Stable rank of the warp's keys among its keys of the same digit, in (item,
// lane) order: the peers of every item first (independent instructions), then
// the running per-digit counts of the warp (hist: its row of the CTA's table,
// zeroed), kept by each group's leader.  FULL: every lane holds a key.
template <typename K, bool FULL>
__device__ __forceinline__ void rank_warp(const K* key, int shift, int cnt, unsigned* hist, unsigned* rank) {
  constexpr int SIT = Tile<sizeof(K)>::IT;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  unsigned peers[SIT];
  int dig[SIT];
#pragma unroll
  for (int i = 0; i < SIT; ++i) {
    dig[i] = (int)((key[i] >> shift) & 255);
    if (!FULL && w * 32 * SIT + i * 32 + lane >= cnt) dig[i] = RADIX;  // no key
    peers[i] = same_digit_lanes<FULL ? 8 : 9>(dig[i]);
  }
  const unsigned lt = (1u << lane) - 1u;
#pragma unroll
  for (int i = 0; i < SIT; ++i) {
    const int leader = __ffs(peers[i]) - 1;
    unsigned old = 0;
    if (lane == leader && (FULL || dig[i] < RADIX)) {
      old = hist[dig[i]];
      hist[dig[i]] = old + __popc(peers[i]);
    }
    old = __shfl_sync(0xffffffffu, old, leader);
    rank[i] = old + __popc(peers[i] & lt);
    __syncwarp();
  }
}

// ---------------------------------------------------------------------------
// 1. Per-tile digit counts, digit-major.  (Counting 4 tiles per CTA, or into one
// histogram per warp, measured no faster: 5.99 / 6.10 ms against 5.99 ms per sort.)
// ---------------------------------------------------------------------------
template <typename T, int SRC>
__global__ void __launch_bounds__(ST) k_sort_count(const __grid_constant__ SortParams P) {
  using K = typename KeyOf<T>::K;
  constexpr int SIT = Tile<sizeof(K)>::IT;
  __shared__ unsigned h[RADIX];
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  if (tid < RADIX) h[tid] = 0;
  const int64_t tile = blockIdx.x;
  K key[SIT];
  const int cnt = load_tile<T, SRC>(P, tile, key);
  const int shift = 8 * P.pass;
  __syncthreads();
#pragma unroll
  for (int i = 0; i < SIT; ++i)
    if (w * 32 * SIT + i * 32 + lane < cnt) atomicAdd(&h[(int)((key[i] >> shift) & 255)], 1u);
  __syncthreads();
  if (tid < RADIX) P.counts[(int64_t)tid * P.ntiles + tile] = h[tid];
}

// ---------------------------------------------------------------------------
// 3. Stable rank and scatter.  SRC 0 / 1: keys from the view's pieces (first
// pass); SRC 2: key bits from P.src.  DST 0: key bits to P.dst; DST 1: values
// to the output segments (last pass).
// ---------------------------------------------------------------------------
template <typename T, int SRC, int DST>
__global__ void DR_SORT_SCATTER_BOUNDS k_sort_scatter(const __grid_constant__ SortParams P) {
  using KO = KeyOf<T>;
  using K = typename KO::K;
  constexpr int SIT = Tile<sizeof(K)>::IT, STILE = Tile<sizeof(K)>::N;
  __shared__ K skeys[STILE];
  __shared__ unsigned whist[SW][RADIX];
  __shared__ unsigned dstart[RADIX];
  __shared__ int dshift[RADIX];  // global start of digit d here minus its tile start
  __shared__ unsigned wsum[SW];
  __shared__ int64_t ostart[DST == 1 ? kMaxPieces : 1];
  // last pass: per digit run, the output segment holding its first key, as the
  // address of global index 0 in that segment's frame and the segment's end
  __shared__ unsigned long long dbase[DST == 1 ? RADIX : 1];
  __shared__ unsigned dsegend[DST == 1 ? RADIX : 1];

  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int shift = 8 * P.pass;
  const int64_t tile = blockIdx.x;
  for (int i = tid; i < SW * RADIX; i += ST) (&whist[0][0])[i] = 0;
  if constexpr (DST == 1)
    for (int i = tid; i < P.npout; i += ST) ostart[i] = P.out[i].start;
  // scanned counts: global position of the tile's first key of digit tid (< 2^30)
  const unsigned gstart = tid < RADIX ? P.counts[(int64_t)tid * P.ntiles + tile] : 0u;
  K key[SIT];
  const int cnt = load_tile<T, SRC>(P, tile, key);
  __syncthreads();
  unsigned rank[SIT];
  if (cnt == STILE) rank_warp<K, true>(key, shift, cnt, &whist[w][0], rank);
  else rank_warp<K, false>(key, shift, cnt, &whist[w][0], rank);
  __syncthreads();

  // thread d: digit d's exclusive prefix over warps and the tile's count of d;
  // the tile's digit runs start at the exclusive scan of those counts
  const int d = tid;
  unsigned tot = 0;
  if (d < RADIX) {
#pragma unroll
    for (int k = 0; k < SW; ++k) {
      const unsigned c = whist[k][d];
      whist[k][d] = tot;
      tot += c;
    }
  }
  unsigned tile_all;
  const unsigned ds = cta_excl_scan(tot, wsum, &tile_all);  // threads >= RADIX add 0
  if (d < RADIX) {
    dstart[d] = ds;
    dshift[d] = (int)gstart - (int)ds;
    if constexpr (DST == 1) {
      int lo = 0, hi = P.npout - 1;
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (ostart[mid] <= (int64_t)gstart) lo = mid;
        else hi = mid - 1;
      }
      dbase[d] = (unsigned long long)P.out[lo].p - (unsigned long long)ostart[lo] * sizeof(T);
      dsegend[d] = lo + 1 < P.npout ? (unsigned)ostart[lo + 1] : (unsigned)P.n;
    }
  }
  __syncthreads();

#pragma unroll
  for (int i = 0; i < SIT; ++i) {
    if (cnt == STILE || w * 32 * SIT + i * 32 + lane < cnt) {
      const int di = (int)((key[i] >> shift) & 255);
      const unsigned at = dstart[di] + whist[w][di] + rank[i];
      if (chk(at < (unsigned)STILE, 500, P.status)) skeys[at] = key[i];
    }
  }
  __syncthreads();
  for (int j = tid; j < cnt; j += ST) {
    const K k = skeys[j];
    const int dd = (int)((k >> shift) & 255);
    const unsigned g = (unsigned)(dshift[dd] + j);
    if (g >= (unsigned)P.n) continue;  // only if the counts' scan gave up a wait
    if constexpr (DST == 0) {
      reinterpret_cast<K*>(P.dst)[g] = k;
    } else if (g >= (unsigned)(dshift[dd] + (int)dstart[dd]) && g < dsegend[dd]) {
      // the run's segment (a run crosses into the next segment only at a boundary)
      *reinterpret_cast<T*>(dbase[dd] + (unsigned long long)g * sizeof(T)) = KO::from(k);
    } else {
      int lo = 0, hi = P.npout - 1;
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (ostart[mid] <= (int64_t)g) lo = mid;
        else hi = mid - 1;
      }
      const int64_t seg_end = lo + 1 < P.npout ? ostart[lo + 1] : P.n;
      if (chk((int64_t)g >= ostart[lo] && (int64_t)g < seg_end, 501, P.status))
        reinterpret_cast<T*>(P.out[lo].p)[(int64_t)g - ostart[lo]] = KO::from(k);
    }
  }
}

template <typename T, int SRC>
cudaError_t run_sort(SortParams& p, const SortLaunch& L, cudaStream_t s) {
  using K = typename KeyOf<T>::K;
  const int np = (int)sizeof(K);
  for (int pass = 0; pass < np; ++pass) {
    p.pass = pass;
    p.ntiles = pass == 0 ? L.ntiles0 : L.ntiles;
    p.src = pass == 0 ? nullptr : L.tmp[(pass - 1) & 1];
    p.dst = pass == np - 1 ? nullptr : L.tmp[pass & 1];
    const unsigned grid = (unsigned)p.ntiles;
    if (pass == 0) k_sort_count<T, SRC><<<grid, ST, 0, s>>>(p);
    else k_sort_count<T, 2><<<grid, ST, 0, s>>>(p);
    if (cudaError_t e = cudaGetLastError()) return e;
    // exclusive scan of the 256 x ntiles counts, in place
    ScanParams& sp = *L.scan;
    std::memset(&sp, 0, sizeof sp);
    sp.vc.kind = 0;
    sp.vc.nleaf = 1;
    sp.op = DR_PLUS;
    sp.dtype = DR_I32;
    sp.npieces = 1;
    sp.exclusive = 1;
    sp.ws = L.scan_ws;
    sp.status = p.status;
    sp.spin_limit = p.spin_limit;
    sp.skip_tile = -1;
    sp.pc[0].a = reinterpret_cast<const char*>(p.counts);
    sp.pc[0].o = reinterpret_cast<char*>(p.counts);
    sp.pc[0].len = (int64_t)RADIX * p.ntiles;
    sp.pc[0].tile_begin = 0;
    sp.pc[0].vec_ok = 1;
    sp.ntiles = (sp.pc[0].len + scan_tile_elems(DR_I32) - 1) / scan_tile_elems(DR_I32);
    if (cudaError_t e = launch_scan(sp, false, scan_grid(DR_I32, sp.ntiles), s)) return e;
    if (pass == 0 && pass == np - 1) k_sort_scatter<T, SRC, 1><<<grid, ST, 0, s>>>(p);
    else if (pass == 0) k_sort_scatter<T, SRC, 0><<<grid, ST, 0, s>>>(p);
    else if (pass == np - 1) k_sort_scatter<T, 2, 1><<<grid, ST, 0, s>>>(p);
    else k_sort_scatter<T, 2, 0><<<grid, ST, 0, s>>>(p);
    if (cudaError_t e = cudaGetLastError()) return e;
  }
  return cudaSuccess;
}

template <typename T>
cudaError_t run_sort_t(SortParams& p, const SortLaunch& L, cudaStream_t s) {
  return p.vc.kind == 0 ? run_sort<T, 0>(p, L, s) : run_sort<T, 1>(p, L, s);
}

}  // namespace

int sort_tile_elems(int dtype) { return (dtype == DR_F32 || dtype == DR_I32) ? Tile<4>::N : Tile<8>::N; }
int sort_passes(int dtype) { return (dtype == DR_F32 || dtype == DR_I32) ? 4 : 8; }

cudaError_t launch_sort(SortParams& p, const SortLaunch& L, cudaStream_t s) {
  switch (p.dtype) {
    case DR_F32: return run_sort_t<float>(p, L, s);
    case DR_F64: return run_sort_t<double>(p, L, s);
    case DR_I32: return run_sort_t<int>(p, L, s);
    case DR_I64: return run_sort_t<long long>(p, L, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace dr
