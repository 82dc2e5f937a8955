// inclusive_scan / exclusive_scan / reverse scan over a fused view, across
// segment boundaries (Sec. 4.3 "inclusive_scan", Algorithm 4).
//
// Algorithm 4 scans every segment locally, gathers the segments' last elements,
// scans them, and makes a second pass that adds each segment's offset: four
// accesses per element (Sec. 5, "Inclusive Scan" blames that second pass for
// the 1 -> 2 tile drop).  Here all segments are pieces of one global tile
// order (32 KB tiles, cut per piece) and the carry crosses segment boundaries
// inside one pass: decoupled lookback, two HBM accesses per element.
//
// Lookahead pipeline (persistent CTAs, tiles handed out by an atomic ticket).
// Iteration k of a CTA handles two tiles:
//   R phase, tile t_k: its loads were issued during iteration k-1 (so they
//     overlap a whole iteration); fold the view, run the thread / warp / block
//     scan tree and publish the tile aggregate.  The loads for t_{k+1} go out
//     at once, the ticket for t_{k+2} is taken.
//   S phase, tile t_{k-1}: warp 0 looks back over the predecessors (all of them
//     published their aggregates at least an iteration ago, so the walk rarely
//     waits), publishes the inclusive prefix, and the CTA re-reads the tile --
//     from L2: the R-phase loads carry an evict_last policy, the re-read and the
//     output stores evict_first -- scans it with the same tree plus the carry
//     and stores it.
// Waiting on a predecessor that is still loading stalls nothing but warp 0's
// walk for a tile whose data arrived an iteration ago, which is what keeps
// HBM busy; with one tile per CTA in flight the CTA idles during every walk.
//
// Forward progress: a CTA consumes its tickets in increasing order, so the
// smallest unfinished tile belongs to a CTA whose predecessors have all
// published.  Every wait is bounded (dr_set_spin_limit) and reports
// DR_E_TIMEOUT instead of hanging.
#pragma once
#include "dr_device.cuh"

namespace dr {
namespace kscan {

constexpr int ST = 256;           // threads per CTA
constexpr int SCH = 8;            // 16-byte chunks per thread per tile (32 KB tiles)
constexpr int SNW = ST / 32;      // warps
constexpr int SQ = SCH * SNW;     // warp-chunk totals per tile
constexpr int SR = SQ / 32;       // totals per lane of warp 0
constexpr int kLookbackG = 4;     // lookback slots per lane per round (128 tiles per round trip)
constexpr int kMinBlocks = 2;     // resident CTAs per SM
static_assert(SQ % 32 == 0, "block-level scan assumes a multiple of 32 totals");

template <typename T>
__host__ __device__ constexpr int stile() {
  return ST * SCH * (16 / (int)sizeof(T));
}

__device__ __forceinline__ int find_piece(const KPiece* pc, int n, int64_t tile) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (pc[mid].tile_begin <= tile) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// Where a logical tile lives.
struct TileRef {
  const KPiece* pc;
  int64_t base;  // element offset of the tile inside its piece
  bool full;     // a whole, 16-byte aligned tile: 128-bit path
};

template <typename T, bool REV>
__device__ __forceinline__ TileRef tile_ref(const ScanParams& P, long long lt) {
  const int64_t pt = REV ? P.ntiles - 1 - lt : lt;
  const KPiece* pc = &P.pc[find_piece(P.pc, P.npieces, pt)];
  const int64_t base = (pt - pc->tile_begin) * stile<T>();
  return TileRef{pc, base, pc->vec_ok && pc->len - base >= stile<T>()};
}

// 128-bit loads of a full tile (operand a, and b for a two-leaf view).
template <typename T>
__device__ __forceinline__ void load_full(const TileRef& r, bool two, int tid, unsigned long long pol,
                                          V16<T> (&xa)[SCH], V16<T> (&xb)[SCH]) {
  constexpr int V = 16 / sizeof(T);
#pragma unroll
  for (int c = 0; c < SCH; ++c)
    xa[c] = ld16_hint<T>(r.pc->a + (r.base + (int64_t)(c * ST + tid) * V) * (int64_t)sizeof(T), pol);
  if (two) {
#pragma unroll
    for (int c = 0; c < SCH; ++c)
      xb[c] = ld16_hint<T>(r.pc->b + (r.base + (int64_t)(c * ST + tid) * V) * (int64_t)sizeof(T), pol);
  }
}

// The tile's view values in registers: from the raw 128-bit loads of a full
// tile, or element by element (identity past the end) for a ragged one.
template <typename T, int KIND, typename VE>
__device__ __forceinline__ void tile_values(const TileRef& r, bool two, int tid, const VE& ve, T ident,
                                            const V16<T> (&xa)[SCH], const V16<T> (&xb)[SCH],
                                            T (&x)[SCH][16 / sizeof(T)]) {
  constexpr int V = 16 / sizeof(T);
  if (r.full) {
#pragma unroll
    for (int c = 0; c < SCH; ++c)
#pragma unroll
      for (int e = 0; e < V; ++e) {
        if constexpr (KIND == 0) x[c][e] = xa[c].v[e];
        else x[c][e] = ve(xa[c].v[e], two ? xb[c].v[e] : T(0));
      }
  } else {
#pragma unroll
    for (int c = 0; c < SCH; ++c)
#pragma unroll
      for (int e = 0; e < V; ++e) {
        const int64_t idx = r.base + (int64_t)(c * ST + tid) * V + e;
        if (idx < r.pc->len) {
          const T a = ld1<T>(r.pc->a + idx * (int64_t)sizeof(T));
          if constexpr (KIND == 0) x[c][e] = a;
          else x[c][e] = ve(a, two ? ld1<T>(r.pc->b + idx * (int64_t)sizeof(T)) : T(0));
        } else {
          x[c][e] = ident;
        }
      }
  }
}

// Thread-local and warp scans of a tile in the scan direction; warp totals go
// to s_tot in scan order.  The same tree runs in the R and the S phase, so the
// published aggregate equals the tile's last output exactly.
template <typename T, int OP, bool REV>
__device__ __forceinline__ void local_scan(T (&x)[SCH][16 / sizeof(T)], T (&wexc)[SCH], T* s_tot, int lane,
                                           int warp, T ident) {
  constexpr int V = 16 / sizeof(T);
  using O = Op<OP>;
  T tsum[SCH];
#pragma unroll
  for (int c = 0; c < SCH; ++c) {
    if constexpr (!REV) {
#pragma unroll
      for (int e = 1; e < V; ++e) x[c][e] = O::apply(x[c][e - 1], x[c][e]);
      tsum[c] = x[c][V - 1];
    } else {
#pragma unroll
      for (int e = V - 2; e >= 0; --e) x[c][e] = O::apply(x[c][e + 1], x[c][e]);
      tsum[c] = x[c][0];
    }
  }
#pragma unroll
  for (int c = 0; c < SCH; ++c) {
    const T wi = warp_inclusive<T, OP, REV>(tsum[c], lane);
    T we = REV ? __shfl_down_sync(0xffffffffu, wi, 1) : __shfl_up_sync(0xffffffffu, wi, 1);
    if (lane == (REV ? 31 : 0)) we = ident;
    wexc[c] = we;
    const T wt = __shfl_sync(0xffffffffu, wi, REV ? 0 : 31);
    const int q = REV ? SQ - 1 - (c * SNW + warp) : c * SNW + warp;
    if (lane == 0) s_tot[q] = wt;
  }
}

// Warp 0: block-level inclusive scan of the SQ totals (SR consecutive per lane).
// Returns the tile aggregate; exc = exclusive prefix of this lane's group.
template <typename T, int OP>
__device__ __forceinline__ T block_totals(const T* s_tot, int lane, T (&loc)[SR], T& exc) {
  using O = Op<OP>;
  T lsum = s_tot[lane * SR];
  loc[0] = lsum;
#pragma unroll
  for (int r = 1; r < SR; ++r) {
    loc[r] = s_tot[lane * SR + r];
    lsum = O::apply(lsum, loc[r]);
  }
  const T inc = warp_inclusive<T, OP, false>(lsum, lane);
  exc = __shfl_up_sync(0xffffffffu, inc, 1);
  return __shfl_sync(0xffffffffu, inc, 31);
}

// KIND: 0 = one leaf, no ops (PLUS only); 2 = generic fused view.
// REV: scan from the last element to the first (reverse inclusive scan).
// EXCL: exclusive scan with init.
template <typename T, int OP, int KIND, bool REV, bool EXCL>
__global__ void __launch_bounds__(ST, kMinBlocks) k_scan(const __grid_constant__ ScanParams P) {
  constexpr int V = 16 / sizeof(T);
  using O = Op<OP>;
  __shared__ T s_totR[SQ], s_totS[SQ], s_off[SQ];
  __shared__ long long s_t;
  __shared__ T s_agg;

  WsHeader* hdr = reinterpret_cast<WsHeader*>(P.ws);
  Slots<T> slots;
  slots.bind(P.ws + sizeof(WsHeader), P.ntiles);
  const unsigned tag = (ld_relaxed_u32(&hdr->epoch) & 0x3fffffffu) << 2;

  ViewEval<T> ve;
  if constexpr (KIND == 2) ve.init(P.vc);
  const bool two = KIND == 2 && P.vc.nleaf == 2;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const T ident = O::template identity<T>();
  const unsigned long long keep = l2_policy_evict_last(), drop = l2_policy_evict_first();

  // prologue: first tile and its loads, ticket of the second
  if (tid == 0) s_t = (long long)atomicAdd(&hdr->ticket, 1ull);
  __syncthreads();
  long long t = s_t, tprev = -1;
  __syncthreads();
  if (tid == 0 && t < P.ntiles) s_t = (long long)atomicAdd(&hdr->ticket, 1ull);
  V16<T> ra[SCH], rb[SCH];
  if (t < P.ntiles) {
    const TileRef r = tile_ref<T, REV>(P, t);
    if (r.full) load_full<T>(r, two, tid, keep, ra, rb);
  }
  __syncthreads();
  long long tnext = t < P.ntiles ? s_t : t;
  T aggprev = ident;  // warp 0: aggregate of tprev

  while (t < P.ntiles || tprev >= 0) {
    const bool haveR = t < P.ntiles, haveS = tprev >= 0;
    const TileRef rs = haveS ? tile_ref<T, REV>(P, tprev) : TileRef{nullptr, 0, false};

    // S-phase loads (L2 hits) go out first
    V16<T> sa[SCH], sb[SCH];
    if (haveS && rs.full) load_full<T>(rs, two, tid, drop, sa, sb);

    // ---- R phase: aggregate of tile t
    if (haveR) {
      const TileRef rr = tile_ref<T, REV>(P, t);
      T x[SCH][V], wx[SCH];
      tile_values<T, KIND>(rr, two, tid, ve, ident, ra, rb, x);
      local_scan<T, OP, REV>(x, wx, s_totR, lane, warp, ident);
    }
    __syncthreads();
    // the next tile's loads overlap this whole iteration; take the ticket after it
    if (tnext < P.ntiles) {
      const TileRef rn = tile_ref<T, REV>(P, tnext);
      if (rn.full) load_full<T>(rn, two, tid, keep, ra, rb);
    }
    long long tnn = tnext;
    if (tid == 0 && tnext < P.ntiles) tnn = (long long)atomicAdd(&hdr->ticket, 1ull);

    T prefix = ident;
    if (warp == 0) {
      if (haveR) {
        T loc[SR], exc;
        const T agg = block_totals<T, OP>(s_totR, lane, loc, exc);
        if (lane == 0 && t != P.skip_tile) slots.publish(t, tag, t == 0 ? kStateP : kStateA, agg);
        if (lane == 0) s_agg = agg;
      }
      // ---- S phase carry: lookback for tprev
      if (haveS && tprev > 0) {
        prefix = lookback<T, O, kLookbackG>(slots, tprev - 1, 0, tag, lane, P.spin_limit, P.status);
        if (lane == 0 && tprev != P.skip_tile) slots.publish(tprev, tag, kStateP, O::apply(prefix, aggprev));
      }
    }

    // ---- S phase: scan tile tprev with its carry and store it
    if (haveS) {
      T x[SCH][V], wexc[SCH];
      tile_values<T, KIND>(rs, two, tid, ve, ident, sa, sb, x);
      local_scan<T, OP, REV>(x, wexc, s_totS, lane, warp, ident);
      __syncthreads();
      if (warp == 0) {
        T loc[SR], exc;
        block_totals<T, OP>(s_totS, lane, loc, exc);
        if (lane == 0) exc = ident;
        T o = O::apply(prefix, exc);
#pragma unroll
        for (int r = 0; r < SR; ++r) {
          s_off[lane * SR + r] = o;
          o = O::apply(o, loc[r]);
        }
      }
      __syncthreads();
      const T init = from_bits<T>(P.init_bits);
#pragma unroll
      for (int c = 0; c < SCH; ++c) {
        const int q = REV ? SQ - 1 - (c * SNW + warp) : c * SNW + warp;
        const T pre = O::apply(s_off[q], wexc[c]);
        T y[V];
#pragma unroll
        for (int e = 0; e < V; ++e) {
          if constexpr (!EXCL) {
            y[e] = O::apply(pre, x[c][e]);
          } else {
            static_assert(!REV, "reverse exclusive scan not instantiated");
            y[e] = O::apply(init, e == 0 ? pre : O::apply(pre, x[c][e - 1]));
          }
        }
        const int64_t off = rs.base + (int64_t)(c * ST + tid) * V;
        if (rs.full) {
          V16<T> o;
#pragma unroll
          for (int e = 0; e < V; ++e) o.v[e] = y[e];
          st16_hint<T>(rs.pc->o + off * (int64_t)sizeof(T), o, drop);
        } else {
#pragma unroll
          for (int e = 0; e < V; ++e)
            if (off + e < rs.pc->len) reinterpret_cast<T*>(rs.pc->o)[off + e] = y[e];
        }
      }
    }
    if (tid == 0) s_t = tnn;
    __syncthreads();  // s_t, s_agg published; shared totals free
    if (warp == 0) aggprev = s_agg;
    tprev = haveR ? t : -1;
    t = tnext;
    tnext = s_t;
    __syncthreads();
  }

  // ---- exit: the last CTA restores the header for the next launch
  if (tid == 0) {
    __threadfence();
    if (atomicAdd(&hdr->done, 1u) == gridDim.x - 1) {
      hdr->ticket = 0;
      hdr->done = 0;
      hdr->epoch = hdr->epoch + 1;
      __threadfence();
    }
  }
}

template <typename T, int OP, int KIND, bool REV, bool EXCL>
cudaError_t go(const ScanParams& p, int grid, cudaStream_t s) {
  static int per_sm = 0;
  if (!per_sm) {
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_scan<T, OP, KIND, REV, EXCL>, ST, 0);
    if (per_sm <= 0) per_sm = 1;
  }
  if (grid <= 0) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    grid = sms * per_sm;
  }
  if (p.ntiles < grid) grid = (int)(p.ntiles > 0 ? p.ntiles : 1);
  k_scan<T, OP, KIND, REV, EXCL><<<grid, ST, 0, s>>>(p);
  return cudaGetLastError();
}

template <typename T, int OP>
cudaError_t dispatch_op(const ScanParams& p, int grid, cudaStream_t s) {
  if (p.exclusive) return go<T, OP, 2, false, true>(p, grid, s);
  if (OP == DR_PLUS && p.vc.kind == 0) return go<T, DR_PLUS, 0, false, false>(p, grid, s);
  return go<T, OP, 2, false, false>(p, grid, s);
}

template <typename T>
cudaError_t dispatch(const ScanParams& p, bool reverse, int grid, cudaStream_t s) {
  if (reverse) {
    if (p.vc.kind == 0) return go<T, DR_PLUS, 0, true, false>(p, grid, s);
    return go<T, DR_PLUS, 2, true, false>(p, grid, s);
  }
  switch (p.op) {
    case DR_PLUS: return dispatch_op<T, DR_PLUS>(p, grid, s);
    case DR_MIN: return dispatch_op<T, DR_MIN>(p, grid, s);
    default: return dispatch_op<T, DR_MAX>(p, grid, s);
  }
}

}  // namespace kscan
}  // namespace dr
