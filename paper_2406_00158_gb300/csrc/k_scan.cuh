// inclusive_scan / exclusive_scan / reverse scan over a fused view, across
// segment boundaries (Sec. 4.3 "inclusive_scan", Algorithm 4).
//
// Algorithm 4 scans every segment locally, gathers the segments' last elements,
// scans them, and makes a second pass that adds each segment's offset: four
// accesses per element (Sec. 5, "Inclusive Scan" blames that second pass for
// the 1 -> 2 tile drop).  Here all segments are pieces of one global tile
// order (32 KB tiles, 12 KB for fused views, cut per piece) and the carry
// crosses segment boundaries inside one pass: decoupled lookback, two HBM
// accesses per element.
//
// Lookahead pipeline (persistent CTAs, tiles handed out by an atomic ticket).
// Iteration k of a CTA handles two tiles:
//   R phase, tile t_k: its bytes were copied into a shared-memory stage by one
//     TMA bulk copy (cp.async.bulk, completing on the stage's mbarrier) issued
//     one iteration earlier; fold the view, reduce the tile (thread, warp,
//     block: the aggregate needs no scan) and publish the aggregate.  The freed
//     stage is refilled with the next ticketed tile.
//   S phase, tile t_{k-1}: warp 0 looks back over the predecessors (all of them
//     published their aggregates at least an iteration ago, so the walk rarely
//     waits), publishes the inclusive prefix, and the CTA re-reads the tile --
//     mostly an L2 hit: the re-read and the output stores carry an
//     evict_first policy so they do not push the staged tiles out -- scans it
//     (thread, warp, block; every warp scans the block's chunk totals itself)
//     with the carry and stores it.
// Measured on GB300 (2^28 fp32): with one tile per CTA in flight a CTA spent
// ~1.8 us loading and ~7 us waiting in lookback for predecessors still loading;
// the lookahead order removes most of that wait, L2 eviction policies keep the
// re-read in L2, and the shared-memory prefetch (two stages) frees the
// registers that held the prefetched tile so that three CTAs fit per SM.  Deeper prefetch was slower: a tile ticketed long before it is
// reduced publishes its aggregate late for its successors.
//
// Forward progress: a CTA consumes its tickets in increasing order, so the
// smallest unfinished tile belongs to a CTA whose predecessors have all
// published.  Every wait is bounded (dr_set_spin_limit) and reports
// DR_E_TIMEOUT instead of hanging.
#pragma once
#include "dr_device.cuh"

namespace dr {
namespace kscan {

#ifndef DR_SCAN_CHUNKS
#define DR_SCAN_CHUNKS 8
#endif
#ifndef DR_SCAN_MINB
#define DR_SCAN_MINB 3
#endif
#ifndef DR_SCAN_LOOKBACK_G
#define DR_SCAN_LOOKBACK_G 1
#endif
#ifndef DR_SCAN_THREADS
#define DR_SCAN_THREADS 256
#endif
#ifndef DR_SCAN_VIEW_CHUNKS
#define DR_SCAN_VIEW_CHUNKS 3
#endif
constexpr int ST = DR_SCAN_THREADS;  // threads per CTA
constexpr int SCH = DR_SCAN_CHUNKS;  // 16-byte chunks per thread per tile (8: 32 KB tiles)
constexpr int SNW = ST / 32;      // warps
constexpr int SQ = SCH * SNW;     // warp-chunk totals per tile
constexpr int SR = (SQ + 31) / 32;  // totals per lane in the block scan
constexpr int kLookbackG = DR_SCAN_LOOKBACK_G;  // lookback slots per lane per round
constexpr int kMinBlocks = DR_SCAN_MINB;        // resident CTAs per SM
constexpr int kStages = 2;        // tiles ticketed ahead: the tile being reduced + the next
constexpr int kTileBytes = ST * SCH * 16;
constexpr int kViewChunks = DR_SCAN_VIEW_CHUNKS;  // chunks per thread of a fused view's tile
#ifndef DR_SCAN_VIEW_MINB
#define DR_SCAN_VIEW_MINB 6
#endif
constexpr int kViewMinBlocks = DR_SCAN_VIEW_MINB;  // resident CTAs per SM of the fused-view kernels

// Tile geometry for CH 16-byte chunks per thread.
template <int CH>
struct Geo {
  static constexpr int SQ = CH * SNW;        // warp-chunk totals per tile
  static constexpr int SR = (SQ + 31) / 32;  // totals per lane in the block scan
  static constexpr int TB = ST * CH * 16;    // tile bytes
};

// A fused view (KIND 2, 3) keeps the view's values of a reduced tile in its
// stage until the tile's S phase, instead of re-reading its leaves from L2 and
// evaluating the view again: one more stage (the tile being reduced, the next
// one, and the one awaiting its S phase).  Its tiles are short (12 KB), so the
// three stages (36 KB) let six CTAs share an SM (compiled for 40 registers).
// Measured (2^28 fp32, zip·mul / one-leaf view): 16 KB tiles at 3 CTAs/SM 0.720 /
// 0.662 ms, at 4 CTAs/SM 0.600 / 0.552 ms; 12 KB tiles at 5 CTAs/SM 0.640 /
// 0.591 ms, at 6 CTAs/SM 0.580 / 0.548 ms.
template <int KIND>
__host__ __device__ constexpr int chunks() { return KIND != 0 ? kViewChunks : SCH; }
template <int KIND>
__host__ __device__ constexpr bool keeps_view() { return KIND != 0; }
template <int KIND>
__host__ __device__ constexpr int smem_stages() { return keeps_view<KIND>() ? kStages + 1 : kStages; }
template <int KIND>
__host__ __device__ constexpr int smem_bytes() { return smem_stages<KIND>() * Geo<chunks<KIND>()>::TB; }

template <typename T, int CH = SCH>
__host__ __device__ constexpr int stile() {
  return ST * CH * (16 / (int)sizeof(T));
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


// The piece table of a launch: inline in the kernel parameters (read through
// the constant cache), or, with EXT, in device memory (a call of more than
// kMaxPieces pieces).  A compile-time choice, so that each kernel knows the
// address space of every piece access.
template <bool EXT>
__device__ __forceinline__ const KPiece* piece_table(const ScanParams& P) {
  if constexpr (EXT) return P.pc_ext;
  else return P.pc;
}

// Where a logical tile lives.
struct TileRef {
  const KPiece* pc;
  int64_t base;  // element offset of the tile inside its piece
  bool full;     // a whole, 16-byte aligned tile: 128-bit path
};

template <typename T, bool REV, bool EXT, int CH = SCH>
__device__ __forceinline__ TileRef tile_ref(const ScanParams& P, long long lt) {
  const KPiece* tab = piece_table<EXT>(P);
  const int64_t pt = REV ? P.ntiles - 1 - lt : lt;
  const int k = find_piece(tab, P.npieces, pt);
  const KPiece* pc = &tab[k];
  const int64_t base = (pt - pc->tile_begin) * stile<T, CH>();
  const bool ok = chk(lt >= 0 && lt < P.ntiles && k >= 0 && k < P.npieces && base >= 0 && base < pc->len, 100,
                      P.status);
  return TileRef{pc, base, ok && pc->vec_ok && pc->len - base >= stile<T, CH>()};
}

// 128-bit loads of a full tile (operand a, and b for a two-leaf view).
template <typename T, int CH = SCH>
__device__ __forceinline__ void load_full(const TileRef& r, bool two, int tid, unsigned long long pol,
                                          V16<T> (&xa)[CH], V16<T> (&xb)[CH], unsigned* status = nullptr) {
  constexpr int V = 16 / sizeof(T);
#pragma unroll
  for (int c = 0; c < CH; ++c) {
    const int64_t e0 = r.base + (int64_t)(c * ST + tid) * V;
    const char* src = r.pc->a + e0 * (int64_t)sizeof(T);
    if (chk(e0 >= 0 && e0 + V <= r.pc->len && ((uintptr_t)src & 15) == 0, 104, status))
      xa[c] = ld16_hint<T>(src, pol);
  }
  if (two) {
#pragma unroll
    for (int c = 0; c < CH; ++c)
      xb[c] = ld16_hint<T>(r.pc->b + (r.base + (int64_t)(c * ST + tid) * V) * (int64_t)sizeof(T), pol);
  }
}

// The tile's view values in registers: from the raw 128-bit loads of a full
// tile, or element by element (identity past the end) for a ragged one.
template <typename T, int KIND, int CH, typename VE>
__device__ __forceinline__ void tile_values(const TileRef& r, bool two, int tid, const VE& ve, T ident,
                                            const V16<T> (&xa)[CH], const V16<T> (&xb)[CH],
                                            T (&x)[CH][16 / sizeof(T)]) {
  constexpr int V = 16 / sizeof(T);
  if (r.full) {
#pragma unroll
    for (int c = 0; c < CH; ++c) {
      T y[V];
#pragma unroll
      for (int e = 0; e < V; ++e) {
        x[c][e] = xa[c].v[e];
        y[e] = two ? xb[c].v[e] : T(0);
      }
      if constexpr (KIND != 0) ve.template eval_all<V>(&x[c][0], y);
    }
  } else {
#pragma unroll
    for (int c = 0; c < CH; ++c)
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
template <typename T, int OP, bool REV, int CH = SCH>
__device__ __forceinline__ void local_scan(T (&x)[CH][16 / sizeof(T)], T (&wexc)[CH], T* s_tot, int lane,
                                           int warp, T ident) {
  constexpr int V = 16 / sizeof(T);
  constexpr int Q = Geo<CH>::SQ;
  using O = Op<OP>;
  T tsum[CH];
#pragma unroll
  for (int c = 0; c < CH; ++c) {
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
  for (int c = 0; c < CH; ++c) {
    const T wi = warp_inclusive<T, OP, REV>(tsum[c], lane);
    T we = REV ? __shfl_down_sync(0xffffffffu, wi, 1) : __shfl_up_sync(0xffffffffu, wi, 1);
    if (lane == (REV ? 31 : 0)) we = ident;
    wexc[c] = we;
    const int q = REV ? Q - 1 - (c * SNW + warp) : c * SNW + warp;
    if (lane == (REV ? 0 : 31)) s_tot[q] = wi;  // the lane holding the warp's total
  }
}

// The R phase needs only the tile's aggregate: each thread folds its values (a
// tree), the warp folds the threads; one total per warp (ops are commutative).
template <typename T, int OP, int CH = SCH>
__device__ __forceinline__ void tile_reduce(const T (&x)[CH][16 / sizeof(T)], T* s_tot, int lane, int warp) {
  constexpr int V = 16 / sizeof(T);
  using O = Op<OP>;
  T c[CH];
#pragma unroll
  for (int q = 0; q < CH; ++q) {
    T a = x[q][0];
#pragma unroll
    for (int e = 1; e < V; ++e) a = O::apply(a, x[q][e]);
    c[q] = a;
  }
  if constexpr ((CH & (CH - 1)) == 0) {
#pragma unroll
    for (int w = CH / 2; w >= 1; w >>= 1)
#pragma unroll
      for (int q = 0; q < w; ++q) c[q] = O::apply(c[q], c[q + w]);
  } else {  // pairwise over any count
#pragma unroll
    for (int w = 1; w < CH; w <<= 1)
#pragma unroll
      for (int q = 0; q + w < CH; q += 2 * w) c[q] = O::apply(c[q], c[q + w]);
  }
  const T s = warp_reduce<T, OP>(c[0]);
  if (lane == 0) s_tot[warp] = s;
}

// Warp 0: block-level inclusive scan of the SQ totals (SR consecutive per lane).
// Returns the tile aggregate; exc = exclusive prefix of this lane's group.
template <typename T, int OP, int CH = SCH>
__device__ __forceinline__ T block_totals(const T* s_tot, int lane, T (&loc)[Geo<CH>::SR], T& exc) {
  using O = Op<OP>;
  constexpr int R = Geo<CH>::SR, Q = Geo<CH>::SQ;
  const T ident = O::template identity<T>();
  // lanes past the Q totals (when Q is not a multiple of 32) contribute the identity
  T lsum = (Q % 32 == 0 || lane * R < Q) ? s_tot[lane * R] : ident;
  loc[0] = lsum;
#pragma unroll
  for (int r = 1; r < R; ++r) {
    loc[r] = (Q % 32 == 0 || lane * R + r < Q) ? s_tot[lane * R + r] : ident;
    lsum = O::apply(lsum, loc[r]);
  }
  const T inc = warp_inclusive<T, OP, false>(lsum, lane);
  exc = __shfl_up_sync(0xffffffffu, inc, 1);
  return __shfl_sync(0xffffffffu, inc, 31);
}

// Thread 0: starts the load of tile `lt` into stage `st` (one bulk copy of a full
// tile, completing on the stage's mbarrier), or completes the barrier's phase
// without a copy (ragged tile, or no tile).  One arrival per call either way, so
// a stage's barrier phase counts its uses.
// With two leaves (a zip view), the tile's range of leaf b is prefetched into
// L2 at the same time, so the R phase's loads of b hit L2.
template <typename T, bool REV, bool EXT, int CH = SCH>
__device__ __forceinline__ void stage_issue(const ScanParams& P, long long lt, char* stage,
                                            unsigned long long* bar, bool two = false) {
  constexpr int TB = Geo<CH>::TB;
  if (lt < P.ntiles) {
    const TileRef r = tile_ref<T, REV, EXT, CH>(P, lt);
    if (r.full) {
      mbar_expect_tx(bar, TB);
      bulk_g2s(stage, r.pc->a + r.base * (int64_t)sizeof(T), TB, bar);
      if (two) bulk_prefetch_l2(r.pc->b + r.base * (int64_t)sizeof(T), TB);
      return;
    }
  }
  mbar_arrive(bar);
}

// KIND: 0 = one leaf, no ops; 2 = generic fused view of one leaf; 3 = generic
// fused view of two leaves (a zip; the only one that needs the second tile's
// registers, so the one-leaf view keeps the plain kernel's occupancy).
// REV: scan from the last element to the first (reverse inclusive scan).
// EXCL: exclusive scan with init.
template <typename T, int OP, int KIND, bool REV, bool EXCL, bool EXT>
__global__ void __launch_bounds__(ST, KIND != 0 ? kViewMinBlocks : kMinBlocks) k_scan(const __grid_constant__ ScanParams P) {
  constexpr int V = 16 / sizeof(T);
  constexpr bool KEEP = keeps_view<KIND>();
  constexpr int NST = smem_stages<KIND>();
  constexpr int CH = chunks<KIND>();        // 16-byte chunks per thread per tile
  constexpr int TB = Geo<CH>::TB, Q = Geo<CH>::SQ, R = Geo<CH>::SR;
  using O = Op<OP>;
  extern __shared__ __align__(128) char s_stage[];  // NST x TB
  __shared__ __align__(8) unsigned long long s_bar[NST];
  __shared__ T s_totR[SNW], s_totS[Q];
  __shared__ long long s_tk[kStages + 2];
  __shared__ T s_agg, s_pref;

  WsHeader* hdr = reinterpret_cast<WsHeader*>(P.ws);
  Slots<T> slots;
  slots.bind(P.ws + sizeof(WsHeader), P.ntiles);
  const unsigned tag = (ld_relaxed_u32(&hdr->epoch) & 0x3fffffffu) << 2;

  ViewEval<T> ve;
  if constexpr (KIND >= 2) ve.init(P.vc);
  const bool two = KIND == 3 && P.vc.nleaf == 2;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const T ident = O::template identity<T>();
  const unsigned long long keep = l2_policy_evict_last(), drop = l2_policy_evict_first();
  (void)keep;
  // Carry-in from device memory (e.g. the total of the part of the range held by
  // lower-ranked GPUs): an inclusive scan's chain starts from it, an exclusive
  // scan takes it as its initial value.
  T chain0 = ident, init = from_bits<T>(P.init_bits);
  if (P.carry) {
    if constexpr (EXCL) init = *reinterpret_cast<const T*>(P.carry);
    else if constexpr (!REV) chain0 = *reinterpret_cast<const T*>(P.carry);
  }

  // prologue: tickets of the first kStages tiles (in order) and their loads
  if (tid == 0) {
    for (int d = 0; d < NST; ++d) mbar_init(&s_bar[d], 1);
    fence_mbar_init();
    for (int d = 0; d < kStages; ++d) {
      s_tk[d] = (long long)atomicAdd(&hdr->ticket, 1ull);
      stage_issue<T, REV, EXT, CH>(P, s_tk[d], s_stage + d * TB, &s_bar[d], two);
    }
  }
  __syncthreads();
  long long tk[kStages];  // tickets of the staged tiles, oldest first
#pragma unroll
  for (int d = 0; d < kStages; ++d) tk[d] = s_tk[d];
  unsigned parity = 0;    // bit d: phase parity of stage d's next completion
  unsigned pend = (1u << kStages) - 1;  // bit d: stage d has an issue not yet consumed
  long long tprev = -1;
  T aggprev = ident;  // warp 0: aggregate of tprev
  int sidx = 0;       // stage of tk[0]
  unsigned it = 0;    // iteration parity: the s_tk slot of this iteration's ticket

  while (tk[0] < P.ntiles || tprev >= 0) {
    const long long t = tk[0];
    const bool haveR = t < P.ntiles, haveS = tprev >= 0;

    // ---- R phase: aggregate of tile t (from its stage; ragged tiles load directly)
    bool copy_lost = false;  // this thread's wait for the stage's bulk copy expired
    if (haveR) {
      const TileRef rr = tile_ref<T, REV, EXT, CH>(P, t);
      T x[CH][V], wx[CH];
      if (rr.full) {
        copy_lost = !mbar_wait(&s_bar[sidx], (parity >> sidx) & 1u, kCopyWaitPolls, P.status);
        const char* st = s_stage + sidx * TB;
#pragma unroll
        for (int c = 0; c < CH; ++c) {
          V16<T> va;
          const char* sp = st + (c * ST + tid) * 16;
          if (chk(sidx >= 0 && sidx < NST && ((uintptr_t)sp & 15) == 0, 103, P.status))
            va = *reinterpret_cast<const V16<T>*>(sp);
          V16<T> vb;
          if (two) vb = ld16_hint<T>(rr.pc->b + (rr.base + (int64_t)(c * ST + tid) * V) * (int64_t)sizeof(T), keep);
          T y[V];
#pragma unroll
          for (int e = 0; e < V; ++e) {
            x[c][e] = va.v[e];
            y[e] = two ? vb.v[e] : T(0);
          }
          if constexpr (KIND != 0) ve.template eval_all<V>(&x[c][0], y);
        }
      } else {
        V16<T> na[CH], nb[CH];
        tile_values<T, KIND, CH>(rr, two, tid, ve, ident, na, nb, x);
      }
      if constexpr (KEEP) {
        // the view's values stay in the stage (each thread its own chunks) for the
        // tile's S phase in the next iteration
        char* st = s_stage + sidx * TB;
#pragma unroll
        for (int c = 0; c < CH; ++c) {
          V16<T> v;
#pragma unroll
          for (int e = 0; e < V; ++e) v.v[e] = x[c][e];
          *reinterpret_cast<V16<T>*>(st + (c * ST + tid) * 16) = v;
        }
      }
      tile_reduce<T, OP, CH>(x, s_totR, lane, warp);
    }
    // the ticket after the staged ones (needed only at the end of the iteration)
    const long long tlast = tk[kStages - 1];
    long long tnew = P.ntiles;
    if (tid == 0 && tlast < P.ntiles) tnew = (long long)atomicAdd(&hdr->ticket, 1ull);
    if (__syncthreads_or(copy_lost)) {
      // A bulk copy did not complete within its bound (DR_E_TIMEOUT is recorded):
      // no stage is read or re-armed any more; wait, again bounded, for the
      // copies that may still be in flight into either stage, then leave.
      if (tid == 0)
        for (int d = 0; d < NST; ++d)
          if (pend >> d & 1u) mbar_wait(&s_bar[d], (parity >> d) & 1u, kCopyWaitPolls, P.status);
      __syncthreads();
      break;
    }

    T prefix = (haveS && tprev == 0) ? chain0 : ident;
    if (warp == 0) {
      if (haveR) {
        const T agg = warp_reduce<T, OP>(lane < SNW ? s_totR[lane] : ident);
        if (lane == 0 && t != P.skip_tile)
          slots.publish(t, tag, t == 0 ? kStateP : kStateA, t == 0 ? O::apply(chain0, agg) : agg);
        if (lane == 0) s_agg = agg;
      }
      // ---- S phase carry: lookback for tprev
      if (haveS && tprev > 0) {
        prefix = lookback<T, O, kLookbackG>(slots, tprev - 1, 0, tag, lane, P.spin_limit, P.status);
        if (lane == 0 && tprev != P.skip_tile) slots.publish(tprev, tag, kStateP, O::apply(prefix, aggprev));
      }
      if (lane == 0) s_pref = prefix;
    }

    // ---- S phase: tile tprev again -- re-read from L2, or (a zip view) its view
    // values from the stage the R phase left them in -- scanned with its carry, stored
    if (haveS) {
      const TileRef rs = tile_ref<T, REV, EXT, CH>(P, tprev);
      T x[CH][V], wexc[CH];
      if constexpr (KEEP) {
        const char* st = s_stage + ((sidx + NST - 1) % NST) * TB;
#pragma unroll
        for (int c = 0; c < CH; ++c) {
          const V16<T> v = *reinterpret_cast<const V16<T>*>(st + (c * ST + tid) * 16);
#pragma unroll
          for (int e = 0; e < V; ++e) x[c][e] = v.v[e];
        }
        fence_proxy_async_smem();  // generic writes above precede the stage's next bulk copy
      } else {
        V16<T> sa[CH], sb[CH];
        if (rs.full) load_full<T, CH>(rs, two, tid, drop, sa, sb, P.status);
        tile_values<T, KIND, CH>(rs, two, tid, ve, ident, sa, sb, x);
      }
      local_scan<T, OP, REV, CH>(x, wexc, s_totS, lane, warp, ident);
      if (tid == 0) s_tk[kStages + (it & 1)] = tnew;  // the next ticket, published by this barrier
      __syncthreads();
      // every warp scans the Q chunk totals itself (no second barrier for a table
      // of offsets): the carry-in of each of this thread's chunks' warp segments
      T cbase[CH];
      {
        T loc[R], exc, offs[R];
        block_totals<T, OP, CH>(s_totS, lane, loc, exc);
        if (lane == 0) exc = ident;
        offs[0] = O::apply(s_pref, exc);
#pragma unroll
        for (int r = 1; r < R; ++r) offs[r] = O::apply(offs[r - 1], loc[r - 1]);
#pragma unroll
        for (int c = 0; c < CH; ++c) {
          const int q = REV ? Q - 1 - (c * SNW + warp) : c * SNW + warp;
          T sel = offs[0];
#pragma unroll
          for (int r = 1; r < R; ++r)
            if (q % R == r) sel = offs[r];
          cbase[c] = __shfl_sync(0xffffffffu, sel, q / R);
        }
      }
#pragma unroll
      for (int c = 0; c < CH; ++c) {
        const T pre = O::apply(cbase[c], wexc[c]);
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
          char* dst = rs.pc->o + off * (int64_t)sizeof(T);
          if (chk(off >= 0 && off + V <= rs.pc->len && ((uintptr_t)dst & 15) == 0, 105, P.status))
            st16_hint<T>(dst, o, drop);
        } else {
#pragma unroll
          for (int e = 0; e < V; ++e)
            if (off + e < rs.pc->len) reinterpret_cast<T*>(rs.pc->o)[off + e] = y[e];
        }
      }
    }
    if (!haveS) {  // no S-phase barrier: publish the ticket, and keep s_totR until warp 0 read it
      if (tid == 0) s_tk[kStages + (it & 1)] = tnew;
      __syncthreads();
    }
    // refill the stage whose tile is done -- the one read in this R phase, or for a
    // zip view the one read in this S phase -- with the next ticketed tile (all
    // reads of it happened before the last barrier); it is reduced two iterations
    // from now.  Two barriers per iteration: s_tk is double-buffered (a slot is
    // rewritten two iterations later, after the next iteration's first barrier)
    const long long tn = tlast < P.ntiles ? s_tk[kStages + (it & 1)] : P.ntiles;
    ++it;
    const int fill = (sidx + kStages) % NST;
    if (tid == 0) {
      fence_proxy_async_smem();
      stage_issue<T, REV, EXT, CH>(P, tn, s_stage + fill * TB, &s_bar[fill], two);
    }
    parity ^= 1u << sidx;
    pend = (pend & ~(1u << sidx)) | (1u << fill);
    if (warp == 0) aggprev = s_agg;
    tprev = haveR ? t : -1;
#pragma unroll
    for (int d = 0; d < kStages - 1; ++d) tk[d] = tk[d + 1];
    tk[kStages - 1] = tn;
    sidx = (sidx + 1) % NST;
    // no barrier here: every shared value read since the last barrier is next
    // written after the next iteration's first barrier
  }

  // ---- exit (no copy is in flight: every staged ticket left is past the end, or
  // the abort path above drained both stages): the last CTA restores the header
  // for the next launch
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

// ---------------------------------------------------------------------------
// One wave: a plain forward scan whose tiles all fit in one wave of resident
// CTAs (e.g. 2^20 int64 = 256 tiles).  Every tile is in flight at once, so the
// lookahead pipeline above only adds latency (a bulk copy, a second ticket, a
// re-read of the tile); here a CTA takes one ticket, keeps its tile in
// registers, publishes the aggregate, folds the aggregates of all its
// predecessors (every thread polls one or two of them: one L2 round trip, where
// a lookback would wait for inclusive prefixes to spread from tile 0) and stores
// the results straight from registers.
// ---------------------------------------------------------------------------
template <typename T, int OP, bool EXCL, bool EXT>
__global__ void __launch_bounds__(ST) k_scan_wave(const __grid_constant__ ScanParams P) {
  constexpr int V = 16 / sizeof(T);
  using O = Op<OP>;
  __shared__ T s_tot[SQ], s_red[SNW];
  __shared__ long long s_t;

  WsHeader* hdr = reinterpret_cast<WsHeader*>(P.ws);
  Slots<T> slots;
  slots.bind(P.ws + sizeof(WsHeader), P.ntiles);
  const unsigned tag = (ld_relaxed_u32(&hdr->epoch) & 0x3fffffffu) << 2;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const T ident = O::template identity<T>();
  T chain0 = ident, init = from_bits<T>(P.init_bits);
  if (P.carry) {
    if constexpr (EXCL) init = *reinterpret_cast<const T*>(P.carry);
    else chain0 = *reinterpret_cast<const T*>(P.carry);
  }
  if (tid == 0) s_t = (long long)atomicAdd(&hdr->ticket, 1ull);
  __syncthreads();
  const long long t = s_t;
  if (t < P.ntiles) {
    const TileRef r = tile_ref<T, false, EXT>(P, t);
    V16<T> xa[SCH], xb[SCH];
    if (r.full) load_full<T>(r, false, tid, l2_policy_evict_first(), xa, xb, P.status);
    T x[SCH][V], wexc[SCH];
    ViewEval<T> ve;
    tile_values<T, 0, SCH>(r, false, tid, ve, ident, xa, xb, x);
    local_scan<T, OP, false>(x, wexc, s_tot, lane, warp, ident);
    __syncthreads();
    // every warp scans the chunk totals (the same order in each); thread 0
    // publishes the aggregate (tile 0's with the carry-in folded in)
    T loc[SR], exc;
    const T agg = block_totals<T, OP>(s_tot, lane, loc, exc);
    if (tid == 0 && t != P.skip_tile) slots.publish(t, tag, kStateA, t == 0 ? O::apply(chain0, agg) : agg);
    // the carry: the fold of every predecessor's aggregate, all of them polled at
    // once by the whole CTA (one L2 round trip, no chain of inclusive prefixes)
    T part = ident;
    for (long long i = tid; i < t; i += ST) {
      T v;
      wait_slot<T, Slots<T>, O>(slots, t - 1 - i, tag, v, P.spin_limit, P.status);
      part = O::apply(part, v);
    }
    part = warp_reduce<T, OP>(part);
    if (lane == 0) s_red[warp] = part;
    __syncthreads();
    const T prefix = t == 0 ? chain0 : warp_reduce<T, OP>(lane < SNW ? s_red[lane] : ident);
    T cbase[SCH];
    {
      T offs[SR];
      offs[0] = O::apply(prefix, lane == 0 ? ident : exc);
#pragma unroll
      for (int q = 1; q < SR; ++q) offs[q] = O::apply(offs[q - 1], loc[q - 1]);
#pragma unroll
      for (int c = 0; c < SCH; ++c) {
        const int q = c * SNW + warp;
        T sel = offs[0];
#pragma unroll
        for (int k = 1; k < SR; ++k)
          if (q % SR == k) sel = offs[k];
        cbase[c] = __shfl_sync(0xffffffffu, sel, q / SR);
      }
    }
    char* out = r.pc->o;
    const int64_t len = r.pc->len;
#pragma unroll
    for (int c = 0; c < SCH; ++c) {
      const T pre = O::apply(cbase[c], wexc[c]);
      T y[V];
#pragma unroll
      for (int e = 0; e < V; ++e) {
        if constexpr (!EXCL) y[e] = O::apply(pre, x[c][e]);
        else y[e] = O::apply(init, e == 0 ? pre : O::apply(pre, x[c][e - 1]));
      }
      const int64_t off = r.base + (int64_t)(c * ST + tid) * V;
      if (r.full) {
        V16<T> ov;
#pragma unroll
        for (int e = 0; e < V; ++e) ov.v[e] = y[e];
        char* dst = out + off * (int64_t)sizeof(T);
        if (chk(off >= 0 && off + V <= len && ((uintptr_t)dst & 15) == 0, 106, P.status)) st16<T>(dst, ov);
      } else {
#pragma unroll
        for (int e = 0; e < V; ++e)
          if (off + e < len) reinterpret_cast<T*>(out)[off + e] = y[e];
      }
    }
  }
  // the last CTA restores the header for the next launch
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

template <typename T, int OP, int KIND, bool REV, bool EXCL, bool EXT>
cudaError_t go(const ScanParams& p, int grid, cudaStream_t s) {
  if constexpr (KIND == 0 && !REV) {
    // every tile in one wave of the one-wave kernel: take it
    static OccCache occw;
    const int per = resident_ctas(occw, k_scan_wave<T, OP, EXCL, EXT>, ST, 0);
    if (per > 0 && p.ntiles <= (int64_t)current_sm_count() * per) {
      k_scan_wave<T, OP, EXCL, EXT><<<(unsigned)(p.ntiles > 0 ? p.ntiles : 1), ST, 0, s>>>(p);
      return cudaGetLastError();
    }
  }
  static OccCache occ;
  const int per_sm = resident_ctas(occ, k_scan<T, OP, KIND, REV, EXCL, EXT>, ST, smem_bytes<KIND>());
  if (per_sm <= 0) return cudaErrorInvalidConfiguration;
  if (grid <= 0) grid = current_sm_count() * per_sm;
  if (p.ntiles < grid) grid = (int)(p.ntiles > 0 ? p.ntiles : 1);
  k_scan<T, OP, KIND, REV, EXCL, EXT><<<grid, ST, smem_bytes<KIND>(), s>>>(p);
  return cudaGetLastError();
}

template <typename T, int OP, bool EXT>
cudaError_t dispatch_op(const ScanParams& p, int grid, cudaStream_t s) {
  // KIND 0 (a plain vector) for every operator; the interpreted view otherwise
  const bool zip = p.vc.nleaf == 2;
  if (p.exclusive) {
    if (p.vc.kind == 0) return go<T, OP, 0, false, true, EXT>(p, grid, s);
    return zip ? go<T, OP, 3, false, true, EXT>(p, grid, s) : go<T, OP, 2, false, true, EXT>(p, grid, s);
  }
  if (p.vc.kind == 0) return go<T, OP, 0, false, false, EXT>(p, grid, s);
  return zip ? go<T, OP, 3, false, false, EXT>(p, grid, s) : go<T, OP, 2, false, false, EXT>(p, grid, s);
}

// EXT: the call's piece table is in device memory (more than kMaxPieces pieces).
template <typename T, bool EXT>
cudaError_t dispatch(const ScanParams& p, bool reverse, int grid, cudaStream_t s) {
  if (reverse) {
    if (p.vc.kind == 0) return go<T, DR_PLUS, 0, true, false, EXT>(p, grid, s);
    return p.vc.nleaf == 2 ? go<T, DR_PLUS, 3, true, false, EXT>(p, grid, s)
                           : go<T, DR_PLUS, 2, true, false, EXT>(p, grid, s);
  }
  switch (p.op) {
    case DR_PLUS: return dispatch_op<T, DR_PLUS, EXT>(p, grid, s);
    case DR_MIN: return dispatch_op<T, DR_MIN, EXT>(p, grid, s);
    default: return dispatch_op<T, DR_MAX, EXT>(p, grid, s);
  }
}

}  // namespace kscan
}  // namespace dr
