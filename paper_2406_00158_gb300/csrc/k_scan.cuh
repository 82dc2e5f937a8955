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
//   R phase, tile t_k: its bytes were copied into a shared-memory stage by one
//     TMA bulk copy (cp.async.bulk, completing on the stage's mbarrier) issued
//     one iteration earlier; fold the view, run the thread / warp / block scan
//     tree and publish the tile aggregate.  The freed stage is refilled with the
//     next ticketed tile.
//   S phase, tile t_{k-1}: warp 0 looks back over the predecessors (all of them
//     published their aggregates at least an iteration ago, so the walk rarely
//     waits), publishes the inclusive prefix, and the CTA re-reads the tile --
//     mostly an L2 hit: the re-read and the output stores carry an
//     evict_first policy so they do not push the staged tiles out -- scans it
//     with the same tree plus the carry and stores it.
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
constexpr int ST = 256;           // threads per CTA
constexpr int SCH = DR_SCAN_CHUNKS;  // 16-byte chunks per thread per tile (8: 32 KB tiles)
constexpr int SNW = ST / 32;      // warps
constexpr int SQ = SCH * SNW;     // warp-chunk totals per tile
constexpr int SR = SQ / 32;       // totals per lane of warp 0
constexpr int kLookbackG = DR_SCAN_LOOKBACK_G;  // lookback slots per lane per round
constexpr int kMinBlocks = DR_SCAN_MINB;        // resident CTAs per SM
constexpr int kStages = 2;        // shared-memory stages: the tile being reduced + the next
constexpr int kTileBytes = ST * SCH * 16;

constexpr int smem_bytes() { return kStages * kTileBytes; }
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
  // search the inline table (kernel parameters: constant-cache loads) or the
  // device table in separate branches, so that each keeps its address space
  int k;
  const KPiece* pc;
  if (P.pc_ext) {
    k = find_piece(P.pc_ext, P.npieces, pt);
    pc = &P.pc_ext[k];
  } else {
    k = find_piece(P.pc, P.npieces, pt);
    pc = &P.pc[k];
  }
  const int64_t base = (pt - pc->tile_begin) * stile<T>();
  const bool ok = chk(lt >= 0 && lt < P.ntiles && k >= 0 && k < P.npieces && base >= 0 && base < pc->len, 100,
                      P.status);
  return TileRef{pc, base, ok && pc->vec_ok && pc->len - base >= stile<T>()};
}

// 128-bit loads of a full tile (operand a, and b for a two-leaf view).
template <typename T>
__device__ __forceinline__ void load_full(const TileRef& r, bool two, int tid, unsigned long long pol,
                                          V16<T> (&xa)[SCH], V16<T> (&xb)[SCH], unsigned* status = nullptr) {
  constexpr int V = 16 / sizeof(T);
#pragma unroll
  for (int c = 0; c < SCH; ++c) {
    const int64_t e0 = r.base + (int64_t)(c * ST + tid) * V;
    const char* src = r.pc->a + e0 * (int64_t)sizeof(T);
    if (chk(e0 >= 0 && e0 + V <= r.pc->len && ((uintptr_t)src & 15) == 0, 104, status))
      xa[c] = ld16_hint<T>(src, pol);
  }
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
    for (int c = 0; c < SCH; ++c) {
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

// Thread 0: starts the load of tile `lt` into stage `st` (one bulk copy of a full
// tile, completing on the stage's mbarrier), or completes the barrier's phase
// without a copy (ragged tile, or no tile).  One arrival per call either way, so
// a stage's barrier phase counts its uses.
// With two leaves (a zip view), the tile's range of leaf b is prefetched into
// L2 at the same time, so the R phase's loads of b hit L2.
template <typename T, bool REV>
__device__ __forceinline__ void stage_issue(const ScanParams& P, long long lt, char* stage,
                                            unsigned long long* bar, bool two = false) {
  if (lt < P.ntiles) {
    const TileRef r = tile_ref<T, REV>(P, lt);
    if (r.full) {
      mbar_expect_tx(bar, kTileBytes);
      bulk_g2s(stage, r.pc->a + r.base * (int64_t)sizeof(T), kTileBytes, bar);
      if (two) bulk_prefetch_l2(r.pc->b + r.base * (int64_t)sizeof(T), kTileBytes);
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
template <typename T, int OP, int KIND, bool REV, bool EXCL>
__global__ void __launch_bounds__(ST, KIND == 3 ? 2 : kMinBlocks) k_scan(const __grid_constant__ ScanParams P) {
  constexpr int V = 16 / sizeof(T);
  using O = Op<OP>;
  extern __shared__ __align__(128) char s_stage[];  // kStages x kTileBytes
  __shared__ __align__(8) unsigned long long s_bar[kStages];
  __shared__ T s_totR[SQ], s_totS[SQ], s_off[SQ];
  __shared__ long long s_tk[kStages + 1];
  __shared__ T s_agg;

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
    for (int d = 0; d < kStages; ++d) mbar_init(&s_bar[d], 1);
    fence_mbar_init();
    for (int d = 0; d < kStages; ++d) {
      s_tk[d] = (long long)atomicAdd(&hdr->ticket, 1ull);
      stage_issue<T, REV>(P, s_tk[d], s_stage + d * kTileBytes, &s_bar[d], two);
    }
  }
  __syncthreads();
  long long tk[kStages];  // tickets of the staged tiles, oldest first
#pragma unroll
  for (int d = 0; d < kStages; ++d) tk[d] = s_tk[d];
  unsigned parity = 0;    // bit d: phase parity of stage d's next completion
  long long tprev = -1;
  T aggprev = ident;  // warp 0: aggregate of tprev
  int sidx = 0;       // stage of tk[0]

  while (tk[0] < P.ntiles || tprev >= 0) {
    const long long t = tk[0];
    const bool haveR = t < P.ntiles, haveS = tprev >= 0;

    // ---- R phase: aggregate of tile t (from its stage; ragged tiles load directly)
    bool copy_lost = false;  // this thread's wait for the stage's bulk copy expired
    if (haveR) {
      const TileRef rr = tile_ref<T, REV>(P, t);
      T x[SCH][V], wx[SCH];
      if (rr.full) {
        copy_lost = !mbar_wait(&s_bar[sidx], (parity >> sidx) & 1u, kCopyWaitPolls, P.status);
        const char* st = s_stage + sidx * kTileBytes;
#pragma unroll
        for (int c = 0; c < SCH; ++c) {
          V16<T> va;
          const char* sp = st + (c * ST + tid) * 16;
          if (chk(sidx >= 0 && sidx < kStages && ((uintptr_t)sp & 15) == 0, 103, P.status))
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
        V16<T> na[SCH], nb[SCH];
        tile_values<T, KIND>(rr, two, tid, ve, ident, na, nb, x);
      }
      local_scan<T, OP, REV>(x, wx, s_totR, lane, warp, ident);
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
        for (int d = 0; d < kStages; ++d) mbar_wait(&s_bar[d], (parity >> d) & 1u, kCopyWaitPolls, P.status);
      __syncthreads();
      break;
    }

    T prefix = (haveS && tprev == 0) ? chain0 : ident;
    if (warp == 0) {
      if (haveR) {
        T loc[SR], exc;
        const T agg = block_totals<T, OP>(s_totR, lane, loc, exc);
        if (lane == 0 && t != P.skip_tile)
          slots.publish(t, tag, t == 0 ? kStateP : kStateA, t == 0 ? O::apply(chain0, agg) : agg);
        if (lane == 0) s_agg = agg;
      }
      // ---- S phase carry: lookback for tprev
      if (haveS && tprev > 0) {
        prefix = lookback<T, O, kLookbackG>(slots, tprev - 1, 0, tag, lane, P.spin_limit, P.status);
        if (lane == 0 && tprev != P.skip_tile) slots.publish(tprev, tag, kStateP, O::apply(prefix, aggprev));
      }
    }

    // ---- S phase: re-read tile tprev (L2), scan it with its carry and store it
    if (haveS) {
      const TileRef rs = tile_ref<T, REV>(P, tprev);
      V16<T> sa[SCH], sb[SCH];
      if (rs.full) load_full<T>(rs, two, tid, drop, sa, sb, P.status);
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
    if (tid == 0) s_tk[kStages] = tnew;
    __syncthreads();  // s_tk, s_agg published; shared totals free
    // refill the stage read in this R phase with the next ticketed tile (all reads
    // of it happened before the barriers above)
    const long long tn = tlast < P.ntiles ? s_tk[kStages] : P.ntiles;
    if (tid == 0) {
      fence_proxy_async_smem();
      stage_issue<T, REV>(P, tn, s_stage + sidx * kTileBytes, &s_bar[sidx], two);
    }
    parity ^= 1u << sidx;
    if (warp == 0) aggprev = s_agg;
    tprev = haveR ? t : -1;
#pragma unroll
    for (int d = 0; d < kStages - 1; ++d) tk[d] = tk[d + 1];
    tk[kStages - 1] = tn;
    sidx = (sidx + 1) % kStages;
    __syncthreads();
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

template <typename T, int OP, int KIND, bool REV, bool EXCL>
cudaError_t go(const ScanParams& p, int grid, cudaStream_t s) {
  static OccCache occ;
  const int per_sm = resident_ctas(occ, k_scan<T, OP, KIND, REV, EXCL>, ST, smem_bytes());
  if (per_sm <= 0) return cudaErrorInvalidConfiguration;
  if (grid <= 0) grid = current_sm_count() * per_sm;
  if (p.ntiles < grid) grid = (int)(p.ntiles > 0 ? p.ntiles : 1);
  k_scan<T, OP, KIND, REV, EXCL><<<grid, ST, smem_bytes(), s>>>(p);
  return cudaGetLastError();
}

template <typename T, int OP>
cudaError_t dispatch_op(const ScanParams& p, int grid, cudaStream_t s) {
  // KIND 0 (a plain vector) for every operator; the interpreted view otherwise
  const bool zip = p.vc.nleaf == 2;
  if (p.exclusive) {
    if (p.vc.kind == 0) return go<T, OP, 0, false, true>(p, grid, s);
    return zip ? go<T, OP, 3, false, true>(p, grid, s) : go<T, OP, 2, false, true>(p, grid, s);
  }
  if (p.vc.kind == 0) return go<T, OP, 0, false, false>(p, grid, s);
  return zip ? go<T, OP, 3, false, false>(p, grid, s) : go<T, OP, 2, false, false>(p, grid, s);
}

template <typename T>
cudaError_t dispatch(const ScanParams& p, bool reverse, int grid, cudaStream_t s) {
  if (reverse) {
    if (p.vc.kind == 0) return go<T, DR_PLUS, 0, true, false>(p, grid, s);
    return p.vc.nleaf == 2 ? go<T, DR_PLUS, 3, true, false>(p, grid, s) : go<T, DR_PLUS, 2, true, false>(p, grid, s);
  }
  switch (p.op) {
    case DR_PLUS: return dispatch_op<T, DR_PLUS>(p, grid, s);
    case DR_MIN: return dispatch_op<T, DR_MIN>(p, grid, s);
    default: return dispatch_op<T, DR_MAX>(p, grid, s);
  }
}

}  // namespace kscan
}  // namespace dr
