// inclusive_scan / exclusive_scan / reverse scan over a fused view, across
// segment boundaries (Sec. 4.3 "inclusive_scan", Algorithm 4).
//
// Algorithm 4 scans every segment locally, gathers the segments' last elements,
// scans them, and makes a second pass that adds each segment's offset: four
// accesses per element (Sec. 5, "Inclusive Scan" blames that second pass for
// the 1 -> 2 tile drop).  Here all segments are pieces of one global tile
// order and the carry crosses segment boundaries inside one pass (decoupled
// lookback): a persistent CTA takes the next tile from an atomic ticket, loads
// it (128-bit, view fused), publishes the tile's aggregate, then warp 0 walks
// back over its predecessors' published aggregates / inclusive prefixes (32 at
// a time) until it meets an inclusive prefix, publishes its own inclusive
// prefix, and the CTA writes the scanned tile: two accesses per element.
//
// Forward progress: tickets are taken in order by CTAs that are already
// running, so every predecessor a CTA waits on is resident.  Every wait is
// bounded (dr_set_spin_limit) and reports DR_E_TIMEOUT instead of hanging.
#pragma once
#include "dr_device.cuh"

namespace dr {
namespace kscan {

constexpr int ST = 256;            // threads per CTA
constexpr int SCH = 4;             // 16-byte chunks per thread per tile
constexpr int SNW = ST / 32;       // warps
constexpr int SQ = SCH * SNW;      // warp-chunk totals per tile (== 32: one per lane of warp 0)
static_assert(SQ == 32, "block-level scan assumes 32 entries");

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

// KIND: 0 = one leaf, no ops (PLUS only); 2 = generic fused view.
// REV: scan from the last element to the first (reverse inclusive scan).
// EXCL: exclusive scan with init.
template <typename T, int OP, int KIND, bool REV, bool EXCL>
__global__ void __launch_bounds__(ST) k_scan(const __grid_constant__ ScanParams P) {
  constexpr int V = 16 / sizeof(T);
  constexpr int TILE = stile<T>();
  using O = Op<OP>;
  __shared__ T s_tot[SQ];
  __shared__ T s_off[SQ];
  __shared__ long long s_ticket;

  WsHeader* hdr = reinterpret_cast<WsHeader*>(P.ws);
  Slots<T> slots;
  slots.bind(P.ws + sizeof(WsHeader), P.ntiles);
  const unsigned tag = (ld_relaxed_u32(&hdr->epoch) & 0x3fffffffu) << 2;

  ViewEval<T> ve;
  if constexpr (KIND == 2) ve.init(P.vc);
  const bool two = KIND == 2 && P.vc.nleaf == 2;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const T ident = O::template identity<T>();

  while (true) {
    if (tid == 0) s_ticket = (long long)atomicAdd(&hdr->ticket, 1ull);
    __syncthreads();
    const int64_t lt = s_ticket;  // logical tile: the order of the carry chain
    if (lt >= P.ntiles) break;
    const int64_t pt = REV ? P.ntiles - 1 - lt : lt;  // physical tile
    const KPiece& pc = P.pc[find_piece(P.pc, P.npieces, pt)];
    const int64_t base = (pt - pc.tile_begin) * TILE;
    const bool full = pc.vec_ok && pc.len - base >= TILE;

    // ---- load (striped: chunk c of thread tid is 16 bytes at (c*ST + tid)*V)
    T x[SCH][V];
    if (full) {
      V16<T> ra[SCH], rb[SCH];
#pragma unroll
      for (int c = 0; c < SCH; ++c)
        ra[c] = ld16<T>(pc.a + (base + (int64_t)(c * ST + tid) * V) * (int64_t)sizeof(T));
      if (two) {
#pragma unroll
        for (int c = 0; c < SCH; ++c)
          rb[c] = ld16<T>(pc.b + (base + (int64_t)(c * ST + tid) * V) * (int64_t)sizeof(T));
      }
#pragma unroll
      for (int c = 0; c < SCH; ++c)
#pragma unroll
        for (int e = 0; e < V; ++e) {
          if constexpr (KIND == 0) x[c][e] = ra[c].v[e];
          else x[c][e] = ve(ra[c].v[e], two ? rb[c].v[e] : T(0));
        }
    } else {
#pragma unroll
      for (int c = 0; c < SCH; ++c)
#pragma unroll
        for (int e = 0; e < V; ++e) {
          const int64_t idx = base + (int64_t)(c * ST + tid) * V + e;
          if (idx < pc.len) {
            T a = ld1<T>(pc.a + idx * (int64_t)sizeof(T));
            if constexpr (KIND == 0) x[c][e] = a;
            else x[c][e] = ve(a, two ? ld1<T>(pc.b + idx * (int64_t)sizeof(T)) : T(0));
          } else {
            x[c][e] = ident;
          }
        }
    }

    // ---- thread-local scan of each chunk (in the scan direction)
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

    // ---- warp scan of the chunk sums; warp totals to shared memory in scan order
    T wexc[SCH];
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
    __syncthreads();

    // ---- warp 0: tile aggregate, lookback, publish
    if (warp == 0) {
      const T v = s_tot[lane];
      const T inc = warp_inclusive<T, OP, false>(v, lane);
      const T agg = __shfl_sync(0xffffffffu, inc, 31);
      T exc = __shfl_up_sync(0xffffffffu, inc, 1);
      if (lane == 0) exc = ident;
      const bool publish = lt != P.skip_tile;
      T prefix = ident;  // combination of all tiles before lt in scan order
      if (lt == 0) {
        if (lane == 0 && publish) slots.publish(0, tag, kStateP, agg);
      } else {
        if (lane == 0 && publish) slots.publish(lt, tag, kStateA, agg);
        int64_t pred = lt - 1;
        T run = ident;
        while (true) {
          const int64_t i = pred - lane;  // lane 0 = nearest predecessor
          T val = ident;
          unsigned st = kStateP;          // before tile 0: identity
          if (i >= 0) st = slots.poll(i, tag, val);
          // only lanes nearer than the nearest inclusive prefix need to wait
          unsigned pm = __ballot_sync(0xffffffffu, st == kStateP);
          const int lim = pm ? __ffs(pm) - 1 : 32;
          if (st == 0 && lane < lim)
            st = wait_slot<T, Slots<T>, O>(slots, i, tag, val, P.spin_limit, P.status);
          __syncwarp();
          pm = __ballot_sync(0xffffffffu, st == kStateP);
          const int first = pm ? __ffs(pm) - 1 : 31;
          const T w = warp_reduce<T, OP>(lane <= first ? val : ident);
          run = O::apply(w, run);
          if (pm) break;
          pred -= 32;
        }
        prefix = run;
        if (lane == 0 && publish) slots.publish(lt, tag, kStateP, O::apply(prefix, agg));
      }
      s_off[lane] = O::apply(prefix, exc);
    }
    __syncthreads();

    // ---- combine and store
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
      const int64_t off = base + (int64_t)(c * ST + tid) * V;
      if (full) {
        V16<T> o;
#pragma unroll
        for (int e = 0; e < V; ++e) o.v[e] = y[e];
        st16<T>(pc.o + off * (int64_t)sizeof(T), o);
      } else {
#pragma unroll
        for (int e = 0; e < V; ++e)
          if (off + e < pc.len) reinterpret_cast<T*>(pc.o)[off + e] = y[e];
      }
    }
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
  if (grid <= 0) {
    if (!per_sm) {
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_scan<T, OP, KIND, REV, EXCL>, ST, 0);
      if (per_sm <= 0) per_sm = 1;
    }
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
