// Batched execution: for many independent segmented fp32 vectors, y_v =
// inclusive_scan(x_v) and dots[v] = <x_v, p_v>, all in ONE persistent launch.
//
// The single-range kernels need one launch per vector per algorithm; with
// thousands of short vectors that is launch-bound (cf. the launch fan-out cost
// of a single-process runtime, Sec. 5 "Reduce").  Here every vector is cut into
// tiles (per segment, as in the single-range kernels) and all tiles form one
// global order, vector after vector, each described by one flat descriptor
// (pointers at the tile, its length, the vector's first tile and tile count).
// Persistent CTAs take tiles from an atomic ticket; each tile reads x and p once
// (128-bit), writes y once: 12 B / element for both algorithms together.
//  * scan carry: decoupled lookback over the tile's predecessors *within its
//    vector* (the vector's first tile publishes its inclusive prefix directly);
//  * dot: each tile writes its partial; the vector's last tile to finish
//    (per-vector counter) combines the partials in tile order: deterministic.
// Launch shape (kernel variant, threads per CTA, elements per thread, CTAs
// per SM) is a template / launch parameter chosen by the autotuner.
#include "dr_batch.h"
#include "dr_device.cuh"

namespace dr {
namespace {

__device__ __forceinline__ float fadd(float a, float b) { return a + b; }

// One tile descriptor: three independent 16-byte loads.
__device__ __forceinline__ BDesc load_desc(const BDesc* d) {
  const uint4* s = reinterpret_cast<const uint4*>(d);
  const uint4 a = __ldg(s), b = __ldg(s + 1), c = __ldg(s + 2);
  BDesc r;
  memcpy(reinterpret_cast<char*>(&r), &a, 16);
  memcpy(reinterpret_cast<char*>(&r) + 16, &b, 16);
  memcpy(reinterpret_cast<char*>(&r) + 32, &c, 16);
  return r;
}

// Workspace layout: header | per-vector counters | lookback slots | per-tile dot
// partials (counters first: their offset does not depend on the tile count).
struct BatchWs {
  WsHeader* hdr;
  unsigned* vcount;
  Slots<float> slots;
  float* dotpart;
  __device__ BatchWs(const BatchParams& P) {
    hdr = reinterpret_cast<WsHeader*>(P.ws);
    vcount = reinterpret_cast<unsigned*>(P.ws + sizeof(WsHeader));
    char* slot_base = P.ws + sizeof(WsHeader) + ((size_t)P.nvec * 4 + 15) / 16 * 16;
    slots.bind(slot_base, P.ntiles);
    dotpart = reinterpret_cast<float*>(slot_base + Slots<float>::bytes(P.ntiles));
  }
};

// The vector's last tile to finish folds the dot partials in tile order (one
// warp); `last` must be uniform across the warp.
__device__ __forceinline__ void fold_dot(const BatchParams& P, const BatchWs& W, int vec, int64_t first,
                                         int ntiles, int lane) {
  __threadfence();
  float acc = 0.f;
  for (int64_t i = first + lane; i < first + ntiles; i += 32)
    acc += __int_as_float((int)ld_relaxed_u32(reinterpret_cast<const unsigned*>(W.dotpart + i)));
  acc = warp_reduce<float, DR_PLUS>(acc);
  if (lane == 0) {
    P.dots[vec] = acc;
    W.vcount[vec] = 0;
  }
}

__device__ __forceinline__ void finish_launch(const BatchWs& W) {
  __threadfence();
  if (atomicAdd(&W.hdr->done, 1u) == gridDim.x - 1) {
    W.hdr->ticket = 0;
    W.hdr->done = 0;
    W.hdr->epoch = W.hdr->epoch + 1;
    __threadfence();
  }
}

// ---------------------------------------------------------------------------
// Variant 0: one tile per CTA and iteration, held in registers.
// ---------------------------------------------------------------------------
template <int THREADS, int CH>
__global__ void __launch_bounds__(THREADS) k_batch(const __grid_constant__ BatchParams P) {
  constexpr int NW = THREADS / 32;
  constexpr int Q = CH * NW;             // warp-chunk totals per tile
  constexpr int R = (Q + 31) / 32;       // entries per lane in warp 0
  using O = Op<DR_PLUS>;
  __shared__ float s_tot[R * 32];
  __shared__ float s_off[R * 32];
  __shared__ float s_dot[NW];
  __shared__ long long s_ticket;
  __shared__ int s_last;

  BatchWs W(P);
  const unsigned tag = (ld_relaxed_u32(&W.hdr->epoch) & 0x3fffffffu) << 2;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

  while (true) {
    if (tid == 0) s_ticket = (long long)atomicAdd(&W.hdr->ticket, 1ull);
    __syncthreads();
    const int64_t t = s_ticket;
    if (t >= P.ntiles) break;
    const BDesc d = load_desc(P.desc + t);

    float x[CH][4], pr[CH][4];
    if (d.full) {
#pragma unroll
      for (int c = 0; c < CH; ++c) {
        const int e0 = (c * THREADS + tid) * 4;
        V16<float> a, b;
        if (chk_vec(e0, 4, d.len, d.x + e0, 600, P.status) && chk_vec(e0, 4, d.len, d.p + e0, 601, P.status)) {
          a = ld16<float>(d.x + e0);
          b = ld16<float>(d.p + e0);
        }
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          x[c][e] = a.v[e];
          pr[c][e] = b.v[e];
        }
      }
    } else {
#pragma unroll
      for (int c = 0; c < CH; ++c)
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int i = (c * THREADS + tid) * 4 + e;
          const bool in = i < d.len;
          x[c][e] = in ? __ldg(d.x + i) : 0.f;
          pr[c][e] = in ? __ldg(d.p + i) : 0.f;
        }
    }

    // dot partial of the tile (fixed order)
    float d0 = 0.f, d1 = 0.f, d2 = 0.f, d3 = 0.f;
#pragma unroll
    for (int c = 0; c < CH; ++c) {
      d0 = __fmaf_rn(x[c][0], pr[c][0], d0);
      d1 = __fmaf_rn(x[c][1], pr[c][1], d1);
      d2 = __fmaf_rn(x[c][2], pr[c][2], d2);
      d3 = __fmaf_rn(x[c][3], pr[c][3], d3);
    }
    float dsum = warp_reduce<float, DR_PLUS>((d0 + d1) + (d2 + d3));
    if (lane == 0) s_dot[warp] = dsum;

    // thread-local and warp scans of x
    float tsum[CH], wexc[CH];
#pragma unroll
    for (int c = 0; c < CH; ++c) {
      x[c][1] = fadd(x[c][0], x[c][1]);
      x[c][2] = fadd(x[c][1], x[c][2]);
      x[c][3] = fadd(x[c][2], x[c][3]);
      tsum[c] = x[c][3];
    }
#pragma unroll
    for (int c = 0; c < CH; ++c) {
      const float wi = warp_inclusive<float, DR_PLUS, false>(tsum[c], lane);
      float we = __shfl_up_sync(0xffffffffu, wi, 1);
      if (lane == 0) we = 0.f;
      wexc[c] = we;
      const float wt = __shfl_sync(0xffffffffu, wi, 31);
      if (lane == 0) s_tot[c * NW + warp] = wt;
    }
    __syncthreads();

    if (warp == 0) {
      // the tile's dot partial
      if (lane == 0) {
        float dt = 0.f;
#pragma unroll
        for (int w = 0; w < NW; ++w) dt += s_dot[w];
        W.dotpart[t] = dt;
      }
      // block-level scan of the Q warp-chunk totals: R consecutive entries per lane
      float loc[R];
      float lsum = 0.f;
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int q = lane * R + r;
        loc[r] = q < Q ? s_tot[q] : 0.f;
        lsum = r == 0 ? loc[0] : fadd(lsum, loc[r]);
      }
      const float inc = warp_inclusive<float, DR_PLUS, false>(lsum, lane);
      const float agg = __shfl_sync(0xffffffffu, inc, 31);
      float exc = __shfl_up_sync(0xffffffffu, inc, 1);
      if (lane == 0) exc = 0.f;

      float prefix = 0.f;
      if (t == d.first_tile) {
        if (lane == 0) W.slots.publish(t, tag, kStateP, agg);
      } else {
        if (lane == 0) W.slots.publish(t, tag, kStateA, agg);
        const float run = lookback<float, O, 4>(W.slots, t - 1, d.first_tile, tag, lane, P.spin_limit, P.status);
        prefix = run;
        if (lane == 0) W.slots.publish(t, tag, kStateP, prefix + agg);
      }
      float o = fadd(prefix, exc);
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int q = lane * R + r;
        if (q < Q) s_off[q] = o;
        o = fadd(o, loc[r]);
      }
    }
    __syncthreads();

#pragma unroll
    for (int c = 0; c < CH; ++c) {
      const float pre = fadd(s_off[c * NW + warp], wexc[c]);
      float y[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) y[e] = fadd(pre, x[c][e]);
      const int off = (c * THREADS + tid) * 4;
      if (d.full) {
        V16<float> q;
#pragma unroll
        for (int e = 0; e < 4; ++e) q.v[e] = y[e];
        if (chk_vec(off, 4, d.len, d.y + off, 602, P.status)) st16<float>(d.y + off, q);
      } else {
#pragma unroll
        for (int e = 0; e < 4; ++e)
          if (off + e < d.len) d.y[off + e] = y[e];
      }
    }

    // the vector's last tile to finish combines the dot partials in tile order
    if (tid == 0) {
      __threadfence();
      s_last = atomicAdd(W.vcount + d.vec, 1u) == (unsigned)d.ntiles - 1;
    }
    __syncthreads();
    if (s_last && warp == 0) fold_dot(P, W, d.vec, d.first_tile, d.ntiles, lane);
    __syncthreads();
  }
  if (tid == 0) finish_launch(W);
}

// ---------------------------------------------------------------------------
// Variant 1: the lookahead pipeline of the single-range scan, per vector.
// Iteration k of a persistent CTA:
//   R phase, tile t_k: x and p arrive in a shared-memory stage by two TMA bulk
//     copies issued two iterations earlier (full tiles; ragged ones load
//     directly), with the tile's descriptor beside them; the dot partial and the
//     sum of x (a reduction: the aggregate needs no scan) run, and the tile
//     aggregate is published (the vector's first tile publishes its inclusive
//     prefix).
//   S phase, tile t_{k-1}: warp 0 looks back within the vector, publishes the
//     inclusive prefix, and the CTA re-reads x (an L2 hit), scans it with the
//     carry and stores y.
// Roles off warp 0's path (the lookback): warp 1 lane 0 takes tickets, loads
// their descriptors and issues the bulk copies; warp 2 writes the dot partial
// and, for the vector's last tile to finish, folds the vector's dot.
// 12 B / element: x and p read once from HBM, y written once.
// ---------------------------------------------------------------------------
constexpr int LT = 256;  // threads per CTA
constexpr int LNW = LT / 32;
constexpr int kProducer = 32;  // warp 1, lane 0
constexpr int kDotWarp = 2;

template <int CH>
struct LaGeom {
  static constexpr int TILE = LT * CH * 4;       // elements per tile
  static constexpr int XB = TILE * 4;            // bytes of x (and of p) per tile
  static constexpr int STAGE = 2 * XB;           // x then p
  static constexpr int SMEM = 2 * STAGE;         // two stages
  static constexpr int SQ = CH * LNW;
  static constexpr int SR = (SQ + 31) / 32;
};

struct LaTile {  // what the S phase needs of the previous tile
  const float* x;
  float* y;
  int64_t first;
  int len;
  bool full;
};

// Producer: loads tile t's descriptor into the stage's slot and starts the bulk
// copies of x and p (full tiles), or completes the stage's barrier phase without
// a copy.  One arrival per call either way, so the phase counts the stage's uses.
template <int CH>
__device__ __forceinline__ void la_fill(const BatchParams& P, long long t, char* stage, unsigned long long* bar,
                                        BDesc* slot) {
  using G = LaGeom<CH>;
  if (t < P.ntiles) {
    const BDesc d = load_desc(P.desc + t);
    *slot = d;
    if (d.full && chk(d.len == G::TILE && ((uintptr_t)d.x & 15) == 0 && ((uintptr_t)d.p & 15) == 0, 605,
                      P.status)) {
      mbar_expect_tx(bar, G::STAGE);
      bulk_g2s(stage, d.x, G::XB, bar);
      bulk_g2s(stage + G::XB, d.p, G::XB, bar);
      return;
    }
  }
  mbar_arrive(bar);
}

template <int CH>
__device__ __forceinline__ void la_local_scan(float (&x)[CH][4], float (&wexc)[CH], float* s_tot, int lane,
                                              int warp) {
  float tsum[CH];
#pragma unroll
  for (int c = 0; c < CH; ++c) {
    x[c][1] = fadd(x[c][0], x[c][1]);
    x[c][2] = fadd(x[c][1], x[c][2]);
    x[c][3] = fadd(x[c][2], x[c][3]);
    tsum[c] = x[c][3];
  }
#pragma unroll
  for (int c = 0; c < CH; ++c) {
    const float wi = warp_inclusive<float, DR_PLUS, false>(tsum[c], lane);
    float we = __shfl_up_sync(0xffffffffu, wi, 1);
    if (lane == 0) we = 0.f;
    wexc[c] = we;
    if (lane == 31) s_tot[c * LNW + warp] = wi;  // the lane holding the warp's total
  }
}

// The R phase needs only the tile's aggregate: a tree over the thread's values,
// then over the warp; one total per warp.
template <int CH>
__device__ __forceinline__ void la_reduce(const float (&x)[CH][4], float* s_tot, int lane, int warp) {
  float c[CH];
#pragma unroll
  for (int q = 0; q < CH; ++q) c[q] = fadd(fadd(x[q][0], x[q][1]), fadd(x[q][2], x[q][3]));
  if constexpr ((CH & (CH - 1)) == 0) {
#pragma unroll
    for (int w = CH / 2; w >= 1; w >>= 1)
#pragma unroll
      for (int q = 0; q < w; ++q) c[q] = fadd(c[q], c[q + w]);
  } else {  // pairwise over any count
#pragma unroll
    for (int w = 1; w < CH; w <<= 1)
#pragma unroll
      for (int q = 0; q + w < CH; q += 2 * w) c[q] = fadd(c[q], c[q + w]);
  }
  const float s = warp_reduce<float, DR_PLUS>(c[0]);
  if (lane == 0) s_tot[warp] = s;
}

template <int CH>
__device__ __forceinline__ float la_block_totals(const float* s_tot, int lane, float (&loc)[LaGeom<CH>::SR],
                                                 float& exc) {
  using G = LaGeom<CH>;
  float lsum = 0.f;
#pragma unroll
  for (int r = 0; r < G::SR; ++r) {
    const int q = lane * G::SR + r;
    loc[r] = q < G::SQ ? s_tot[q] : 0.f;
    lsum = r == 0 ? loc[0] : fadd(lsum, loc[r]);
  }
  const float inc = warp_inclusive<float, DR_PLUS, false>(lsum, lane);
  exc = __shfl_up_sync(0xffffffffu, inc, 1);
  if (lane == 0) exc = 0.f;
  return __shfl_sync(0xffffffffu, inc, 31);
}

template <int CH, int MINB>
__global__ void __launch_bounds__(LT, MINB) k_batch_la(const __grid_constant__ BatchParams P) {
  using G = LaGeom<CH>;
  using O = Op<DR_PLUS>;
  extern __shared__ __align__(128) char s_stage[];  // 2 stages x (x tile | p tile)
  __shared__ __align__(8) unsigned long long s_bar[2];
  __shared__ __align__(16) BDesc s_desc[2];         // descriptor of the tile in stage d
  __shared__ float s_totR[G::SR * 32], s_totS[G::SR * 32], s_off[G::SR * 32], s_dot[LNW];
  __shared__ long long s_tk[4];  // [0], [1]: first tickets; [2 + stage]: the ticket an iteration takes
  __shared__ float s_agg;

  BatchWs W(P);
  const unsigned tag = (ld_relaxed_u32(&W.hdr->epoch) & 0x3fffffffu) << 2;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const unsigned long long drop = l2_policy_evict_first();

  if (tid == 0) {
    mbar_init(&s_bar[0], 1);
    mbar_init(&s_bar[1], 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (tid == kProducer) {
    for (int d = 0; d < 2; ++d) {
      s_tk[d] = (long long)atomicAdd(&W.hdr->ticket, 1ull);
      la_fill<CH>(P, s_tk[d], s_stage + d * G::STAGE, &s_bar[d], &s_desc[d]);
    }
  }
  __syncthreads();
  long long tk0 = s_tk[0], tk1 = s_tk[1], tprev = -1;
  unsigned parity = 0;
  int sidx = 0;
  float aggprev = 0.f;  // warp 0
  LaTile prev{nullptr, nullptr, 0, 0, false};

  while (tk0 < P.ntiles || tprev >= 0) {
    const long long t = tk0;
    const bool haveR = t < P.ntiles, haveS = tprev >= 0;
    // the producer takes the next ticket now (used after barrier A)
    long long tnew = P.ntiles;
    if (tid == kProducer && tk1 < P.ntiles) tnew = (long long)atomicAdd(&W.hdr->ticket, 1ull);
    LaTile cur{nullptr, nullptr, 0, 0, false};
    int vec = 0, vtiles = 0;

    // ---- R phase: dot partial and scan aggregate of tile t
    bool copy_lost = false;  // this thread's wait for the stage's bulk copies expired
    if (haveR) {
      const BDesc d = s_desc[sidx];
      vec = d.vec;
      vtiles = d.ntiles;
      cur = LaTile{d.x, d.y, d.first_tile, d.len, d.full != 0};
      float x[CH][4], pr[CH][4];
      if (cur.full) {
        copy_lost = !mbar_wait(&s_bar[sidx], (parity >> sidx) & 1u, kCopyWaitPolls, P.status);
        const char* st = s_stage + sidx * G::STAGE;
#pragma unroll
        for (int c = 0; c < CH; ++c) {
          const V16<float> a = *reinterpret_cast<const V16<float>*>(st + (c * LT + tid) * 16);
          const V16<float> b = *reinterpret_cast<const V16<float>*>(st + G::XB + (c * LT + tid) * 16);
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            x[c][e] = a.v[e];
            pr[c][e] = b.v[e];
          }
        }
      } else {
#pragma unroll
        for (int c = 0; c < CH; ++c)
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const int i = (c * LT + tid) * 4 + e;
            const bool in = i < d.len;
            x[c][e] = in ? __ldg(d.x + i) : 0.f;
            pr[c][e] = in ? __ldg(d.p + i) : 0.f;
          }
      }
      float d0 = 0.f, d1 = 0.f, d2 = 0.f, d3 = 0.f;
#pragma unroll
      for (int c = 0; c < CH; ++c) {
        d0 = __fmaf_rn(x[c][0], pr[c][0], d0);
        d1 = __fmaf_rn(x[c][1], pr[c][1], d1);
        d2 = __fmaf_rn(x[c][2], pr[c][2], d2);
        d3 = __fmaf_rn(x[c][3], pr[c][3], d3);
      }
      const float dsum = warp_reduce<float, DR_PLUS>((d0 + d1) + (d2 + d3));
      if (lane == 0) s_dot[warp] = dsum;
      la_reduce<CH>(x, s_totR, lane, warp);
    }
    if (__syncthreads_or(copy_lost)) {  // ---- barrier A: s_totR, s_dot; the R stage is read
      // A bulk copy did not complete within its bound (DR_E_TIMEOUT is recorded):
      // no stage is read or re-armed any more; wait, again bounded, for copies
      // that may still be in flight into either stage, then leave.
      if (tid == 0)
        for (int d = 0; d < 2; ++d) mbar_wait(&s_bar[d], (parity >> d) & 1u, kCopyWaitPolls, P.status);
      __syncthreads();
      break;
    }
#ifndef DR_BATCH_LATE_REFILL
#define DR_BATCH_LATE_REFILL 0
#endif
    if (!DR_BATCH_LATE_REFILL && tid == kProducer) {
      // every read of the stage consumed in this R phase happened before barrier A
      s_tk[2 + sidx] = tnew;
      fence_proxy_async_smem();
      la_fill<CH>(P, tnew, s_stage + sidx * G::STAGE, &s_bar[sidx], &s_desc[sidx]);
    }

    float prefix = 0.f;
    if (warp == 0) {
      if (haveR) {
        const float agg = warp_reduce<float, DR_PLUS>(lane < LNW ? s_totR[lane] : 0.f);
        if (lane == 0) {
          W.slots.publish(t, tag, t == cur.first ? kStateP : kStateA, agg);
          s_agg = agg;
        }
      }
      if (haveS && tprev != prev.first) {
        prefix = lookback<float, O, 1>(W.slots, tprev - 1, prev.first, tag, lane, P.spin_limit, P.status);
        if (lane == 0) W.slots.publish(tprev, tag, kStateP, prefix + aggprev);
      }
    } else if (warp == kDotWarp && haveR) {
      int last = 0;
      if (lane == 0) {
        float dt = 0.f;
#pragma unroll
        for (int w = 0; w < LNW; ++w) dt += s_dot[w];
        W.dotpart[t] = dt;
        __threadfence();
        last = atomicAdd(W.vcount + vec, 1u) == (unsigned)vtiles - 1;
      }
      if (__shfl_sync(0xffffffffu, last, 0)) fold_dot(P, W, vec, cur.first, vtiles, lane);
    }

    // ---- S phase: y of tile tprev
    if (haveS) {
      float x[CH][4], wexc[CH];
      if (prev.full) {
#pragma unroll
        for (int c = 0; c < CH; ++c) {
          const int e0 = (c * LT + tid) * 4;
          V16<float> a;
          if (chk_vec(e0, 4, prev.len, prev.x + e0, 604, P.status)) a = ld16_hint<float>(prev.x + e0, drop);
#pragma unroll
          for (int e = 0; e < 4; ++e) x[c][e] = a.v[e];
        }
      } else {
#pragma unroll
        for (int c = 0; c < CH; ++c)
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const int i = (c * LT + tid) * 4 + e;
            x[c][e] = i < prev.len ? __ldg(prev.x + i) : 0.f;
          }
      }
      la_local_scan<CH>(x, wexc, s_totS, lane, warp);
      __syncthreads();  // ---- barrier B: s_totS
      if (warp == 0) {
        float loc[G::SR], exc;
        la_block_totals<CH>(s_totS, lane, loc, exc);
        float o = fadd(prefix, exc);
#pragma unroll
        for (int r = 0; r < G::SR; ++r) {
          const int q = lane * G::SR + r;
          if (q < G::SQ) s_off[q] = o;
          o = fadd(o, loc[r]);
        }
      }
      __syncthreads();  // ---- barrier C: s_off
#pragma unroll
      for (int c = 0; c < CH; ++c) {
        const float pre = fadd(s_off[c * LNW + warp], wexc[c]);
        const int off = (c * LT + tid) * 4;
        if (prev.full) {
          V16<float> q;
#pragma unroll
          for (int e = 0; e < 4; ++e) q.v[e] = fadd(pre, x[c][e]);
          if (chk_vec(off, 4, prev.len, prev.y + off, 603, P.status)) st16_hint<float>(prev.y + off, q, drop);
        } else {
#pragma unroll
          for (int e = 0; e < 4; ++e)
            if (off + e < prev.len) prev.y[off + e] = fadd(pre, x[c][e]);
        }
      }
    } else {
      __syncthreads();  // the reads of s_totR and s_dot end before the next R phase rewrites them
    }
    if (DR_BATCH_LATE_REFILL) {
      if (tid == kProducer) {
        s_tk[2 + sidx] = tnew;
        fence_proxy_async_smem();
        la_fill<CH>(P, tnew, s_stage + sidx * G::STAGE, &s_bar[sidx], &s_desc[sidx]);
      }
      __syncthreads();
    }
    parity ^= 1u << sidx;
    if (warp == 0) aggprev = haveR ? s_agg : 0.f;
    prev = cur;
    tprev = haveR ? t : -1;
    tk0 = tk1;
    tk1 = s_tk[2 + sidx];  // written by the producer before barrier B (or the plain barrier)
    sidx ^= 1;
  }
  if (tid == 0) finish_launch(W);
}

template <int CH, int MINB>
cudaError_t go_la(const BatchParams& p, int ctas_per_sm, int sms, cudaStream_t s) {
  using G = LaGeom<CH>;
  static OccCache occ;
  const int per = resident_ctas(occ, k_batch_la<CH, MINB>, LT, G::SMEM);
  if (per <= 0) return cudaErrorInvalidConfiguration;
  const int k = ctas_per_sm < per ? ctas_per_sm : per;
  int64_t grid = (int64_t)sms * (k > 0 ? k : 1);
  if (grid > p.ntiles) grid = p.ntiles > 0 ? p.ntiles : 1;
  k_batch_la<CH, MINB><<<(unsigned)grid, LT, G::SMEM, s>>>(p);
  return cudaGetLastError();
}

template <int THREADS, int CH>
cudaError_t go(const BatchParams& p, int ctas_per_sm, int sms, cudaStream_t s) {
  static OccCache occ;
  const int per = resident_ctas(occ, k_batch<THREADS, CH>, THREADS, 0);
  if (per <= 0) return cudaErrorInvalidConfiguration;
  const int k = ctas_per_sm < per ? ctas_per_sm : per;
  int64_t grid = (int64_t)sms * (k > 0 ? k : 1);
  if (grid > p.ntiles) grid = p.ntiles > 0 ? p.ntiles : 1;
  k_batch<THREADS, CH><<<(unsigned)grid, THREADS, 0, s>>>(p);
  return cudaGetLastError();
}

}  // namespace

bool batch_shape_supported(int variant, int threads, int items) {
  if (variant == 1) return threads == LT && (items == 12 || items == 16 || items == 32);
  return variant == 0 && (threads == 128 || threads == 256 || threads == 512) && (items == 8 || items == 16);
}

size_t batch_ws_bytes(int64_t ntiles, int nvec) {
  return sizeof(WsHeader) + ((size_t)nvec * 4 + 15) / 16 * 16 + Slots<float>::bytes(ntiles) +
         (size_t)ntiles * 4;
}

cudaError_t launch_batch(const BatchParams& p, const dr_tune& t, int sms, cudaStream_t s) {
  if (p.ntiles <= 0) return cudaSuccess;
  const int ch = t.items / 4;
  if (t.variant == 1) {
    if (ch == 3) return go_la<3, 4>(p, t.ctas_per_sm, sms, s);
    if (ch == 4) return go_la<4, 3>(p, t.ctas_per_sm, sms, s);
    if (ch == 8) return go_la<8, 1>(p, t.ctas_per_sm, sms, s);
    return cudaErrorInvalidValue;
  }
  if (t.threads == 128 && ch == 2) return go<128, 2>(p, t.ctas_per_sm, sms, s);
  if (t.threads == 128 && ch == 4) return go<128, 4>(p, t.ctas_per_sm, sms, s);
  if (t.threads == 256 && ch == 2) return go<256, 2>(p, t.ctas_per_sm, sms, s);
  if (t.threads == 256 && ch == 4) return go<256, 4>(p, t.ctas_per_sm, sms, s);
  if (t.threads == 512 && ch == 2) return go<512, 2>(p, t.ctas_per_sm, sms, s);
  if (t.threads == 512 && ch == 4) return go<512, 4>(p, t.ctas_per_sm, sms, s);
  return cudaErrorInvalidValue;
}

}  // namespace dr
