// reduce / transform_reduce over a fused view (Sec. 4.3, Algorithm 3; the dot
// product of Algorithm 1 is the zip-multiply instance).
//
// Algorithm 3 reduces every segment locally, then combines the per-segment
// partials.  On one GPU the segments become pieces of one global tile list, so
// one launch covers all of them: CTAs stride over tiles (128-bit loads of up to
// two operands, the view applied in registers, V independent accumulators per
// thread), reduce with warp shuffles, write one partial per CTA, and the last
// CTA to finish combines the partials in a fixed tree order.  The reduction
// tree depends only on the grid size, so results are run-to-run reproducible.
#include <type_traits>

#pragma once
#include "dr_device.cuh"

namespace dr {
namespace kreduce {

constexpr int RT = 256;  // threads per CTA
constexpr int RCH = 4;   // 16-byte chunks per operand per thread per tile
constexpr int RCTAS = 4; // resident CTAs per SM (fixed: the grid fixes the reduction tree)

template <typename T>
__host__ __device__ constexpr int rtile() {
  return RT * RCH * (16 / (int)sizeof(T));
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

template <typename T>
__device__ __forceinline__ T mul_add(T a, T b, T acc) {
  if constexpr (std::is_same<T, float>::value) return __fmaf_rn(a, b, acc);
  else if constexpr (std::is_same<T, double>::value) return __fma_rn(a, b, acc);
  else return wrap_add(acc, wrap_mul(a, b));
}

template <typename T, int OP>
__device__ __forceinline__ T block_reduce(T v, T* s_w) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  v = warp_reduce<T, OP>(v);
  if (lane == 0) s_w[warp] = v;
  __syncthreads();
  T x = Op<OP>::template identity<T>();
  if (warp == 0) {
    if (lane < RT / 32) x = s_w[lane];
    x = warp_reduce<T, OP>(x);
  }
  __syncthreads();
  return x;  // valid in warp 0
}

// KIND: 0 one leaf, no ops; 1 zip(a, b) | multiply, PLUS only; 2 generic view.
// EXT: the piece table is in device memory (more pieces than the kernel
// parameters hold) -- a compile-time choice, so that every piece access keeps
// its address space (the inline table is read through the constant cache).
template <typename T, int OP, int KIND, bool EXT>
__global__ void __launch_bounds__(RT, RCTAS) k_reduce(const __grid_constant__ ReduceParams P) {
  constexpr int V = 16 / sizeof(T);
  constexpr int TILE = rtile<T>();
  using O = Op<OP>;
  __shared__ T s_w[RT / 32];
  __shared__ int s_last;

  ViewEval<T> ve;
  if constexpr (KIND == 2) ve.init(P.vc);
  const bool two = (KIND == 1) || (KIND == 2 && P.vc.nleaf == 2);
  const int tid = threadIdx.x;

  T acc[V];
#pragma unroll
  for (int e = 0; e < V; ++e) acc[e] = O::template identity<T>();

  for (int64_t tile = blockIdx.x; tile < P.ntiles; tile += gridDim.x) {
    const KPiece* tab;
    if constexpr (EXT) tab = P.pc_ext;
    else tab = P.pc;
    const int k = find_piece(tab, P.npieces, tile);
    const KPiece& pc = tab[k];
    const int64_t base = (tile - pc.tile_begin) * TILE;
    if (!chk(k >= 0 && k < P.npieces && base >= 0 && base < pc.len, 200, P.status)) continue;
    if (pc.vec_ok && pc.len - base >= TILE) {
      V16<T> ra[RCH], rb[RCH];
#pragma unroll
      for (int c = 0; c < RCH; ++c) {
        const int64_t e0 = base + (int64_t)(c * RT + tid) * V;
        const char* pa = pc.a + e0 * (int64_t)sizeof(T);
        if (chk_vec(e0, V, pc.len, pa, 201, P.status)) ra[c] = ld16<T>(pa);
      }
      if (two) {
#pragma unroll
        for (int c = 0; c < RCH; ++c) {
          const int64_t e0 = base + (int64_t)(c * RT + tid) * V;
          const char* pb = pc.b + e0 * (int64_t)sizeof(T);
          if (chk_vec(e0, V, pc.len, pb, 202, P.status)) rb[c] = ld16<T>(pb);
        }
      }
      if constexpr (KIND == 2) {
        T xa[RCH][V], xb[RCH][V];
#pragma unroll
        for (int c = 0; c < RCH; ++c)
#pragma unroll
          for (int e = 0; e < V; ++e) {
            xa[c][e] = ra[c].v[e];
            xb[c][e] = two ? rb[c].v[e] : T(0);
          }
        ve.template eval_all<RCH * V>(&xa[0][0], &xb[0][0]);
#pragma unroll
        for (int c = 0; c < RCH; ++c)
#pragma unroll
          for (int e = 0; e < V; ++e) acc[e] = O::apply(acc[e], xa[c][e]);
      } else {
#pragma unroll
        for (int c = 0; c < RCH; ++c)
#pragma unroll
          for (int e = 0; e < V; ++e) {
            if constexpr (KIND == 0) acc[e] = O::apply(acc[e], ra[c].v[e]);
            else acc[e] = mul_add(ra[c].v[e], rb[c].v[e], acc[e]);
          }
      }
    } else {
#pragma unroll
      for (int c = 0; c < RCH; ++c)
#pragma unroll
        for (int e = 0; e < V; ++e) {
          const int64_t idx = base + (int64_t)(c * RT + tid) * V + e;
          if (idx < pc.len) {
            T a = ld1<T>(pc.a + idx * (int64_t)sizeof(T));
            T b = two ? ld1<T>(pc.b + idx * (int64_t)sizeof(T)) : T(0);
            if constexpr (KIND == 0) acc[e] = O::apply(acc[e], a);
            else if constexpr (KIND == 1) acc[e] = mul_add(a, b, acc[e]);
            else acc[e] = O::apply(acc[e], ve(a, b));
          }
        }
    }
  }

  T v = acc[0];
#pragma unroll
  for (int e = 1; e < V; ++e) v = O::apply(v, acc[e]);
  v = block_reduce<T, OP>(v, s_w);

  WsHeader* hdr = reinterpret_cast<WsHeader*>(P.ws);
  unsigned long long* part = reinterpret_cast<unsigned long long*>(P.ws + sizeof(WsHeader));
  if (tid == 0) {
    if (chk(blockIdx.x < (P.ws_partials ? P.ws_partials : gridDim.x), 203, P.status)) part[blockIdx.x] = to_bits(v);
    __threadfence();
    s_last = atomicAdd(&hdr->done, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  T x = O::template identity<T>();
  for (int i = tid; i < (int)gridDim.x; i += RT) x = O::apply(x, from_bits<T>(ld_relaxed_u64(part + i)));
  x = block_reduce<T, OP>(x, s_w);
  if (tid == 0) {
    *reinterpret_cast<T*>(P.result) = O::apply(from_bits<T>(P.init_bits), x);
    hdr->done = 0;
  }
}

template <typename T, int OP, int KIND>
cudaError_t go(const ReduceParams& p, int grid, cudaStream_t s) {
  if (p.ntiles < grid) grid = (int)(p.ntiles > 0 ? p.ntiles : 1);
  if (p.pc_ext) k_reduce<T, OP, KIND, true><<<grid, RT, 0, s>>>(p);
  else k_reduce<T, OP, KIND, false><<<grid, RT, 0, s>>>(p);
  return cudaGetLastError();
}

template <typename T>
cudaError_t dispatch(const ReduceParams& p, int grid, cudaStream_t s) {
  const int kind = p.vc.kind;
  if (p.op == DR_PLUS && kind == 1) return go<T, DR_PLUS, 1>(p, grid, s);
  switch (p.op) {
    case DR_PLUS: return kind == 0 ? go<T, DR_PLUS, 0>(p, grid, s) : go<T, DR_PLUS, 2>(p, grid, s);
    case DR_MUL: return kind == 0 ? go<T, DR_MUL, 0>(p, grid, s) : go<T, DR_MUL, 2>(p, grid, s);
    case DR_MIN: return kind == 0 ? go<T, DR_MIN, 0>(p, grid, s) : go<T, DR_MIN, 2>(p, grid, s);
    default: return kind == 0 ? go<T, DR_MAX, 0>(p, grid, s) : go<T, DR_MAX, 2>(p, grid, s);
  }
}

}  // namespace kreduce
}  // namespace dr
