// for_each with a 5-point Jacobi update over a row-block segmented 2-D array
// (Sec. 4.3 "for_each" over the block_row partition of Sec. 4.2.2), with the
// halo exchange fused into the producing step, plus the stand-alone halo
// exchange used before the first step.
//
// Layout: block k is one allocation of (rows_k + 2) x cols fp32, row 0 and row
// rows_k + 1 being ghost copies of the neighbours' boundary rows.  A CTA owns
// 4*TX columns x RB rows of one block and marches down its rows keeping the
// rows above / at / below the current one in registers (each thread 4
// consecutive columns as one float4), so every cell is read from HBM once per
// step (plus 2 halo rows per RB rows) and written once: 8 B / cell / step.
// West / east neighbours come from the adjacent lanes by warp shuffle; lanes 0
// and 31 read the one missing column with a scalar load (an L1/L2 hit: the
// neighbouring warp loads that line).  Rows are fetched G at a time so G
// independent 16-byte loads per thread are in flight.  Measured on GB300
// (16384^2, 8 blocks): G = 4 with 8 resident CTAs per SM (58 registers) moves
// 6.2 TB/s; G = 8 (>100 registers) 5.5 TB/s; 10 CTAs per SM 4.8 TB/s.  The epilogue also
// writes a block's first / last own row into the neighbouring blocks' ghost
// rows of the output, which is the halo exchange for the next step.
//
// Arithmetic (fixed order, no contraction): s = (N + S) + (W + E);
// r = wn * s; and if wc != 0, r = r + wc * C.  Outside the grid is 0.
#include "dr_device.cuh"

namespace dr {
namespace {

constexpr int TX = kStencilThreads;
constexpr int RB = kStencilRowsPerCta;
#ifndef DR_STENCIL_GROUP
#define DR_STENCIL_GROUP 4
#endif
#ifndef DR_STENCIL_MINB
#define DR_STENCIL_MINB 8  // resident CTAs per SM asked of the register allocator (<= 64 registers)
#endif
constexpr int G = DR_STENCIL_GROUP;  // rows fetched per group

__device__ __forceinline__ int find_seg(const StencilParams& P, int64_t rb) {
  int lo = 0, hi = P.nseg - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (P.seg[mid].rb_begin <= rb) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

template <int VW>
struct Row {
  float v[VW];
  float w, e;  // west of v[0] (lane 0 only), east of v[VW-1] (lane 31 only)
};

// Row g (0 .. nrows-1, ghost rows included) of a block allocation of nrows x C.
template <int VW>
__device__ __forceinline__ void load_row(Row<VW>& r, const float* in, int64_t g, int64_t C, int64_t c,
                                         bool zero_row, int lane, int64_t nrows, unsigned* status) {
  const bool load = !zero_row && c < C &&
                    chk(g >= 0 && g < nrows && c + VW <= C && (VW == 1 || ((uintptr_t)(in + g * C + c) & 15) == 0),
                        300, status);
  if (!load) {
#pragma unroll
    for (int e = 0; e < VW; ++e) r.v[e] = 0.f;
  } else if constexpr (VW == 4) {
    V16<float> q = ld16<float>(in + g * C + c);
#pragma unroll
    for (int e = 0; e < 4; ++e) r.v[e] = q.v[e];
  } else {
    r.v[0] = __ldg(in + g * C + c);
  }
  r.w = 0.f;
  r.e = 0.f;
  if (load) {
    if (lane == 0 && c > 0) r.w = __ldg(in + g * C + c - 1);
    if (lane == 31 && c + VW < C) r.e = __ldg(in + g * C + c + VW);
  }
}

template <int VW>
__device__ __forceinline__ float upd(float n, float s, float w, float e, float ctr, float wc, float wn) {
  const float sum = __fadd_rn(__fadd_rn(n, s), __fadd_rn(w, e));
  float r = __fmul_rn(wn, sum);
  if (wc != 0.f) r = __fadd_rn(r, __fmul_rn(wc, ctr));
  return r;
}

// WGRAD: the backward step of the weight gradients.  `in` holds u_bar_t, the
// output is u_bar_{t-1} = A^T u_bar_t (= A u_bar_t), and with the forward state
// u_{t-1} read from `prev` the kernel also accumulates <u_bar_t, u_{t-1}> (the
// wc term) and <N(u_bar_t), u_{t-1}> (the wn term; N = neighbour sum, and
// <u_bar, N u> = <N u_bar, u> because N is symmetric) into acc[0], acc[1].
template <int VW, bool WGRAD>
__global__ void __launch_bounds__(TX, DR_STENCIL_MINB) k_stencil5(const __grid_constant__ StencilParams P) {
  const int64_t rb = P.outer_only ? (blockIdx.y == 0 ? 0 : P.nrb - 1) : P.rb_lo + (int64_t)blockIdx.y;
  const int s = find_seg(P, rb);
  const StencilSeg& S = P.seg[s];
  const int64_t C = P.cols;
  const int64_t r0 = 1 + (rb - S.rb_begin) * RB;                   // first own row (1-based)
  const int64_t r1 = min(r0 + RB, S.rows + 1);                      // one past the last
  const int lane = threadIdx.x & 31;
  const int64_t c = ((int64_t)blockIdx.x * TX + threadIdx.x) * VW;
  const bool act = c < C;
  // zero rows outside the grid, unless the outer ghost rows hold a neighbour's rows
  const bool top = s == 0 && !P.ext_top, bot = s == P.nseg - 1 && !P.ext_bot;
  const float wc = P.wc, wn = P.wn;

  float gwc = 0.f, gwn = 0.f;  // weight-gradient partials (WGRAD)
  Row<VW> up, cur;
  const int64_t nrows = S.rows + 2;
  if (!chk(s >= 0 && s < P.nseg && r0 >= 1 && r0 <= S.rows, 301, P.status)) return;
  load_row<VW>(up, S.in, r0 - 1, C, c, top && r0 - 1 == 0, lane, nrows, P.status);
  load_row<VW>(cur, S.in, r0, C, c, false, lane, nrows, P.status);

  for (int64_t r = r0; r < r1; r += G) {
    Row<VW> nx[G];
#pragma unroll
    for (int k = 0; k < G; ++k) {
      const int64_t g = r + 1 + k;
      if (g <= r1) load_row<VW>(nx[k], S.in, g, C, c, bot && g == S.rows + 1, lane, nrows, P.status);
    }
#pragma unroll
    for (int k = 0; k < G; ++k) {
      const int64_t row = r + k;
      if (row < r1) {
        // west / east neighbours along the row
        float wv = __shfl_up_sync(0xffffffffu, cur.v[VW - 1], 1);
        float ev = __shfl_down_sync(0xffffffffu, cur.v[0], 1);
        if (lane == 0) wv = cur.w;
        if (lane == 31) ev = cur.e;
        float o[VW];
        float pv[VW];
        if constexpr (WGRAD) {
          if (act && chk(row >= 1 && row <= S.rows && c + VW <= C, 302, P.status)) {
            if constexpr (VW == 4) {
              const V16<float> q = ld16<float>(S.prev + row * C + c);
#pragma unroll
              for (int e = 0; e < 4; ++e) pv[e] = q.v[e];
            } else {
              pv[0] = __ldg(S.prev + row * C + c);
            }
          } else {
#pragma unroll
            for (int e = 0; e < VW; ++e) pv[e] = 0.f;
          }
        }
#pragma unroll
        for (int e = 0; e < VW; ++e) {
          const float W = e == 0 ? wv : cur.v[e - 1];
          const float E = e == VW - 1 ? ev : cur.v[e + 1];
          o[e] = upd<VW>(up.v[e], nx[k].v[e], W, E, cur.v[e], wc, wn);
          if constexpr (WGRAD) {
            const float nsum = __fadd_rn(__fadd_rn(up.v[e], nx[k].v[e]), __fadd_rn(W, E));
            gwc = __fmaf_rn(cur.v[e], pv[e], gwc);
            gwn = __fmaf_rn(nsum, pv[e], gwn);
          }
        }
        if (act && chk(row >= 1 && row <= S.rows && c + VW <= C &&
                           (VW == 1 || ((uintptr_t)(S.out + row * C + c) & 15) == 0), 303, P.status)) {
          float* dst = S.out + row * C + c;
          // a block's first / last own row also goes to the neighbours' ghost rows
          float* g_up = (row == 1 && S.out_prev) ? S.out_prev + (S.prev_rows + 1) * C + c : nullptr;
          float* g_dn = (row == S.rows && S.out_next) ? S.out_next + c : nullptr;
          if constexpr (VW == 4) {
            V16<float> q;
#pragma unroll
            for (int e = 0; e < 4; ++e) q.v[e] = o[e];
            st16<float>(dst, q);
            if (g_up) st16<float>(g_up, q);
            if (g_dn) st16<float>(g_dn, q);
          } else {
            *dst = o[0];
            if (g_up) *g_up = o[0];
            if (g_dn) *g_dn = o[0];
          }
        }
        up = cur;
        cur = nx[k];
      }
    }
  }
  if constexpr (WGRAD) {
    __shared__ float s_g[2][TX / 32];
    gwc = warp_reduce<float, DR_PLUS>(gwc);
    gwn = warp_reduce<float, DR_PLUS>(gwn);
    if (lane == 0) {
      s_g[0][threadIdx.x >> 5] = gwc;
      s_g[1][threadIdx.x >> 5] = gwn;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double a = 0.0, b = 0.0;
#pragma unroll
      for (int w = 0; w < TX / 32; ++w) {
        a += s_g[0][w];
        b += s_g[1][w];
      }
      atomicAdd(P.acc, a);
      atomicAdd(P.acc + 1, b);
    }
  }
}

__global__ void k_halo(const __grid_constant__ HaloParams P) {
  const auto& b = P.b[blockIdx.y];
  const float* src = blockIdx.z == 0 ? b.src_last : b.src_first;
  float* dst = blockIdx.z == 0 ? b.dst_top_ghost : b.dst_bot_ghost;
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < P.cols; j += (int64_t)gridDim.x * blockDim.x)
    dst[j] = src[j];
}

}  // namespace

cudaError_t launch_stencil(const StencilParams& p, int64_t nrb_launch, cudaStream_t s) {
  if (nrb_launch <= 0) return cudaSuccess;
  const int vw = p.vec_ok ? 4 : 1;
  dim3 grid((unsigned)((p.cols + (int64_t)TX * vw - 1) / ((int64_t)TX * vw)), (unsigned)nrb_launch);
  if (p.acc) {
    if (p.vec_ok) k_stencil5<4, true><<<grid, TX, 0, s>>>(p);
    else k_stencil5<1, true><<<grid, TX, 0, s>>>(p);
  } else {
    if (p.vec_ok) k_stencil5<4, false><<<grid, TX, 0, s>>>(p);
    else k_stencil5<1, false><<<grid, TX, 0, s>>>(p);
  }
  return cudaGetLastError();
}

cudaError_t launch_halo(const HaloParams& p, cudaStream_t s) {
  if (p.nbound <= 0) return cudaSuccess;
  const int threads = 256;
  unsigned gx = (unsigned)std::min<int64_t>((p.cols + threads - 1) / threads, 64);
  k_halo<<<dim3(gx, p.nbound, 2), threads, 0, s>>>(p);
  return cudaGetLastError();
}

}  // namespace dr
