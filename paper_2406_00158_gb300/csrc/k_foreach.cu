// for_each over a k-ary zip with a built-in element function (Sec. 4.3
// "for_each"; Sec. 5's STREAM and Black-Scholes benchmarks), and transform:
// a fused view written out to a vector.
//
// Both are pure streams: every element is read once and written once, so the
// kernels are HBM-bound and shaped like the other streaming kernels here: a
// tile is FT threads x FCH 16-byte vectors per operand, grid-stride over tiles
// with a grid of resident CTAs, 128-bit accesses on aligned full tiles and
// scalar accesses on the ragged end of a piece.  Loads are coherent (a written
// operand may be the very storage of a read one: in place) and, like the
// stores, carry an L2 evict-first policy: nothing is reused.
#include "dr_device.cuh"

namespace dr {
namespace {

constexpr int FT = 256;
constexpr int FCH = 4;

template <typename T>
__host__ __device__ constexpr int ftile() {
  return FT * FCH * (16 / (int)sizeof(T));
}

template <typename T>
__device__ __forceinline__ V16<T> ld16_stream(const void* p, unsigned long long pol) {
  uint4 r;
  asm volatile("ld.global.L1::no_allocate.L2::cache_hint.v4.u32 {%0,%1,%2,%3}, [%4], %5;"
               : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
               : "l"(p), "l"(pol)
               : "memory");
  V16<T> o;
  memcpy(&o, &r, 16);
  return o;
}

// ---------------------------------------------------------------------------
// Element functions.  in(j) / out(o): the zip operand of the j-th input / o-th output.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }

template <typename T, int FN>
struct Fn;

template <typename T>
struct Fn<T, DR_FE_COPY> {  // zip(a, c): c = a
  static constexpr int NIN = 1, NOUT = 1;
  static __device__ __forceinline__ int in(int) { return 0; }
  static __device__ __forceinline__ int out(int) { return 1; }
  __device__ __forceinline__ void init(const double*) {}
  __device__ __forceinline__ void operator()(const T* x, T* y) const { y[0] = x[0]; }
};

template <typename T>
struct Fn<T, DR_FE_SCALE> {  // zip(b, c): b = q * c
  static constexpr int NIN = 1, NOUT = 1;
  static __device__ __forceinline__ int in(int) { return 1; }
  static __device__ __forceinline__ int out(int) { return 0; }
  T q;
  __device__ __forceinline__ void init(const double* a) { q = (T)a[0]; }
  __device__ __forceinline__ void operator()(const T* x, T* y) const { y[0] = mul_rn(q, x[0]); }
};

template <typename T>
struct Fn<T, DR_FE_ADD> {  // zip(a, b, c): c = a + b
  static constexpr int NIN = 2, NOUT = 1;
  static __device__ __forceinline__ int in(int j) { return j; }
  static __device__ __forceinline__ int out(int) { return 2; }
  __device__ __forceinline__ void init(const double*) {}
  __device__ __forceinline__ void operator()(const T* x, T* y) const { y[0] = add_rn(x[0], x[1]); }
};

template <typename T>
struct Fn<T, DR_FE_TRIAD> {  // zip(a, b, c): a = b + q * c  (two roundings)
  static constexpr int NIN = 2, NOUT = 1;
  static __device__ __forceinline__ int in(int j) { return 1 + j; }
  static __device__ __forceinline__ int out(int) { return 0; }
  T q;
  __device__ __forceinline__ void init(const double* a) { q = (T)a[0]; }
  __device__ __forceinline__ void operator()(const T* x, T* y) const { y[0] = add_rn(x[0], mul_rn(q, x[1])); }
};

// Black-Scholes-Merton European call and put for spot S, strike X, expiry T
// (this generic form is the fp64 one; fp32 is specialised below):
//   d1 = (ln(S/X) + (r + sigma^2/2) T) / (sigma sqrt T),  d2 = d1 - sigma sqrt T,
//   C = S N(d1) - X e^{-rT} N(d2),  P = X e^{-rT} N(-d2) - S N(-d1).
// N(d) and N(-d) come from one complementary error function value: with
// e = erfc(|d| / sqrt 2) / 2 = N(-|d|) <= 1/2, the pair is (1 - e, e) ordered by
// the sign of d, so both keep full relative accuracy in the tails.
__device__ __forceinline__ float bs_log(float x) { return logf(x); }
__device__ __forceinline__ double bs_log(double x) { return log(x); }
__device__ __forceinline__ float bs_exp(float x) { return expf(x); }
__device__ __forceinline__ double bs_exp(double x) { return exp(x); }
__device__ __forceinline__ float bs_sqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ double bs_sqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float bs_erfc(float x) { return erfcf(x); }
__device__ __forceinline__ double bs_erfc(double x) { return erfc(x); }

template <typename T>
struct Fn<T, DR_FE_BLACK_SCHOLES> {  // zip(S, X, T, C, P)
  static constexpr int NIN = 3, NOUT = 2;
  static __device__ __forceinline__ int in(int j) { return j; }
  static __device__ __forceinline__ int out(int o) { return 3 + o; }
  T r, sigma, drift;
  __device__ __forceinline__ void init(const double* a) {
    r = (T)a[0];
    sigma = (T)a[1];
    drift = r + (T)0.5 * sigma * sigma;
  }
  static __device__ __forceinline__ void cdf_pair(T d, T& n_pos, T& n_neg) {
    const T e = (T)0.5 * bs_erfc(fabs(d) * (T)0.70710678118654752440);
    const T c = (T)1 - e;
    n_pos = d >= (T)0 ? c : e;  // N(d)
    n_neg = d >= (T)0 ? e : c;  // N(-d)
  }
  __device__ __forceinline__ void operator()(const T* x, T* y) const {
    const T S = x[0], X = x[1], t = x[2];
    const T sv = sigma * bs_sqrt(t);
    const T d1 = (bs_log(S / X) + drift * t) / sv;
    const T d2 = d1 - sv;
    const T K = X * bs_exp(-r * t);
    T n1, m1, n2, m2;
    cdf_pair(d1, n1, m1);
    cdf_pair(d2, n2, m2);
    y[0] = S * n1 - K * n2;
    y[1] = K * m2 - S * m1;
  }
};

// fp32 evaluation for throughput: the division, logarithm, exponential and
// square root use the hardware approximations (relative error a few ulp;
// lg2.approx absolute error 2^-22.6 on [0.5, 2]), and N comes from the
// Zelen-Severo polynomial (Abramowitz & Stegun, Handbook of Mathematical
// Functions, 26.2.17): for x >= 0,
//   N(-x) = phi(x) (b1 t + b2 t^2 + b3 t^3 + b4 t^4 + b5 t^5),  t = 1 / (1 + p x),
// phi the standard normal density, with absolute error below 7.5e-8 (1.3 fp32
// ulp of 1), so every quantity stays within 8 ulp of its exact value.
template <>
struct Fn<float, DR_FE_BLACK_SCHOLES> {
  static constexpr int NIN = 3, NOUT = 2;
  static __device__ __forceinline__ int in(int j) { return j; }
  static __device__ __forceinline__ int out(int o) { return 3 + o; }
  float r, sigma, inv_sigma, drift;
  __device__ __forceinline__ void init(const double* a) {
    r = (float)a[0];
    sigma = (float)a[1];
    inv_sigma = 1.0f / sigma;
    drift = r + 0.5f * sigma * sigma;
  }
  static __device__ __forceinline__ void cdf_pair(float d, float& n_pos, float& n_neg) {
    const float x = fabsf(d);
    const float t = __fdividef(1.0f, fmaf(0.2316419f, x, 1.0f));
    const float phi = 0.3989422804014327f * __expf(-0.5f * x * x);
    float poly = fmaf(t, 1.330274429f, -1.821255978f);
    poly = fmaf(t, poly, 1.781477937f);
    poly = fmaf(t, poly, -0.356563782f);
    poly = fmaf(t, poly, 0.319381530f);
    const float e = phi * (poly * t);  // N(-|d|)
    const float c = 1.0f - e;
    n_pos = d >= 0.0f ? c : e;
    n_neg = d >= 0.0f ? e : c;
  }
  __device__ __forceinline__ void operator()(const float* x, float* y) const {
    const float S = x[0], X = x[1], t = x[2];
    const float rs = rsqrtf(t);
    const float sv = sigma * t * rs;  // sigma sqrt(t)
    const float lnr = __log2f(__fdividef(S, X)) * 0.6931471805599453f;
    const float d1 = fmaf(drift, t, lnr) * (inv_sigma * rs);
    const float d2 = d1 - sv;
    const float K = X * __expf(-r * t);
    float n1, m1, n2, m2;
    cdf_pair(d1, n1, m1);
    cdf_pair(d2, n2, m2);
    y[0] = S * n1 - K * n2;
    y[1] = K * m2 - S * m1;
  }
};

// The piece holding `tile`, from a table of n pieces sorted by first tile.
template <typename PC>
__device__ __forceinline__ int find_tile_piece(const PC* pc, int n, int64_t tile) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (pc[mid].tile_begin <= tile) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// The piece table: inline in the kernel parameters (read through the constant
// cache), or, with EXT, in device memory (more pieces than the parameters hold).
// A compile-time choice, so that every piece access keeps its address space.
template <bool EXT, typename PP>
__device__ __forceinline__ const auto* fe_table(const PP& P) {
  if constexpr (EXT) return P.pc_ext;
  else return P.pc;
}

template <typename T, int FN, bool EXT>
__global__ void __launch_bounds__(FT) k_for_each(const __grid_constant__ ForEachParams P) {
  using F = Fn<T, FN>;
  constexpr int VN = 16 / sizeof(T);
  constexpr int TILE = ftile<T>();
  F f;
  f.init(P.arg);
  const unsigned long long pol = l2_policy_evict_first();
  const int tid = threadIdx.x;
  for (int64_t tile = blockIdx.x; tile < P.ntiles; tile += gridDim.x) {
    const auto* tab = fe_table<EXT>(P);
    const int k = find_tile_piece(tab, P.npieces, tile);
    const FePiece& pc = tab[k];
    const int64_t base = (tile - pc.tile_begin) * TILE;
    if (!chk(k >= 0 && k < P.npieces && base >= 0 && base < pc.len, 400, P.status)) continue;
    if (pc.vec_ok && pc.len - base >= TILE) {
      V16<T> xv[FCH][F::NIN];
#pragma unroll
      for (int c = 0; c < FCH; ++c) {
        const int64_t e0 = base + (int64_t)(c * FT + tid) * VN;
        const int64_t off = e0 * (int64_t)sizeof(T);
#pragma unroll
        for (int j = 0; j < F::NIN; ++j)
          if (chk_vec(e0, VN, pc.len, pc.p[F::in(j)] + off, 401, P.status))
            xv[c][j] = ld16_stream<T>(pc.p[F::in(j)] + off, pol);
      }
#pragma unroll
      for (int c = 0; c < FCH; ++c) {
        const int64_t off = (base + (int64_t)(c * FT + tid) * VN) * (int64_t)sizeof(T);
        V16<T> yv[F::NOUT];
#pragma unroll
        for (int e = 0; e < VN; ++e) {
          T xi[F::NIN], yo[F::NOUT];
#pragma unroll
          for (int j = 0; j < F::NIN; ++j) xi[j] = xv[c][j].v[e];
          f(xi, yo);
#pragma unroll
          for (int o = 0; o < F::NOUT; ++o) yv[o].v[e] = yo[o];
        }
#pragma unroll
        for (int o = 0; o < F::NOUT; ++o)
          if (chk_vec(off / (int64_t)sizeof(T), VN, pc.len, pc.p[F::out(o)] + off, 402, P.status))
            st16_hint<T>(pc.p[F::out(o)] + off, yv[o], pol);
      }
    } else {
      const int64_t end = min(base + (int64_t)TILE, pc.len);
      for (int64_t i = base + tid; i < end; i += FT) {
        if (!chk_at(i, pc.len, 403, P.status)) continue;
        T xi[F::NIN], yo[F::NOUT];
#pragma unroll
        for (int j = 0; j < F::NIN; ++j) xi[j] = reinterpret_cast<const T*>(pc.p[F::in(j)])[i];
        f(xi, yo);
#pragma unroll
        for (int o = 0; o < F::NOUT; ++o) reinterpret_cast<T*>(pc.p[F::out(o)])[i] = yo[o];
      }
    }
  }
}

// ---------------------------------------------------------------------------
// transform: out = view (KIND 0: one plain leaf; 1: a * b; 2: interpreted chain)
// ---------------------------------------------------------------------------
template <typename T, int KIND>
__device__ __forceinline__ T tr_eval(const ViewEval<T>& ve, T a, T b) {
  if constexpr (KIND == 0) return a;
  else if constexpr (KIND == 1) return wrap_mul(a, b);
  else return ve(a, b);
}

template <typename T, int KIND, bool EXT>
__global__ void __launch_bounds__(FT) k_transform(const __grid_constant__ TransformParams P) {
  constexpr int VN = 16 / sizeof(T);
  constexpr int TILE = ftile<T>();
  ViewEval<T> ve;
  ve.init(P.vc);
  const bool two = P.vc.nleaf == 2;
  const unsigned long long pol = l2_policy_evict_first();
  const int tid = threadIdx.x;
  for (int64_t tile = blockIdx.x; tile < P.ntiles; tile += gridDim.x) {
    const auto* tab = fe_table<EXT>(P);
    const int k = find_tile_piece(tab, P.npieces, tile);
    const KPiece& pc = tab[k];
    const int64_t base = (tile - pc.tile_begin) * TILE;
    if (!chk(k >= 0 && k < P.npieces && base >= 0 && base < pc.len, 410, P.status)) continue;
    if (pc.vec_ok && pc.len - base >= TILE) {
      V16<T> av[FCH], bv[FCH];
#pragma unroll
      for (int c = 0; c < FCH; ++c) {
        const int64_t e0 = base + (int64_t)(c * FT + tid) * VN;
        const int64_t off = e0 * (int64_t)sizeof(T);
        if (chk_vec(e0, VN, pc.len, pc.a + off, 411, P.status)) av[c] = ld16_stream<T>(pc.a + off, pol);
        if (two && chk_vec(e0, VN, pc.len, pc.b + off, 412, P.status)) bv[c] = ld16_stream<T>(pc.b + off, pol);
      }
      if constexpr (KIND == 2) {
        T xa[FCH][VN], xb[FCH][VN];
#pragma unroll
        for (int c = 0; c < FCH; ++c)
#pragma unroll
          for (int e = 0; e < VN; ++e) {
            xa[c][e] = av[c].v[e];
            xb[c][e] = two ? bv[c].v[e] : T(0);
          }
        ve.template eval_all<FCH * VN>(&xa[0][0], &xb[0][0]);
#pragma unroll
        for (int c = 0; c < FCH; ++c)
#pragma unroll
          for (int e = 0; e < VN; ++e) av[c].v[e] = xa[c][e];
      }
#pragma unroll
      for (int c = 0; c < FCH; ++c) {
        const int64_t off = (base + (int64_t)(c * FT + tid) * VN) * (int64_t)sizeof(T);
        V16<T> o;
#pragma unroll
        for (int e = 0; e < VN; ++e)
          o.v[e] = KIND == 2 ? av[c].v[e] : tr_eval<T, KIND>(ve, av[c].v[e], two ? bv[c].v[e] : T(0));
        if (chk_vec(off / (int64_t)sizeof(T), VN, pc.len, pc.o + off, 413, P.status)) st16_hint<T>(pc.o + off, o, pol);
      }
    } else {
      const int64_t end = min(base + (int64_t)TILE, pc.len);
      for (int64_t i = base + tid; i < end; i += FT) {
        if (!chk_at(i, pc.len, 414, P.status)) continue;
        const T a = reinterpret_cast<const T*>(pc.a)[i];
        const T b = two ? reinterpret_cast<const T*>(pc.b)[i] : T(0);
        reinterpret_cast<T*>(pc.o)[i] = tr_eval<T, KIND>(ve, a, b);
      }
    }
  }
}

// Resident-CTA grid of a kernel (occupancy queried once per kernel instance and
// device), capped by the tile count.
template <typename K>
int resident_grid(OccCache& occ, K* kernel, int64_t ntiles) {
  const int per = resident_ctas(occ, kernel, FT, 0);
  const int64_t g = (int64_t)current_sm_count() * (per > 0 ? per : 1);
  return (int)(ntiles < g ? ntiles : g);
}

template <typename T, int FN>
cudaError_t run_fe(const ForEachParams& p, cudaStream_t s) {
  static OccCache occ, occx;
  if (p.pc_ext) {
    const int grid = resident_grid(occx, k_for_each<T, FN, true>, p.ntiles);
    k_for_each<T, FN, true><<<grid, FT, 0, s>>>(p);
  } else {
    const int grid = resident_grid(occ, k_for_each<T, FN, false>, p.ntiles);
    k_for_each<T, FN, false><<<grid, FT, 0, s>>>(p);
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t run_fe_t(const ForEachParams& p, cudaStream_t s) {
  switch (p.fn) {
    case DR_FE_COPY: return run_fe<T, DR_FE_COPY>(p, s);
    case DR_FE_SCALE: return run_fe<T, DR_FE_SCALE>(p, s);
    case DR_FE_ADD: return run_fe<T, DR_FE_ADD>(p, s);
    case DR_FE_TRIAD: return run_fe<T, DR_FE_TRIAD>(p, s);
    case DR_FE_BLACK_SCHOLES: return run_fe<T, DR_FE_BLACK_SCHOLES>(p, s);
  }
  return cudaErrorInvalidValue;
}

template <typename T, int KIND>
cudaError_t run_tr(const TransformParams& p, cudaStream_t s) {
  static OccCache occ, occx;
  if (p.pc_ext) {
    const int grid = resident_grid(occx, k_transform<T, KIND, true>, p.ntiles);
    k_transform<T, KIND, true><<<grid, FT, 0, s>>>(p);
  } else {
    const int grid = resident_grid(occ, k_transform<T, KIND, false>, p.ntiles);
    k_transform<T, KIND, false><<<grid, FT, 0, s>>>(p);
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t run_tr_t(const TransformParams& p, cudaStream_t s) {
  switch (p.vc.kind) {
    case 0: return run_tr<T, 0>(p, s);
    case 1: return run_tr<T, 1>(p, s);
    default: return run_tr<T, 2>(p, s);
  }
}

}  // namespace

int foreach_tile_elems(int dtype) {
  return (dtype == DR_F32 || dtype == DR_I32) ? ftile<float>() : ftile<double>();
}

cudaError_t launch_for_each(const ForEachParams& p, cudaStream_t s) {
  if (p.ntiles <= 0) return cudaSuccess;
  return p.dtype == DR_F32 ? run_fe_t<float>(p, s) : run_fe_t<double>(p, s);
}

cudaError_t launch_transform(const TransformParams& p, cudaStream_t s) {
  if (p.ntiles <= 0) return cudaSuccess;
  switch (p.dtype) {
    case DR_F32: return run_tr_t<float>(p, s);
    case DR_F64: return run_tr_t<double>(p, s);
    case DR_I64: return run_tr_t<long long>(p, s);
    case DR_I32: return run_tr_t<int>(p, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace dr
