// CPU oracle for the segmented-range hot path of "Distributed Ranges"
// (Brock et al., arXiv 2406.00158).
//
// TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the benchmark's
// CPU-baseline leg may load this library.  It shares no code, header, table or
// helper with the CUDA path; both only see inputs from the seeded generator.
//
// Every function here is a plain, sequential, obviously-correct statement of
// what the method computes:
//   * A distributed range is the concatenation of its segments in segment order
//     (Sec. 3, "Distributed Range"), so the oracle's scan and reduce work on the
//     concatenated array; segmentation must not change any result (up to the
//     floating-point rounding order), which the tests check on the GPU side.
//   * Floating-point sums accumulate in FP64 in index order; integer sums are
//     exact (two's-complement, mod 2^64).
//   * Algorithms 3 and 4 (per-segment reduce / scan + carry) are also written
//     out step by step for integers, so that the tests can confirm the paper's
//     segmented procedure equals the plain definition.
//   * The 5-point stencil and its transpose, the reverse scan (adjoint of the
//     inclusive scan) and the dot-product adjoint are written from their
//     definitions; the stencil's transpose is written in scatter form so that
//     the symmetry of the operator is checked, never assumed.
//   * for_each's element functions (the STREAM kernels, Black-Scholes pricing)
//     are written from their textbook definitions.
//
// Build: g++ -O2 -std=c++17 -fPIC -shared -ffp-contract=off (no fast-math).
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <functional>
#include <numeric>
#include <vector>

extern "C" {

// --------------------------------------------------------------------------
// inclusive_scan: y_i = x_0 + ... + x_i over the concatenation of segments
// (Sec. 4.3 "inclusive_scan"; plain definition = std::inclusive_scan).
// --------------------------------------------------------------------------

// int64 with wrap-around addition: the sum is taken in uint64 (mod 2^64).
void oracle_inclusive_scan_i64(const int64_t* x, int64_t n, int64_t* y) {
  std::vector<uint64_t> ux(x, x + n), uy(n);
  std::inclusive_scan(ux.begin(), ux.end(), uy.begin());
  std::memcpy(y, uy.data(), sizeof(uint64_t) * n);
}

// fp32 input, FP64 sequential accumulation.  Also returns s_i = sum_{j<=i} |x_j|,
// the scale of the rounding-error bound.
void oracle_inclusive_scan_f32_f64(const float* x, int64_t n, double* y, double* abs_prefix) {
  double s = 0.0, a = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    s += (double)x[i];
    a += std::fabs((double)x[i]);
    y[i] = s;
    if (abs_prefix) abs_prefix[i] = a;
  }
}

// FP64 input and output (used for adjoint / gradient references).
void oracle_inclusive_scan_f64(const double* x, int64_t n, double* y) {
  std::inclusive_scan(x, x + n, y);
}

// fp32 sequential scan in fp32 (context only: the error of the naive CPU scan).
void oracle_inclusive_scan_f32_seq(const float* x, int64_t n, float* y) {
  float s = 0.0f;
  for (int64_t i = 0; i < n; ++i) {
    s = s + x[i];
    y[i] = s;
  }
}

// Algorithm 4 written out for int64 (Sec. 4.3): a local scan of every segment,
// the last element of each segment collected into partial_sums (one entry per
// segment; an empty segment contributes 0), a scan of partial_sums, then
// segment k > 0 adds partial_sums[k-1].
void oracle_segmented_scan_alg4_i64(int nseg, const int64_t* lens, const int64_t* x,
                                    int64_t* y) {
  std::vector<uint64_t> partial(nseg, 0);
  int64_t off = 0;
  for (int k = 0; k < nseg; ++k) {
    uint64_t s = 0;
    for (int64_t i = 0; i < lens[k]; ++i) {
      s += (uint64_t)x[off + i];
      y[off + i] = (int64_t)s;
    }
    partial[k] = s;  // == *(out.end()-1), or the identity for an empty segment
    off += lens[k];
  }
  std::inclusive_scan(partial.begin(), partial.end(), partial.begin());
  off = 0;
  for (int k = 0; k < nseg; ++k) {
    uint64_t add = k > 0 ? partial[k - 1] : 0;
    for (int64_t i = 0; i < lens[k]; ++i) y[off + i] = (int64_t)((uint64_t)y[off + i] + add);
    off += lens[k];
  }
}

// --------------------------------------------------------------------------
// Scans and reduces with the other associative operators of Sec. 4.3 (the
// footnote to "reduce": any such operator; the last paragraph of
// "inclusive_scan": exclusive_scan is the same algorithm shifted by one, with
// an initial value).  op: 0 = plus, 2 = min, 3 = max (1 = multiply, reduce
// only).  min(a, b) selects b only when b < a, max(a, b) selects b only when
// a < b.  Integer plus and multiply wrap in the unsigned type of the same
// width.  mode 0: inclusive, y_i = init op x_0 op ... op x_i (the identity as
// init gives the plain inclusive scan); mode 1: exclusive, y_0 = init,
// y_i = init op x_0 op ... op x_{i-1}.
// --------------------------------------------------------------------------
}  // extern "C"

template <typename T, typename U>
static T op_apply(int op, T a, T b) {
  switch (op) {
    case 0: return (T)(U)((U)a + (U)b);
    case 1: return (T)(U)((U)a * (U)b);
    case 2: return b < a ? b : a;
    default: return a < b ? b : a;
  }
}

template <typename T, typename U>
static void scan_op(const T* x, int64_t n, int op, int mode, T init, T* y) {
  T acc = init;
  for (int64_t i = 0; i < n; ++i) {
    if (mode == 1) {
      y[i] = acc;
      acc = op_apply<T, U>(op, acc, x[i]);
    } else {
      acc = op_apply<T, U>(op, acc, x[i]);
      y[i] = acc;
    }
  }
}

template <typename T, typename U>
static T reduce_op(const T* x, int64_t n, int op, T init) {
  T acc = init;
  for (int64_t i = 0; i < n; ++i) acc = op_apply<T, U>(op, acc, x[i]);
  return acc;
}

// Floating-point operators in FP64 (plus rounds at every step; min / max select).
struct F64U {};
template <>
double op_apply<double, F64U>(int op, double a, double b) {
  switch (op) {
    case 0: return a + b;
    case 1: return a * b;
    case 2: return b < a ? b : a;
    default: return a < b ? b : a;
  }
}

extern "C" {

void oracle_scan_i64(const int64_t* x, int64_t n, int op, int mode, int64_t init, int64_t* y) {
  scan_op<int64_t, uint64_t>(x, n, op, mode, init, y);
}
void oracle_scan_i32(const int32_t* x, int64_t n, int op, int mode, int32_t init, int32_t* y) {
  scan_op<int32_t, uint32_t>(x, n, op, mode, init, y);
}
void oracle_scan_f64(const double* x, int64_t n, int op, int mode, double init, double* y) {
  scan_op<double, F64U>(x, n, op, mode, init, y);
}
int64_t oracle_reduce_i64(const int64_t* x, int64_t n, int op, int64_t init) {
  return reduce_op<int64_t, uint64_t>(x, n, op, init);
}
int32_t oracle_reduce_i32(const int32_t* x, int64_t n, int op, int32_t init) {
  return reduce_op<int32_t, uint32_t>(x, n, op, init);
}
double oracle_reduce_f64(const double* x, int64_t n, int op, double init) {
  return reduce_op<double, F64U>(x, n, op, init);
}

// The exact sum of n doubles as a non-overlapping expansion (J. R. Shewchuk,
// "Adaptive precision floating-point arithmetic and fast robust geometric
// predicates", Discrete Comput. Geom. 18, 1997: Grow-Expansion with zero
// elimination).  Each new term is added into the list of partials by
// error-free two-sums (hi = a + b rounded; lo = the exact rounding error,
// recovered with the magnitude-ordered Fast-Two-Sum); nonzero errors stay in
// the list, so sum(partials) equals sum(x) exactly, barring overflow.  Writes
// at most `cap` partials (smallest first) and returns their count, or -1 if
// more would be needed.
int64_t oracle_sum_expansion_f64(const double* x, int64_t n, double* partials, int64_t cap) {
  std::vector<double> p;
  for (int64_t i = 0; i < n; ++i) {
    double v = x[i];
    size_t k = 0;
    for (size_t j = 0; j < p.size(); ++j) {
      double a = v, b = p[j];
      if (std::fabs(a) < std::fabs(b)) std::swap(a, b);
      const double hi = a + b;
      const double lo = b - (hi - a);
      if (lo != 0.0) p[k++] = lo;
      v = hi;
    }
    p.resize(k);
    p.push_back(v);
  }
  if ((int64_t)p.size() > cap) return -1;
  for (size_t j = 0; j < p.size(); ++j) partials[j] = p[j];
  return (int64_t)p.size();
}

// --------------------------------------------------------------------------
// Reverse inclusive scan (adjoint of inclusive_scan):
//   g_x[j] = sum_{i >= j} g_y[i]
// --------------------------------------------------------------------------
void oracle_reverse_inclusive_scan_f64(const double* g, int64_t n, double* out) {
  double s = 0.0;
  for (int64_t j = n - 1; j >= 0; --j) {
    s += g[j];
    out[j] = s;
  }
}

// --------------------------------------------------------------------------
// transform_reduce(zip(x, y), multiply, plus): the dot product of Algorithm 1,
// reduced as in Algorithm 3.  Products of two fp32 values are exact in FP64; the
// sum runs in index order in FP64.  abs_dot = sum |x_i y_i| (error-bound scale).
// --------------------------------------------------------------------------
void oracle_dot_f64(const float* x, const float* y, int64_t n, double* dot, double* abs_dot) {
  *dot = std::inner_product(x, x + n, y, 0.0, std::plus<double>(),
                            [](float a, float b) { return (double)a * (double)b; });
  if (abs_dot)
    *abs_dot = std::inner_product(x, x + n, y, 0.0, std::plus<double>(),
                                  [](float a, float b) { return std::fabs((double)a * (double)b); });
}

// Algorithm 3 written out for int64: one local reduce per segment, partials
// combined in segment order.
int64_t oracle_segmented_reduce_alg3_i64(int nseg, const int64_t* lens, const int64_t* x) {
  uint64_t init = 0;
  int64_t off = 0;
  for (int k = 0; k < nseg; ++k) {
    uint64_t local = 0;
    for (int64_t i = 0; i < lens[k]; ++i) local += (uint64_t)x[off + i];
    init += local;
    off += lens[k];
  }
  return (int64_t)init;
}

// Adjoint of d = <x, y> for an incoming gradient g: (g*y, g*x), in FP64.
void oracle_dot_adjoint_f64(const float* x, const float* y, int64_t n, double g, double* gx,
                            double* gy) {
  for (int64_t i = 0; i < n; ++i) {
    gx[i] = g * (double)y[i];
    gy[i] = g * (double)x[i];
  }
}

// --------------------------------------------------------------------------
// 5-point Jacobi stencil for_each over an R x C row-major grid:
//   u'[i][j] = wc*u[i][j] + wn*(u[i-1][j] + u[i+1][j] + u[i][j-1] + u[i][j+1]),
// every cell updated, u = 0 outside [0,R) x [0,C) (zero ghost ring).  The
// segmentation into row blocks and the halo exchange do not appear: the state
// after each step does not depend on them.
// --------------------------------------------------------------------------
static inline double at_f64(const double* u, int64_t R, int64_t C, int64_t i, int64_t j) {
  return (i < 0 || i >= R || j < 0 || j >= C) ? 0.0 : u[i * C + j];
}

static void stencil5_f64_step(const double* a, double* b, int64_t R, int64_t C, double wc,
                              double wn) {
  for (int64_t i = 0; i < R; ++i)
    for (int64_t j = 0; j < C; ++j) {
      double nbr = at_f64(a, R, C, i - 1, j) + at_f64(a, R, C, i + 1, j) + at_f64(a, R, C, i, j - 1) +
                   at_f64(a, R, C, i, j + 1);
      b[i * C + j] = wc * a[i * C + j] + wn * nbr;
    }
}

void oracle_stencil5_f64(const double* u0, int64_t R, int64_t C, int steps, double wc, double wn,
                         double* out) {
  std::vector<double> a(u0, u0 + R * C), b(R * C);
  for (int t = 0; t < steps; ++t) {
    stencil5_f64_step(a.data(), b.data(), R, C, wc, wn);
    std::swap(a, b);
  }
  std::memcpy(out, a.data(), sizeof(double) * R * C);
}

// The same stencil in fp32 with one fixed evaluation order, for bit-exact
// comparison: s = (N + S) + (W + E); r = wn * s; and, only when wc != 0,
// r = r + wc * C.  Every operation is a separately rounded fp32 add or
// multiply (built with -ffp-contract=off, so nothing is fused).
static inline float at_f32(const float* u, int64_t R, int64_t C, int64_t i, int64_t j) {
  return (i < 0 || i >= R || j < 0 || j >= C) ? 0.0f : u[i * C + j];
}

static void stencil5_f32_step(const float* a, float* b, int64_t R, int64_t C, float wc, float wn) {
  for (int64_t i = 0; i < R; ++i)
    for (int64_t j = 0; j < C; ++j) {
      float ns = at_f32(a, R, C, i - 1, j) + at_f32(a, R, C, i + 1, j);
      float we = at_f32(a, R, C, i, j - 1) + at_f32(a, R, C, i, j + 1);
      float s = ns + we;
      float r = wn * s;
      if (wc != 0.0f) r = r + wc * a[i * C + j];
      b[i * C + j] = r;
    }
}

void oracle_stencil5_f32(const float* u0, int64_t R, int64_t C, int steps, float wc, float wn,
                         float* out) {
  std::vector<float> a(u0, u0 + R * C), b(R * C);
  for (int t = 0; t < steps; ++t) {
    stencil5_f32_step(a.data(), b.data(), R, C, wc, wn);
    std::swap(a, b);
  }
  std::memcpy(out, a.data(), sizeof(float) * R * C);
}

// Values of the stencil after `steps` steps at selected cells only.  One step
// reads neighbours at distance 1, so the value at (i,j) after t steps depends
// only on u0 within distance t.  For each requested cell the plain stencil is
// run on the window [i-t, i+t] x [j-t, j+t] clipped to the grid; outside the
// window (but inside the grid) the window sees zeros, which corrupts cells at
// distance d from the window edge only from step d+1 on, so the centre is exact.
// The per-cell arithmetic is identical to the full-grid functions above.
void oracle_stencil5_f32_at(const float* u0, int64_t R, int64_t C, int steps, float wc, float wn,
                            const int64_t* cells, int64_t ncells, float* out) {
  for (int64_t q = 0; q < ncells; ++q) {
    int64_t ci = cells[2 * q], cj = cells[2 * q + 1];
    int64_t i0 = std::max<int64_t>(0, ci - steps), i1 = std::min<int64_t>(R, ci + steps + 1);
    int64_t j0 = std::max<int64_t>(0, cj - steps), j1 = std::min<int64_t>(C, cj + steps + 1);
    int64_t wr = i1 - i0, wcn = j1 - j0;
    std::vector<float> a(wr * wcn), b(wr * wcn);
    for (int64_t i = 0; i < wr; ++i)
      for (int64_t j = 0; j < wcn; ++j) a[i * wcn + j] = u0[(i0 + i) * C + (j0 + j)];
    for (int t = 0; t < steps; ++t) {
      stencil5_f32_step(a.data(), b.data(), wr, wcn, wc, wn);
      std::swap(a, b);
    }
    out[q] = a[(ci - i0) * wcn + (cj - j0)];
  }
}

void oracle_stencil5_f64_at(const double* u0, int64_t R, int64_t C, int steps, double wc,
                            double wn, const int64_t* cells, int64_t ncells, double* out) {
  for (int64_t q = 0; q < ncells; ++q) {
    int64_t ci = cells[2 * q], cj = cells[2 * q + 1];
    int64_t i0 = std::max<int64_t>(0, ci - steps), i1 = std::min<int64_t>(R, ci + steps + 1);
    int64_t j0 = std::max<int64_t>(0, cj - steps), j1 = std::min<int64_t>(C, cj + steps + 1);
    int64_t wr = i1 - i0, wcn = j1 - j0;
    std::vector<double> a(wr * wcn), b(wr * wcn);
    for (int64_t i = 0; i < wr; ++i)
      for (int64_t j = 0; j < wcn; ++j) a[i * wcn + j] = u0[(i0 + i) * C + (j0 + j)];
    for (int t = 0; t < steps; ++t) {
      stencil5_f64_step(a.data(), b.data(), wr, wcn, wc, wn);
      std::swap(a, b);
    }
    out[q] = a[(ci - i0) * wcn + (cj - j0)];
  }
}

// Transposed stencil A^T, applied `steps` times, in scatter form: each cell
// (k,l) sends wc*v[k][l] to itself and wn*v[k][l] to each in-grid neighbour,
// i.e. column (k,l) of A^T is row (k,l) of A.
void oracle_stencil5_T_f64(const double* v0, int64_t R, int64_t C, int steps, double wc,
                           double wn, double* out) {
  std::vector<double> a(v0, v0 + R * C), b(R * C);
  const int64_t di[4] = {-1, 1, 0, 0}, dj[4] = {0, 0, -1, 1};
  for (int t = 0; t < steps; ++t) {
    std::fill(b.begin(), b.end(), 0.0);
    for (int64_t k = 0; k < R; ++k)
      for (int64_t l = 0; l < C; ++l) {
        double v = a[k * C + l];
        b[k * C + l] += wc * v;
        for (int d = 0; d < 4; ++d) {
          int64_t i = k + di[d], j = l + dj[d];
          if (i >= 0 && i < R && j >= 0 && j < C) b[i * C + j] += wn * v;
        }
      }
    std::swap(a, b);
  }
  std::memcpy(out, a.data(), sizeof(double) * R * C);
}

// --------------------------------------------------------------------------
// for_each over a zip of k vectors with an element function (Sec. 4.3
// "for_each"; Sec. 5's STREAM and Black-Scholes benchmarks).
//
// STREAM (McCalpin's four kernels), over zip(a, b, c) in the element type with
// one IEEE rounding per operation -- the plain definition (no FMA contraction):
//   copy:  c_i = a_i          scale: b_i = q * c_i
//   add:   c_i = a_i + b_i    triad: a_i = b_i + q * c_i
// --------------------------------------------------------------------------
}  // extern "C"

template <typename T>
static void stream_op(int fn, int64_t n, T* a, T* b, T* c, T q) {
  for (int64_t i = 0; i < n; ++i) {
    switch (fn) {
      case 0: c[i] = a[i]; break;
      case 1: b[i] = q * c[i]; break;
      case 2: c[i] = a[i] + b[i]; break;
      case 3: {
        const T qc = q * c[i];
        a[i] = b[i] + qc;
        break;
      }
    }
  }
}

extern "C" {

void oracle_stream_f32(int fn, int64_t n, float* a, float* b, float* c, float q) {
  stream_op<float>(fn, n, a, b, c, q);
}
void oracle_stream_f64(int fn, int64_t n, double* a, double* b, double* c, double q) {
  stream_op<double>(fn, n, a, b, c, q);
}

// European option prices under the Black-Scholes-Merton model (F. Black and
// M. Scholes, J. Political Economy 81(3), 1973; R. C. Merton, Bell J. Econ. 4(1),
// 1973), for spot S, strike X, time to expiry T (years), risk-free rate r and
// volatility sigma, in FP64:
//   d1 = (ln(S/X) + (r + sigma^2/2) T) / (sigma sqrt(T)),   d2 = d1 - sigma sqrt(T)
//   call = S N(d1) - X e^{-rT} N(d2),   put = X e^{-rT} N(-d2) - S N(-d1)
// with N the standard normal CDF, N(x) = erfc(-x / sqrt(2)) / 2.
// Also returns, per option, the first-order error scale of an fp32 evaluation:
// phi(d1) and phi(d2) (the normal density), d1, and K = X e^{-rT}.
static double norm_cdf(double x) { return 0.5 * std::erfc(-x / std::sqrt(2.0)); }
static double norm_pdf(double x) { return std::exp(-0.5 * x * x) / std::sqrt(2.0 * M_PI); }

void oracle_black_scholes_f64(int64_t n, const double* S, const double* X, const double* T, double r,
                              double sigma, double* call, double* put, double* aux /* n x 4 or NULL */) {
  for (int64_t i = 0; i < n; ++i) {
    const double sqt = std::sqrt(T[i]);
    const double d1 = (std::log(S[i] / X[i]) + (r + 0.5 * sigma * sigma) * T[i]) / (sigma * sqt);
    const double d2 = d1 - sigma * sqt;
    const double K = X[i] * std::exp(-r * T[i]);
    call[i] = S[i] * norm_cdf(d1) - K * norm_cdf(d2);
    put[i] = K * norm_cdf(-d2) - S[i] * norm_cdf(-d1);
    if (aux) {
      aux[4 * i + 0] = norm_pdf(d1);
      aux[4 * i + 1] = norm_pdf(d2);
      aux[4 * i + 2] = d1;
      aux[4 * i + 3] = K;
    }
  }
}

// --------------------------------------------------------------------------
// sort (Sec. 4.3 "sort"): the elements of the range in ascending order,
// written back over the same segmentation (C++'s sort is in place).  The plain
// definition is a sort of the concatenation.  Floating-point keys use the IEEE
// 754 totalOrder (-NaN < -inf < ... < -0 < +0 < ... < +inf < +NaN, NaNs by
// payload), so that the sorted sequence is unique bit for bit.
// --------------------------------------------------------------------------
}  // extern "C"

static bool total_less_f64(double a, double b) {
  int64_t x, y;
  std::memcpy(&x, &a, 8);
  std::memcpy(&y, &b, 8);
  // negative values order by decreasing magnitude bits
  if (x < 0) x = INT64_MIN - x - 1;  // maps sign-magnitude to two's complement order
  if (y < 0) y = INT64_MIN - y - 1;
  return x < y;
}
static bool total_less_f32(float a, float b) {
  int32_t x, y;
  std::memcpy(&x, &a, 4);
  std::memcpy(&y, &b, 4);
  if (x < 0) x = INT32_MIN - x - 1;
  if (y < 0) y = INT32_MIN - y - 1;
  return x < y;
}

extern "C" {

void oracle_sort_f32(float* x, int64_t n) { std::sort(x, x + n, total_less_f32); }
void oracle_sort_f64(double* x, int64_t n) { std::sort(x, x + n, total_less_f64); }
void oracle_sort_i32(int32_t* x, int64_t n) { std::sort(x, x + n); }
void oracle_sort_i64(int64_t* x, int64_t n) { std::sort(x, x + n); }

// The paper's distributed partition sort written out step by step for int64
// over p segments (lens[k] elements each, concatenated in x; result in out, the
// same segmentation):
//   1. each segment is sorted in place;
//   2. p-1 "medians" are taken from every sorted segment: the elements at
//      ranks floor(j * len / p), j = 1..p-1 (none from an empty segment);
//   3. all samples are sorted and the p-1 splitters are taken at ranks
//      floor(j * m / p), j = 1..p-1, of the m samples;
//   4. every segment counts its elements per chunk: chunk c (0 <= c < p) holds
//      the values v with splitter[c-1] <= v < splitter[c] (open ends at 0 and
//      p-1); the counts summed over segments give each chunk's size;
//   5. the elements are redistributed into the chunks (segment order within a
//      chunk), each chunk is sorted, and the chunks, concatenated in order,
//      are copied into the output range.
void oracle_partition_sort_i64(int p, const int64_t* lens, const int64_t* x, int64_t* out) {
  std::vector<std::vector<int64_t>> seg(p);
  int64_t off = 0;
  for (int k = 0; k < p; ++k) {
    seg[k].assign(x + off, x + off + lens[k]);
    off += lens[k];
    std::sort(seg[k].begin(), seg[k].end());
  }
  std::vector<int64_t> samples;
  for (int k = 0; k < p; ++k) {
    const int64_t L = (int64_t)seg[k].size();
    if (L == 0) continue;
    for (int j = 1; j < p; ++j) samples.push_back(seg[k][(j * L) / p]);
  }
  std::sort(samples.begin(), samples.end());
  const int64_t m = (int64_t)samples.size();
  std::vector<int64_t> split;
  if (m > 0)
    for (int j = 1; j < p; ++j) split.push_back(samples[(j * m) / p]);
  const int nchunk = (int)split.size() + 1;
  auto chunk_of = [&](int64_t v) {
    return (int)(std::upper_bound(split.begin(), split.end(), v) - split.begin());
  };
  std::vector<int64_t> size(nchunk, 0);
  for (int k = 0; k < p; ++k)
    for (int64_t v : seg[k]) size[chunk_of(v)]++;
  std::vector<std::vector<int64_t>> chunk(nchunk);
  for (int c = 0; c < nchunk; ++c) chunk[c].reserve(size[c]);
  for (int k = 0; k < p; ++k)
    for (int64_t v : seg[k]) chunk[chunk_of(v)].push_back(v);
  int64_t o = 0;
  for (int c = 0; c < nchunk; ++c) {
    std::sort(chunk[c].begin(), chunk[c].end());
    for (int64_t v : chunk[c]) out[o++] = v;
  }
}

}  // extern "C"
