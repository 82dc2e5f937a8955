// Device-side helpers shared by the kernels of the segmented-range library:
// element types and operators, 128-bit access, memory-model-explicit flag
// loads/stores (PTX), bounded waits and warp-level scan / reduce building blocks.
#pragma once

#include <cstdint>
#include <mutex>
#include <cuda_runtime.h>

#include "dr_kernels.h"

namespace dr {

// --------------------------------------------------------------------------
// operators
// --------------------------------------------------------------------------
template <typename T>
struct Lim;
template <>
struct Lim<float> {
  static __device__ __forceinline__ float lowest() { return -__int_as_float(0x7f800000); }
  static __device__ __forceinline__ float highest() { return __int_as_float(0x7f800000); }
};
template <>
struct Lim<double> {
  static __device__ __forceinline__ double lowest() { return -__longlong_as_double(0x7ff0000000000000ll); }
  static __device__ __forceinline__ double highest() { return __longlong_as_double(0x7ff0000000000000ll); }
};
template <>
struct Lim<long long> {
  static __device__ __forceinline__ long long lowest() { return (long long)0x8000000000000000ull; }
  static __device__ __forceinline__ long long highest() { return 0x7fffffffffffffffll; }
};
template <>
struct Lim<int> {
  static __device__ __forceinline__ int lowest() { return (int)0x80000000u; }
  static __device__ __forceinline__ int highest() { return 0x7fffffff; }
};

// Integer adds and multiplies wrap (done in the unsigned type).
template <typename T>
__device__ __forceinline__ T wrap_add(T a, T b) { return a + b; }
template <>
__device__ __forceinline__ long long wrap_add(long long a, long long b) {
  return (long long)((unsigned long long)a + (unsigned long long)b);
}
template <>
__device__ __forceinline__ int wrap_add(int a, int b) { return (int)((unsigned)a + (unsigned)b); }
template <typename T>
__device__ __forceinline__ T wrap_mul(T a, T b) { return a * b; }
template <>
__device__ __forceinline__ long long wrap_mul(long long a, long long b) {
  return (long long)((unsigned long long)a * (unsigned long long)b);
}
template <>
__device__ __forceinline__ int wrap_mul(int a, int b) { return (int)((unsigned)a * (unsigned)b); }

template <int OP>
struct Op {
  static constexpr int kOp = OP;
  template <typename T>
  static __device__ __forceinline__ T apply(T a, T b) {
    if constexpr (OP == DR_PLUS) return wrap_add(a, b);
    else if constexpr (OP == DR_MUL) return wrap_mul(a, b);
    else if constexpr (OP == DR_MIN) return b < a ? b : a;
    else return a < b ? b : a;
  }
  template <typename T>
  static __device__ __forceinline__ T identity() {
    if constexpr (OP == DR_PLUS) return T(0);
    else if constexpr (OP == DR_MUL) return T(1);
    else if constexpr (OP == DR_MIN) return Lim<T>::highest();
    else return Lim<T>::lowest();
  }
};

template <typename T>
__device__ __forceinline__ T binop_rt(int op, T a, T b) {
  switch (op) {
    case DR_PLUS: return wrap_add(a, b);
    case DR_MUL: return wrap_mul(a, b);
    case DR_MIN: return b < a ? b : a;
    default: return a < b ? b : a;
  }
}

template <typename T>
__device__ __forceinline__ T unop_rt(int op, T x, T a) {
  switch (op) {
    case DR_U_SCALE: return wrap_mul(a, x);
    case DR_U_ADD: return wrap_add(x, a);
    case DR_U_NEG: return wrap_mul(T(-1), x);
    case DR_U_ABS: return x < T(0) ? wrap_mul(T(-1), x) : x;
    default: return wrap_mul(x, x);
  }
}

// The fused view of a kernel: nleaf operands, each with a chain of unary ops,
// combined by zipop (if two), then a chain of unary ops.  The view code stays
// where the launch put it (the kernel's __grid_constant__ parameters): its
// fields are uniform across the grid and read from there, so evaluating a view
// costs no registers beyond the values themselves.
template <typename T>
__device__ __forceinline__ T view_arg(const double* d, const float* f, const long long* i, int k) {
  if constexpr (sizeof(T) == 4 && T(0.5) != T(0)) return f[k];       // float
  else if constexpr (T(0.5) != T(0)) return d[k];                    // double
  else return (T)i[k];                                               // int, long long
}

// One op applied to N register values (the switch taken once for all of them);
// the same arithmetic as unop_rt / binop_rt.
template <typename T, int N>
__device__ __forceinline__ void unop_all(int op, T a, T* x) {
  switch (op) {
    case DR_U_SCALE:
#pragma unroll
      for (int i = 0; i < N; ++i) x[i] = wrap_mul(a, x[i]);
      break;
    case DR_U_ADD:
#pragma unroll
      for (int i = 0; i < N; ++i) x[i] = wrap_add(x[i], a);
      break;
    case DR_U_NEG:
#pragma unroll
      for (int i = 0; i < N; ++i) x[i] = wrap_mul(T(-1), x[i]);
      break;
    case DR_U_ABS:
#pragma unroll
      for (int i = 0; i < N; ++i) x[i] = x[i] < T(0) ? wrap_mul(T(-1), x[i]) : x[i];
      break;
    default:
#pragma unroll
      for (int i = 0; i < N; ++i) x[i] = wrap_mul(x[i], x[i]);
  }
}
template <typename T, int N>
__device__ __forceinline__ void binop_all(int op, T* x, const T* y) {
  switch (op) {
    case DR_PLUS:
#pragma unroll
      for (int i = 0; i < N; ++i) x[i] = wrap_add(x[i], y[i]);
      break;
    case DR_MUL:
#pragma unroll
      for (int i = 0; i < N; ++i) x[i] = wrap_mul(x[i], y[i]);
      break;
    case DR_MIN:
#pragma unroll
      for (int i = 0; i < N; ++i) x[i] = y[i] < x[i] ? y[i] : x[i];
      break;
    default:
#pragma unroll
      for (int i = 0; i < N; ++i) x[i] = x[i] < y[i] ? y[i] : x[i];
  }
}

template <typename T>
struct ViewEval {
  const KViewCode* c;

  __device__ __forceinline__ void init(const KViewCode& code) { c = &code; }

  // The view over N values of each leaf held in registers: a (leaf 0) becomes
  // the view's values; b (leaf 1, used when the view has two leaves) is scratch.
  // Op by op over the whole array, so a chain costs one branch per op per call.
  template <int N>
  __device__ __forceinline__ void eval_all(T* a, T* b) const {
#pragma unroll 1
    for (int k = 0; k < c->npre[0]; ++k)
      unop_all<T, N>(c->pre_op[0][k], view_arg<T>(c->pre_arg[0], c->pre_argf[0], c->pre_argi[0], k), a);
    if (c->nleaf == 2) {
#pragma unroll 1
      for (int k = 0; k < c->npre[1]; ++k)
        unop_all<T, N>(c->pre_op[1][k], view_arg<T>(c->pre_arg[1], c->pre_argf[1], c->pre_argi[1], k), b);
      binop_all<T, N>(c->zipop, a, b);
    }
#pragma unroll 1
    for (int k = 0; k < c->npost; ++k)
      unop_all<T, N>(c->post_op[k], view_arg<T>(c->post_arg, c->post_argf, c->post_argi, k), a);
  }
  __device__ __forceinline__ T operator()(T a, T b) const {
#pragma unroll
    for (int k = 0; k < kMaxChain; ++k)
      if (k < c->npre[0]) a = unop_rt(c->pre_op[0][k], a, view_arg<T>(c->pre_arg[0], c->pre_argf[0], c->pre_argi[0], k));
    if (c->nleaf == 2) {
#pragma unroll
      for (int k = 0; k < kMaxChain; ++k)
        if (k < c->npre[1])
          b = unop_rt(c->pre_op[1][k], b, view_arg<T>(c->pre_arg[1], c->pre_argf[1], c->pre_argi[1], k));
      a = binop_rt(c->zipop, a, b);
    }
#pragma unroll
    for (int k = 0; k < kMaxChain; ++k)
      if (k < c->npost) a = unop_rt(c->post_op[k], a, view_arg<T>(c->post_arg, c->post_argf, c->post_argi, k));
    return a;
  }
};

// --------------------------------------------------------------------------
// 128-bit access
// --------------------------------------------------------------------------
template <typename T>
struct V16 {
  static constexpr int N = 16 / sizeof(T);
  T v[N];
};

template <typename T>
__device__ __forceinline__ V16<T> ld16(const void* p) {
  uint4 r;
  asm volatile("ld.global.nc.L1::no_allocate.v4.u32 {%0,%1,%2,%3}, [%4];"
               : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
               : "l"(p));
  V16<T> o;
  memcpy(&o, &r, 16);
  return o;
}

template <typename T>
__device__ __forceinline__ void st16(void* p, const V16<T>& o) {
  uint4 r;
  memcpy(&r, &o, 16);
  asm volatile("st.global.v4.u32 [%0], {%1,%2,%3,%4};" ::"l"(p), "r"(r.x), "r"(r.y), "r"(r.z),
               "r"(r.w)
               : "memory");
}

// L2 eviction-priority policies (createpolicy) and 128-bit accesses carrying them.
__device__ __forceinline__ unsigned long long l2_policy_evict_last() {
  unsigned long long p;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ unsigned long long l2_policy_evict_first() {
  unsigned long long p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
template <typename T>
__device__ __forceinline__ V16<T> ld16_hint(const void* p, unsigned long long pol) {
  uint4 r;
  asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.u32 {%0,%1,%2,%3}, [%4], %5;"
               : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
               : "l"(p), "l"(pol));
  V16<T> o;
  memcpy(&o, &r, 16);
  return o;
}
template <typename T>
__device__ __forceinline__ void st16_hint(void* p, const V16<T>& o, unsigned long long pol) {
  uint4 r;
  memcpy(&r, &o, 16);
  asm volatile("st.global.L2::cache_hint.v4.u32 [%0], {%1,%2,%3,%4}, %5;" ::"l"(p), "r"(r.x), "r"(r.y),
               "r"(r.z), "r"(r.w), "l"(pol)
               : "memory");
}

template <typename T>
__device__ __forceinline__ T ld1(const void* p) {
  return __ldg(reinterpret_cast<const T*>(p));
}

// --------------------------------------------------------------------------
// memory-model-explicit accesses (gpu scope)
// --------------------------------------------------------------------------
__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_u32(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned ld_relaxed_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

template <typename T>
__device__ __forceinline__ unsigned long long to_bits(T v) {
  if constexpr (sizeof(T) == 4) {
    unsigned u;
    memcpy(&u, &v, 4);
    return u;
  } else {
    unsigned long long u;
    memcpy(&u, &v, 8);
    return u;
  }
}
template <typename T>
__device__ __forceinline__ T from_bits(unsigned long long u) {
  T v;
  if constexpr (sizeof(T) == 4) {
    unsigned w = (unsigned)u;
    memcpy(&v, &w, 4);
  } else {
    memcpy(&v, &u, 8);
  }
  return v;
}

// --------------------------------------------------------------------------
// Lookback slots.  Tile i publishes (state, value): state A = the tile's own
// aggregate, state P = the inclusive prefix through the tile.  A flag is
// (epoch << 2) | state and is valid only for the current launch's epoch, so the
// slots never need clearing between launches.
//   4-byte T: flag and value packed in one 64-bit word (single-copy atomic).
//   8-byte T: a 32-bit flag published with release after the value; readers
//             load the flag with acquire, then the value.
// --------------------------------------------------------------------------
constexpr unsigned kStateA = 1, kStateP = 2;
// One slot per 128-byte line: hundreds of CTAs poll the slots just behind their
// tiles, and packing 16 slots into a line turns those polls (and the publishers'
// stores queued behind them) into an L2 hot spot.
constexpr int kSlotBytes = 128;

template <typename T, bool PACKED = (sizeof(T) == 4)>
struct Slots;

template <typename T>
struct Slots<T, true> {  // [flag:32 | value bits:32] in one 64-bit word
  char* base;
  static __host__ __device__ size_t bytes(int64_t ntiles) { return (size_t)ntiles * kSlotBytes; }
  __device__ void bind(char* b, int64_t) { base = b; }
  __device__ __forceinline__ unsigned long long* word(int64_t i) const {
    return reinterpret_cast<unsigned long long*>(base + i * kSlotBytes);
  }
  __device__ __forceinline__ void publish(int64_t i, unsigned tag, unsigned state, T v) {
    st_relaxed_u64(word(i), ((unsigned long long)(tag | state) << 32) | to_bits(v));
  }
  // returns the state (0 if not yet valid for this epoch)
  __device__ __forceinline__ unsigned poll(int64_t i, unsigned tag, T& v) const {
    unsigned long long x = ld_relaxed_u64(word(i));
    unsigned f = (unsigned)(x >> 32);
    if ((f & ~3u) != tag) return 0;
    v = from_bits<T>(x & 0xffffffffull);
    return f & 3u;
  }
};

// 8-byte values: two 64-bit words, each [flag:32 | one half of the value:32].
// Each word is written and read single-copy atomically; a reader accepts the
// pair only when both words carry the same flag (epoch and state): a state is
// published once per epoch, so matching flags identify one publication (an
// A -> P overwrite in flight shows as a mismatch and is polled again).  One L2
// round trip per poll, as for 4-byte values, instead of an acquire load of the
// flag followed by a dependent load of the value.
template <typename T>
struct Slots<T, false> {
  char* base;
  static __host__ __device__ size_t bytes(int64_t ntiles) { return (size_t)ntiles * kSlotBytes; }
  __device__ void bind(char* b, int64_t) { base = b; }
  __device__ __forceinline__ unsigned long long* word(int64_t i) const {
    return reinterpret_cast<unsigned long long*>(base + i * kSlotBytes);
  }
  __device__ __forceinline__ void publish(int64_t i, unsigned tag, unsigned state, T v) {
    const unsigned long long bits = to_bits(v), f = (unsigned long long)(tag | state) << 32;
    st_relaxed_u64(word(i), f | (bits & 0xffffffffull));
    st_relaxed_u64(word(i) + 1, f | (bits >> 32));
  }
  __device__ __forceinline__ unsigned poll(int64_t i, unsigned tag, T& v) const {
    const unsigned long long w0 = ld_relaxed_u64(word(i)), w1 = ld_relaxed_u64(word(i) + 1);
    const unsigned f0 = (unsigned)(w0 >> 32), f1 = (unsigned)(w1 >> 32);
    if (f0 != f1 || (f0 & ~3u) != tag) return 0;
    v = from_bits<T>((w0 & 0xffffffffull) | (w1 << 32));
    return f0 & 3u;
  }
};

// Records a device-side failure in the status word (first writer wins).
__device__ __forceinline__ void raise_status(unsigned* status, unsigned code, unsigned info) {
  if (atomicCAS(status, 0u, code) == 0u) atomicExch(status + 1, info);
}

// Range-checked builds (-DDR_CHECKED=1): every global address a kernel forms is
// checked against the bounds of the piece (segment, row block, tile) it belongs
// to -- and, for a 16-byte access, its alignment -- before the access.  A
// violation records DR_E_BOUNDS with the check's id in the device status word
// (read by dr_sync_status) and the access is skipped instead of faulting.
// Release builds compile the checks away.  Ids: scan 1xx, reduce 2xx, stencil
// 3xx, for_each / transform 4xx, sort 5xx, batched 6xx.
#ifndef DR_CHECKED
#define DR_CHECKED 0
#endif
__device__ __forceinline__ bool chk(bool ok, unsigned id, unsigned* status) {
  if (DR_CHECKED && !ok) raise_status(status, DR_E_BOUNDS, id);
  return !DR_CHECKED || ok;
}
// A 16-byte access of elements [e0, e0 + n) of a piece of `len` elements at p.
__device__ __forceinline__ bool chk_vec(int64_t e0, int n, int64_t len, const void* p, unsigned id,
                                        unsigned* status) {
  return chk(e0 >= 0 && e0 + n <= len && ((uintptr_t)p & 15) == 0, id, status);
}
// An access of element e of a piece of `len` elements.
__device__ __forceinline__ bool chk_at(int64_t e, int64_t len, unsigned id, unsigned* status) {
  return chk(e >= 0 && e < len, id, status);
}

// Polls slot i until it is valid for this epoch.  Bounded: gives up after
// `limit` polls (or as soon as another wait on the device has given up),
// records DR_E_TIMEOUT and returns P with the identity so the caller finishes.
template <typename T, typename S, typename OPT>
__device__ __forceinline__ unsigned wait_slot(const S& slots, int64_t i, unsigned tag, T& v,
                                              int64_t limit, unsigned* status) {
  unsigned s = slots.poll(i, tag, v);
  if (s) return s;
  unsigned ns = 16;
  for (int64_t polls = 1;; ++polls) {
    if (polls > 4) {  // the predecessor is usually a few hundred ns away: spin first
      __nanosleep(ns);
      if (ns < 512) ns <<= 1;
    }
    s = slots.poll(i, tag, v);
    if (s) return s;
    if (polls >= limit) {
      raise_status(status, DR_E_TIMEOUT, (unsigned)i);
      break;
    }
    if ((polls & 31) == 0 && ld_relaxed_u32(status) != 0u) break;
  }
  v = OPT::template identity<T>();
  return kStateP;
}

// --------------------------------------------------------------------------
// TMA bulk copies (cp.async.bulk, 1-D: 16-byte aligned addresses, size a
// multiple of 16) completing on a shared-memory mbarrier
// --------------------------------------------------------------------------
__device__ __forceinline__ unsigned smem_addr(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned long long* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}
// Bulk prefetch of [src, src + bytes) into L2 (16-byte aligned address, size a
// multiple of 16); a hint: nothing waits on it.
__device__ __forceinline__ void bulk_prefetch_l2(const void* src, unsigned bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait for an mbarrier phase; records DR_E_TIMEOUT and returns false on expiry.
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity, int64_t limit,
                                          unsigned* status) {
  for (int64_t k = 0; k < limit; ++k)
    if (mbar_try_wait(bar, parity)) return true;
  raise_status(status, DR_E_TIMEOUT, 0xffffffffu);
  return false;
}

// Polls of a wait for a bulk copy's completion.  A copy of a few tens of KB
// lands within microseconds; this bound (each try_wait may suspend for a
// hardware time slice) only ends a wait for a copy that never completes.  It
// is separate from the lookback poll limit (dr_set_spin_limit), which tests
// shorten on purpose: a CTA whose copy wait expired must neither read nor
// re-arm that stage, and must not exit while the copy may still be writing.
constexpr int64_t kCopyWaitPolls = int64_t(1) << 22;

// --------------------------------------------------------------------------
// warp building blocks
// --------------------------------------------------------------------------
template <typename T, int OP>
__device__ __forceinline__ T warp_reduce(T v) {
#pragma unroll
  for (int d = 16; d >= 1; d >>= 1) v = Op<OP>::apply(v, __shfl_xor_sync(0xffffffffu, v, d));
  return v;
}

// Inclusive scan across the lanes of a warp; REV = from lane 31 down to lane 0.
template <typename T, int OP, bool REV>
__device__ __forceinline__ T warp_inclusive(T v, int lane) {
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    if constexpr (!REV) {
      T y = __shfl_up_sync(0xffffffffu, v, d);
      if (lane >= d) v = Op<OP>::apply(y, v);
    } else {
      T y = __shfl_down_sync(0xffffffffu, v, d);
      if (lane + d < 32) v = Op<OP>::apply(y, v);
    }
  }
  return v;
}

// --------------------------------------------------------------------------
// Warp-wide decoupled lookback.  Returns the combination of the published
// values of tiles (pred, pred-1, ...) down to and including the nearest one in
// the inclusive-prefix state; tiles before `lo` count as an inclusive prefix
// equal to the identity.  Each round polls gr <= G slots per lane (32*gr tiles,
// nearest first: lane l holds pred - l*gr - g), waits only for unpublished slots
// nearer than the nearest inclusive prefix, and moves on by 32*gr if there is
// none.  One round costs one L2 round trip; covering 32*gr tiles per round keeps
// the walk short when hundreds of tiles are in flight at once.
// --------------------------------------------------------------------------
template <typename T, typename OPT, int G, typename S>
__device__ __forceinline__ T lookback(const S& slots, int64_t pred, int64_t lo, unsigned tag, int lane,
                                      int64_t limit, unsigned* status, int gr = G) {
  // gr (1 <= gr <= G, uniform across the warp): slots polled per lane per round
  const T ident = OPT::template identity<T>();
  T run = ident;
  while (true) {
    T val[G];
    unsigned st[G];
#pragma unroll
    for (int g = 0; g < G; ++g) {
      const int64_t i = pred - (int64_t)(lane * gr + g);
      val[g] = ident;
      st[g] = kStateP;
      if (g < gr && i >= lo) st[g] = slots.poll(i, tag, val[g]);
    }
    int gp = G;  // this lane's nearest inclusive prefix
#pragma unroll
    for (int g = G - 1; g >= 0; --g)
      if (g < gr && st[g] == kStateP) gp = g;
    unsigned pm = __ballot_sync(0xffffffffu, gp < G);
    int fl = pm ? __ffs(pm) - 1 : 32;
    if (lane <= fl) {
#pragma unroll
      for (int g = 0; g < G; ++g)
        if (g < gr && st[g] == 0 && (lane < fl || g < gp)) {
          const int64_t i = pred - (int64_t)(lane * gr + g);
          st[g] = wait_slot<T, S, OPT>(slots, i, tag, val[g], limit, status);
        }
    }
    __syncwarp();
    gp = G;
#pragma unroll
    for (int g = G - 1; g >= 0; --g)
      if (g < gr && st[g] == kStateP) gp = g;
    pm = __ballot_sync(0xffffffffu, gp < G);
    fl = pm ? __ffs(pm) - 1 : 32;
    T c = ident;
#pragma unroll
    for (int g = 0; g < G; ++g)
      if (g < gr && (lane < fl || (lane == fl && g <= gp))) c = OPT::apply(c, val[g]);
    run = OPT::apply(warp_reduce<T, OPT::kOp>(c), run);
    if (pm) break;
    pred -= 32 * gr;
  }
  return run;
}

// ---------------------------------------------------------------------------
// Host: resident CTAs per SM of a kernel on the current device.  Launch
// attributes (the dynamic shared-memory opt-in) are per device, so they are set
// once per device, with the result cached per device, under a lock.
// ---------------------------------------------------------------------------
struct OccCache {
  std::mutex mu;
  int per_sm[64] = {};
};

// Returns the resident CTAs per SM (>= 1), or 0 if the device index is out of
// range or the attribute could not be set (the caller reports a launch error).
template <typename K>
int resident_ctas(OccCache& c, K* kernel, int threads, int dyn_smem) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
  std::lock_guard<std::mutex> g(c.mu);
  if (!c.per_sm[dev]) {
    // the opt-in is needed once static + dynamic shared memory passes 48 KB, so
    // any kernel with dynamic shared memory sets it (to exactly what it launches with)
    if (dyn_smem > 0 &&
        cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn_smem) != cudaSuccess)
      return 0;
    int per = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, threads, dyn_smem) != cudaSuccess) return 0;
    c.per_sm[dev] = per > 0 ? per : 1;
  }
  return c.per_sm[dev];
}

inline int current_sm_count() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms > 0 ? sms : 1;
}

}  // namespace dr
