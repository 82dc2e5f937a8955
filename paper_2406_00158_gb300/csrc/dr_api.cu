// Host side of the C ABI (dr.h): handles, view composition and flattening,
// re-segmentation, argument validation, and the algorithm entry points that
// fill kernel parameters and launch.  No entry point throws or aborts.
#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>

#include "dr_host.h"

namespace dr {

// ---------------------------------------------------------------------------
// errors, per-device status word, knobs
// ---------------------------------------------------------------------------
static thread_local std::string t_msg;

int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  t_msg = buf;
  return code;
}

int cuda_fail(cudaError_t e, const char* what) {
  return fail(DR_E_CUDA, "%s: %s (%s)", what, cudaGetErrorString(e), cudaGetErrorName(e));
}

void clear_error() { t_msg.clear(); }

int esize(int dtype) {
  switch (dtype) {
    case DR_F32:
    case DR_I32: return 4;
    case DR_F64:
    case DR_I64: return 8;
    default: return 0;
  }
}

bool valid_dtype(int dtype) { return esize(dtype) != 0; }

// [0] = first failure code, [1] = its info (tile / item index)
__device__ unsigned g_status[4];

static std::mutex g_mu;
static constexpr int kMaxDevices = 64;
static unsigned* g_status_addr[kMaxDevices];
static std::atomic<int64_t> g_spin{int64_t(1) << 21};
static std::atomic<int64_t> g_skip{-1};

unsigned* status_word() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return nullptr;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_status_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_status) != cudaSuccess) return nullptr;
    g_status_addr[dev] = static_cast<unsigned*>(p);
  }
  return g_status_addr[dev];
}

int64_t spin_limit() { return g_spin.load(); }
int64_t take_skip_publish() { return g_skip.exchange(-1); }

int sm_count() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms > 0 ? sms : 1;
}

namespace {
// Per device: the library's stream-ordered memory pool (memory stays cached in
// the pool: release threshold unbounded) and a stream for frees of workspaces
// whose last use is unknown.
struct DevPool {
  cudaMemPool_t pool = nullptr;
  cudaStream_t free_stream = nullptr;
};
DevPool* dev_pool(int dev) {
  static std::mutex m;
  static DevPool pools[64];
  if (dev < 0 || dev >= 64) return nullptr;
  std::lock_guard<std::mutex> g(m);
  DevPool& d = pools[dev];
  if (!d.pool) {
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t p = nullptr;
    if (cudaMemPoolCreate(&p, &props) != cudaSuccess) return nullptr;
    uint64_t thr = ~uint64_t(0);
    cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &thr);
    cudaStream_t fs = nullptr;
    if (cudaStreamCreateWithFlags(&fs, cudaStreamNonBlocking) != cudaSuccess) {
      cudaMemPoolDestroy(p);
      return nullptr;
    }
    d.pool = p;
    d.free_stream = fs;
  }
  return &d;
}
}  // namespace

int Workspace::ensure(size_t need, cudaStream_t s, size_t zero) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (ptr && bytes >= need && device == dev) return DR_OK;
  if (ptr) release();  // behind its last use; the pool orders any reuse after the free
  DevPool* dp = dev_pool(dev);
  if (!dp) return fail(DR_E_CUDA, "workspace pool for device %d could not be created", dev);
  need = (need + 255) / 256 * 256;
  e = cudaMallocFromPoolAsync(&ptr, need, dp->pool, s);
  if (e != cudaSuccess) {
    ptr = nullptr;
    return fail(DR_E_NOMEM, "workspace allocation of %zu bytes failed: %s", need, cudaGetErrorString(e));
  }
  e = cudaMemsetAsync(ptr, 0, zero < need ? zero : need, s);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(workspace)");
  bytes = need;
  device = dev;
  marked = false;
  return DR_OK;
}

void Workspace::mark(cudaStream_t s) {
  if (!ptr) return;
  last = s;
  marked = true;
}

void Workspace::release() {
  if (ptr) {
    int cur = 0;
    cudaGetDevice(&cur);
    if (cur != device) cudaSetDevice(device);
    if (marked) {
      cudaFreeAsync(ptr, last);  // after the work queued on the stream of the last use
    } else {
      cudaDeviceSynchronize();   // unknown last use: kernels on any stream may still use it
      DevPool* dp = dev_pool(device);
      cudaFreeAsync(ptr, dp ? dp->free_stream : nullptr);
    }
    if (cur != device) cudaSetDevice(cur);
  }
  last = nullptr;
  marked = false;
  ptr = nullptr;
  bytes = 0;
  device = -1;
}

// ---------------------------------------------------------------------------
// re-segmentation (Sec. 4.4 "Zip")
// ---------------------------------------------------------------------------
std::vector<Piece> resegment(const std::vector<std::vector<Seg>>& ops, int esz) {
  const size_t k = std::min<size_t>(ops.size(), kMaxZip);  // callers pass at most kMaxZip
  std::vector<Piece> out;
  std::vector<size_t> si(k, 0);
  std::vector<int64_t> used(k, 0);
  int64_t pos = 0;
  while (true) {
    bool done = false;
    for (size_t o = 0; o < k; ++o) {
      while (si[o] < ops[o].size() && used[o] >= ops[o][si[o]].len) {
        ++si[o];
        used[o] = 0;
      }
      if (si[o] == ops[o].size()) done = true;
    }
    if (done || k == 0) break;
    int64_t take = INT64_MAX;
    for (size_t o = 0; o < k; ++o) take = std::min(take, ops[o][si[o]].len - used[o]);
    Piece pc{};
    pc.start = pos;
    pc.len = take;
    for (size_t o = 0; o < k; ++o) {
      const Seg& s = ops[o][si[o]];
      pc.p[o] = s.p + used[o] * esz;
      pc.seg[o] = s.idx;
      pc.off[o] = s.off + used[o];
      used[o] += take;
    }
    out.push_back(pc);
    pos += take;
  }
  return out;
}

}  // namespace dr

using namespace dr;

std::vector<Seg> dr_vec::window(int64_t lo, int64_t hi) const {
  std::vector<Seg> out;
  for (size_t k = 0; k < ptr.size(); ++k) {
    const int64_t a = std::max(lo, start[k]), b = std::min(hi, start[k] + len[k]);
    if (b > a) out.push_back(Seg{ptr[k] + (a - start[k]) * esz, b - a, (int32_t)k, a - start[k]});
  }
  return out;
}

void dr_view::recompute() {
  std::vector<std::vector<Seg>> ops;
  size = INT64_MAX;
  for (int l = 0; l < nleaf; ++l) {
    ops.push_back(leaf[l].vec->window(leaf[l].lo, leaf[l].hi));
    size = std::min(size, leaf[l].hi - leaf[l].lo);
  }
  if (size < 0) size = 0;
  pieces = resegment(ops, esize(dtype));
}

KViewCode dr_view::code() const {
  KViewCode c{};
  c.nleaf = nleaf;
  c.zipop = zipop < 0 ? DR_PLUS : zipop;
  c.npost = npost;
  // integer views take the scalar truncated toward zero (as a C cast), fp32 views rounded
  auto to_i = [](double v) {
    if (!(v == v)) return 0LL;
    if (v >= 9.2233720368547758e18) return (long long)0x7fffffffffffffffLL;
    if (v <= -9.2233720368547758e18) return (long long)0x8000000000000000LL;
    return (long long)v;
  };
  for (int l = 0; l < 2; ++l) {
    c.npre[l] = npre[l];
    for (int k = 0; k < kMaxChain; ++k) {
      c.pre_op[l][k] = pre_op[l][k];
      c.pre_arg[l][k] = pre_arg[l][k];
      c.pre_argf[l][k] = (float)pre_arg[l][k];
      c.pre_argi[l][k] = to_i(pre_arg[l][k]);
    }
  }
  for (int k = 0; k < kMaxChain; ++k) {
    c.post_op[k] = post_op[k];
    c.post_arg[k] = post_arg[k];
    c.post_argf[k] = (float)post_arg[k];
    c.post_argi[k] = to_i(post_arg[k]);
  }
  if (nleaf == 1 && npre[0] == 0 && npost == 0) c.kind = 0;
  else if (nleaf == 2 && zipop == DR_MUL && npre[0] == 0 && npre[1] == 0 && npost == 0) c.kind = 1;
  else c.kind = 2;
  return c;
}

// ---------------------------------------------------------------------------
// status
// ---------------------------------------------------------------------------
extern "C" const char* dr_last_error(void) { return t_msg.c_str(); }

extern "C" int dr_version(void) { return 1; }

extern "C" int dr_sync_status(dr_stream_t stream) {
  clear_error();
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
  unsigned h[4] = {0, 0, 0, 0};
  e = cudaMemcpyFromSymbol(h, g_status, sizeof h);
  if (e != cudaSuccess) return cuda_fail(e, "reading the device status word");
  if (h[0] != 0) {
    const unsigned z[4] = {0, 0, 0, 0};
    cudaMemcpyToSymbol(g_status, z, sizeof z);
    if (h[0] == DR_E_TIMEOUT)
      return fail(DR_E_TIMEOUT, "a bounded device wait expired (tile/item %u); results of the kernels "
                                "launched since the last check are invalid", h[1]);
    return fail((int)h[0], "device reported status %u (info %u)", h[0], h[1]);
  }
  return DR_OK;
}

extern "C" int dr_kernel_geometry(int kernel, int dtype, int64_t* tile_elems, int* ctas_per_sm) {
  clear_error();
  if (!valid_dtype(dtype)) return fail(DR_E_DTYPE, "dr_kernel_geometry: unknown dtype %d", dtype);
  int64_t t = 0;
  int per = 0;
  switch (kernel) {
    case DR_K_SCAN: t = scan_tile_elems(dtype); break;
    case DR_K_SCAN_VIEW: t = scan_tile_elems(dtype, true); break;
    case DR_K_REDUCE:
      t = reduce_tile_elems(dtype);
      per = reduce_ctas_per_sm();
      break;
    case DR_K_FOREACH: t = foreach_tile_elems(dtype); break;
    case DR_K_SORT: t = sort_tile_elems(dtype); break;
    default: return fail(DR_E_INVAL, "dr_kernel_geometry: unknown kernel family %d", kernel);
  }
  if (tile_elems) *tile_elems = t;
  if (ctas_per_sm) *ctas_per_sm = per;
  return DR_OK;
}

extern "C" int dr_set_spin_limit(int64_t polls) {
  clear_error();
  if (polls < 1) return fail(DR_E_INVAL, "spin limit must be >= 1 (got %lld)", (long long)polls);
  g_spin.store(polls);
  return DR_OK;
}

extern "C" int dr_debug_skip_publish(int64_t tile) {
  clear_error();
  g_skip.store(tile < 0 ? -1 : tile);
  return DR_OK;
}

// ---------------------------------------------------------------------------
// segmented vector
// ---------------------------------------------------------------------------
extern "C" int dr_block_lengths(int64_t n, int p, int64_t* lens_out) {
  clear_error();
  if (n < 0 || p < 1 || !lens_out) return fail(DR_E_INVAL, "dr_block_lengths: need n >= 0, p >= 1, lens_out");
  const int64_t b = (n + p - 1) / p;
  int64_t left = n;
  for (int k = 0; k < p; ++k) {
    lens_out[k] = std::min(b, left);
    left -= lens_out[k];
  }
  return DR_OK;
}

extern "C" int dr_vec_create(int dtype, int nseg, const int64_t* lens, void* const* seg_ptrs,
                             dr_vec** out) {
  clear_error();
  if (!out) return fail(DR_E_INVAL, "dr_vec_create: out is NULL");
  *out = nullptr;
  if (!valid_dtype(dtype)) return fail(DR_E_DTYPE, "dr_vec_create: unknown dtype %d", dtype);
  if (nseg < 1 || !lens || !seg_ptrs) return fail(DR_E_INVAL, "dr_vec_create: need nseg >= 1, lens, seg_ptrs");
  const int esz = esize(dtype);
  for (int k = 0; k < nseg; ++k) {
    if (lens[k] < 0) return fail(DR_E_INVAL, "dr_vec_create: segment %d has negative length", k);
    if (lens[k] > 0 && !seg_ptrs[k]) return fail(DR_E_INVAL, "dr_vec_create: segment %d pointer is NULL", k);
    if ((uintptr_t)seg_ptrs[k] % esz)
      return fail(DR_E_ALIGN, "dr_vec_create: segment %d pointer not aligned to %d bytes", k, esz);
  }
  dr_vec* v = new (std::nothrow) dr_vec();
  if (!v) return fail(DR_E_NOMEM, "dr_vec_create: out of host memory");
  v->dtype = dtype;
  v->esz = esz;
  int64_t s = 0;
  for (int k = 0; k < nseg; ++k) {
    v->ptr.push_back(static_cast<char*>(seg_ptrs[k]));
    v->len.push_back(lens[k]);
    v->start.push_back(s);
    s += lens[k];
  }
  v->n = s;
  *out = v;
  return DR_OK;
}

extern "C" int dr_vec_rebind(dr_vec* v, void* const* seg_ptrs) {
  clear_error();
  if (!v || !seg_ptrs) return fail(DR_E_INVAL, "dr_vec_rebind: NULL argument");
  for (size_t k = 0; k < v->ptr.size(); ++k) {
    if (v->len[k] > 0 && !seg_ptrs[k]) return fail(DR_E_INVAL, "dr_vec_rebind: segment %zu pointer is NULL", k);
    if ((uintptr_t)seg_ptrs[k] % v->esz)
      return fail(DR_E_ALIGN, "dr_vec_rebind: segment %zu pointer not aligned to %d bytes", k, v->esz);
  }
  for (size_t k = 0; k < v->ptr.size(); ++k) v->ptr[k] = static_cast<char*>(seg_ptrs[k]);
  return DR_OK;
}

extern "C" int dr_vec_destroy(dr_vec* v) {
  clear_error();
  delete v;
  return DR_OK;
}

extern "C" int dr_vec_info(const dr_vec* v, int* dtype, int* nseg, int64_t* n) {
  clear_error();
  if (!v) return fail(DR_E_INVAL, "dr_vec_info: NULL vector");
  if (dtype) *dtype = v->dtype;
  if (nseg) *nseg = (int)v->ptr.size();
  if (n) *n = v->n;
  return DR_OK;
}

extern "C" int dr_vec_segment(const dr_vec* v, int k, void** ptr, int64_t* len, int64_t* start) {
  clear_error();
  if (!v) return fail(DR_E_INVAL, "dr_vec_segment: NULL vector");
  if (k < 0 || k >= (int)v->ptr.size()) return fail(DR_E_BOUNDS, "dr_vec_segment: no segment %d", k);
  if (ptr) *ptr = v->ptr[k];
  if (len) *len = v->len[k];
  if (start) *start = v->start[k];
  return DR_OK;
}

extern "C" int dr_vec_locate(const dr_vec* v, int64_t i, int* seg, int64_t* off) {
  clear_error();
  if (!v) return fail(DR_E_INVAL, "dr_vec_locate: NULL vector");
  if (i < 0 || i >= v->n) return fail(DR_E_BOUNDS, "dr_vec_locate: index %lld outside [0, %lld)", (long long)i, (long long)v->n);
  // last segment whose start is <= i; empty segments share starts, step back over them
  auto it = std::upper_bound(v->start.begin(), v->start.end(), i);
  int k = (int)(it - v->start.begin()) - 1;
  while (k > 0 && (v->len[k] == 0 || i >= v->start[k] + v->len[k])) --k;
  if (seg) *seg = k;
  if (off) *off = i - v->start[k];
  return DR_OK;
}

static int copy_vec(const dr_vec* v, void* host, bool to_host, cudaStream_t s) {
  for (size_t k = 0; k < v->ptr.size(); ++k) {
    if (!v->len[k]) continue;
    char* h = static_cast<char*>(host) + v->start[k] * v->esz;
    cudaError_t e = to_host ? cudaMemcpyAsync(h, v->ptr[k], v->len[k] * v->esz, cudaMemcpyDeviceToHost, s)
                            : cudaMemcpyAsync(v->ptr[k], h, v->len[k] * v->esz, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_fail(e, to_host ? "copy segment to host" : "copy segment from host");
  }
  return DR_OK;
}

extern "C" int dr_vec_copy_from_host(dr_vec* v, const void* host, dr_stream_t stream) {
  clear_error();
  if (!v || (!host && v->n)) return fail(DR_E_INVAL, "dr_vec_copy_from_host: NULL argument");
  return copy_vec(v, const_cast<void*>(host), false, (cudaStream_t)stream);
}

extern "C" int dr_vec_copy_to_host(const dr_vec* v, void* host, dr_stream_t stream) {
  clear_error();
  if (!v || (!host && v->n)) return fail(DR_E_INVAL, "dr_vec_copy_to_host: NULL argument");
  return copy_vec(v, host, true, (cudaStream_t)stream);
}

// ---------------------------------------------------------------------------
// row-block 2-D array
// ---------------------------------------------------------------------------
extern "C" int dr_md2_create(int dtype, int64_t rows, int64_t cols, int nseg, const int64_t* seg_rows,
                             void* const* seg_ptrs, dr_md2** out) {
  clear_error();
  if (!out) return fail(DR_E_INVAL, "dr_md2_create: out is NULL");
  *out = nullptr;
  if (dtype != DR_F32) return fail(DR_E_DTYPE, "dr_md2_create: only DR_F32 is supported");
  if (rows < 1 || cols < 1 || nseg < 1 || nseg > kMaxPieces || !seg_rows || !seg_ptrs)
    return fail(DR_E_INVAL, "dr_md2_create: need rows, cols >= 1, 1 <= nseg <= %d, seg_rows, seg_ptrs", kMaxPieces);
  int64_t sum = 0;
  for (int k = 0; k < nseg; ++k) {
    if (seg_rows[k] < 1) return fail(DR_E_INVAL, "dr_md2_create: block %d has %lld rows", k, (long long)seg_rows[k]);
    if (!seg_ptrs[k]) return fail(DR_E_INVAL, "dr_md2_create: block %d pointer is NULL", k);
    if ((uintptr_t)seg_ptrs[k] % 4) return fail(DR_E_ALIGN, "dr_md2_create: block %d pointer not 4-byte aligned", k);
    sum += seg_rows[k];
  }
  if (sum != rows) return fail(DR_E_INVAL, "dr_md2_create: block rows sum to %lld, not %lld", (long long)sum, (long long)rows);
  dr_md2* m = new (std::nothrow) dr_md2();
  if (!m) return fail(DR_E_NOMEM, "dr_md2_create: out of host memory");
  m->dtype = dtype;
  m->rows = rows;
  m->cols = cols;
  for (int k = 0; k < nseg; ++k) {
    m->ptr.push_back(static_cast<char*>(seg_ptrs[k]));
    m->srows.push_back(seg_rows[k]);
  }
  *out = m;
  return DR_OK;
}

extern "C" int dr_md2_destroy(dr_md2* m) {
  clear_error();
  delete m;
  return DR_OK;
}

static int exchange_halos(const dr_md2* m, cudaStream_t s) {
  if (m->ptr.size() < 2) return DR_OK;
  HaloParams p{};
  p.nbound = (int)m->ptr.size() - 1;
  p.cols = m->cols;
  for (int k = 0; k < p.nbound; ++k) {
    float* a = reinterpret_cast<float*>(m->ptr[k]);
    float* b = reinterpret_cast<float*>(m->ptr[k + 1]);
    p.b[k].src_last = a + m->srows[k] * m->cols;
    p.b[k].dst_top_ghost = b;
    p.b[k].src_first = b + m->cols;
    p.b[k].dst_bot_ghost = a + (m->srows[k] + 1) * m->cols;
  }
  cudaError_t e = launch_halo(p, s);
  return e == cudaSuccess ? DR_OK : cuda_fail(e, "halo exchange launch");
}

extern "C" int dr_md2_exchange_halos(dr_md2* m, dr_stream_t stream) {
  clear_error();
  if (!m) return fail(DR_E_INVAL, "dr_md2_exchange_halos: NULL array");
  return exchange_halos(m, (cudaStream_t)stream);
}

// ---------------------------------------------------------------------------
// views
// ---------------------------------------------------------------------------
extern "C" int dr_view_of(const dr_vec* v, dr_view** out) {
  clear_error();
  if (!v || !out) return fail(DR_E_INVAL, "dr_view_of: NULL argument");
  dr_view* w = new (std::nothrow) dr_view();
  if (!w) return fail(DR_E_NOMEM, "dr_view_of: out of host memory");
  w->dtype = v->dtype;
  w->arity = 1;
  w->nleaf = 1;
  w->leaf[0] = {v, 0, v->n};
  w->recompute();
  *out = w;
  return DR_OK;
}

static dr_view* clone_view(const dr_view* b) {
  dr_view* w = new (std::nothrow) dr_view();
  if (!w) return nullptr;
  w->dtype = b->dtype;
  w->arity = b->arity;
  w->nleaf = b->nleaf;
  for (int l = 0; l < kMaxZip; ++l) w->leaf[l] = b->leaf[l];
  std::memcpy(w->npre, b->npre, sizeof w->npre);
  std::memcpy(w->pre_op, b->pre_op, sizeof w->pre_op);
  std::memcpy(w->pre_arg, b->pre_arg, sizeof w->pre_arg);
  w->zipop = b->zipop;
  w->npost = b->npost;
  std::memcpy(w->post_op, b->post_op, sizeof w->post_op);
  std::memcpy(w->post_arg, b->post_arg, sizeof w->post_arg);
  w->size = b->size;
  w->pieces = b->pieces;
  return w;
}

extern "C" int dr_view_transform(const dr_view* base, int op, double arg, dr_view** out) {
  clear_error();
  if (!base || !out) return fail(DR_E_INVAL, "dr_view_transform: NULL argument");
  if (base->arity != 1)
    return fail(DR_E_INVAL, "dr_view_transform: base is a raw zip; use dr_view_zip_transform first");
  if (op < DR_U_SCALE || op > DR_U_SQUARE) return fail(DR_E_INVAL, "dr_view_transform: unknown op %d", op);
  if (base->npost >= kMaxChain)
    return fail(DR_E_UNSUPPORTED, "dr_view_transform: more than %d chained transforms", kMaxChain);
  dr_view* w = clone_view(base);
  if (!w) return fail(DR_E_NOMEM, "dr_view_transform: out of host memory");
  w->post_op[w->npost] = op;
  w->post_arg[w->npost] = arg;
  w->npost++;
  *out = w;
  return DR_OK;
}

// Aligned operands (Sec. 4.4 "Zip"): the same number of (non-empty) segments
// over the views' windows, with corresponding segments of equal size.
static bool aligned(const dr_view* a, const dr_view* b) {
  const std::vector<Seg> sa = a->leaf[0].vec->window(a->leaf[0].lo, a->leaf[0].hi);
  const std::vector<Seg> sb = b->leaf[0].vec->window(b->leaf[0].lo, b->leaf[0].hi);
  if (sa.size() != sb.size()) return false;
  for (size_t k = 0; k < sa.size(); ++k)
    if (sa[k].len != sb[k].len) return false;
  return true;
}

extern "C" int dr_view_zip_ex(const dr_view* a, const dr_view* b, int flags, dr_view** out) {
  clear_error();
  if (!a || !b || !out) return fail(DR_E_INVAL, "dr_view_zip_ex: NULL argument");
  if (flags & ~DR_ZIP_STRICT_ALIGN) return fail(DR_E_INVAL, "dr_view_zip_ex: unknown flags 0x%x", flags);
  if (a->arity != 1 || b->arity != 1 || a->nleaf != 1 || b->nleaf != 1)
    return fail(DR_E_UNSUPPORTED, "dr_view_zip_ex: operands must be (transformed) views of one vector each");
  if ((flags & DR_ZIP_STRICT_ALIGN) && !aligned(a, b))
    return fail(DR_E_ALIGN, "dr_view_zip_ex: operands are not aligned (segment counts or sizes differ) and "
                            "strict alignment was requested");
  return dr_view_zip(a, b, out);
}

extern "C" int dr_view_zip(const dr_view* a, const dr_view* b, dr_view** out) {
  clear_error();
  if (!a || !b || !out) return fail(DR_E_INVAL, "dr_view_zip: NULL argument");
  if (a->arity != 1 || b->arity != 1 || a->nleaf != 1 || b->nleaf != 1)
    return fail(DR_E_UNSUPPORTED, "dr_view_zip: operands must be (transformed) views of one vector each");
  if (a->dtype != b->dtype) return fail(DR_E_DTYPE, "dr_view_zip: operand dtypes differ");
  dr_view* w = new (std::nothrow) dr_view();
  if (!w) return fail(DR_E_NOMEM, "dr_view_zip: out of host memory");
  w->dtype = a->dtype;
  w->arity = 2;
  w->nleaf = 2;
  w->leaf[0] = a->leaf[0];
  w->leaf[1] = b->leaf[0];
  w->npre[0] = a->npost;
  w->npre[1] = b->npost;
  for (int k = 0; k < kMaxChain; ++k) {
    w->pre_op[0][k] = a->post_op[k];
    w->pre_arg[0][k] = a->post_arg[k];
    w->pre_op[1][k] = b->post_op[k];
    w->pre_arg[1][k] = b->post_arg[k];
  }
  w->recompute();
  *out = w;
  return DR_OK;
}

extern "C" int dr_view_zipn(int k, const dr_view* const* leaves, dr_view** out) {
  clear_error();
  const char* who = "dr_view_zipn";
  if (!leaves || !out) return fail(DR_E_INVAL, "%s: NULL argument", who);
  if (k < 2 || k > kMaxZip) return fail(DR_E_UNSUPPORTED, "%s: k = %d outside [2, %d]", who, k, kMaxZip);
  for (int l = 0; l < k; ++l) {
    const dr_view* v = leaves[l];
    if (!v) return fail(DR_E_INVAL, "%s: leaf %d is NULL", who, l);
    if (v->arity != 1 || v->nleaf != 1 || v->npost != 0 || v->npre[0] != 0)
      return fail(DR_E_UNSUPPORTED, "%s: leaf %d is not an untransformed view of one vector", who, l);
    if (v->dtype != leaves[0]->dtype) return fail(DR_E_DTYPE, "%s: leaf dtypes differ", who);
  }
  dr_view* w = new (std::nothrow) dr_view();
  if (!w) return fail(DR_E_NOMEM, "%s: out of host memory", who);
  w->dtype = leaves[0]->dtype;
  w->arity = k;
  w->nleaf = k;
  for (int l = 0; l < k; ++l) w->leaf[l] = leaves[l]->leaf[0];
  w->recompute();
  *out = w;
  return DR_OK;
}

extern "C" int dr_view_zip_transform(const dr_view* zip, int op, dr_view** out) {
  clear_error();
  if (!zip || !out) return fail(DR_E_INVAL, "dr_view_zip_transform: NULL argument");
  if (zip->arity != 2) return fail(DR_E_INVAL, "dr_view_zip_transform: base is not a zip");
  if (op < DR_PLUS || op > DR_MAX) return fail(DR_E_INVAL, "dr_view_zip_transform: unknown op %d", op);
  dr_view* w = clone_view(zip);
  if (!w) return fail(DR_E_NOMEM, "dr_view_zip_transform: out of host memory");
  w->arity = 1;
  w->zipop = op;
  *out = w;
  return DR_OK;
}

static int trim(const dr_view* base, int64_t lo_add, int64_t new_size, dr_view** out) {
  dr_view* w = clone_view(base);
  if (!w) return fail(DR_E_NOMEM, "take/drop: out of host memory");
  for (int l = 0; l < w->nleaf; ++l) {
    w->leaf[l].lo += lo_add;
    w->leaf[l].hi = std::min(w->leaf[l].hi, w->leaf[l].lo + new_size);
  }
  w->recompute();
  *out = w;
  return DR_OK;
}

extern "C" int dr_view_take(const dr_view* base, int64_t l, dr_view** out) {
  clear_error();
  if (!base || !out) return fail(DR_E_INVAL, "dr_view_take: NULL argument");
  l = std::max<int64_t>(0, std::min(l, base->size));
  return trim(base, 0, l, out);
}

extern "C" int dr_view_drop(const dr_view* base, int64_t f, dr_view** out) {
  clear_error();
  if (!base || !out) return fail(DR_E_INVAL, "dr_view_drop: NULL argument");
  f = std::max<int64_t>(0, std::min(f, base->size));
  return trim(base, f, base->size - f, out);
}

extern "C" int dr_view_destroy(dr_view* v) {
  clear_error();
  if (v) {
    v->ws_scan.release();
    v->ws_reduce.release();
    v->ws_sort.release();
    v->ws_table.release();
  }
  delete v;
  return DR_OK;
}

extern "C" int dr_view_info(const dr_view* v, int64_t* size, int* arity, int* dtype, int* npieces) {
  clear_error();
  if (!v) return fail(DR_E_INVAL, "dr_view_info: NULL view");
  if (size) *size = v->size;
  if (arity) *arity = v->arity;
  if (dtype) *dtype = v->dtype;
  if (npieces) *npieces = (int)v->pieces.size();
  return DR_OK;
}

extern "C" int dr_view_segments(const dr_view* v, int max_pieces, dr_piece* out) {
  clear_error();
  if (!v || (!out && max_pieces > 0)) return fail(DR_E_INVAL, "dr_view_segments: NULL argument");
  const int n = std::min<int>(max_pieces, (int)v->pieces.size());
  for (int i = 0; i < n; ++i) {
    const Piece& p = v->pieces[i];
    out[i].start = p.start;
    out[i].len = p.len;
    for (int l = 0; l < 2; ++l) {
      out[i].seg[l] = l < v->nleaf ? p.seg[l] : -1;
      out[i].off[l] = l < v->nleaf ? p.off[l] : 0;
    }
  }
  return DR_OK;
}

// ---------------------------------------------------------------------------
// algorithms
// ---------------------------------------------------------------------------

// A table of more pieces than a launch carries inline goes to the view's device
// table, uploaded on `s` (a stream-ordered copy from pageable memory: the call
// waits for the stream's earlier work, and cannot be captured in a graph).
template <typename P>
static int place_pieces(dr_view* v, const std::vector<P>& pcs, P* inline_pc, const P** ext, cudaStream_t s) {
  if (pcs.size() <= (size_t)kMaxPieces) {
    std::copy(pcs.begin(), pcs.end(), inline_pc);
    *ext = nullptr;
    return DR_OK;
  }
  const size_t bytes = pcs.size() * sizeof(P);
  if (int r = v->ws_table.ensure(bytes, s, 0)) return r;
  cudaError_t e = cudaMemcpyAsync(v->ws_table.ptr, pcs.data(), bytes, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return cuda_fail(e, "piece table upload");
  v->ws_table.mark(s);
  *ext = static_cast<const P*>(v->ws_table.ptr);
  return DR_OK;
}

// The pieces of a call: the view's leaves (and the output, if any) re-segmented
// together, each cut into tiles of `tile` elements.
static std::vector<KPiece> build_pieces(const dr_view* in, const dr_vec* out, int tile, int64_t* ntiles) {
  std::vector<std::vector<Seg>> ops;
  for (int l = 0; l < in->nleaf; ++l) ops.push_back(in->leaf[l].vec->window(in->leaf[l].lo, in->leaf[l].hi));
  if (out) ops.push_back(out->window(0, in->size));
  const std::vector<Piece> ps = resegment(ops, esize(in->dtype));
  std::vector<KPiece> v(ps.size());
  int64_t t = 0;
  for (size_t i = 0; i < ps.size(); ++i) {
    KPiece& k = v[i];
    k.a = ps[i].p[0];
    k.b = in->nleaf == 2 ? ps[i].p[1] : nullptr;
    k.o = out ? ps[i].p[in->nleaf] : nullptr;
    k.len = ps[i].len;
    k.tile_begin = t;
    k.vec_ok = ((uintptr_t)k.a % 16 == 0) && ((uintptr_t)k.b % 16 == 0) && ((uintptr_t)k.o % 16 == 0);
    t += (ps[i].len + tile - 1) / tile;
  }
  *ntiles = t;
  return v;
}

// build_pieces, then up to kMaxPieces inline in `pc`; more go to the view's
// device table (*ext), or are refused when ext == NULL.
static int call_pieces(dr_view* in, const dr_vec* out, int tile, KPiece* pc, const KPiece** ext, int* npieces,
                       int64_t* ntiles, cudaStream_t s) {
  const std::vector<KPiece> v = build_pieces(in, out, tile, ntiles);
  if (!ext && (int)v.size() > kMaxPieces)
    return fail(DR_E_UNSUPPORTED, "call spans %zu segments after re-segmentation (limit %d)", v.size(), kMaxPieces);
  *npieces = (int)v.size();
  if (!ext) {
    std::copy(v.begin(), v.end(), pc);
    return DR_OK;
  }
  return place_pieces(in, v, pc, ext, s);
}

// True when [p, p + n) and [q, q + n) overlap but do not coincide.
static bool partial_overlap(const char* p, const char* q, int64_t nbytes) {
  return p != q && p < q + nbytes && q < p + nbytes;
}

static int check_single(const dr_view* in, const char* who) {
  if (!in) return fail(DR_E_INVAL, "%s: NULL input view", who);
  if (in->arity != 1) return fail(DR_E_INVAL, "%s: input is a raw zip; apply dr_view_zip_transform", who);
  return DR_OK;
}

static int do_scan(const char* who, const dr_view* in_c, dr_vec* out, int op, bool reverse, bool exclusive,
                   const void* init, cudaStream_t s, const void* dev_carry = nullptr) {
  clear_error();
  if (int r = check_single(in_c, who)) return r;
  dr_view* in = const_cast<dr_view*>(in_c);
  if (!out) return fail(DR_E_INVAL, "%s: NULL output", who);
  if (out->dtype != in->dtype) return fail(DR_E_DTYPE, "%s: output dtype differs from input", who);
  if (out->n < in->size)
    return fail(DR_E_INVAL, "%s: output has %lld elements, input %lld", who, (long long)out->n, (long long)in->size);
  if (op != DR_PLUS && op != DR_MIN && op != DR_MAX) return fail(DR_E_INVAL, "%s: op must be PLUS, MIN or MAX", who);
  if (exclusive && !init && !dev_carry) return fail(DR_E_INVAL, "%s: NULL init", who);
  if (dev_carry && (uintptr_t)dev_carry % esize(in->dtype))
    return fail(DR_E_ALIGN, "%s: carry pointer not aligned to the element size", who);
  if (in->size == 0) return DR_OK;
  static thread_local ScanParams p;
  std::memset(&p, 0, sizeof p);
  p.vc = in->code();
  p.op = op;
  p.dtype = in->dtype;
  p.exclusive = exclusive ? 1 : 0;
  // the kernels the dispatch picks for a fused view (vc.kind != 0) have shorter tiles
  const bool fused = p.vc.kind != 0;
  if (int r = call_pieces(in, out, scan_tile_elems(in->dtype, fused), p.pc, &p.pc_ext, &p.npieces, &p.ntiles, s))
    return r;
  if (int r = in->ws_scan.ensure(scan_ws_bytes(p.ntiles, in->dtype), s)) return r;
  p.ws = static_cast<char*>(in->ws_scan.ptr);
  p.status = status_word();
  if (!p.status) return fail(DR_E_CUDA, "%s: no device status word", who);
  p.spin_limit = spin_limit();
  p.skip_tile = take_skip_publish();
  if (exclusive && init) std::memcpy(&p.init_bits, init, esize(in->dtype));
  p.carry = dev_carry;
  cudaError_t e = launch_scan(p, reverse, scan_grid(in->dtype, p.ntiles), s);
  in->ws_scan.mark(s);
  return e == cudaSuccess ? DR_OK : cuda_fail(e, who);
}

extern "C" int dr_inclusive_scan(const dr_view* in, dr_vec* out, int op, dr_stream_t stream) {
  return do_scan("dr_inclusive_scan", in, out, op, false, false, nullptr, (cudaStream_t)stream);
}

extern "C" int dr_exclusive_scan(const dr_view* in, dr_vec* out, int op, const void* init, dr_stream_t stream) {
  return do_scan("dr_exclusive_scan", in, out, op, false, true, init, (cudaStream_t)stream);
}

extern "C" int dr_scan_with_carry(const dr_view* in, dr_vec* out, int op, int exclusive, const void* dev_carry,
                                  dr_stream_t stream) {
  if (!dev_carry) {
    clear_error();
    return fail(DR_E_INVAL, "dr_scan_with_carry: NULL carry");
  }
  return do_scan("dr_scan_with_carry", in, out, op, false, exclusive != 0, nullptr, (cudaStream_t)stream, dev_carry);
}

extern "C" int dr_reverse_inclusive_scan(const dr_view* in, dr_vec* out, dr_stream_t stream) {
  return do_scan("dr_reverse_inclusive_scan", in, out, DR_PLUS, true, false, nullptr, (cudaStream_t)stream);
}

extern "C" int dr_transform_reduce(const dr_view* in_c, int op, const void* init, void* dev_result,
                                   dr_stream_t stream) {
  clear_error();
  const char* who = "dr_transform_reduce";
  if (int r = check_single(in_c, who)) return r;
  dr_view* in = const_cast<dr_view*>(in_c);
  if (op < DR_PLUS || op > DR_MAX) return fail(DR_E_INVAL, "%s: unknown op %d", who, op);
  if (!init || !dev_result) return fail(DR_E_INVAL, "%s: NULL init or result", who);
  if ((uintptr_t)dev_result % esize(in->dtype)) return fail(DR_E_ALIGN, "%s: result pointer misaligned", who);
  cudaStream_t s = (cudaStream_t)stream;
  static thread_local ReduceParams p;
  std::memset(&p, 0, sizeof p);
  p.vc = in->code();
  p.op = op;
  p.dtype = in->dtype;
  p.result = dev_result;
  std::memcpy(&p.init_bits, init, esize(in->dtype));
  if (int r = call_pieces(in, nullptr, reduce_tile_elems(in->dtype), p.pc, &p.pc_ext, &p.npieces, &p.ntiles, s))
    return r;
  const int grid = reduce_grid(in->dtype);
  if (int r = in->ws_reduce.ensure(reduce_ws_bytes(grid), s)) return r;
  p.ws = static_cast<char*>(in->ws_reduce.ptr);
  p.ws_partials = grid;
  p.status = status_word();
  if (!p.status) return fail(DR_E_CUDA, "%s: no device status word", who);
  cudaError_t e = launch_reduce(p, grid, s);
  in->ws_reduce.mark(s);
  return e == cudaSuccess ? DR_OK : cuda_fail(e, who);
}

extern "C" int dr_scale_by_partner(const dr_vec* x, const dr_vec* y, const float* dev_g, dr_vec* gx,
                                   dr_vec* gy, dr_stream_t stream) {
  clear_error();
  const char* who = "dr_scale_by_partner";
  if (!x || !y || !dev_g) return fail(DR_E_INVAL, "%s: NULL argument", who);
  if (!gx && !gy) return DR_OK;
  if (x->dtype != DR_F32 || y->dtype != DR_F32 || (gx && gx->dtype != DR_F32) || (gy && gy->dtype != DR_F32))
    return fail(DR_E_DTYPE, "%s: fp32 vectors only", who);
  const int64_t n = x->n;
  if (y->n != n || (gx && gx->n != n) || (gy && gy->n != n))
    return fail(DR_E_INVAL, "%s: vectors must have equal length", who);
  if (n == 0) return DR_OK;
  std::vector<std::vector<Seg>> ops = {x->window(0, n), y->window(0, n)};
  if (gx) ops.push_back(gx->window(0, n));
  if (gy) ops.push_back(gy->window(0, n));
  const std::vector<Piece> ps = resegment(ops, 4);
  if ((int)ps.size() > kMaxPieces) return fail(DR_E_UNSUPPORTED, "%s: more than %d pieces", who, kMaxPieces);
  static thread_local ScaleParams p;
  std::memset(&p, 0, sizeof p);
  p.g = dev_g;
  p.npieces = (int)ps.size();
  const int tile = scale_tile_elems();
  int64_t t = 0;
  for (size_t i = 0; i < ps.size(); ++i) {
    auto& k = p.pc[i];
    k.x = ps[i].p[0];
    k.y = ps[i].p[1];
    int o = 2;
    k.gx = gx ? ps[i].p[o++] : nullptr;
    k.gy = gy ? ps[i].p[o++] : nullptr;
    k.len = ps[i].len;
    k.tile_begin = t;
    k.vec_ok = (uintptr_t)k.x % 16 == 0 && (uintptr_t)k.y % 16 == 0 && (uintptr_t)k.gx % 16 == 0 &&
               (uintptr_t)k.gy % 16 == 0;
    t += (k.len + tile - 1) / tile;
  }
  p.ntiles = t;
  cudaError_t e = launch_scale(p, 0, (cudaStream_t)stream);
  return e == cudaSuccess ? DR_OK : cuda_fail(e, who);
}

// ---------------------------------------------------------------------------
// for_each over a k-ary zip, and transform
// ---------------------------------------------------------------------------
namespace {
struct FeSig {
  int arity, nargs;
  unsigned written;  // bit l: operand l is written
};
bool fe_sig(int fn, FeSig* s) {
  switch (fn) {
    case DR_FE_COPY: *s = {2, 0, 1u << 1}; return true;
    case DR_FE_SCALE: *s = {2, 1, 1u << 0}; return true;
    case DR_FE_ADD: *s = {3, 0, 1u << 2}; return true;
    case DR_FE_TRIAD: *s = {3, 1, 1u << 0}; return true;
    case DR_FE_BLACK_SCHOLES: *s = {5, 2, (1u << 3) | (1u << 4)}; return true;
  }
  return false;
}
}  // namespace

extern "C" int dr_for_each(const dr_view* zip, int fn, const double* args, int nargs, dr_stream_t stream) {
  clear_error();
  const char* who = "dr_for_each";
  if (!zip) return fail(DR_E_INVAL, "%s: NULL zip", who);
  FeSig sig;
  if (!fe_sig(fn, &sig)) return fail(DR_E_INVAL, "%s: unknown function %d", who, fn);
  if (zip->arity != sig.arity || zip->nleaf != sig.arity)
    return fail(DR_E_INVAL, "%s: function %d takes a zip of %d vectors (got arity %d)", who, fn, sig.arity,
                zip->arity);
  if (zip->dtype != DR_F32 && zip->dtype != DR_F64) return fail(DR_E_DTYPE, "%s: fp32 or fp64 only", who);
  if (nargs < sig.nargs || (sig.nargs > 0 && !args))
    return fail(DR_E_INVAL, "%s: function %d needs %d scalar arguments", who, fn, sig.nargs);
  const int esz = esize(zip->dtype);
  const_cast<dr_view*>(zip)->recompute();  // its vectors may have been rebound to new storage
  static thread_local ForEachParams p;
  std::memset(&p, 0, sizeof p);
  p.fn = fn;
  p.dtype = zip->dtype;
  for (int a = 0; a < sig.nargs; ++a) p.arg[a] = args[a];
  const int tile = foreach_tile_elems(zip->dtype);
  int64_t t = 0;
  std::vector<FePiece> tab;
  tab.reserve(zip->pieces.size());
  for (const Piece& q : zip->pieces) {
    if (q.len == 0) continue;
    for (int w = 0; w < sig.arity; ++w) {
      if (!(sig.written >> w & 1)) continue;
      for (int l = 0; l < sig.arity; ++l)
        if (l != w && partial_overlap(q.p[w], q.p[l], q.len * esz))
          return fail(DR_E_INVAL, "%s: written operand %d overlaps operand %d", who, w, l);
    }
    tab.emplace_back();
    FePiece& k = tab.back();
    bool al = true;
    for (int l = 0; l < sig.arity; ++l) {
      k.p[l] = q.p[l];
      al = al && (uintptr_t)q.p[l] % 16 == 0;
    }
    k.len = q.len;
    k.tile_begin = t;
    k.vec_ok = al;
    t += (q.len + tile - 1) / tile;
  }
  p.npieces = (int)tab.size();
  p.ntiles = t;
  if (t == 0) return DR_OK;
  p.status = status_word();
  if (!p.status) return fail(DR_E_CUDA, "%s: no device status word", who);
  if (int r = place_pieces(const_cast<dr_view*>(zip), tab, p.pc, &p.pc_ext, (cudaStream_t)stream)) return r;
  cudaError_t e = launch_for_each(p, (cudaStream_t)stream);
  return e == cudaSuccess ? DR_OK : cuda_fail(e, who);
}

extern "C" int dr_transform(const dr_view* in, dr_vec* out, dr_stream_t stream) {
  clear_error();
  const char* who = "dr_transform";
  if (int r = check_single(in, who)) return r;
  if (!out) return fail(DR_E_INVAL, "%s: NULL output", who);
  if (out->dtype != in->dtype) return fail(DR_E_DTYPE, "%s: output dtype differs from input", who);
  if (out->n < in->size)
    return fail(DR_E_INVAL, "%s: output has %lld elements, input %lld", who, (long long)out->n, (long long)in->size);
  if (in->size == 0) return DR_OK;
  static thread_local TransformParams p;
  std::memset(&p, 0, sizeof p);
  p.vc = in->code();
  p.dtype = in->dtype;
  const std::vector<KPiece> tab = build_pieces(in, out, foreach_tile_elems(in->dtype), &p.ntiles);
  const int esz = esize(in->dtype);
  for (const KPiece& k : tab) {
    if (partial_overlap(k.o, k.a, k.len * esz) || (k.b && partial_overlap(k.o, k.b, k.len * esz)))
      return fail(DR_E_INVAL, "%s: output overlaps an operand of the view", who);
  }
  p.npieces = (int)tab.size();
  p.status = status_word();
  if (!p.status) return fail(DR_E_CUDA, "%s: no device status word", who);
  if (int r = place_pieces(const_cast<dr_view*>(in), tab, p.pc, &p.pc_ext, (cudaStream_t)stream)) return r;
  cudaError_t e = launch_transform(p, (cudaStream_t)stream);
  return e == cudaSuccess ? DR_OK : cuda_fail(e, who);
}

extern "C" int dr_sort(const dr_view* in_c, dr_vec* out, dr_stream_t stream) {
  clear_error();
  const char* who = "dr_sort";
  if (int r = check_single(in_c, who)) return r;
  dr_view* in = const_cast<dr_view*>(in_c);
  if (!out) return fail(DR_E_INVAL, "%s: NULL output", who);
  if (out->dtype != in->dtype) return fail(DR_E_DTYPE, "%s: output dtype differs from input", who);
  if (out->n < in->size)
    return fail(DR_E_INVAL, "%s: output has %lld elements, input %lld", who, (long long)out->n, (long long)in->size);
  const int64_t n = in->size;
  if (n == 0) return DR_OK;
  if (n >= (int64_t(1) << 30)) return fail(DR_E_UNSUPPORTED, "%s: %lld elements (limit 2^30 - 1)", who, (long long)n);
  cudaStream_t s = (cudaStream_t)stream;
  static thread_local SortParams p;
  std::memset(&p, 0, sizeof p);
  p.vc = in->code();
  p.dtype = in->dtype;
  p.n = n;
  SortLaunch L{};
  if (int r = call_pieces(in, nullptr, sort_tile_elems(in->dtype), p.in, nullptr, &p.npin, &L.ntiles0, s)) return r;
  const std::vector<Seg> os = out->window(0, n);
  if ((int)os.size() > kMaxPieces) return fail(DR_E_UNSUPPORTED, "%s: output has more than %d segments", who, kMaxPieces);
  int64_t g = 0;
  for (size_t i = 0; i < os.size(); ++i) {
    p.out[i].p = os[i].p;
    p.out[i].start = g;
    g += os[i].len;
  }
  p.npout = (int)os.size();
  const int tile = sort_tile_elems(in->dtype), esz = esize(in->dtype);
  L.ntiles = (n + tile - 1) / tile;
  const int64_t maxt = std::max(L.ntiles0, L.ntiles);
  auto up = [](size_t b) { return (b + 255) / 256 * 256; };
  const int64_t ncounts = 256 * maxt;
  const size_t scan_b = up(scan_ws_bytes((ncounts + scan_tile_elems(DR_I32) - 1) / scan_tile_elems(DR_I32), DR_I32));
  const size_t counts_b = up((size_t)ncounts * 4), tmp_b = up((size_t)n * esz);
  // the scan's workspace comes first so that it keeps its (self-cleaning) state when
  // the workspace is reused; it is zeroed once, when allocated
  if (int r = in->ws_sort.ensure(scan_b + counts_b + 2 * tmp_b, s, scan_b)) return r;
  char* ws = static_cast<char*>(in->ws_sort.ptr);
  L.scan_ws = ws;
  p.counts = reinterpret_cast<unsigned*>(ws + scan_b);
  L.tmp[0] = ws + scan_b + counts_b;
  L.tmp[1] = L.tmp[0] + tmp_b;
  static thread_local ScanParams sp;
  L.scan = &sp;
  p.status = status_word();
  if (!p.status) return fail(DR_E_CUDA, "%s: no device status word", who);
  p.spin_limit = spin_limit();
  cudaError_t e = cudaSuccess;
  e = launch_sort(p, L, s);
  in->ws_sort.mark(s);
  return e == cudaSuccess ? DR_OK : cuda_fail(e, who);
}

static int do_stencil(const char* who, dr_md2* in, dr_md2* out, dr_md2* tmp, int steps, double wc, double wn,
                      cudaStream_t s, const dr_md2* prev = nullptr, double* acc = nullptr, int part = DR_ROWS_ALL) {
  clear_error();
  if (!in || !out) return fail(DR_E_INVAL, "%s: NULL array", who);
  if (steps < 1) return fail(DR_E_INVAL, "%s: steps must be >= 1", who);
  if (part < DR_ROWS_ALL || part > DR_ROWS_OUTER) return fail(DR_E_INVAL, "%s: unknown row part %d", who, part);
  if (steps > 1 && (in->ext_top || in->ext_bot))
    return fail(DR_E_INVAL, "%s: an array with external halos needs an exchange between steps: one step per call",
                who);
  if (out->ext_top != in->ext_top || out->ext_bot != in->ext_bot)
    return fail(DR_E_INVAL, "%s: in and out differ in their external halos", who);
  if (steps > 1 && !tmp) return fail(DR_E_INVAL, "%s: tmp is required when steps > 1", who);
  auto same = [&](const dr_md2* m) {
    return m->rows == in->rows && m->cols == in->cols && m->srows == in->srows;
  };
  if (!same(out) || (tmp && !same(tmp))) return fail(DR_E_INVAL, "%s: arrays differ in shape or blocking", who);
  if (in == out || in == tmp || out == tmp) return fail(DR_E_INVAL, "%s: in, out, tmp must be distinct", who);
  if (acc && (!prev || !same(prev) || steps != 1))
    return fail(DR_E_INVAL, "%s: needs one step and a forward state of the same shape", who);
  for (size_t k = 0; k < in->ptr.size(); ++k)
    if (out->ptr[k] == in->ptr[k] || (tmp && (tmp->ptr[k] == in->ptr[k] || tmp->ptr[k] == out->ptr[k])))
      return fail(DR_E_INVAL, "%s: in, out, tmp share storage", who);
  const int nseg = (int)in->ptr.size();
  int64_t nrb = 0;
  for (int k = 0; k < nseg; ++k) nrb += (in->srows[k] + kStencilRowsPerCta - 1) / kStencilRowsPerCta;
  if (nrb > 65535) return fail(DR_E_UNSUPPORTED, "%s: more than 65535 row blocks", who);
  if (int r = exchange_halos(in, s)) return r;
  static thread_local StencilParams p;
  bool vec = in->cols % 4 == 0;
  for (const dr_md2* m : {(const dr_md2*)in, (const dr_md2*)out, (const dr_md2*)tmp, prev})
    if (m)
      for (char* q : m->ptr) vec = vec && (uintptr_t)q % 16 == 0;
  const dr_md2* src = in;
  unsigned* status = status_word();
  if (!status) return fail(DR_E_CUDA, "%s: no device status word", who);
  for (int t = 0; t < steps; ++t) {
    dr_md2* dst = ((steps - 1 - t) % 2 == 0) ? out : tmp;
    std::memset(&p, 0, sizeof p);
    p.status = status;
    p.nseg = nseg;
    p.cols = in->cols;
    p.nrb = nrb;
    p.ext_top = in->ext_top;
    p.ext_bot = in->ext_bot;
    p.wc = (float)wc;
    p.wn = (float)wn;
    p.vec_ok = vec ? 1 : 0;
    p.acc = acc;
    int64_t rb = 0;
    for (int k = 0; k < nseg; ++k) {
      StencilSeg& g = p.seg[k];
      g.in = reinterpret_cast<const float*>(src->ptr[k]);
      g.prev = prev ? reinterpret_cast<const float*>(prev->ptr[k]) : nullptr;
      g.out = reinterpret_cast<float*>(dst->ptr[k]);
      g.out_prev = k > 0 ? reinterpret_cast<float*>(dst->ptr[k - 1]) : nullptr;
      g.out_next = k + 1 < nseg ? reinterpret_cast<float*>(dst->ptr[k + 1]) : nullptr;
      g.rows = in->srows[k];
      g.prev_rows = k > 0 ? in->srows[k - 1] : 0;
      g.rb_begin = rb;
      rb += (in->srows[k] + kStencilRowsPerCta - 1) / kStencilRowsPerCta;
    }
    // ALL: every row block; OUTER: the first and the last row block (the only ones
    // that read the outer ghost rows); INNER: the others
    int64_t nlaunch = nrb;
    if (part == DR_ROWS_OUTER) {
      p.outer_only = 1;
      nlaunch = nrb > 1 ? 2 : 1;
    } else if (part == DR_ROWS_INNER) {
      p.rb_lo = 1;
      nlaunch = nrb > 2 ? nrb - 2 : 0;
    }
    cudaError_t e = launch_stencil(p, nlaunch, s);
    if (e != cudaSuccess) return cuda_fail(e, who);
    src = dst;
  }
  return DR_OK;
}

extern "C" int dr_stencil5(dr_md2* in, dr_md2* out, dr_md2* tmp, int steps, double wc, double wn,
                           dr_stream_t stream) {
  return do_stencil("dr_stencil5", in, out, tmp, steps, wc, wn, (cudaStream_t)stream);
}

extern "C" int dr_stencil5_part(dr_md2* in, dr_md2* out, int part, double wc, double wn, dr_stream_t stream) {
  return do_stencil("dr_stencil5_part", in, out, nullptr, 1, wc, wn, (cudaStream_t)stream, nullptr, nullptr, part);
}

extern "C" int dr_md2_set_external_halos(dr_md2* m, int top, int bottom) {
  clear_error();
  if (!m) return fail(DR_E_INVAL, "dr_md2_set_external_halos: NULL array");
  m->ext_top = top ? 1 : 0;
  m->ext_bot = bottom ? 1 : 0;
  return DR_OK;
}

// A^T of the zero-ghost-ring 5-point operator: column (k,l) of A^T is row (k,l)
// of A, i.e. wc on the diagonal and wn on the in-grid neighbours, which is A.
extern "C" int dr_stencil5_T(dr_md2* in, dr_md2* out, dr_md2* tmp, int steps, double wc, double wn,
                             dr_stream_t stream) {
  return do_stencil("dr_stencil5_T", in, out, tmp, steps, wc, wn, (cudaStream_t)stream);
}

// One backward step of the stencil chain with the gradients of the weights:
// out = A^T in, acc[0] += <in, prev>, acc[1] += <N(in), prev>.
extern "C" int dr_stencil5_T_wgrad(dr_md2* in, dr_md2* out, const dr_md2* prev, double wc, double wn,
                                   double* dev_acc, dr_stream_t stream) {
  if (!dev_acc || (uintptr_t)dev_acc % 8) return fail(DR_E_INVAL, "dr_stencil5_T_wgrad: bad accumulator pointer");
  return do_stencil("dr_stencil5_T_wgrad", in, out, nullptr, 1, wc, wn, (cudaStream_t)stream, prev, dev_acc);
}
