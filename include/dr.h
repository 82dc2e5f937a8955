/*
 * dr.h -- C ABI of a GB300-native (sm_103a) implementation of the data-parallel
 * hot path of the Distributed Ranges model (Brock, Cohn, et al., arXiv 2406.00158).
 *
 * Model (Sec. 3): a *distributed range* is a range split into *segments*; each
 * segment is a *remote range* living in one memory locale, and the segments
 * concatenated in order form the whole range.  Here every memory locale is a
 * separate allocation in one GPU's HBM, so a segment is just (device pointer,
 * length).  Containers are built over caller-given segments, *views* are
 * composed lazily (Sec. 4.4: transform, zip of two or k ranges, take / drop)
 * and algorithms (Sec. 4.3: inclusive / exclusive scan, reduce /
 * transform_reduce, for_each, transform, sort; and the 5-point stencil over a
 * row-block array) run over a composition with the view fused into the
 * kernel's loads and stores.  Adjoints (reverse scan, scale-by-partner,
 * transposed stencil) and a batched persistent launch complete the set.
 *
 * Conventions for every entry point:
 *   - Returns an int status (enum dr_status); never throws or aborts across
 *     the ABI.  On failure, dr_last_error() gives a message for this thread.
 *   - Device memory is OWNED BY THE CALLER and never freed by the library.
 *     Handles (dr_vec, dr_md2, dr_view, dr_batch) are owned by the library from
 *     *_create / *_plan until the matching *_destroy.
 *   - Views are non-owning (Sec. 4.4): a view must not outlive the containers
 *     (or views) it was built from.
 *   - Every GPU call is asynchronous on the stream it is given (NULL = the
 *     legacy default stream) and uses the calling thread's current CUDA device.
 *     Device-side failures (a bounded wait that expired) are recorded in a
 *     per-device status word that dr_sync_status() reads and clears.
 *   - A handle that carries device workspace (views passed to algorithms,
 *     batch plans) must not be used by two calls that can overlap on the GPU.
 *     A view's workspace is freed, when the view is destroyed, in the order of
 *     the stream its latest call used: destroy a view before that stream.
 *   - Element types: fp32, fp64, int64, int32.  Integer arithmetic wraps mod
 *     2^bits; floating-point arithmetic is IEEE round-to-nearest, no fast-math.
 */
#ifndef DR_GB300_H
#define DR_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same type as cudaStream_t; NULL is the legacy default stream. */
typedef struct CUstream_st* dr_stream_t;

enum dr_status {
  DR_OK = 0,
  DR_E_INVAL = 1,       /* bad argument: null pointer, negative size, size mismatch */
  DR_E_DTYPE = 2,       /* unsupported or mismatched element type / operation */
  DR_E_ALIGN = 3,       /* pointer not aligned to its element size, or a non-aligned
                           zip where strict alignment was requested (Sec. 4.3) */
  DR_E_CUDA = 4,        /* a CUDA runtime call failed (message has the CUDA error) */
  DR_E_TIMEOUT = 5,     /* a bounded device-side wait expired (see dr_set_spin_limit) */
  DR_E_BOUNDS = 6,      /* index out of range */
  DR_E_NOMEM = 7,       /* workspace allocation failed */
  DR_E_UNSUPPORTED = 8  /* composition or size outside what this build supports */
};

enum dr_dtype { DR_F32 = 0, DR_F64 = 1, DR_I64 = 2, DR_I32 = 3 };

/* Associative binary operations (scan / reduce operators, zip combiners).
 * Sec. 4.3 (footnote to "reduce") allows any such operator; PLUS is the one
 * of Algorithms 1, 3 and 4. */
enum dr_binop { DR_PLUS = 0, DR_MUL = 1, DR_MIN = 2, DR_MAX = 3 };

/* Elementwise functions of a transform view (Sec. 4.4 "Transform");
 * `arg` is the scalar a. */
enum dr_unop {
  DR_U_SCALE = 0,  /* a * x */
  DR_U_ADD = 1,    /* x + a */
  DR_U_NEG = 2,    /* -x */
  DR_U_ABS = 3,    /* |x| */
  DR_U_SQUARE = 4  /* x * x */
};

typedef struct dr_vec dr_vec;
typedef struct dr_md2 dr_md2;
typedef struct dr_view dr_view;
typedef struct dr_batch dr_batch;

/* One piece of a view's segmentation, as reported by dr_view_segments: the
 * piece covers `len` consecutive elements of the view starting at global index
 * `start`; for each operand k (k < arity) it lies in segment seg[k] of that
 * operand's container, starting at element off[k] of that segment. */
typedef struct dr_piece {
  int64_t start;
  int64_t len;
  int32_t seg[2];
  int64_t off[2];
} dr_piece;

/* Launch shape of the batched kernel (chosen by the autotuner or the caller).
 * variant 0: one tile per CTA in registers; threads 128, 256 or 512; items 8 or 16.
 * variant 1: lookahead pipeline with TMA-staged x and p; threads 256; items 12, 16 or 32. */
typedef struct dr_tune {
  int32_t threads;      /* threads per CTA */
  int32_t items;        /* elements per thread per tile (fp32) */
  int32_t ctas_per_sm;  /* persistent CTAs per SM: 1..8 (capped by occupancy) */
  int32_t variant;      /* kernel variant, see above */
} dr_tune;

/* ------------------------------------------------------------------------ */
/* Library status                                                            */
/* ------------------------------------------------------------------------ */

/* Message of the last failed call on this thread (never NULL; "" if none). */
const char* dr_last_error(void);

/* ABI version, currently 1. */
int dr_version(void);

/* Synchronizes `stream`, then reads and clears the current device's status
 * word.  Returns DR_OK, DR_E_TIMEOUT (a bounded wait expired in a kernel
 * launched earlier on this device; its results are invalid) or DR_E_CUDA. */
int dr_sync_status(dr_stream_t stream);

/* Tile geometry of a kernel family (host only; no device needed):
 *   *tile_elems = the elements of `dtype` one tile covers -- the unit of the
 *     scan's carry chain (one lookback hop per tile; DR_K_SCAN_VIEW: the scan
 *     of a fused view -- ops or a zip -- whose tiles are shorter), of the reduce's
 *     per-thread accumulation, of for_each / transform and of a sort pass;
 *   *ctas_per_sm = the CTAs per SM of the kernel's grid when it is fixed by
 *     design (the reduce: its grid fixes the summation tree), else 0 (a
 *     persistent grid sized by occupancy).
 * Either output may be NULL.  Rounding-error bounds are derived from these. */
enum dr_kernel_family { DR_K_SCAN = 0, DR_K_REDUCE = 1, DR_K_FOREACH = 2, DR_K_SORT = 3, DR_K_SCAN_VIEW = 4 };
int dr_kernel_geometry(int kernel, int dtype, int64_t* tile_elems, int* ctas_per_sm);

/* Upper bound on the polls of every device-side wait (scan lookback, batched
 * carry); each poll sleeps at most ~1 us.  Default 1<<21 (~1-2 s).  polls>=1. */
int dr_set_spin_limit(int64_t polls);

/* Test hook for the bounded-wait path: the next scan launch skips publishing
 * the status of tile `tile` (so its successors' waits expire and report
 * DR_E_TIMEOUT instead of hanging).  tile < 0 disarms.  Not for production. */
int dr_debug_skip_publish(int64_t tile);

/* ------------------------------------------------------------------------ */
/* Segmented vector (Sec. 4.2.1 "Distributed Vector")                        */
/* ------------------------------------------------------------------------ */

/* Block partition of Sec. 4.2.1: p segments of ceil(n/p) elements, the last
 * ones shorter or empty.  Writes p lengths to lens_out.  Host only. */
int dr_block_lengths(int64_t n, int p, int64_t* lens_out);

/* Builds a segmented vector over nseg caller-owned device segments:
 * segment k holds lens[k] >= 0 elements of `dtype` at seg_ptrs[k] (which may
 * be NULL only if lens[k] == 0 and must be aligned to the element size;
 * 16-byte alignment enables 128-bit access).  The global order is segment 0,
 * then 1, ... (the concatenation of Sec. 3).  nseg >= 1.  Host only: the
 * pointers are recorded, not dereferenced. */
int dr_vec_create(int dtype, int nseg, const int64_t* lens, void* const* seg_ptrs, dr_vec** out);
int dr_vec_destroy(dr_vec* v);

/* Points the vector's segments at new storage of the same lengths (seg_ptrs:
 * one device pointer per segment, rules as for dr_vec_create).  Views built on
 * the vector follow it -- their next call uses the new storage -- and keep the
 * device workspaces they allocated, so a caller that runs an algorithm on a new
 * set of equally shaped tensors every step (an autograd function, a training
 * loop) allocates no workspace after the first step.  Launches already made
 * keep the storage they were given.  Host only. */
int dr_vec_rebind(dr_vec* v, void* const* seg_ptrs);

/* Shape queries (host only). */
int dr_vec_info(const dr_vec* v, int* dtype, int* nseg, int64_t* n);
int dr_vec_segment(const dr_vec* v, int k, void** ptr, int64_t* len, int64_t* start);

/* Global index arithmetic of operator[] (Sec. 4.2): element i of the vector is
 * element *off of segment *seg.  DR_E_BOUNDS unless 0 <= i < n.  Host only. */
int dr_vec_locate(const dr_vec* v, int64_t i, int* seg, int64_t* off);

/* Copies the whole vector from / to a contiguous host buffer of n elements
 * (pinned memory makes the copies asynchronous), one cudaMemcpyAsync per
 * segment, on `stream` (Sec. 4.1: copy into and out of remote memory). */
int dr_vec_copy_from_host(dr_vec* v, const void* host, dr_stream_t stream);
int dr_vec_copy_to_host(const dr_vec* v, void* host, dr_stream_t stream);

/* ------------------------------------------------------------------------ */
/* Row-block segmented 2-D array (Sec. 4.2.2 "Distributed Matrix", block_row  */
/* partition) with one ghost (halo) row above and below every segment.        */
/* ------------------------------------------------------------------------ */

/* rows x cols array in nseg row blocks; block k has seg_rows[k] >= 1 rows and
 * seg_ptrs[k] points to (seg_rows[k] + 2) * cols contiguous elements: row 0 is
 * the top ghost row, rows 1..seg_rows[k] the block's own rows, row
 * seg_rows[k]+1 the bottom ghost row.  sum(seg_rows) == rows.  Only DR_F32.
 * Ghost rows hold copies of the neighbouring blocks' boundary rows; the
 * ghosts at the two outer edges of the grid are never read (the grid is zero
 * outside).  The library rewrites ghost rows of any array it operates on. */
int dr_md2_create(int dtype, int64_t rows, int64_t cols, int nseg, const int64_t* seg_rows,
                  void* const* seg_ptrs, dr_md2** out);
int dr_md2_destroy(dr_md2* m);

/* Halo exchange: copies each block's first / last own row into the ghost row
 * of the neighbouring block, on `stream`. */
int dr_md2_exchange_halos(dr_md2* m, dr_stream_t stream);

/* ------------------------------------------------------------------------ */
/* Views (Sec. 4.4).  Lazy, non-owning, composable.                          */
/* ------------------------------------------------------------------------ */

/* The view of a whole vector. */
int dr_view_of(const dr_vec* v, dr_view** out);

/* transform: applies `op` (enum dr_unop, scalar `arg`) to every element of a
 * single-valued view.  Its segments are the base's segments, transformed. */
int dr_view_transform(const dr_view* base, int op, double arg, dr_view** out);

/* zip of two single-valued views of the same dtype: element i is the pair
 * (a_i, b_i), length min(|a|, |b|).  If the operands are not aligned (same
 * segment count and sizes) the segments are re-cut at the union of both
 * operands' boundaries (Sec. 4.4 "Zip").  A zip is not single-valued until a
 * binary function is applied with dr_view_zip_transform. */
int dr_view_zip(const dr_view* a, const dr_view* b, dr_view** out);

/* zip with flags.  DR_ZIP_STRICT_ALIGN refuses operands that are not aligned
 * with DR_E_ALIGN instead of re-cutting them: the distributed-memory runtime of
 * Sec. 4.3 ("inclusive_scan") and Sec. 4.4 ("Zip") prohibits zips of
 * non-aligned ranges, where aligned means the same number of segments with
 * corresponding segments of the same size (and memory locale; here every
 * segment is in one GPU's memory).  The segments compared are those the views
 * cover (after take / drop), empty segments not counted.  flags 0 is
 * dr_view_zip. */
#define DR_ZIP_STRICT_ALIGN 1
int dr_view_zip_ex(const dr_view* a, const dr_view* b, int flags, dr_view** out);

/* transform of a zip with a binary function: element i = op(a_i, b_i), e.g.
 * DR_MUL for the dot product of Algorithm 1. */
int dr_view_zip_transform(const dr_view* zip, int op, dr_view** out);

/* k-ary zip (Sec. 4.4 "Zip" over k ranges; 2 <= k <= DR_MAX_ZIP) of
 * untransformed views (dr_view_of, possibly trimmed by take / drop) of one
 * dtype: element i is the k-tuple of the operands' i-th elements, length the
 * shortest operand's; the segments are re-cut at the union of all operands'
 * boundaries.  Its elements are references: dr_for_each writes through them.
 * `leaves` is a host array of k views; the zip refers to their vectors, not to
 * the leaf handles, which may be destroyed afterwards. */
#define DR_MAX_ZIP 6
int dr_view_zipn(int k, const dr_view* const* leaves, dr_view** out);

/* take / drop (Sec. 4.4 "Take and Drop"): the first l elements, or all but the
 * first f, via trimmed segments.  l and f are clamped to [0, size]. */
int dr_view_take(const dr_view* base, int64_t l, dr_view** out);
int dr_view_drop(const dr_view* base, int64_t f, dr_view** out);

int dr_view_destroy(dr_view* v);

/* Queries (host only): size, arity (1 for single-valued, k for a raw k-ary
 * zip), element type, number of pieces of the (re-)segmentation, and the
 * pieces (dr_piece reports the first two operands of a zip). */
int dr_view_info(const dr_view* v, int64_t* size, int* arity, int* dtype, int* npieces);
int dr_view_segments(const dr_view* v, int max_pieces, dr_piece* out);

/* ------------------------------------------------------------------------ */
/* Algorithms (Sec. 4.3)                                                      */
/* ------------------------------------------------------------------------ */

/* inclusive_scan (Sec. 4.3, Algorithm 4): out_i = in_0 op in_1 op ... op in_i
 * over the whole range, across segment boundaries, op in {PLUS, MIN, MAX}.
 * `in` is single-valued; `out` has in's dtype and at least |in| elements; out
 * may be the same storage as in's base vector (in place).  Single pass: each
 * tile's carry comes from its predecessors' published aggregates (decoupled
 * lookback) instead of Algorithm 4's second pass over the data.  The first
 * call on a view allocates its workspace (do it outside stream capture). */
int dr_inclusive_scan(const dr_view* in, dr_vec* out, int op, dr_stream_t stream);

/* exclusive_scan (Sec. 4.3, last paragraph of "inclusive_scan"): out_0 = init,
 * out_i = init op in_0 op ... op in_{i-1}.  `init` points to one host value of
 * the view's dtype. */
int dr_exclusive_scan(const dr_view* in, dr_vec* out, int op, const void* init,
                      dr_stream_t stream);

/* Scan with a carry-in read from device memory.  Algorithm 4 (Sec. 4.3) adds
 * to each segment the total of everything before it; when the segments before
 * this range live on other GPUs (a range sharded over ranks), that total
 * arrives as a device value, e.g. from a collective, and is passed here
 * without a host round trip.  op in {PLUS, MIN, MAX}.
 *   exclusive == 0: out_i = carry op in_0 op ... op in_i
 *   exclusive != 0: out_0 = carry, out_i = carry op in_0 op ... op in_{i-1}
 * dev_carry: one element of the view's dtype in device memory, aligned to its
 * size, read by the kernel (so earlier work on `stream` may produce it).
 * Otherwise as dr_inclusive_scan (same kernel, same workspace rules). */
int dr_scan_with_carry(const dr_view* in, dr_vec* out, int op, int exclusive, const void* dev_carry,
                       dr_stream_t stream);

/* Reverse inclusive scan: out_j = in_j + in_{j+1} + ... + in_{n-1}.  This is
 * the adjoint of the PLUS inclusive scan (gradient of y = scan(x) is
 * x_bar = reverse_scan(y_bar)). */
int dr_reverse_inclusive_scan(const dr_view* in, dr_vec* out, dr_stream_t stream);

/* reduce / transform_reduce (Sec. 4.3, Algorithm 3; Algorithm 1's dot product
 * is transform_reduce over zip_transform(zip(x, y), MUL) with PLUS):
 * *dev_result = init op in_0 op ... op in_{n-1}.  `init` points to one host
 * value of the view's dtype; dev_result to one device element.  One kernel:
 * per-CTA partials combined by the last CTA in a fixed order (deterministic
 * for a given device).  Workspace as for dr_inclusive_scan. */
int dr_transform_reduce(const dr_view* in, int op, const void* init, void* dev_result,
                        dr_stream_t stream);

/* for_each (Sec. 4.3 "for_each") over a raw k-ary zip with a built-in element
 * function; Sec. 5's STREAM and Black-Scholes benchmarks are for_each over a
 * zip of their arrays.  The roles of the zip's operands, in order:
 *   DR_FE_COPY          zip(a, c):           c = a
 *   DR_FE_SCALE         zip(b, c):           b = q * c              args {q}
 *   DR_FE_ADD           zip(a, b, c):        c = a + b
 *   DR_FE_TRIAD         zip(a, b, c):        a = b + q * c          args {q}
 *   DR_FE_BLACK_SCHOLES zip(S, X, T, C, P):  C, P = European call and put
 *                       prices under the Black-Scholes-Merton model for spot S,
 *                       strike X, expiry T (years)     args {r, sigma}
 * dtype fp32 or fp64; args (nargs >= the function's count) are host doubles
 * converted to the dtype.  STREAM functions round once per operation (no
 * fused multiply-add), so results are bit-exact against a plain loop in the
 * dtype.  Black-Scholes in fp64 calls CUDA's log, exp, sqrt and erfc; in fp32
 * it uses the hardware approximations of division, log2, exp and 1/sqrt and
 * the Zelen-Severo polynomial for the normal CDF (Abramowitz & Stegun 26.2.17,
 * absolute error < 7.5e-8), every intermediate within 8 ulp of exact.
 * A written operand may be the very same elements as another operand
 * (in place, e.g. zip(b, b) for b = q * b); any other overlap between a
 * written operand and another operand is DR_E_INVAL.  One launch, no
 * workspace, graph-capturable. */
enum dr_foreach_fn {
  DR_FE_COPY = 0,
  DR_FE_SCALE = 1,
  DR_FE_ADD = 2,
  DR_FE_TRIAD = 3,
  DR_FE_BLACK_SCHOLES = 4
};
int dr_for_each(const dr_view* zip, int fn, const double* args, int nargs, dr_stream_t stream);

/* transform / copy of a view into a vector (Sec. 4.3: algorithms write their
 * results through a range; Sec. 4.4: views are lazy until then):
 * out_i = in_i for i < |in|, with in's fused transform / zip_transform chain
 * evaluated in the load.  `out` has in's dtype and at least |in| elements; it
 * may be the very storage of one of in's operands (in place); other overlap
 * is DR_E_INVAL.  One launch, no workspace, graph-capturable. */
int dr_transform(const dr_view* in, dr_vec* out, dr_stream_t stream);

/* sort (Sec. 4.3 "sort"): out_0 <= out_1 <= ... <= out_{n-1} are the n = |in|
 * elements of the single-valued view `in` (its transforms evaluated) in
 * ascending order, written over out's segments (its first n elements).
 * Integers by value; fp32 / fp64 by the IEEE 754 totalOrder (-NaN < -inf <
 * ... < -0 < +0 < ... < +inf < +NaN, NaNs by payload), so the result is
 * unique bit for bit.  out may be the storage of in's vector (in place, as
 * C++'s sort).  n <= 2^30 - 1 (DR_E_UNSUPPORTED beyond).  The paper sorts with
 * a distributed partition sort (sampled splitters, per-chunk counts,
 * redistribution, local sorts); on one GPU the partition is a radix pass, so
 * this is a least-significant-digit radix sort over the segment table: one
 * histogram read plus one pass per 8-bit digit (4 passes for 32-bit keys, 8 for
 * 64-bit), each pass one kernel with decoupled lookback.  The view's workspace
 * holds two scratch copies of the keys plus counters (allocated by the first
 * call, as for dr_inclusive_scan); each call clears its counters on `stream`. */
int dr_sort(const dr_view* in, dr_vec* out, dr_stream_t stream);

/* The dot product of dr_transform_reduce(zip(x, y) | DR_MUL, DR_PLUS) for callers
 * that cannot allocate device memory at the call (a framework that owns all device
 * memory through its own pool; a latency-critical loop that cannot pay for
 * cudaMalloc, or for the device-wide synchronization of cudaFree).  The paper has
 * no counterpart: this is an allocation-free variant of the same reduce kernel.
 * x and y share one segmentation: segment k has lens[k] >= 0 fp32 elements at
 * x_segs[k] and y_segs[k] (device pointers, 4-byte aligned; 16-byte aligned for
 * 128-bit access; host arrays of nseg entries, 1 <= nseg <= 128).
 * *dev_result = init + sum_i x_i*y_i (one device fp32).  Its scratch (32,832
 * bytes: a counter header and one partial per CTA) is a fixed device array of
 * the library, present on every device that loads it until the process exits;
 * nothing is allocated.  The first call on a device looks up that array's
 * device address (make it before any stream capture).  Every call shares the
 * array: each clears its counter header on `stream` first, and calls that can
 * overlap on the GPU race.  DR_E_UNSUPPORTED if nseg > 128 or the device needs
 * more than 4096 CTAs' partials. */
int dr_dot_f32_noalloc(int nseg, const int64_t* lens, const float* const* x_segs,
                       const float* const* y_segs, float init, float* dev_result,
                       dr_stream_t stream);

/* Adjoint of d = <x, y> (dot product): gx = g * y and gy = g * x elementwise,
 * with g read from device memory (dev_g, one fp32).  Either output may be
 * NULL.  fp32 vectors of equal length; segmentations may differ. */
int dr_scale_by_partner(const dr_vec* x, const dr_vec* y, const float* dev_g, dr_vec* gx,
                        dr_vec* gy, dr_stream_t stream);

/* for_each with a 5-point Jacobi update (a halo-exchanging stencil over the
 * row-block array; Sec. 4.3 "for_each" over Sec. 4.2.2's block-row matrix):
 *   u'[i][j] = wc*u[i][j] + wn*(u[i-1][j] + u[i+1][j] + u[i][j-1] + u[i][j+1])
 * on every cell, with u = 0 outside the grid, evaluated in fp32 as
 * s = (N + S) + (W + E); r = wn*s; if wc != 0: r = r + wc*C (no fusion).
 * Runs `steps` >= 1 steps from `in`; the result lands in `out`; `tmp` (same
 * shape; may be NULL when steps == 1) holds intermediate states.  The first
 * step re-exchanges in's halos; every step writes its blocks' boundary rows
 * into the neighbours' ghost rows of its output.  in, out, tmp distinct. */
int dr_stencil5(dr_md2* in, dr_md2* out, dr_md2* tmp, int steps, double wc, double wn,
                dr_stream_t stream);

/* Marks a row-block array as one rank's share of a taller grid split by rows
 * over several GPUs (Sec. 4.2.2's block_row partition with blocks on
 * different memory locales): with top (bottom) != 0 the first block's top
 * (the last block's bottom) ghost row holds the row just above (below) the
 * share -- written by the caller before each step, e.g. received from the
 * neighbouring rank -- and the stencil reads it instead of the zero outside the
 * grid.  Default: both 0 (the array is the whole grid).  Such an array is
 * stepped one step per call (the caller exchanges the outer rows in between);
 * in and out of a call must agree on these flags.  Host only. */
int dr_md2_set_external_halos(dr_md2* m, int top, int bottom);

/* One step of dr_stencil5 restricted to a part of the row blocks (64 rows
 * each, per block), so that an exchange of the outer ghost rows can overlap
 * the update of the rows that do not read them:
 *   DR_ROWS_ALL   every row block (= dr_stencil5 with steps == 1);
 *   DR_ROWS_INNER all but the array's first and last row block;
 *   DR_ROWS_OUTER the first and the last row block (the only ones that read
 *                 the outer ghost rows).
 * INNER then OUTER (or OUTER then INNER) on one stream is one full step. */
enum dr_rows_part { DR_ROWS_ALL = 0, DR_ROWS_INNER = 1, DR_ROWS_OUTER = 2 };
int dr_stencil5_part(dr_md2* in, dr_md2* out, int part, double wc, double wn, dr_stream_t stream);

/* The transposed operator A^T applied `steps` times (adjoint of dr_stencil5
 * for the gradient w.r.t. the initial state).  With a zero ghost ring the
 * operator is symmetric, so this runs the same update. */
int dr_stencil5_T(dr_md2* in, dr_md2* out, dr_md2* tmp, int steps, double wc, double wn,
                  dr_stream_t stream);

/* One backward step of the stencil chain that also yields the gradients of
 * the weights.  With u_t = wc*u_{t-1} + wn*N(u_{t-1}) (N = sum of the 4
 * neighbours) and in = u_bar_t (the gradient w.r.t. u_t): out = A^T in
 * (= u_bar_{t-1}), and, with prev = the forward state u_{t-1},
 *   dev_acc[0] += <u_bar_t, u_{t-1}>      (dL/dwc contribution of step t)
 *   dev_acc[1] += <N(u_bar_t), u_{t-1}>   (dL/dwn contribution; N is symmetric)
 * accumulated in FP64 (fp32 per-thread partials, one FP64 atomic per CTA and
 * accumulator).  prev's ghost rows are not read.  dev_acc: 2 device doubles. */
int dr_stencil5_T_wgrad(dr_md2* in, dr_md2* out, const dr_md2* prev, double wc, double wn,
                        double* dev_acc, dr_stream_t stream);

/* ------------------------------------------------------------------------ */
/* Batched execution: many independent segmented vectors in one launch        */
/* ------------------------------------------------------------------------ */

/* Plans y_v = inclusive_scan(x_v) and dots[v] = <x_v, p_v> (PLUS) for nvec
 * independent fp32 vectors in ONE persistent launch.  x[v], p[v], y[v] are
 * vectors of equal length (segmentations may differ); dev_dots has nvec fp32
 * slots.  `tune` NULL = the default launch shape (see dr_batch_set_tune).  The
 * plan allocates its device tables and workspace. */
int dr_batch_plan(int nvec, const dr_vec* const* x, const dr_vec* const* p, dr_vec* const* y,
                  float* dev_dots, const dr_tune* tune, dr_batch** out);
int dr_batch_destroy(dr_batch* b);

/* Changes the launch shape (invalidates a captured graph). */
int dr_batch_set_tune(dr_batch* b, const dr_tune* tune);
int dr_batch_get_tune(const dr_batch* b, dr_tune* tune);

/* Runs the plan: one kernel launch, no allocation, no synchronization (safe to
 * capture into a CUDA graph). */
int dr_batch_run(dr_batch* b, dr_stream_t stream);

/* Captures dr_batch_run into a CUDA graph once (on a private stream) and
 * replays it on `stream`. */
int dr_batch_run_graph(dr_batch* b, dr_stream_t stream);

/* Baseline: the same work as one dr_inclusive_scan-kernel launch plus one
 * transform_reduce-kernel launch per vector (2*nvec launches). */
int dr_batch_run_per_range(dr_batch* b, dr_stream_t stream);

/* The same 2*nvec launches captured once into a CUDA graph (on a private
 * stream; the first call captures, later calls replay on `stream`): the
 * per-range baseline without the host's per-launch cost, which separates the
 * persistent launch's gain from saved launch overhead. */
int dr_batch_run_per_range_graph(dr_batch* b, dr_stream_t stream);

/* Autotuner: times every candidate launch shape on the plan `calib` (its
 * inputs must be initialized; its outputs are overwritten), picks the fastest
 * and stores it in the JSON cache at cache_path (NULL = $DR_TUNE_CACHE, else
 * no file), keyed by device name, SM count and a size bucket of the plan.
 * mode 0: use a cached entry if present, else tune; mode 1: always re-tune.
 * Writes the choice to *chosen and applies it to `calib`. */
int dr_batch_autotune(dr_batch* calib, int mode, const char* cache_path, dr_tune* chosen);

#ifdef __cplusplus
}
#endif

#endif /* DR_GB300_H */
