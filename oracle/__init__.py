"""CPU oracle for the segmented-range hot path (arXiv 2406.00158).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by ``__graft_entry__.smoke()``
and by the benchmark's CPU-baseline / reference leg, never by the product path.
It shares no code with the CUDA library.

The heavy functions are plain sequential C++ (``dr_oracle.cpp``) loaded with
ctypes; the zip re-segmentation oracle is a brute-force Python loop over
element ownership (small inputs only).  Each function cites the passage it
follows; see ``dr_oracle.cpp`` for the arithmetic.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from fractions import Fraction

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dr_oracle.cpp")
_LIB = os.path.join(_HERE, "libdr_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with g++ (no fast-math, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-ffp-contract=off",
                               "-fno-fast-math", _SRC, "-o", tmp])
        os.replace(tmp, _LIB)
    return _LIB


_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_SIGS = {
    "oracle_inclusive_scan_i64": (None, [_P, _I64, _P]),
    "oracle_inclusive_scan_f32_f64": (None, [_P, _I64, _P, _P]),
    "oracle_inclusive_scan_f64": (None, [_P, _I64, _P]),
    "oracle_inclusive_scan_f32_seq": (None, [_P, _I64, _P]),
    "oracle_segmented_scan_alg4_i64": (None, [ctypes.c_int, _P, _P, _P]),
    "oracle_reverse_inclusive_scan_f64": (None, [_P, _I64, _P]),
    "oracle_dot_f64": (None, [_P, _P, _I64, _P, _P]),
    "oracle_segmented_reduce_alg3_i64": (_I64, [ctypes.c_int, _P, _P]),
    "oracle_dot_adjoint_f64": (None, [_P, _P, _I64, ctypes.c_double, _P, _P]),
    "oracle_stencil5_f64": (None, [_P, _I64, _I64, ctypes.c_int, ctypes.c_double, ctypes.c_double, _P]),
    "oracle_stencil5_f32": (None, [_P, _I64, _I64, ctypes.c_int, ctypes.c_float, ctypes.c_float, _P]),
    "oracle_stencil5_f32_at": (None, [_P, _I64, _I64, ctypes.c_int, ctypes.c_float, ctypes.c_float,
                                      _P, _I64, _P]),
    "oracle_stencil5_f64_at": (None, [_P, _I64, _I64, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                      _P, _I64, _P]),
    "oracle_stencil5_T_f64": (None, [_P, _I64, _I64, ctypes.c_int, ctypes.c_double, ctypes.c_double, _P]),
    "oracle_stream_f32": (None, [ctypes.c_int, _I64, _P, _P, _P, ctypes.c_float]),
    "oracle_stream_f64": (None, [ctypes.c_int, _I64, _P, _P, _P, ctypes.c_double]),
    "oracle_black_scholes_f64": (None, [_I64, _P, _P, _P, ctypes.c_double, ctypes.c_double, _P, _P, _P]),
    "oracle_sort_f32": (None, [_P, _I64]),
    "oracle_sort_f64": (None, [_P, _I64]),
    "oracle_sort_i32": (None, [_P, _I64]),
    "oracle_sort_i64": (None, [_P, _I64]),
    "oracle_partition_sort_i64": (None, [ctypes.c_int, _P, _P, _P]),
    "oracle_scan_i64": (None, [_P, _I64, ctypes.c_int, ctypes.c_int, ctypes.c_int64, _P]),
    "oracle_scan_i32": (None, [_P, _I64, ctypes.c_int, ctypes.c_int, ctypes.c_int32, _P]),
    "oracle_scan_f64": (None, [_P, _I64, ctypes.c_int, ctypes.c_int, ctypes.c_double, _P]),
    "oracle_reduce_i64": (ctypes.c_int64, [_P, _I64, ctypes.c_int, ctypes.c_int64]),
    "oracle_reduce_i32": (ctypes.c_int32, [_P, _I64, ctypes.c_int, ctypes.c_int32]),
    "oracle_reduce_f64": (ctypes.c_double, [_P, _I64, ctypes.c_int, ctypes.c_double]),
    "oracle_sum_expansion_f64": (_I64, [_P, _I64, _P, _I64]),
}


def lib():
    global _lib
    with _lock:
        if _lib is None:
            l = ctypes.CDLL(build())
            for name, (res, args) in _SIGS.items():
                f = getattr(l, name)
                f.restype = res
                f.argtypes = args
            _lib = l
    return _lib


def _c(a: np.ndarray, dtype) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=dtype)


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


# ---------------------------------------------------------------------------
# inclusive_scan over the concatenation of segments (Sec. 3 "Distributed Range";
# Sec. 4.3 "inclusive_scan")
# ---------------------------------------------------------------------------

def inclusive_scan_i64(x) -> np.ndarray:
    x = _c(x, np.int64)
    y = np.empty_like(x)
    lib().oracle_inclusive_scan_i64(_p(x), x.size, _p(y))
    return y


def inclusive_scan_f32_f64(x):
    """FP64 sequential scan of fp32 input; returns (y, abs_prefix)."""
    x = _c(x, np.float32)
    y = np.empty(x.size, np.float64)
    a = np.empty(x.size, np.float64)
    lib().oracle_inclusive_scan_f32_f64(_p(x), x.size, _p(y), _p(a))
    return y, a


def inclusive_scan_f64(x) -> np.ndarray:
    x = _c(x, np.float64)
    y = np.empty_like(x)
    lib().oracle_inclusive_scan_f64(_p(x), x.size, _p(y))
    return y


def inclusive_scan_f32_seq(x) -> np.ndarray:
    x = _c(x, np.float32)
    y = np.empty_like(x)
    lib().oracle_inclusive_scan_f32_seq(_p(x), x.size, _p(y))
    return y


def segmented_scan_alg4_i64(lens, x) -> np.ndarray:
    """Algorithm 4 step by step (local scans, partial sums, offsets)."""
    lens = _c(lens, np.int64)
    x = _c(x, np.int64)
    assert int(lens.sum()) == x.size
    y = np.empty_like(x)
    lib().oracle_segmented_scan_alg4_i64(int(lens.size), _p(lens), _p(x), _p(y))
    return y


def reverse_inclusive_scan_f64(g) -> np.ndarray:
    """Adjoint of inclusive_scan: out[j] = sum_{i>=j} g[i]."""
    g = _c(g, np.float64)
    out = np.empty_like(g)
    lib().oracle_reverse_inclusive_scan_f64(_p(g), g.size, _p(out))
    return out


# ---------------------------------------------------------------------------
# transform_reduce(zip(x, y), multiply, plus) -- Algorithm 1 / Algorithm 3
# ---------------------------------------------------------------------------

def dot_f64(x, y):
    """Returns (dot, sum |x_i y_i|) in FP64."""
    x = _c(x, np.float32)
    y = _c(y, np.float32)
    assert x.size == y.size
    d = ctypes.c_double()
    a = ctypes.c_double()
    lib().oracle_dot_f64(_p(x), _p(y), x.size, ctypes.byref(d), ctypes.byref(a))
    return d.value, a.value


def segmented_reduce_alg3_i64(lens, x) -> int:
    lens = _c(lens, np.int64)
    x = _c(x, np.int64)
    return int(lib().oracle_segmented_reduce_alg3_i64(int(lens.size), _p(lens), _p(x)))


def dot_adjoint_f64(x, y, g: float):
    x = _c(x, np.float32)
    y = _c(y, np.float32)
    gx = np.empty(x.size, np.float64)
    gy = np.empty(x.size, np.float64)
    lib().oracle_dot_adjoint_f64(_p(x), _p(y), x.size, float(g), _p(gx), _p(gy))
    return gx, gy


# ---------------------------------------------------------------------------
# 5-point Jacobi stencil (zero outside the grid) and its transpose
# ---------------------------------------------------------------------------

def stencil5_f64(u0, steps: int, wc: float = 0.0, wn: float = 0.25) -> np.ndarray:
    u0 = _c(u0, np.float64)
    R, C = u0.shape
    out = np.empty_like(u0)
    lib().oracle_stencil5_f64(_p(u0), R, C, int(steps), float(wc), float(wn), _p(out))
    return out


def stencil5_f32(u0, steps: int, wc: float = 0.0, wn: float = 0.25) -> np.ndarray:
    """fp32, fixed evaluation order ((N+S)+(W+E))*wn [+ wc*C]."""
    u0 = _c(u0, np.float32)
    R, C = u0.shape
    out = np.empty_like(u0)
    lib().oracle_stencil5_f32(_p(u0), R, C, int(steps), float(wc), float(wn), _p(out))
    return out


def stencil5_f32_at(u0, steps: int, cells, wc: float = 0.0, wn: float = 0.25) -> np.ndarray:
    u0 = _c(u0, np.float32)
    R, C = u0.shape
    cells = _c(cells, np.int64).reshape(-1, 2)
    out = np.empty(cells.shape[0], np.float32)
    lib().oracle_stencil5_f32_at(_p(u0), R, C, int(steps), float(wc), float(wn), _p(cells),
                                 cells.shape[0], _p(out))
    return out


def stencil5_f64_at(u0, steps: int, cells, wc: float = 0.0, wn: float = 0.25) -> np.ndarray:
    u0 = _c(u0, np.float64)
    R, C = u0.shape
    cells = _c(cells, np.int64).reshape(-1, 2)
    out = np.empty(cells.shape[0], np.float64)
    lib().oracle_stencil5_f64_at(_p(u0), R, C, int(steps), float(wc), float(wn), _p(cells),
                                 cells.shape[0], _p(out))
    return out


def stencil5_T_f64(v0, steps: int, wc: float = 0.0, wn: float = 0.25) -> np.ndarray:
    v0 = _c(v0, np.float64)
    R, C = v0.shape
    out = np.empty_like(v0)
    lib().oracle_stencil5_T_f64(_p(v0), R, C, int(steps), float(wc), float(wn), _p(out))
    return out


# ---------------------------------------------------------------------------
# zip re-segmentation (Sec. 4.4 "Zip"), brute force over element ownership
# ---------------------------------------------------------------------------

def zip_segments_bruteforce(lens_a, lens_b):
    """For each global index i < min(|a|, |b|) find (segment of a, segment of b)
    holding element i; the zipped segments are the maximal runs of indices with
    the same pair.  Returns a list of (seg_a, off_in_a, seg_b, off_in_b, length).
    Empty segments own no index and produce no piece.  Pure-Python loop: small
    inputs only."""
    def owners(lens):
        out = []
        for k, L in enumerate(lens):
            out.extend((k, j) for j in range(int(L)))
        return out

    oa, ob = owners(lens_a), owners(lens_b)
    n = min(len(oa), len(ob))
    pieces = []
    for i in range(n):
        (ka, ja), (kb, jb) = oa[i], ob[i]
        if pieces and pieces[-1][0] == ka and pieces[-1][2] == kb:
            p = pieces[-1]
            pieces[-1] = (p[0], p[1], p[2], p[3], p[4] + 1)
        else:
            pieces.append((ka, ja, kb, jb, 1))
    return pieces


def zip_segments_bruteforce_k(lens_list):
    """k-ary form of zip_segments_bruteforce: the maximal runs of global indices
    whose k owners (segment of each operand) stay the same.  Returns a list of
    (segs, offs, length) with segs / offs k-tuples.  Small inputs only."""
    owners = []
    for lens in lens_list:
        o = []
        for k, L in enumerate(lens):
            o.extend((k, j) for j in range(int(L)))
        owners.append(o)
    n = min(len(o) for o in owners)
    pieces = []
    for i in range(n):
        segs = tuple(o[i][0] for o in owners)
        if pieces and pieces[-1][0] == segs:
            pieces[-1] = (segs, pieces[-1][1], pieces[-1][2] + 1)
        else:
            pieces.append((segs, tuple(o[i][1] for o in owners), 1))
    return pieces


# ---------------------------------------------------------------------------
# central finite differences in FP64 (gradient checks)
# ---------------------------------------------------------------------------

def fd_gradient(loss, x, h: float = 2.0 ** -10) -> np.ndarray:
    """g_j = (L(x + h e_j) - L(x - h e_j)) / (2h), FP64, one coordinate at a time."""
    x = np.array(x, dtype=np.float64)
    g = np.empty(x.size)
    flat = x.reshape(-1)
    for j in range(flat.size):
        old = flat[j]
        flat[j] = old + h
        lp = loss(x)
        flat[j] = old - h
        lm = loss(x)
        flat[j] = old
        g[j] = (lp - lm) / (2.0 * h)
    return g.reshape(x.shape)


# ---------------------------------------------------------------------------
# for_each element functions (Sec. 4.3 "for_each"; Sec. 5 STREAM, Black-Scholes)
# ---------------------------------------------------------------------------

STREAM_FNS = {"copy": 0, "scale": 1, "add": 2, "triad": 3}


def stream(fn: str, a, b, c, q: float = 0.0):
    """One STREAM kernel over zip(a, b, c) in the arrays' dtype (fp32 or fp64),
    one rounding per operation: copy c=a; scale b=q*c; add c=a+b; triad a=b+q*c.
    Returns new arrays (a, b, c) with the written one updated."""
    dt = np.asarray(a).dtype
    assert dt in (np.float32, np.float64)
    a, b, c = (np.array(v, dtype=dt, copy=True) for v in (a, b, c))
    assert a.size == b.size == c.size
    f = lib().oracle_stream_f32 if dt == np.float32 else lib().oracle_stream_f64
    f(STREAM_FNS[fn], a.size, _p(a), _p(b), _p(c), float(q))
    return a, b, c


def black_scholes_f64(S, X, T, r: float, sigma: float, aux: bool = False):
    """European call and put prices in FP64.  With aux=True also returns an
    (n, 4) array of (phi(d1), phi(d2), d1, X e^{-rT}) for error bounds."""
    S, X, T = (_c(v, np.float64) for v in (S, X, T))
    assert S.size == X.size == T.size
    call = np.empty_like(S)
    put = np.empty_like(S)
    ax = np.empty((S.size, 4), np.float64) if aux else None
    lib().oracle_black_scholes_f64(S.size, _p(S), _p(X), _p(T), float(r), float(sigma), _p(call), _p(put),
                                   _p(ax) if aux else None)
    return (call, put, ax) if aux else (call, put)


# ---------------------------------------------------------------------------
# sort (Sec. 4.3 "sort")
# ---------------------------------------------------------------------------

_SORTS = {np.dtype(np.float32): "oracle_sort_f32", np.dtype(np.float64): "oracle_sort_f64",
          np.dtype(np.int32): "oracle_sort_i32", np.dtype(np.int64): "oracle_sort_i64"}


def sort(x) -> np.ndarray:
    """Ascending sort of the concatenation; floats in IEEE totalOrder."""
    x = np.array(x, copy=True)
    getattr(lib(), _SORTS[x.dtype])(_p(x), x.size)
    return x


def partition_sort_i64(lens, x) -> np.ndarray:
    """The paper's distributed partition sort, step by step (int64)."""
    lens = _c(lens, np.int64)
    x = _c(x, np.int64)
    assert int(lens.sum()) == x.size
    out = np.empty_like(x)
    lib().oracle_partition_sort_i64(int(lens.size), _p(lens), _p(x), _p(out))
    return out


# ---------------------------------------------------------------------------
# the other associative operators (Sec. 4.3: the footnote to "reduce"; the last
# paragraph of "inclusive_scan" for exclusive_scan)
# ---------------------------------------------------------------------------

OPS = {"plus": 0, "mul": 1, "min": 2, "max": 3}


def identity(op: str, dtype):
    """The identity element of op for an element type (min / max: the type's
    largest / lowest value, infinities for floats)."""
    dt = np.dtype(dtype)
    if op == "plus":
        return dt.type(0)
    if op == "mul":
        return dt.type(1)
    if np.issubdtype(dt, np.floating):
        return dt.type(np.inf if op == "min" else -np.inf)
    info = np.iinfo(dt)
    return dt.type(info.max if op == "min" else info.min)


def scan(x, op: str = "plus", exclusive: bool = False, init=None):
    """Sequential scan of the concatenation with op in {plus, min, max}:
    inclusive y_i = init op x_0 op ... op x_i (init defaults to the identity),
    exclusive y_0 = init, y_i = init op x_0 op ... op x_{i-1}.  int64 / int32
    wrap for plus; fp32 / fp64 run in FP64 (plus rounds in FP64 at every step,
    min / max select exactly) and return FP64."""
    x = np.asarray(x)
    if init is None:
        init = identity(op, x.dtype)
    mode = 1 if exclusive else 0
    if x.dtype == np.int64:
        xc = _c(x, np.int64)
        y = np.empty_like(xc)
        lib().oracle_scan_i64(_p(xc), xc.size, OPS[op], mode, int(init), _p(y))
    elif x.dtype == np.int32:
        xc = _c(x, np.int32)
        y = np.empty_like(xc)
        lib().oracle_scan_i32(_p(xc), xc.size, OPS[op], mode, int(init), _p(y))
    else:
        xc = _c(x, np.float64)
        y = np.empty_like(xc)
        lib().oracle_scan_f64(_p(xc), xc.size, OPS[op], mode, float(init), _p(y))
    return y


def reduce(x, op: str = "plus", init=None):
    """init op x_0 op ... op x_{n-1} over the concatenation (Algorithm 3's
    result).  Integers: exact (wrapping plus / multiply).  Floats: min / max
    exact; plus returns the EXACT sum as a Fraction (see sum_exact)."""
    x = np.asarray(x)
    if init is None:
        init = identity(op, x.dtype)
    if x.dtype == np.int64:
        xc = _c(x, np.int64)
        return int(lib().oracle_reduce_i64(_p(xc), xc.size, OPS[op], int(init)))
    if x.dtype == np.int32:
        xc = _c(x, np.int32)
        return int(lib().oracle_reduce_i32(_p(xc), xc.size, OPS[op], int(init)))
    if op == "plus":
        return sum_exact(np.concatenate([[float(init)], np.asarray(x, np.float64)]))
    xc = _c(x, np.float64)
    return float(lib().oracle_reduce_f64(_p(xc), xc.size, OPS[op], float(init)))


def sum_exact(x) -> Fraction:
    """The exact sum of the doubles x (a rational): the oracle builds a
    non-overlapping expansion with error-free two-sums (Shewchuk's
    Grow-Expansion) and the expansion's terms are added as Fractions."""
    xc = _c(x, np.float64)
    cap = 2100  # a double expansion has at most ~2098 non-overlapping terms
    parts = np.empty(cap, np.float64)
    k = lib().oracle_sum_expansion_f64(_p(xc), xc.size, _p(parts), cap)
    assert k >= 0
    return sum((Fraction(float(v)) for v in parts[:k]), Fraction(0))


# ---------------------------------------------------------------------------
# take / drop (Sec. 4.4 "Take and Drop": both trim the segment list)
# ---------------------------------------------------------------------------

def trim_segments(lens, f: int, l: int):
    """The segments of a range restricted to its elements [f, l): for every
    segment k covering global indices [s_k, s_k + len_k), the part inside
    [f, l) as (k, offset in segment k, length); segments left empty are
    dropped.  Bounds are clamped to [0, n]."""
    n = int(sum(int(v) for v in lens))
    f = max(0, min(int(f), n))
    l = max(f, min(int(l), n))
    out, s = [], 0
    for k, L in enumerate(lens):
        L = int(L)
        a, b = max(f, s), min(l, s + L)
        if b > a:
            out.append((k, a - s, b - a))
        s += L
    return out


def take_segments(lens, l: int):
    """take(l): the first l elements (trim to [0, l))."""
    return trim_segments(lens, 0, l)


def drop_segments(lens, f: int):
    """drop(f): all but the first f elements (trim to [f, n))."""
    return trim_segments(lens, f, sum(int(v) for v in lens))


def gather_segments(x, lens, pieces):
    """The elements of the concatenation x (segment sizes lens) that the pieces
    (segment, offset, length) name, in order."""
    starts = np.concatenate([[0], np.cumsum(np.asarray(lens, np.int64))])
    parts = [np.asarray(x)[starts[k] + o: starts[k] + o + L] for k, o, L in pieces]
    return np.concatenate(parts) if parts else np.asarray(x)[:0]
