"""Seeded synthetic inputs shared by the CUDA path's callers and the CPU oracle's tests.

This module holds no arithmetic of the segmented-range method itself: it only
draws numbers.  Every draw comes from one counter-based generator, SplitMix64
(G. L. Steele, D. Lea, C. H. Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014; the public-domain ``splitmix64.c`` of S. Vigna):

    r_i(key) = mix64(key + (i + 1) * 0x9E3779B97F4A7C15)   (mod 2^64)
    mix64(z) = z ^= z >> 30; z *= 0xBF58476D1CE4E5B9;
               z ^= z >> 27; z *= 0x94D049BB133111EB; z ^ (z >> 31)

so ``r_i(key)`` is the i-th output of a SplitMix64 stream seeded with ``key``.
Values are derived from ``r`` only through exact integer / power-of-two maps:

* integers in [lo, hi):  lo + ((r >> 32) * (hi - lo)) >> 32
* fp32 in [0, 1):        (r >> 40) * 2^-24      (exact in fp32)
* fp32 in [-1, 1):       (r >> 40) * 2^-23 - 1  (exact in fp32)

The paper's benchmarks are synthetic (dot product, scan, STREAM-style
kernels; no dataset), so these draws are the whole input recipe.
"""
from __future__ import annotations

import math
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np

GOLDEN_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_CHUNK = 1 << 21

# Seeds of the five workloads (base 2406 + index; one stream per array).
SEED_SCAN_I64 = 2406
SEED_DOT_X = 2407
SEED_DOT_Y = 2408
SEED_STENCIL = 2409
SEED_GRAD = 2410
SEED_BATCH = 2411     # batch shapes
SEED_BATCH_X = 3411   # batch values x
SEED_BATCH_P = 4411   # batch partner values p
SEED_STREAM = 2412    # STREAM arrays a, b, c: streams 2412, 2413, 2414
SEED_BS = 2415        # Black-Scholes S, X, T: streams 2415, 2416, 2417
SEED_SORT = 2418      # sort keys

# Black-Scholes option batch (the paper gives no sizes or ranges): spot S in
# [5, 30), strike X in [1, 100), expiry T in [0.25, 10) years, fp32; rate and
# volatility are scalars (r = 0.02, sigma = 0.30 rounded to fp32).
BS_S_RANGE = (5.0, 30.0)
BS_X_RANGE = (1.0, 100.0)
BS_T_RANGE = (0.25, 10.0)
BS_R = 0.02
BS_SIGMA = 0.30


def _mix64(z: np.ndarray) -> np.ndarray:
    z = z ^ (z >> np.uint64(30))
    z = z * _M1
    z = z ^ (z >> np.uint64(27))
    z = z * _M2
    return z ^ (z >> np.uint64(31))


def _raw_chunk(key: int, start: int, count: int) -> np.ndarray:
    i = np.arange(start + 1, start + 1 + count, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return _mix64(np.uint64(key & 0xFFFFFFFFFFFFFFFF) + i * GOLDEN_GAMMA)


def _fill(n: int, dtype, fn) -> np.ndarray:
    """Evaluate ``fn(start, count) -> array`` over [0, n) in chunks, in threads."""
    out = np.empty(n, dtype=dtype)
    if n <= _CHUNK:
        if n:
            out[:] = fn(0, n)
        return out
    starts = range(0, n, _CHUNK)

    def work(s):
        c = min(_CHUNK, n - s)
        out[s:s + c] = fn(s, c)

    with ThreadPoolExecutor(max_workers=min(32, os.cpu_count() or 1)) as ex:
        list(ex.map(work, starts))
    return out


def raw_u64(key: int, n: int, start: int = 0) -> np.ndarray:
    """The raw SplitMix64 outputs r_start .. r_{start+n-1} of stream ``key``."""
    return _fill(n, np.uint64, lambda s, c: _raw_chunk(key, start + s, c))


def uniform_int64(key: int, n: int, lo: int = 0, hi: int = 1000) -> np.ndarray:
    span = np.uint64(hi - lo)

    def f(s, c):
        r = _raw_chunk(key, s, c) >> np.uint64(32)
        with np.errstate(over="ignore"):
            return ((r * span) >> np.uint64(32)).astype(np.int64) + lo

    return _fill(n, np.int64, f)


def uniform01_f32(key: int, n: int) -> np.ndarray:
    return _fill(n, np.float32, lambda s, c: (
        (_raw_chunk(key, s, c) >> np.uint64(40)).astype(np.float32) * np.float32(2.0 ** -24)))


def uniform_pm1_f32(key: int, n: int) -> np.ndarray:
    return _fill(n, np.float32, lambda s, c: (
        (_raw_chunk(key, s, c) >> np.uint64(40)).astype(np.float32) * np.float32(2.0 ** -23)
        - np.float32(1.0)))


def uniform01_f64(key: int, n: int) -> np.ndarray:
    """Doubles in [0, 1) with 53 random bits: (r >> 11) * 2^-53."""
    return _fill(n, np.float64, lambda s, c: (
        (_raw_chunk(key, s, c) >> np.uint64(11)).astype(np.float64) * 2.0 ** -53))


# ----------------------------------------------------------------------------------
# Segmentations
# ----------------------------------------------------------------------------------

def proportional_segments(n: int, weights) -> list[int]:
    """Split n into len(weights) segment sizes proportional to ``weights``
    (floor of each share, remainder added to the last)."""
    w = [int(x) for x in weights]
    tot = sum(w)
    sizes = [n * x // tot for x in w]
    sizes[-1] += n - sum(sizes)
    return sizes


def block_segments(n: int, p: int) -> list[int]:
    """Block partition of n over p locales: ceil(n/p) each, the tail shorter
    (possibly empty) -- the distributed vector's default layout."""
    b = -(-n // p) if p else 0
    out = []
    left = n
    for _ in range(p):
        out.append(min(b, left))
        left -= out[-1]
    return out


def random_cut_segments(key: int, n: int, nseg: int) -> list[int]:
    """Cut [0, n) at nseg-1 distinct points drawn uniformly from [1, n-1]
    (rejection of repeats; fewer cuts when n is too small)."""
    want = max(0, min(nseg - 1, n - 1))
    cuts: list[int] = []
    seen = set()
    i = 0
    while len(cuts) < want:
        r = int(raw_u64(key, 1, start=i)[0])
        i += 1
        c = 1 + ((r >> 32) * (n - 1) >> 32)
        if c not in seen:
            seen.add(c)
            cuts.append(c)
    cuts.sort()
    edges = [0] + cuts + [n]
    return [edges[k + 1] - edges[k] for k in range(len(edges) - 1)]


def batch_shapes(key: int, nvec: int, lo: float = 1e3, hi: float = 1e6, max_seg: int = 8):
    """Shapes of a batch of independent segmented vectors: for vector v,
    length L = round(exp(U(ln lo, ln hi))) and s ~ U{1..max_seg} segments cut at
    s-1 distinct uniform points.  Returns a list of per-vector segment-size lists."""
    shapes = []
    la, lb = math.log(lo), math.log(hi)
    for v in range(nvec):
        vkey = key ^ ((v + 1) << 32)
        r = raw_u64(vkey, 2)
        u = float(int(r[0]) >> 11) * 2.0 ** -53
        L = int(round(math.exp(la + u * (lb - la))))
        s = 1 + ((int(r[1]) >> 32) * max_seg >> 32)
        shapes.append(random_cut_segments(vkey ^ 0x5EC5, L, s))
    return shapes


def black_scholes_inputs(n: int, key: int = SEED_BS):
    """fp32 arrays (S, X, T) of n options: lo + (hi - lo) * U[0, 1) per range,
    evaluated in fp32."""
    out = []
    for j, (lo, hi) in enumerate((BS_S_RANGE, BS_X_RANGE, BS_T_RANGE)):
        u = uniform01_f32(key + j, n)
        out.append((np.float32(lo) + np.float32(hi - lo) * u).astype(np.float32))
    return tuple(out)


def stream_inputs(n: int, dtype=np.float64, key: int = SEED_STREAM):
    """STREAM arrays (a, b, c), values in [-1, 1)."""
    if dtype == np.float32:
        return tuple(uniform_pm1_f32(key + j, n) for j in range(3))
    return tuple(2.0 * uniform01_f64(key + j, n) - 1.0 for j in range(3))
