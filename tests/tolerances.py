"""Rounding-error bounds for the fp32 results, derived from the kernels'
summation trees (standard results for recursive / blocked summation: a sum of
terms whose longest chain of dependent roundings has k adds has error at most
gamma_k * sum|terms|, gamma_k = k u / (1 - k u), u = 2^-24 for fp32).

reduce / dot (transform_reduce over zip | multiply): every thread keeps
V = 16 / sizeof(T) independent accumulation chains (one per lane of a 16-byte
vector), each taking RCH = 4 terms per tile (one FMA or add each) over the
tiles its CTA strides over; the V chains are then combined one after the
other (V - 1 roundings), then a warp (5 levels), the block's 8 warps (3
levels), and the last CTA folds the grid's partials (ceil(grid/256)
sequential, then 5 + 3 tree levels), plus init.  The grid is fixed: CTAs per
SM x SMs (capped at the tile count).

scan: inside a tile an element's prefix takes at most 3 (thread) + 5 (warp)
+ 5 (block) + 3 (offset combine) roundings; across tiles the carry is a chain
whose every hop (one tile) adds at most 5 (window reduce) + 1 (own
aggregate) roundings of partial sums bounded by the prefix's |x| sum.
"""
import math

U32 = 2.0 ** -24
U64 = 2.0 ** -53


def gamma(k: int, u: float = U32) -> float:
    return k * u / (1.0 - k * u)


def reduce_chain(n: int, sms: int, esize: int = 4, ctas_per_sm: int = 4, threads: int = 256,
                 rch: int = 4) -> int:
    """Longest chain of dependent roundings in the reduce kernel's tree."""
    v = 16 // esize
    tile = threads * rch * v
    ntiles = max(1, -(-n // tile))
    grid = min(sms * ctas_per_sm, ntiles)
    per_cta = -(-ntiles // grid)
    return per_cta * rch + (v - 1) + 5 + 3 + (-(-grid // threads)) + 5 + 3 + 1


def dot_chain(n: int, sms: int) -> int:
    return reduce_chain(n, sms, 4)


def dot_bound(n: int, abs_sum: float, sms: int) -> float:
    return gamma(dot_chain(n, sms)) * abs_sum


def reduce_bound(n: int, abs_sum: float, sms: int, esize: int) -> float:
    """|computed - exact| for a PLUS reduce of n elements of a float type of
    esize bytes (u = 2^-24 for fp32, 2^-53 for fp64), scaled by sum |x|."""
    u = U32 if esize == 4 else U64
    return gamma(reduce_chain(n, sms, esize), u) * abs_sum


def scan_bound(abs_prefix, tile_of_elem):
    """Per-element bound |y_i - y*_i| <= gamma(7 T_i + 20) * S_i, T_i = 1 + tile index,
    S_i the prefix of |x|: the longest chain of dependent fp32 roundings any input
    passes through on its way to y_i, counted for the scan kernels.  Inside a tile:
    thread scan (<= 3), warp scan (5), the block scan of the chunk totals (<= 7),
    the carry-in and the element's own add (2): <= 20.  An input of an earlier tile:
    its tile's aggregate (a reduction tree: thread 3, chunk tree <= 3, warp 5, block
    5 = 16), then per lookback hop the 5-level warp reduction of the window, the
    combine with the running carry and the published inclusive prefix (7), at most
    one hop per tile, and 4 roundings carrying the prefix into the output:
    16 + 1 + 7 (T - 1) + 4 <= 7 T + 20."""
    import numpy as np
    k = 7.0 * (np.asarray(tile_of_elem, dtype=np.float64) + 1.0) + 20.0
    return k * U32 / (1.0 - k * U32) * np.asarray(abs_prefix)


def stencil_f64_bound(steps: int, max_abs_u0: float) -> float:
    """fp32 vs FP64 after t steps: each step adds at most 3 roundings of values
    bounded by max|u0| (the 1/4-weighted update is a max-norm contraction)."""
    return 3.0 * steps * U32 * max_abs_u0


def black_scholes_bound(S, X, T, r, sigma, aux, u=U32):
    """First-order bound on |price - price*| for the library's Black-Scholes
    element function evaluated with unit roundoff u on the same inputs, against
    the FP64 prices.  Derived for the fp32 kernel's arithmetic (fp64, u = 2^-53,
    calls log / exp / sqrt / erfc, which are within these budgets too):

      q = S / X          __fdividef: 2 ulp                      -> rel 4u
      lnr = log2(q) ln2  __log2f: abs 2^-22.6 on [0.5, 2], else 2 ulp; the
                         multiply by ln2 (constant rounded):
                         |err| <= A = ln2 2^-22.6 + 4u + 6u |ln q|
      num = fma(drift, T, lnr)  drift = r + sigma^2/2 in two roundings
                         (rel 2u); the fma rounds once: |err| <= A + 2u drift T + u |num|
      m = (1/sigma) rsqrtf(T)   division 1u, rsqrtf 2 ulp (4u), product 1u -> rel 6u
      d1 = num m         E1 = (A + 2u drift T) / (sigma sqrt T) + 8u |d1|
      sv = sigma T rsqrtf(T)    rel 6u;  d2 = d1 - sv:  E2 = E1 + 6u sv + u |d2|
      K = X __expf(-rT)  __expf: (2 + floor(1.173 rT)) ulp, rT rounded, product
                         -> E_K = u (5 + 3.4 rT) K
      N(-x), x = |d|     Zelen-Severo (Abramowitz & Stegun 26.2.17): absolute
                         7.5e-8 in exact arithmetic; its fp32 evaluation
                         (t = __fdividef(1, fma(p, x, 1)), phi via __expf with
                         (2 + 1.173 x^2/2) ulp, four Horner fmas, rounded
                         coefficients) is within rel (64 + 3 x^2) u of its
                         value e <= min(1/2, phi(x) / x); N(x) = 1 - e adds u:
                         E_N = 7.5e-8 + u + (64 + 3 x^2) u min(1/2, phi(x) / x)
      C = S N(d1) - K N(d2), P = K N(-d2) - S N(-d1): each price moves by at most
      S (phi(d1) E1 + E_N(d1)) + K (phi(d2) E2 + E_N(d2)) + E_K, plus the two
      products and the subtraction: 2u (S + K).
    aux is the oracle's (phi(d1), phi(d2), d1, K) per option."""
    import numpy as np
    S, X, T = (np.asarray(v, np.float64) for v in (S, X, T))
    phi1, phi2, d1, K = aux[:, 0], aux[:, 1], aux[:, 2], aux[:, 3]
    sq = np.sqrt(T)
    sv = sigma * sq
    d2 = d1 - sv
    drift = r + 0.5 * sigma * sigma
    A = math.log(2.0) * 2.0 ** -22.6 + 4 * u + 6 * u * np.abs(np.log(S / X))
    e1 = (A + 2 * u * drift * T) / sv + 8 * u * np.abs(d1)
    e2 = e1 + 6 * u * sv + u * np.abs(d2)
    eK = u * (5 + 3.4 * r * T) * K

    def e_n(d, phi):
        x = np.abs(d)
        tail = np.minimum(0.5, np.where(x > 0, phi / np.maximum(x, 1e-300), 0.5))
        return 7.5e-8 + u + (64 + 3 * x * x) * u * tail

    return S * (phi1 * e1 + e_n(d1, phi1)) + K * (phi2 * e2 + e_n(d2, phi2)) + eK + 2 * u * (S + K)
