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
    """Per-element bound |y_i - y*_i| <= gamma(6 T_i + 20) * S_i, T_i = 1 + tile index."""
    import numpy as np
    k = 6.0 * (np.asarray(tile_of_elem, dtype=np.float64) + 1.0) + 20.0
    return k * U32 / (1.0 - k * U32) * np.asarray(abs_prefix)


def stencil_f64_bound(steps: int, max_abs_u0: float) -> float:
    """fp32 vs FP64 after t steps: each step adds at most 3 roundings of values
    bounded by max|u0| (the 1/4-weighted update is a max-norm contraction)."""
    return 3.0 * steps * U32 * max_abs_u0


def black_scholes_bound(S, X, T, r, sigma, aux, u=U32):
    """First-order bound on |price - price*| for Black-Scholes evaluated in a
    precision with unit roundoff u (fp32: 2^-24) from the same inputs, against
    the FP64 values.  The kernel's quantities each carry a few roundings and
    one library call (log <= 1 ulp, exp <= 2 ulp, erfc <= 4 ulp for fp32; sqrt
    and division correctly rounded), so 8u bounds each one's relative error:
      d1:   E1 = 8u (1 + |ln(S/X)| + (r + sigma^2/2) T) / (sigma sqrt T) + 8u |d1|
      d2:   E2 = E1 + 8u sigma sqrt T
      N:    8u absolute (N = 1 - e or e with e = erfc(.)/2 <= 1/2)
      K = X e^{-rT}:  8u (1 + rT) K
    and a price S N(+-d1) -+ K N(+-d2) moves by at most the density times the
    argument's error plus N's own error, per term, plus the final 2 roundings.
    aux is the oracle's (phi(d1), phi(d2), d1, K) per option."""
    import numpy as np
    S, X, T = (np.asarray(v, np.float64) for v in (S, X, T))
    phi1, phi2, d1, K = aux[:, 0], aux[:, 1], aux[:, 2], aux[:, 3]
    s = sigma * np.sqrt(T)
    e1 = 8 * u * (1 + np.abs(np.log(S / X)) + (r + 0.5 * sigma * sigma) * T) / s + 8 * u * np.abs(d1)
    e2 = e1 + 8 * u * s
    eK = 8 * u * (1 + r * T) * K
    return S * (phi1 * e1 + 8 * u) + K * (phi2 * e2 + 8 * u) + eK + 4 * u * (S + K)
