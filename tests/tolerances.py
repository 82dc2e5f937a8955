"""Rounding-error bounds for the fp32 results, derived from the kernels'
summation trees (standard results for recursive / blocked summation: a sum of
terms whose longest chain of dependent roundings has k adds has error at most
gamma_k * sum|terms|, gamma_k = k u / (1 - k u), u = 2^-24 for fp32).

dot (transform_reduce over zip | multiply): every thread accumulates V=4
independent FMA chains over its tiles (RCH=4 terms per tile per chain), then
the 4 chains (2 levels), a warp (5 levels), the block's 8 warps (3 levels),
and the last CTA folds the grid's partials (ceil(grid/256) sequential, then 8
tree levels), plus init.

scan: inside a tile an element's prefix takes at most 3 (thread) + 5 (warp)
+ 5 (block) + 3 (offset combine) roundings; across tiles the carry is a chain
whose every hop (one tile) adds at most 5 (window reduce) + 1 (own
aggregate) roundings of partial sums bounded by the prefix's |x| sum.
"""
import math

U32 = 2.0 ** -24


def gamma(k: int, u: float = U32) -> float:
    return k * u / (1.0 - k * u)


def dot_chain(n: int, sms: int, tile: int = 4096, ctas_per_sm: int = 4, threads: int = 256) -> int:
    grid = sms * ctas_per_sm
    ntiles = max(1, -(-n // tile))
    per_cta = -(-ntiles // grid)
    return per_cta * 4 + 2 + 5 + 3 + (-(-grid // threads)) + 5 + 3 + 1


def dot_bound(n: int, abs_sum: float, sms: int) -> float:
    return gamma(dot_chain(n, sms)) * abs_sum


def scan_bound(abs_prefix, tile_of_elem):
    """Per-element bound |y_i - y*_i| <= gamma(6 T_i + 20) * S_i, T_i = 1 + tile index."""
    import numpy as np
    k = 6.0 * (np.asarray(tile_of_elem, dtype=np.float64) + 1.0) + 20.0
    return k * U32 / (1.0 - k * U32) * np.asarray(abs_prefix)


def stencil_f64_bound(steps: int, max_abs_u0: float) -> float:
    """fp32 vs FP64 after t steps: each step adds at most 3 roundings of values
    bounded by max|u0| (the 1/4-weighted update is a max-norm contraction)."""
    return 3.0 * steps * U32 * max_abs_u0
