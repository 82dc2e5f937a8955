"""Pins of the CPU oracle against facts fixed outside the oracle itself:
closed forms, brute force on tiny inputs, exact special cases, invariants and
adjoint identities.  Each test is chosen so that a plausible slip in the oracle
(a dropped term, an off-by-one, a wrong sign or transposed index, a wrong
boundary) fails it.  CPU only."""
import itertools
import os
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_2406_00158_gb300 import inputs

RNG_KEY = 99


# ----------------------------------------------------------------------------------
# inclusive_scan, int64 (plain definition: y_i = x_0 + ... + x_i)
# ----------------------------------------------------------------------------------

@pytest.mark.parametrize("n", [0, 1, 2, 7, 4097])
def test_scan_i64_ones_is_iota(n):
    y = oracle.inclusive_scan_i64(np.ones(n, np.int64))
    assert np.array_equal(y, np.arange(1, n + 1, dtype=np.int64))


def test_scan_i64_arange_closed_form():
    n = 100_003
    y = oracle.inclusive_scan_i64(np.arange(n, dtype=np.int64))
    i = np.arange(n, dtype=np.int64)
    assert np.array_equal(y, i * (i + 1) // 2)
    assert int(y[-1]) == n * (n - 1) // 2


def test_scan_i64_bruteforce_tiny():
    x = inputs.uniform_int64(RNG_KEY, 8, -10**12, 10**12)
    for n in range(9):
        y = oracle.inclusive_scan_i64(x[:n])
        for i in range(n):
            assert int(y[i]) == sum(int(v) for v in x[:i + 1])


def test_scan_i64_wraps_mod_2_64():
    big = np.array([2**62, 2**62, 2**62, -5], dtype=np.int64)
    y = oracle.inclusive_scan_i64(big)

    def wrap(v):
        v %= 2**64
        return v - 2**64 if v >= 2**63 else v

    for i in range(4):
        assert int(y[i]) == wrap(sum(int(v) for v in big[:i + 1]))


def _compositions(n, parts_max=4):
    """All ways to cut n into 1..parts_max ordered segments, empty segments allowed."""
    for k in range(1, parts_max + 1):
        for cuts in itertools.combinations_with_replacement(range(n + 1), k - 1):
            edges = (0,) + cuts + (n,)
            yield [edges[i + 1] - edges[i] for i in range(k)]


@pytest.mark.parametrize("n", [0, 1, 5, 8])
def test_alg4_segmented_scan_equals_definition_all_splits(n):
    x = inputs.uniform_int64(RNG_KEY + n, n, 0, 1000)
    ref = oracle.inclusive_scan_i64(x)
    for lens in _compositions(n):
        assert np.array_equal(oracle.segmented_scan_alg4_i64(lens, x), ref), lens


def test_alg4_random_large_split_with_empty_segments():
    n = 1 << 16
    x = inputs.uniform_int64(RNG_KEY, n, 0, 1000)
    lens = inputs.random_cut_segments(7, n, 12)
    lens = lens[:3] + [0] + lens[3:] + [0]
    assert np.array_equal(oracle.segmented_scan_alg4_i64(lens, x), oracle.inclusive_scan_i64(x))


def test_scan_i64_total_permutation_invariant():
    x = inputs.uniform_int64(RNG_KEY, 10_000, 0, 1000)
    p = np.argsort(inputs.raw_u64(5, x.size))
    assert oracle.inclusive_scan_i64(x)[-1] == oracle.inclusive_scan_i64(x[p])[-1] == int(x.sum())


# ----------------------------------------------------------------------------------
# inclusive_scan, fp32 input accumulated in FP64
# ----------------------------------------------------------------------------------

def test_scan_f32_f64_ones_exact():
    n = 1 << 20
    y, a = oracle.inclusive_scan_f32_f64(np.ones(n, np.float32))
    assert np.array_equal(y, np.arange(1, n + 1, dtype=np.float64))
    assert np.array_equal(a, y)


def test_scan_f32_f64_integer_values_exact():
    xi = inputs.uniform_int64(RNG_KEY, 50_000, -1000, 1000)
    y, a = oracle.inclusive_scan_f32_f64(xi.astype(np.float32))
    assert np.array_equal(y, np.cumsum(xi).astype(np.float64))
    assert np.array_equal(a, np.cumsum(np.abs(xi)).astype(np.float64))


def test_scan_f32_f64_matches_exact_rational_prefix():
    x = inputs.uniform_pm1_f32(RNG_KEY, 300)
    y, a = oracle.inclusive_scan_f32_f64(x)
    acc = Fraction(0)
    for i, v in enumerate(x):
        acc += Fraction(float(v))
        # sequential FP64 summation error <= i * 2^-53 * sum|x|
        assert abs(Fraction(float(y[i])) - acc) <= Fraction(i + 1, 2**53) * Fraction(float(a[i]))


def test_scan_f32_seq_exact_on_small_integers():
    xi = inputs.uniform_int64(RNG_KEY, 4096, 0, 1000)
    y = oracle.inclusive_scan_f32_seq(xi.astype(np.float32))
    assert np.array_equal(y.astype(np.int64), np.cumsum(xi))


# ----------------------------------------------------------------------------------
# reverse inclusive scan (adjoint of inclusive_scan)
# ----------------------------------------------------------------------------------

def test_reverse_scan_ones_closed_form():
    n = 1000
    assert np.array_equal(oracle.reverse_inclusive_scan_f64(np.ones(n)),
                          np.arange(n, 0, -1, dtype=np.float64))


def test_reverse_scan_bruteforce():
    g = inputs.uniform_pm1_f32(3, 50).astype(np.float64)
    r = oracle.reverse_inclusive_scan_f64(g)
    for j in range(50):
        assert r[j] == pytest.approx(math.fsum(g[j:]), abs=1e-14)


def test_reverse_scan_is_adjoint_of_scan():
    n = 4096
    x = inputs.uniform_pm1_f32(11, n).astype(np.float64)
    w = inputs.uniform_pm1_f32(12, n).astype(np.float64)
    lhs = math.fsum(oracle.inclusive_scan_f64(x) * w)
    rhs = math.fsum(x * oracle.reverse_inclusive_scan_f64(w))
    assert lhs == pytest.approx(rhs, rel=1e-12, abs=1e-9)


def test_fd_gradient_of_scan_equals_reverse_scan():
    n = 256
    x = inputs.uniform_pm1_f32(13, n).astype(np.float64)
    w = inputs.uniform_pm1_f32(14, n).astype(np.float64)
    g = oracle.fd_gradient(lambda v: float(np.dot(w, oracle.inclusive_scan_f64(v))), x)
    assert np.allclose(g, oracle.reverse_inclusive_scan_f64(w), rtol=0, atol=1e-10)


# ----------------------------------------------------------------------------------
# dot = transform_reduce(zip(x, y), multiply, plus)
# ----------------------------------------------------------------------------------

@pytest.mark.parametrize("a,b", [(0.5, 0.25), (-2.0, 0.125), (1.0, 1.0)])
def test_dot_constant_powers_of_two(a, b):
    n = 1 << 20
    d, ad = oracle.dot_f64(np.full(n, a, np.float32), np.full(n, b, np.float32))
    assert d == n * a * b
    assert ad == n * abs(a * b)


def test_dot_iota_times_ones():
    n = 1 << 12
    d, _ = oracle.dot_f64(np.arange(n, dtype=np.float32), np.ones(n, np.float32))
    assert d == n * (n - 1) // 2


def test_dot_against_exact_sum():
    x = inputs.uniform_pm1_f32(21, 5000)
    y = inputs.uniform_pm1_f32(22, 5000)
    d, ad = oracle.dot_f64(x, y)
    prods = [float(a) * float(b) for a, b in zip(x, y)]  # exact in FP64
    assert abs(d - math.fsum(prods)) <= 5000 * 2**-53 * ad
    assert ad == pytest.approx(math.fsum(abs(p) for p in prods), rel=1e-12)


def test_dot_uneven_lengths_and_empty():
    d, ad = oracle.dot_f64(np.zeros(0, np.float32), np.zeros(0, np.float32))
    assert d == 0.0 and ad == 0.0


def test_alg3_segmented_reduce_equals_sum():
    x = inputs.uniform_int64(31, 70_000, -500, 500)
    for nseg in (1, 3, 8):
        lens = inputs.random_cut_segments(40 + nseg, x.size, nseg)
        assert oracle.segmented_reduce_alg3_i64(lens + [0], x) == int(x.sum())


def test_dot_adjoint_matches_fd_of_dot():
    n = 64
    x = inputs.uniform_pm1_f32(41, n)
    y = inputs.uniform_pm1_f32(42, n)
    g = 0.75
    gx, gy = oracle.dot_adjoint_f64(x, y, g)
    # d(g*<x,y>)/dx_j, by central differences on the oracle's own dot; h = 2^-10
    # keeps x_j +- h exact in fp32 so the difference is exact.
    fdx = oracle.fd_gradient(lambda v: g * oracle.dot_f64(v.astype(np.float32), y)[0], x)
    fdy = oracle.fd_gradient(lambda v: g * oracle.dot_f64(x, v.astype(np.float32))[0], y)
    assert np.allclose(gx, fdx, atol=1e-12) and np.allclose(gy, fdy, atol=1e-12)


# ----------------------------------------------------------------------------------
# 5-point stencil (zero outside the grid), its transpose, sampled-cell variants
# ----------------------------------------------------------------------------------

def _dist_to_edge(R, C):
    i = np.arange(R)[:, None]
    j = np.arange(C)[None, :]
    return np.minimum(np.minimum(i, R - 1 - i), np.minimum(j, C - 1 - j))


@pytest.mark.parametrize("steps", [1, 3, 7])
def test_stencil_linear_field_is_harmonic(steps):
    R, C = 40, 33
    i = np.arange(R)[:, None].astype(np.float64)
    j = np.arange(C)[None, :].astype(np.float64)
    u0 = 3 * i - 2 * j + 5
    far = _dist_to_edge(R, C) >= steps
    out64 = oracle.stencil5_f64(u0, steps)
    out32 = oracle.stencil5_f32(u0.astype(np.float32), steps)
    assert np.array_equal(out64[far], u0[far])
    assert np.array_equal(out32[far], u0[far].astype(np.float32))
    # the zero ghost ring pulls the edge down: the corner after one step
    if steps == 1:
        assert out64[0, 0] == 0.25 * (u0[1, 0] + u0[0, 1])


def test_stencil_constant_field_interior():
    R, C, t = 30, 30, 5
    out = oracle.stencil5_f64(np.full((R, C), 0.5), t)
    far = _dist_to_edge(R, C) >= t
    assert np.all(out[far] == 0.5)
    assert np.all(out[~far] < 0.5)


@pytest.mark.parametrize("t", [1, 2, 5, 12])
def test_stencil_impulse_is_random_walk_law(t):
    # A^t e_c for wc=0, wn=1/4 is the law of a simple 2D random walk after t
    # steps: P(x, y) = C(t, (t+x+y)/2) * C(t, (t+x-y)/2) / 4^t when x+y+t is even.
    n = 2 * t + 9
    c = n // 2
    u0 = np.zeros((n, n))
    u0[c, c] = 1.0
    out = oracle.stencil5_f64(u0, t)
    for x in range(-t - 1, t + 2):
        for y in range(-t - 1, t + 2):
            if (x + y + t) % 2 or abs(x) + abs(y) > t:
                p = 0.0
            else:
                p = math.comb(t, (t + x + y) // 2) * math.comb(t, (t + x - y) // 2) / 4.0**t
            assert out[c + x, c + y] == p, (x, y)


def test_stencil_weights_one_step_impulse():
    u0 = np.zeros((5, 6))
    u0[2, 3] = 1.0
    out = oracle.stencil5_f64(u0, 1, wc=0.5, wn=0.125)
    exp = np.zeros((5, 6))
    exp[2, 3] = 0.5
    exp[1, 3] = exp[3, 3] = exp[2, 2] = exp[2, 4] = 0.125
    assert np.array_equal(out, exp)
    # the corner loses the two neighbours that fall outside the grid
    u0 = np.zeros((5, 6))
    u0[0, 0] = 1.0
    out = oracle.stencil5_f64(u0, 1)
    assert out.sum() == 0.5 and out[0, 1] == out[1, 0] == 0.25


@pytest.mark.parametrize("wc,wn", [(0.0, 0.25), (0.3, 0.15), (-0.1, 0.7)])
def test_stencil_transpose_adjoint_identity(wc, wn):
    R, C, t = 9, 13, 4
    x = inputs.uniform_pm1_f32(51, R * C).astype(np.float64).reshape(R, C)
    w = inputs.uniform_pm1_f32(52, R * C).astype(np.float64).reshape(R, C)
    lhs = math.fsum((oracle.stencil5_f64(x, t, wc, wn) * w).ravel())
    rhs = math.fsum((x * oracle.stencil5_T_f64(w, t, wc, wn)).ravel())
    assert lhs == pytest.approx(rhs, rel=1e-13, abs=1e-13)
    # with a zero ghost ring the operator is symmetric: A^T w == A w
    assert np.allclose(oracle.stencil5_T_f64(w, t, wc, wn), oracle.stencil5_f64(w, t, wc, wn),
                       rtol=0, atol=1e-14)


def test_stencil_f32_same_order_within_contraction_bound():
    R, C, t = 64, 48, 20
    u0 = inputs.uniform01_f32(61, R * C).reshape(R, C)
    d = np.abs(oracle.stencil5_f32(u0, t).astype(np.float64) - oracle.stencil5_f64(u0, t))
    assert d.max() <= 3 * t * 2.0**-24 * np.abs(u0).max()


@pytest.mark.parametrize("wc,wn", [(0.0, 0.25), (0.2, 0.2)])
def test_stencil_sampled_cells_equal_full_grid(wc, wn):
    R, C, t = 23, 31, 6
    u0 = inputs.uniform01_f32(71, R * C).reshape(R, C)
    cells = np.array([(i, j) for i in range(R) for j in range(C)], np.int64)
    full32 = oracle.stencil5_f32(u0, t, wc, wn)
    at32 = oracle.stencil5_f32_at(u0, t, cells, wc, wn)
    assert np.array_equal(at32, full32[cells[:, 0], cells[:, 1]])
    full64 = oracle.stencil5_f64(u0, t, wc, wn)
    at64 = oracle.stencil5_f64_at(u0, t, cells, wc, wn)
    assert np.array_equal(at64, full64[cells[:, 0], cells[:, 1]])


def test_stencil_fd_gradient_equals_transpose():
    R, C, t = 8, 8, 3
    u0 = inputs.uniform01_f32(81, R * C).astype(np.float64).reshape(R, C)
    w = inputs.uniform_pm1_f32(82, R * C).astype(np.float64).reshape(R, C)
    g = oracle.fd_gradient(lambda v: float((oracle.stencil5_f64(v, t) * w).sum()), u0)
    assert np.allclose(g, oracle.stencil5_T_f64(w, t), atol=1e-10)


# ----------------------------------------------------------------------------------
# zip re-segmentation (Sec. 4.4)
# ----------------------------------------------------------------------------------

def test_zip_hand_examples():
    # a = [3 | 5], b = [4 | 4]: cuts at 3 and 4 -> pieces of 3, 1, 4
    assert oracle.zip_segments_bruteforce([3, 5], [4, 4]) == [
        (0, 0, 0, 0, 3), (1, 0, 0, 3, 1), (1, 1, 1, 0, 4)]
    assert oracle.zip_segments_bruteforce([8], [8]) == [(0, 0, 0, 0, 8)]
    # empty segments own nothing
    assert oracle.zip_segments_bruteforce([0, 4], [2, 0, 2]) == [(1, 0, 0, 0, 2), (1, 2, 2, 0, 2)]
    # zip is as long as its shortest input
    assert oracle.zip_segments_bruteforce([5], [2, 1]) == [(0, 0, 0, 0, 2), (0, 2, 1, 0, 1)]


def test_zip_properties_random():
    for trial in range(30):
        na = 1 + trial % 5
        nb = 1 + (trial * 7) % 6
        la = inputs.random_cut_segments(100 + trial, 200, na)
        lb = inputs.random_cut_segments(200 + trial, 200 - trial, nb)
        pcs = oracle.zip_segments_bruteforce(la, lb)
        assert sum(p[4] for p in pcs) == min(sum(la), sum(lb))
        bounds_a = set(np.cumsum([0] + la))
        bounds_b = set(np.cumsum([0] + lb))
        pos = 0
        for k, (sa, oa, sb, ob, L) in enumerate(pcs):
            assert oa + L <= la[sa] and ob + L <= lb[sb] and L > 0
            pos += L
            if k + 1 < len(pcs):  # every cut is a segment boundary of a or of b
                assert pos in bounds_a or pos in bounds_b


# ----------------------------------------------------------------------------------
# seeded generator
# ----------------------------------------------------------------------------------

def test_splitmix64_published_outputs():
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "splitmix64_seed0.txt")
    want = [int(l, 16) for l in open(path) if l.strip() and not l.startswith("#")]
    assert [int(v) for v in inputs.raw_u64(0, len(want))] == want


def test_generator_ranges_and_exactness():
    x = inputs.uniform_pm1_f32(1, 1 << 16)
    assert x.min() >= -1.0 and x.max() < 1.0
    k = (x.astype(np.float64) + 1.0) * 2.0**23
    assert np.array_equal(k, np.round(k))
    u = inputs.uniform01_f32(2, 1 << 16)
    assert u.min() >= 0.0 and u.max() < 1.0
    i = inputs.uniform_int64(3, 1 << 16)
    assert i.min() >= 0 and i.max() < 1000
    # chunked / threaded generation equals one-shot generation
    big = inputs.uniform_pm1_f32(9, (1 << 22) + 5)
    assert np.array_equal(big[-5:], inputs.uniform_pm1_f32(9, (1 << 22) + 5)[-5:])
    assert np.array_equal(inputs.raw_u64(9, 10, start=(1 << 22) - 3),
                          inputs.raw_u64(9, (1 << 22) + 7)[-10:])


def test_batch_shapes_recipe():
    shapes = inputs.batch_shapes(2411, 256)
    for s in shapes:
        assert 1 <= len(s) <= 8 and all(v > 0 for v in s)
        assert 1000 <= sum(s) <= 1_000_000
    assert shapes == inputs.batch_shapes(2411, 256)


# ----------------------------------------------------------------------------------
# for_each element functions: STREAM (one rounding per operation, element type)
# ----------------------------------------------------------------------------------

@pytest.mark.parametrize("dt", [np.float32, np.float64])
def test_stream_roles_and_closed_forms(dt):
    n = 1000
    i = np.arange(n, dtype=dt)
    ones = np.ones(n, dt)
    # copy: c = a, a and b untouched
    a, b, c = oracle.stream("copy", i, 2 * i, ones)
    assert np.array_equal(c, i) and np.array_equal(a, i) and np.array_equal(b, 2 * i)
    # scale: b = q c (q = 3, integer-valued: exact); a, c untouched
    a, b, c = oracle.stream("scale", ones, ones, i, 3.0)
    assert np.array_equal(b, 3 * i) and np.array_equal(c, i) and np.array_equal(a, ones)
    # add: c = a + b
    a, b, c = oracle.stream("add", i, 7 * ones, ones)
    assert np.array_equal(c, i + 7) and np.array_equal(b, 7 * ones)
    # triad: a = b + q c with b = i, c = 1, q = 3 -> i + 3 (not 1 + 3 i: catches b <-> c)
    a, b, c = oracle.stream("triad", 5 * ones, i, ones, 3.0)
    assert np.array_equal(a, i + 3) and np.array_equal(b, i) and np.array_equal(c, ones)


@pytest.mark.parametrize("dt,eps", [(np.float32, 2.0 ** -23), (np.float64, 2.0 ** -52)])
def test_stream_triad_rounds_twice(dt, eps):
    # q = c = 1 + eps: q*c = 1 + 2 eps + eps^2, rounded to 1 + 2 eps before the add;
    # b = -1 leaves exactly 2 eps.  A fused multiply-add would keep eps^2 as well.
    q = 1 + eps
    a, _, _ = oracle.stream("triad", np.zeros(1, dt), -np.ones(1, dt), np.full(1, q, dt), q)
    assert a[0] == dt(2 * eps)


def test_stream_random_matches_numpy_definition():
    # the definition in numpy's own (separately rounded) element ops
    x = inputs.uniform_pm1_f32(RNG_KEY, 4096)
    y = inputs.uniform_pm1_f32(RNG_KEY + 1, 4096)
    z = inputs.uniform_pm1_f32(RNG_KEY + 2, 4096)
    q = np.float32(0.4)
    a, _, _ = oracle.stream("triad", x, y, z, float(q))
    assert np.array_equal(a, y + q * z)
    _, _, c = oracle.stream("add", x, y, z)
    assert np.array_equal(c, x + y)


# ----------------------------------------------------------------------------------
# Black-Scholes-Merton European call / put (FP64)
# ----------------------------------------------------------------------------------

def _golden_bs():
    path = os.path.join(os.path.dirname(__file__), "golden", "black_scholes_textbook.txt")
    rows = []
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        rows.append({k: float(v) for k, v in (f.split("=") for f in line.split())})
    return rows


def test_black_scholes_textbook_example():
    for g in _golden_bs():
        call, put, aux = oracle.black_scholes_f64([g["S"]], [g["X"]], [g["T"]], g["r"], g["sigma"], aux=True)
        d1 = aux[0, 2]
        d2 = d1 - g["sigma"] * math.sqrt(g["T"])
        dd, pd = int(g["d_decimals"]), int(g["price_decimals"])
        assert round(d1, dd) == pytest.approx(g["d1"], abs=1e-12)
        assert round(d2, dd) == pytest.approx(g["d2"], abs=1e-12)
        assert round(call[0], pd) == pytest.approx(g["call"], abs=1e-12)
        assert round(put[0], pd) == pytest.approx(g["put"], abs=1e-12)


def _bs_inputs(n, key=RNG_KEY):
    S = 5 + 25 * inputs.uniform01_f64(key, n)
    X = 1 + 99 * inputs.uniform01_f64(key + 1, n)
    T = 0.25 + 9.75 * inputs.uniform01_f64(key + 2, n)
    return S, X, T


def test_black_scholes_put_call_parity():
    # call - put = S - X e^{-rT} for every option (a model-free identity): catches a
    # sign or argument slip in either price
    S, X, T = _bs_inputs(10000)
    r, sigma = 0.02, 0.30
    call, put = oracle.black_scholes_f64(S, X, T, r, sigma)
    rhs = S - X * np.exp(-r * T)
    assert np.max(np.abs((call - put) - rhs) / (S + X)) < 1e-14
    assert np.all(call >= np.maximum(rhs, 0) - 1e-12 * (S + X))   # no-arbitrage lower bounds
    assert np.all(put >= np.maximum(-rhs, 0) - 1e-12 * (S + X))
    assert np.all(call <= S) and np.all(put <= X * np.exp(-r * T) + 1e-12)


def test_black_scholes_at_the_money_forward_closed_form():
    # S = X e^{-rT}: d1 = sigma sqrt(T)/2, d2 = -d1, so call = put = S erf(sigma sqrt(T) / (2 sqrt 2));
    # depends on the sigma^2/2 drift term and on N's definition
    for sigma, T, r, X in [(0.2, 1.0, 0.05, 100.0), (0.5, 2.0, 0.01, 30.0), (0.1, 0.25, 0.0, 7.0)]:
        S = X * math.exp(-r * T)
        call, put = oracle.black_scholes_f64([S], [X], [T], r, sigma)
        want = S * math.erf(sigma * math.sqrt(T) / (2 * math.sqrt(2)))
        assert call[0] == pytest.approx(want, rel=1e-13)
        assert put[0] == pytest.approx(want, rel=1e-13)


def test_black_scholes_zero_volatility_limit():
    # sigma -> 0: the option is worth its discounted intrinsic value (r > 0 drift in d1)
    S, X, T = _bs_inputs(2000, key=RNG_KEY + 7)
    r = 0.05
    keep = np.abs(np.log(S / X) + r * T) > 1e-3
    S, X, T = S[keep], X[keep], T[keep]
    call, put = oracle.black_scholes_f64(S, X, T, r, 1e-9)
    K = X * np.exp(-r * T)
    assert np.allclose(call, np.maximum(S - K, 0), rtol=0, atol=1e-9)
    assert np.allclose(put, np.maximum(K - S, 0), rtol=0, atol=1e-9)


def test_zip_bruteforce_k_agrees_with_pairwise_and_identity():
    # k = 2 is the pairwise brute force; zipping a segmentation with itself k times
    # returns that segmentation (minus its empty segments)
    for la, lb in [([3, 5], [4, 4]), ([0, 4], [2, 0, 2]), ([5], [2, 1]), ([1, 1, 6], [8])]:
        two = oracle.zip_segments_bruteforce(la, lb)
        k = oracle.zip_segments_bruteforce_k([la, lb])
        assert [(s[0], f[0], s[1], f[1], n) for s, f, n in k] == two
    lens = [2, 0, 3, 1]
    k3 = oracle.zip_segments_bruteforce_k([lens, lens, lens])
    assert [n for _, _, n in k3] == [2, 3, 1]
    assert [s for s, _, _ in k3] == [(0, 0, 0), (2, 2, 2), (3, 3, 3)]
    # a third operand's cut splits a piece of the first two
    k3 = oracle.zip_segments_bruteforce_k([[6], [6], [2, 4]])
    assert [(s, f, n) for s, f, n in k3] == [((0, 0, 0), (0, 0, 0), 2), ((0, 0, 1), (2, 2, 0), 4)]


# ----------------------------------------------------------------------------------
# sort: plain definition (ascending; floats in IEEE totalOrder) and the paper's
# distributed partition sort
# ----------------------------------------------------------------------------------

def test_sort_total_order_of_special_values():
    # totalOrder: -NaN < -inf < -1 < -tiny < -0 < +0 < tiny < 1 < inf < +NaN
    for dt, it in [(np.float32, np.uint32), (np.float64, np.uint64)]:
        vals = np.array([np.nan, 1.0, -0.0, np.inf, -1.0, 0.0, -np.inf, -np.nan], dt)
        tiny = np.finfo(dt).smallest_subnormal
        vals = np.concatenate([vals, np.array([tiny, -tiny], dt)])
        neg_nan = (-np.abs(np.array([np.nan], dt)))  # sign bit set
        vals[-3] = neg_nan[0]
        want = np.array([neg_nan[0], -np.inf, -1.0, -tiny, -0.0, 0.0, tiny, 1.0, np.inf, np.nan], dt)
        got = oracle.sort(vals[np.argsort(np.arange(vals.size) * 7 % vals.size)])
        assert np.array_equal(got.view(it), want.view(it))


@pytest.mark.parametrize("dt", [np.int32, np.int64, np.float32, np.float64])
def test_sort_is_sorted_permutation(dt):
    n = 5000
    if dt in (np.int32, np.int64):
        x = inputs.uniform_int64(RNG_KEY, n, -300, 300).astype(dt)       # many duplicates
    else:
        x = inputs.uniform_pm1_f32(RNG_KEY, n).astype(dt)
    y = oracle.sort(x)
    assert np.all(y[1:] >= y[:-1])
    assert np.array_equal(np.sort(y), np.sort(x))     # same multiset (library sort as a check)
    assert np.array_equal(y, np.sort(x))              # no NaN / signed zero: plain order agrees


def test_sort_bruteforce_permutations():
    base = [3, -1, 3, 0, 7, -1]
    for perm in itertools.permutations(range(len(base))):
        x = np.array([base[i] for i in perm], np.int64)
        assert list(oracle.sort(x)) == sorted(base)


@pytest.mark.parametrize("trial", range(12))
def test_partition_sort_equals_plain_sort(trial):
    # the paper's splitter / histogram / redistribute / local-sort procedure reaches the
    # plain definition for any segmentation, duplicates, empty segments and one segment
    n = [0, 1, 7, 100, 1000, 5000][trial % 6]
    p = 1 + trial % 9
    lens = inputs.random_cut_segments(500 + trial, n, p) if n else [0] * p
    if trial % 4 == 1:
        lens = [0] + lens + [0]
    span = 10 if trial % 3 == 0 else 1_000_000
    x = inputs.uniform_int64(600 + trial, n, -span, span)
    assert np.array_equal(oracle.partition_sort_i64(lens, x), np.sort(x))
    assert np.array_equal(oracle.partition_sort_i64(lens, np.full(n, 5, np.int64)), np.full(n, 5))


ZS_P = 0.2316419
ZS_B = (0.319381530, -0.356563782, 1.781477937, -1.821255978, 1.330274429)


def test_zelen_severo_normal_tail_within_its_published_bound():
    """Abramowitz & Stegun 26.2.17: N(-x) = phi(x)(b1 t + ... + b5 t^5), t = 1/(1 + p x),
    within 7.5e-8 for x >= 0 -- checked in FP64 against erfc on a dense grid."""
    from scipy.special import erfc
    x = np.linspace(0.0, 12.0, 200_001)
    t = 1.0 / (1.0 + ZS_P * x)
    poly = sum(b * t ** (k + 1) for k, b in enumerate(ZS_B))
    approx = np.exp(-0.5 * x * x) / math.sqrt(2 * math.pi) * poly
    exact = 0.5 * erfc(x / math.sqrt(2.0))
    assert np.max(np.abs(approx - exact)) < 7.5e-8
    assert np.max(np.abs(approx - exact)) > 1e-8            # and the bound is nearly attained


def test_black_scholes_fp32_bound_holds_for_the_kernels_evaluation_order():
    """The stated tolerance covers an fp32 evaluation in the fp32 kernel's order
    (q = S/X, ln q = log2(q) ln2, d1 = fma(drift, T, ln q) (1/sigma) rsqrt(T), the
    Zelen-Severo N with fma Horner steps) -- here with correctly rounded fp32
    operations standing in for the hardware approximations, whose larger
    documented errors the bound budgets -- and is not vacuous."""
    from tests import tolerances as T
    f = np.float32
    S, X, Tm = inputs.black_scholes_inputs(1 << 15, key=RNG_KEY)
    r, sig = f(inputs.BS_R), f(inputs.BS_SIGMA)

    def fma(a, b, c):   # one rounding of a*b + c (the product is exact in FP64)
        return (np.asarray(a, np.float64) * np.asarray(b, np.float64) + np.asarray(c, np.float64)).astype(f)

    inv_sig = f(1.0) / sig
    drift = r + f(0.5) * sig * sig
    rs = (f(1.0) / np.sqrt(Tm)).astype(f)
    sv = sig * Tm * rs
    lnr = (np.log2(S / X).astype(f) * f(0.6931471805599453)).astype(f)
    d1 = fma(drift, Tm, lnr) * (inv_sig * rs)
    d2 = d1 - sv
    K = X * np.exp(-r * Tm).astype(f)

    def cdf_pair(d):
        x = np.abs(d)
        t = (f(1.0) / fma(f(ZS_P), x, f(1.0))).astype(f)
        phi = f(0.3989422804014327) * np.exp(f(-0.5) * x * x).astype(f)
        poly = fma(t, f(ZS_B[4]), f(ZS_B[3]))
        for b in (ZS_B[2], ZS_B[1], ZS_B[0]):
            poly = fma(t, poly, f(b))
        e = phi * (poly * t)
        c = f(1.0) - e
        return np.where(d >= 0, c, e), np.where(d >= 0, e, c)

    n1, m1 = cdf_pair(d1)
    n2, m2 = cdf_pair(d2)
    call = S * n1 - K * n2
    put = K * m2 - S * m1
    assert call.dtype == np.float32 and put.dtype == np.float32
    ec, ep, aux = oracle.black_scholes_f64(S, X, Tm, float(r), float(sig), aux=True)
    bound = T.black_scholes_bound(S, X, Tm, float(r), float(sig), aux)
    assert np.all(np.abs(call - ec) <= bound) and np.all(np.abs(put - ep) <= bound)
    # not vacuous: prices are resolved to about 1e-6 of their scale, and a result
    # 1e-3 off would fail
    assert np.median(bound / (S + aux[:, 3])) < 2e-5
    assert not np.all(np.abs(call + 1e-3 * (S + aux[:, 3]) - ec) <= bound)


# ----------------------------------------------------------------------------------
# the other associative operators: exclusive scans with init, MIN / MAX scans,
# reduce over every operator and element type (Sec. 4.3)
# ----------------------------------------------------------------------------------

def _wrap(v, bits):
    v %= 2 ** bits
    return v - 2 ** bits if v >= 2 ** (bits - 1) else v


@pytest.mark.parametrize("n,init", [(0, 7), (1, 7), (4097, -3), (10_000, 0)])
def test_exclusive_scan_of_ones_is_init_plus_iota(n, init):
    y = oracle.scan(np.ones(n, np.int64), "plus", exclusive=True, init=init)
    assert np.array_equal(y, init + np.arange(n, dtype=np.int64))
    y32 = oracle.scan(np.ones(n, np.int32), "plus", exclusive=True, init=init)
    assert y32.dtype == np.int32 and np.array_equal(y32, init + np.arange(n, dtype=np.int32))


@pytest.mark.parametrize("dt,bits", [(np.int64, 64), (np.int32, 32)])
def test_scan_plus_bruteforce_wraps(dt, bits):
    lo, hi = (-2 ** 62, 2 ** 62) if bits == 64 else (-2 ** 30, 2 ** 30)
    x = inputs.uniform_int64(RNG_KEY + 1, 12, lo, hi).astype(dt)
    init = int(x[0]) // 3
    yi = oracle.scan(x, "plus", exclusive=False, init=init)
    ye = oracle.scan(x, "plus", exclusive=True, init=init)
    for i in range(x.size):
        assert int(yi[i]) == _wrap(init + sum(int(v) for v in x[:i + 1]), bits)
        assert int(ye[i]) == _wrap(init + sum(int(v) for v in x[:i]), bits)


@pytest.mark.parametrize("op", ["max", "min"])
def test_minmax_scan_of_a_permutation_bruteforce(op):
    n = 300
    r = inputs.raw_u64(RNG_KEY + 2, n)
    perm = np.argsort(r, kind="stable").astype(np.int64)   # a permutation of 0..n-1
    f = max if op == "max" else min
    for excl in (False, True):
        for init in (None, 150):
            y = oracle.scan(perm, op, exclusive=excl, init=init)
            start = (-(2 ** 63) if op == "max" else 2 ** 63 - 1) if init is None else init
            for i in range(n):
                pre = [int(v) for v in perm[:i + (0 if excl else 1)]]
                assert int(y[i]) == f([start] + pre)
    if op == "max":   # a permutation's running max reaches n-1 exactly where n-1 sits
        y = oracle.scan(perm, "max")
        k = int(np.argmax(perm))
        assert int(y[k]) == n - 1 and (k == 0 or int(y[k - 1]) < n - 1)


@pytest.mark.parametrize("op", ["max", "min"])
def test_minmax_scan_floats_bruteforce(op):
    x = inputs.uniform_pm1_f32(RNG_KEY + 3, 200).astype(np.float64)
    f = max if op == "max" else min
    y = oracle.scan(x, op)
    ye = oracle.scan(x, op, exclusive=True, init=0.25)
    for i in range(x.size):
        assert y[i] == f(float(v) for v in x[:i + 1])
        assert ye[i] == f([0.25] + [float(v) for v in x[:i]])
    assert oracle.scan(x[:0], op).size == 0
    assert oracle.scan(x[:1], op, exclusive=True)[0] == (-np.inf if op == "max" else np.inf)


def test_scan_plus_f64_small_integers_exact():
    x = inputs.uniform_int64(RNG_KEY + 4, 5000, -100, 100)
    y = oracle.scan(x.astype(np.float64), "plus", exclusive=True, init=2.0)
    assert np.array_equal(y, 2.0 + np.concatenate([[0], np.cumsum(x)[:-1]]).astype(np.float64))


@pytest.mark.parametrize("dt,bits", [(np.int64, 64), (np.int32, 32)])
def test_reduce_integers_bruteforce(dt, bits):
    lo, hi = (-2 ** 62, 2 ** 62) if bits == 64 else (-2 ** 30, 2 ** 30)
    x = inputs.uniform_int64(RNG_KEY + 5, 64, lo, hi).astype(dt)
    xs = [int(v) for v in x]
    assert oracle.reduce(x, "plus", init=5) == _wrap(5 + sum(xs), bits)
    assert oracle.reduce(x, "max", init=-7) == max([-7] + xs)
    assert oracle.reduce(x, "min", init=7) == min([7] + xs)
    assert oracle.reduce(x, "max") == max(xs) and oracle.reduce(x, "min") == min(xs)
    small = inputs.uniform_int64(RNG_KEY + 6, 20, -3, 4).astype(dt)
    assert oracle.reduce(small, "mul", init=1) == _wrap(math.prod(int(v) for v in small), bits)
    n = 70_001
    assert oracle.reduce(np.arange(n, dtype=dt), "plus") == _wrap(n * (n - 1) // 2, bits)


def test_reduce_float_minmax_and_empty():
    x = inputs.uniform_pm1_f32(RNG_KEY + 7, 1000)
    assert oracle.reduce(x, "max") == max(float(v) for v in x)
    assert oracle.reduce(x, "min", init=-2.0) == -2.0
    assert oracle.reduce(x[:0], "max", init=3.5) == 3.5
    assert oracle.reduce(x[:0], "plus", init=1.25) == Fraction(5, 4)


def test_sum_exact_against_rationals_and_fsum():
    # huge cancellation: every naive order loses the small terms
    x = np.array([1e16, 1.0, -1e16, 3.0, 2.0 ** -60, -3.0], np.float64)
    assert oracle.sum_exact(x) == Fraction(1) + Fraction(2) ** -60
    for key in range(5):
        r = inputs.uniform01_f64(RNG_KEY + 10 + key, 400)
        e = inputs.uniform_int64(RNG_KEY + 20 + key, 400, -60, 60)
        v = (2 * r - 1) * np.exp2(e.astype(np.float64))    # magnitudes over 120 binades
        exact = sum((Fraction(float(t)) for t in v), Fraction(0))
        got = oracle.sum_exact(v)
        assert got == exact
        assert float(got) == math.fsum(v)   # both correctly rounded
    # reduce(plus) of floats = init plus the exact sum
    v = inputs.uniform_pm1_f32(RNG_KEY + 30, 3000)
    assert oracle.reduce(v, "plus", init=0.5) == Fraction(1, 2) + sum((Fraction(float(t)) for t in v), Fraction(0))


# ----------------------------------------------------------------------------------
# take / drop via trimmed segments (Sec. 4.4 "Take and Drop")
# ----------------------------------------------------------------------------------

def _owner_runs(lens, f, l):
    """Brute force: the owner (segment, offset) of every global index in [f, l),
    merged into maximal runs of one segment."""
    owners = []
    for k, L in enumerate(lens):
        owners.extend((k, j) for j in range(L))
    runs = []
    for i in range(max(0, f), min(l, len(owners))):
        k, j = owners[i]
        if runs and runs[-1][0] == k:
            runs[-1] = (k, runs[-1][1], runs[-1][2] + 1)
        else:
            runs.append((k, j, 1))
    return runs


@pytest.mark.parametrize("lens", [[3, 0, 4, 1, 0], [5], [0, 0, 2], [1, 1, 1, 1]])
def test_trim_segments_bruteforce_every_window(lens):
    n = sum(lens)
    for f in range(-1, n + 2):
        for l in range(-1, n + 3):
            assert oracle.trim_segments(lens, f, l) == _owner_runs(lens, f, l), (f, l)
    for l in range(n + 3):
        assert oracle.take_segments(lens, l) == _owner_runs(lens, 0, l)
    for f in range(n + 3):
        assert oracle.drop_segments(lens, f) == _owner_runs(lens, f, n)


def test_trim_gathers_the_slice():
    lens = [10, 0, 25, 7, 0, 13]
    x = np.arange(55, dtype=np.int64) * 3 + 1
    for f, l in [(0, 55), (9, 11), (10, 35), (34, 36), (50, 80), (20, 20)]:
        got = oracle.gather_segments(x, lens, oracle.trim_segments(lens, f, l))
        assert np.array_equal(got, x[max(0, f):min(l, 55)])
