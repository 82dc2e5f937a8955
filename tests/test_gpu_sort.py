"""sort (Sec. 4.3) on the GPU, through the C ABI: bit-exact against the CPU
oracle's sort of the concatenation (floats in IEEE totalOrder), for every key
type, segmentation, duplicate pattern and special value; in place and over
transformed views; the benchmark's size checked by properties."""
import numpy as np
import pytest

import oracle
from paper_2406_00158_gb300 import inputs
from tests import gpu_util as G

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TILE = 256 * 15
TDT = {np.float32: torch.float32, np.float64: torch.float64, np.int32: torch.int32, np.int64: torch.int64}
BITS = {np.float32: np.uint32, np.float64: np.uint64, np.int32: np.uint32, np.int64: np.uint64}


@pytest.fixture(scope="module")
def api():
    G.dev()
    from paper_2406_00158_gb300 import api
    return api


def keys(dt, n, seed, kind="random"):
    if kind == "dups":
        return inputs.uniform_int64(seed, n, -4, 5).astype(dt)
    if dt == np.int64:
        return inputs.raw_u64(seed, n).view(np.int64)              # all 64 bits random
    if dt == np.int32:
        return (inputs.raw_u64(seed, n) >> np.uint64(32)).astype(np.uint32).view(np.int32)
    return (inputs.uniform_pm1_f32(seed, n) * 1000).astype(dt)


def check(api, x, lin, lout, dt, offset=0):
    v = G.segvec(x, lin, offset_elems=offset)
    out = G.empty_like_vec(lout, TDT[dt])
    api.sort(v, out)
    api.sync_status()
    got = G.to_np(out)
    exp = oracle.sort(x)
    assert np.array_equal(got.view(BITS[dt]), exp.view(BITS[dt]))


@pytest.mark.parametrize("dt", [np.float32, np.float64, np.int32, np.int64])
@pytest.mark.parametrize("n,lin,lout", [
    (3 * TILE + 17, [1000, 0, 3 * TILE + 17 - 1000], [3 * TILE + 17]),
    (50_000, [50_000], [7, 20_000, 29_993]),
    (TILE, [TILE], [TILE]),
    (TILE + 1, [1, TILE], [TILE, 1]),
    (1, [1], [1]),
    (200_001, [1, 99_999, 0, 100_001], [200_001]),
])
def test_sort_random_bit_exact(api, dt, n, lin, lout):
    check(api, keys(dt, n, 11 + n % 97), lin, lout, dt)


@pytest.mark.parametrize("dt", [np.float32, np.int64])
@pytest.mark.parametrize("kind", ["dups", "sorted", "reversed", "constant"])
def test_sort_patterns(api, dt, kind):
    n = 5 * TILE + 123
    x = keys(dt, n, 21, "dups" if kind == "dups" else "random")
    if kind == "sorted":
        x = oracle.sort(x)
    elif kind == "reversed":
        x = oracle.sort(x)[::-1].copy()
    elif kind == "constant":
        x = np.full(n, x[0], dt)
    check(api, x, [n // 3, n - n // 3], [n], dt, offset=1)


@pytest.mark.parametrize("dt", [np.float32, np.float64])
def test_sort_special_float_values(api, dt):
    n = 2 * TILE + 99
    x = keys(dt, n, 31)
    it = BITS[dt]
    tiny = np.finfo(dt).smallest_subnormal
    neg_nan = (-np.abs(np.array([np.nan], dt)))[0]
    special = np.array([np.nan, neg_nan, np.inf, -np.inf, 0.0, -0.0, tiny, -tiny, 1.0, -1.0], dt)
    idx = inputs.uniform_int64(32, 400, 0, n)
    x[idx] = special[np.arange(400) % special.size]
    # a NaN with another payload
    bits = x.view(it)
    bits[5] = (np.array([0x7F800001], np.uint32) if dt == np.float32 else np.array([0x7FF0000000000001], np.uint64))[0]
    check(api, x, [n], [TILE, n - TILE], dt)


def test_sort_in_place_and_transformed_view(api):
    n = 4 * TILE + 5
    x = keys(np.int64, n, 41)
    v = G.segvec(x, [n // 2, n - n // 2])
    api.sort(v, v)  # in place
    api.sync_status()
    assert np.array_equal(G.to_np(v), np.sort(x))
    # sort(transform(y, neg)) is y in descending order, negated
    y = keys(np.float32, n, 43)
    vy = G.segvec(y, [n])
    out = G.empty_like_vec([n], torch.float32)
    api.sort(vy.view().transform("neg"), out)
    api.sync_status()
    assert np.array_equal(G.to_np(out), oracle.sort(-y))
    # sort of a zip_transform (x * x), and of a take / drop window
    out64 = G.empty_like_vec([n], torch.int64)
    xs = inputs.uniform_int64(44, n, -1000, 1000)
    vx = G.segvec(xs, [100, n - 100])
    api.sort(api.dot_view(vx, vx), out64)
    api.sync_status()
    assert np.array_equal(G.to_np(out64), np.sort(xs * xs))
    part = G.empty_like_vec([5000], torch.int64)
    api.sort(vx.view().drop(77).take(5000), part)
    api.sync_status()
    assert np.array_equal(G.to_np(part), np.sort(xs[77:5077]))


def test_sort_output_longer_than_input_keeps_tail(api):
    n = 10_000
    x = keys(np.int32, n, 51)
    out = G.segvec(np.full(n + 10, 7, np.int32), [n + 10])
    api.sort(G.segvec(x, [n]), out)
    api.sync_status()
    got = G.to_np(out)
    assert np.array_equal(got[:n], np.sort(x)) and np.all(got[n:] == 7)


def test_sort_repeated_calls_reuse_workspace(api):
    n = 3 * TILE + 1
    v = G.segvec(keys(np.float32, n, 61), [n])
    out = G.empty_like_vec([n], torch.float32)
    for seed in (62, 63, 64):
        x = keys(np.float32, n, seed)
        v = G.segvec(x, [n])
        api.sort(v, out)
        api.sync_status()
        assert np.array_equal(G.to_np(out), oracle.sort(x))


def test_sort_full_size_vs_oracle(api):
    """The benchmark's workload (2^28 fp32 keys U[-1, 1) in 8 segments into 8
    output segments, the bench's launch): bit-exact against the oracle's sort."""
    n = 1 << 28
    x = inputs.uniform_pm1_f32(inputs.SEED_SORT, n)
    lens = [n // 8] * 8
    v = G.segvec(x, lens)
    out = G.empty_like_vec(lens, torch.float32)
    api.sort(v, out)
    api.sync_status()
    got = G.to_np(out)
    exp = oracle.sort(x)
    assert np.array_equal(got.view(np.uint32), exp.view(np.uint32))
