"""inclusive / exclusive / reverse scan across segment boundaries on the GPU
(single pass, decoupled lookback), through the C ABI, against the CPU oracle."""
import numpy as np
import pytest

import oracle
from paper_2406_00158_gb300 import inputs
from tests import gpu_util as G
from tests import tolerances as T

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def api():
    G.dev()
    from paper_2406_00158_gb300 import api
    return api


def scan_i64(api, x, lens, out_lens=None, offset=0):
    vx = G.segvec(x, lens, offset_elems=offset)
    out = G.empty_like_vec(out_lens or lens, torch.int64)
    api.inclusive_scan(vx, out)
    api.sync_status()
    return G.to_np(out)


def test_scan_i64_config_2p20_uneven_1_2_3_2(api):
    """int64, n = 2^20, 4 segments 1:2:3:2, values U[0,1000): bit-exact."""
    n = 1 << 20
    lens = inputs.proportional_segments(n, [1, 2, 3, 2])
    assert lens == [131072, 262144, 393216, 262144]
    x = inputs.uniform_int64(inputs.SEED_SCAN_I64, n)
    assert np.array_equal(scan_i64(api, x, lens), oracle.inclusive_scan_i64(x))


@pytest.mark.parametrize("lens", [
    [1 << 16], [1] * 64 + [(1 << 16) - 64], [0, 5, 0, 65_531, 0], [2047, 2049, 4096, 57_344],
    "random", "random_unaligned_out",
])
def test_scan_i64_segment_split_invariance(api, lens):
    n = 1 << 16
    x = inputs.uniform_int64(31, n, 0, 1000)
    out_lens = None
    if lens == "random":
        lens = inputs.random_cut_segments(7, n, 8)
    elif lens == "random_unaligned_out":
        lens = inputs.random_cut_segments(8, n, 5)
        out_lens = inputs.random_cut_segments(9, n, 7)
    assert np.array_equal(scan_i64(api, x, lens, out_lens), oracle.inclusive_scan_i64(x))


def test_scan_i64_all_small_splits(api):
    """Brute force over every split of n = 8 into up to 3 segments (empty allowed)."""
    x = inputs.uniform_int64(37, 8, 0, 1000)
    ref = oracle.inclusive_scan_i64(x)
    for a in range(9):
        for b in range(a, 9):
            lens = [a, b - a, 8 - b]
            lens = [l for l in lens] if sum(lens) == 8 else None
            assert np.array_equal(scan_i64(api, x, lens), ref)


def test_scan_i64_unaligned_and_closed_forms(api):
    n = 100_003
    x = inputs.uniform_int64(41, n, 0, 1000)
    assert np.array_equal(scan_i64(api, x, [50_001, 50_002], offset=1), oracle.inclusive_scan_i64(x))
    ones = np.ones(n, np.int64)
    assert np.array_equal(scan_i64(api, ones, [3, n - 3]), np.arange(1, n + 1))


def test_scan_i64_in_place(api):
    n = 77_777
    x = inputs.uniform_int64(43, n, 0, 1000)
    lens = [30_000, 47_777]
    v = G.segvec(x, lens)
    api.inclusive_scan(v, v)
    api.sync_status()
    assert np.array_equal(G.to_np(v), oracle.inclusive_scan_i64(x))


def test_scan_i64_full_size_roofline_case(api):
    """int64 at n = 2^28 (4 GB per array) in 4 segments 1:2:3:2: bit-exact."""
    n = 1 << 28
    lens = inputs.proportional_segments(n, [1, 2, 3, 2])
    x = inputs.uniform_int64(inputs.SEED_SCAN_I64, n)
    got = scan_i64(api, x, lens)
    assert np.array_equal(got, oracle.inclusive_scan_i64(x))


def check_f32_scan(got, x, lens, tile=None):
    tile = tile or G.scan_tile(torch.float32)
    y, s = oracle.inclusive_scan_f32_f64(x)
    err = np.abs(got.astype(np.float64) - y)
    bound = T.scan_bound(s, G.tile_index(lens, tile))
    assert np.all(err <= bound), (np.argmax(err - bound), err.max())
    return err, s


@pytest.mark.parametrize("n,lens", [(3 * 4096 + 5, None), (100_000, [1, 49_999, 0, 50_000])])
def test_scan_f32_small(api, n, lens):
    x = inputs.uniform_pm1_f32(47, n)
    lens = lens or [n]
    vx = G.segvec(x, lens)
    out = G.empty_like_vec(lens, torch.float32)
    api.inclusive_scan(vx, out)
    api.sync_status()
    check_f32_scan(G.to_np(out), x, lens)


def test_scan_f32_exact_special_cases(api):
    n = 1 << 20
    lens = inputs.block_segments(n, 8)
    ones = G.segvec(np.ones(n, np.float32), lens)
    out = G.empty_like_vec(lens, torch.float32)
    api.inclusive_scan(ones, out)
    api.sync_status()
    assert np.array_equal(G.to_np(out), np.arange(1, n + 1, dtype=np.float32))
    xi = inputs.uniform_int64(53, n, -8, 8).astype(np.float32)  # |prefix| < 2^24: exact
    api.inclusive_scan(G.segvec(xi, lens), out)
    api.sync_status()
    assert np.array_equal(G.to_np(out), oracle.inclusive_scan_i64(xi.astype(np.int64)).astype(np.float32))


def test_scan_f32_full_size_8_segments(api):
    """fp32 inclusive_scan over 2^28 elements in 8 segments (same x as the dot)."""
    n = 1 << 28
    x = inputs.uniform_pm1_f32(inputs.SEED_DOT_X, n)
    lens = inputs.block_segments(n, 8)
    vx = G.segvec(x, lens)
    out = G.empty_like_vec(lens, torch.float32)
    api.inclusive_scan(vx, out)
    api.sync_status()
    got = G.to_np(out)
    err, s = check_f32_scan(got, x, lens)
    seq = oracle.inclusive_scan_f32_seq(x)
    y, _ = oracle.inclusive_scan_f32_f64(x)
    seq_err = np.abs(seq.astype(np.float64) - y)
    print(f"scan f32 2^28: max |err|/S = {np.max(err / np.maximum(s, 1e-30)):.3e}; "
          f"max err {err.max():.3e} vs sequential fp32 {seq_err.max():.3e} "
          f"(ratio {err.max() / max(seq_err.max(), 1e-30):.3f})")
    # the tree-shaped scan must not be less accurate than the naive sequential one
    assert err.max() <= seq_err.max()


# ---------------------------------------------------------------------------
# fp32 at full size, exactly: integer-valued steps in {-1, 0, 1}.  Every partial
# sum the kernel forms (in a thread, a warp, a tile, a lookback window, the
# carry) is the sum of a contiguous range, i.e. a difference of two prefixes of
# the walk; the test checks that the walk's prefixes span less than 2^24, so
# every fp32 addition is exact and the result must equal the int64 oracle bit
# for bit.  At 2^28 elements (32768 tiles over the persistent grid) this covers
# every CTA's multi-tile lookahead and the fp32 lookback slots: a dropped,
# doubled or misplaced tile carry anywhere changes the bits.
# ---------------------------------------------------------------------------
SEED_WALK = 2406 + 100


@pytest.fixture(scope="module")
def walk_2p28():
    n = 1 << 28
    xi = inputs.uniform_int64(SEED_WALK, n, -1, 2)
    ref = oracle.inclusive_scan_i64(xi)
    span = max(int(ref.max()), 0) - min(int(ref.min()), 0)
    assert span < (1 << 24), span
    return xi, ref


def _walk_lens(kind, n):
    if kind == "8_equal":
        return inputs.block_segments(n, 8), inputs.block_segments(n, 8)
    if kind == "1:2:3:2_into_8_equal":
        return inputs.proportional_segments(n, [1, 2, 3, 2]), inputs.block_segments(n, 8)
    cut = inputs.random_cut_segments(SEED_WALK + 1, n, 6)
    lens = cut[:2] + [0] + cut[2:]                      # an empty segment in the middle
    return lens, lens


@pytest.mark.parametrize("kind", ["8_equal", "1:2:3:2_into_8_equal", "random_with_empty"])
def test_scan_f32_full_size_exact_integer_walk(api, walk_2p28, kind):
    xi, ref = walk_2p28
    n = xi.size
    lens, out_lens = _walk_lens(kind, n)
    x = xi.astype(np.float32)
    vx = G.segvec(x, lens)
    out = G.empty_like_vec(out_lens, torch.float32)
    api.inclusive_scan(vx, out)
    api.sync_status()
    got = G.to_np(out)
    bad = np.flatnonzero(got != ref.astype(np.float32))
    assert bad.size == 0, (bad[:5], got[bad[:5]], ref[bad[:5]])
    if kind == "8_equal":
        # the exclusive scan (init 0) and the reverse scan on the same walk, exactly
        api.exclusive_scan(vx, out, init=0.0)
        api.sync_status()
        exp = oracle.scan(xi, "plus", exclusive=True, init=0)
        assert np.array_equal(G.to_np(out), exp.astype(np.float32))
        api.reverse_inclusive_scan(vx, out)
        api.sync_status()
        rev = oracle.reverse_inclusive_scan_f64(xi.astype(np.float64))
        assert np.array_equal(G.to_np(out), rev.astype(np.float32))


def test_exclusive_scan(api):
    n = 60_001
    xi = inputs.uniform_int64(59, n, 0, 1000)
    lens = [20_000, 0, 40_001]
    out = G.empty_like_vec(lens, torch.int64)
    api.exclusive_scan(G.segvec(xi, lens), out, init=7)
    api.sync_status()
    assert np.array_equal(G.to_np(out), oracle.scan(xi, "plus", exclusive=True, init=7))


@pytest.mark.parametrize("op", ["max", "min"])
def test_scan_max_min(api, op):
    n = 50_000
    x = inputs.uniform_pm1_f32(61, n)
    lens = [17, 24_983, 25_000]
    out = G.empty_like_vec(lens, torch.float32)
    api.inclusive_scan(G.segvec(x, lens), out, op=op)
    api.sync_status()
    assert np.array_equal(G.to_np(out), oracle.scan(x, op).astype(np.float32))
    xi = inputs.uniform_int64(62, n, -10**15, 10**15)   # int64: both boundary-crossing and ragged
    out64 = G.empty_like_vec(lens, torch.int64)
    api.inclusive_scan(G.segvec(xi, lens), out64, op=op)
    api.sync_status()
    assert np.array_equal(G.to_np(out64), oracle.scan(xi, op))


def test_scan_over_fused_zip_transform(api):
    """scan(zip(x, y) | multiply) in int64: no intermediate array."""
    n = 40_000
    x = inputs.uniform_int64(67, n, -30, 30)
    y = inputs.uniform_int64(71, n, -30, 30)
    vx, vy = G.segvec(x, [10_000, 30_000]), G.segvec(y, [25_000, 15_000])
    out = G.empty_like_vec([n], torch.int64)
    api.inclusive_scan(api.dot_view(vx, vy), out)
    api.sync_status()
    assert np.array_equal(G.to_np(out), oracle.inclusive_scan_i64(x * y))


@pytest.mark.parametrize("n", [3 * 4096 + 77, 1 << 26])
def test_scan_over_zip_view_exact_integer_valued(api, n):
    """scan(zip(x, y) | multiply) in fp32 with x, y in {-1, 0, 1}: every product is
    exact and every partial sum a range sum of a walk whose prefixes span less than
    2^24 (checked), so the result must equal the oracle's integer scan bit for bit.
    The operands are cut differently (8 equal segments against 1:2:3:2), so the
    zip is re-segmented and tiles break at every union boundary; at 2^26 every
    CTA of the zip kernel runs many tiles (the kept-stage pipeline in steady
    state).  The reverse scan of the same view as well."""
    xi = inputs.uniform_int64(inputs.SEED_DOT_X + 91, n, -1, 2)
    yi = inputs.uniform_int64(inputs.SEED_DOT_Y + 91, n, -1, 2)
    prod = xi * yi
    fwd = oracle.inclusive_scan_i64(prod)
    assert max(int(fwd.max()), 0) - min(int(fwd.min()), 0) < (1 << 24)
    lx, ly = inputs.block_segments(n, 8), inputs.proportional_segments(n, [1, 2, 3, 2])
    view = api.dot_view(G.segvec(xi.astype(np.float32), lx), G.segvec(yi.astype(np.float32), ly))
    out = G.empty_like_vec([n // 2, n - n // 2], torch.float32)
    api.inclusive_scan(view, out)
    api.sync_status()
    assert np.array_equal(G.to_np(out), fwd.astype(np.float32))
    api.reverse_inclusive_scan(view, out)
    api.sync_status()
    assert np.array_equal(G.to_np(out), oracle.reverse_inclusive_scan_f64(prod.astype(np.float64)).astype(np.float32))


@pytest.mark.parametrize("n", [3 * 4096 + 77, 1 << 26])
def test_scan_over_one_leaf_view_exact_integer_valued(api, n):
    """scan(x | scale(-1) | add(0)) in fp32 with x in {-1, 0, 1} (the fused
    one-leaf view kernel, kept view values, 16 KB tiles): exact integer walk,
    bit-exact against the oracle, forward and reverse, over 1:2:3:2 segments."""
    xi = inputs.uniform_int64(inputs.SEED_DOT_X + 93, n, -1, 2)
    fwd = oracle.inclusive_scan_i64(-xi)
    assert max(int(fwd.max()), 0) - min(int(fwd.min()), 0) < (1 << 24)
    lens = inputs.proportional_segments(n, [1, 2, 3, 2])
    view = G.segvec(xi.astype(np.float32), lens).view().transform("scale", -1.0).transform("add", 0.0)
    out = G.empty_like_vec(lens, torch.float32)
    api.inclusive_scan(view, out)
    api.sync_status()
    assert np.array_equal(G.to_np(out), fwd.astype(np.float32))
    api.reverse_inclusive_scan(view, out)
    api.sync_status()
    assert np.array_equal(G.to_np(out), oracle.reverse_inclusive_scan_f64(-xi.astype(np.float64)).astype(np.float32))


def test_reverse_scan(api):
    n = 123_457
    g = inputs.uniform_pm1_f32(73, n)
    lens = [100, 60_000, 63_357]
    out = G.empty_like_vec(lens, torch.float32)
    api.reverse_inclusive_scan(G.segvec(g, lens), out)
    api.sync_status()
    ref = oracle.reverse_inclusive_scan_f64(g.astype(np.float64))
    absref = oracle.reverse_inclusive_scan_f64(np.abs(g).astype(np.float64))
    tiles_from_end = G.tile_index(lens, G.scan_tile(torch.float32))
    tiles_from_end = tiles_from_end.max() - tiles_from_end
    err = np.abs(G.to_np(out).astype(np.float64) - ref)
    assert np.all(err <= T.scan_bound(absref, tiles_from_end))
    gi = inputs.uniform_int64(79, n, -100, 100)
    out64 = G.empty_like_vec(lens, torch.int64)
    api.reverse_inclusive_scan(G.segvec(gi, lens), out64)
    api.sync_status()
    assert np.array_equal(G.to_np(out64), oracle.reverse_inclusive_scan_f64(gi.astype(np.float64)).astype(np.int64))


def test_bounded_wait_reports_timeout_and_recovers(api):
    """A tile that never publishes makes its successors' waits expire: the call
    reports DR_E_TIMEOUT (no hang), and the next call is correct again."""
    from paper_2406_00158_gb300 import _lib as L
    n = 64 * 4096
    x = inputs.uniform_int64(83, n, 0, 1000)
    lens = [n]
    vx = G.segvec(x, lens)
    out = G.empty_like_vec(lens, torch.int64)
    api.set_spin_limit(2000)
    try:
        api.debug_skip_publish(5)
        api.inclusive_scan(vx, out)
        with pytest.raises(L.DRError) as ei:
            api.sync_status()
        assert ei.value.status == L.DR_E_TIMEOUT
    finally:
        api.set_spin_limit(1 << 21)
        api.debug_skip_publish(-1)
    api.inclusive_scan(vx, out)
    api.sync_status()
    assert np.array_equal(G.to_np(out), oracle.inclusive_scan_i64(x))


@pytest.mark.parametrize("op", ["max", "min"])
@pytest.mark.parametrize("dt", [np.int32, np.float64])
def test_exclusive_scan_max_min_plain_and_viewed(api, op, dt):
    """Exclusive MIN / MAX scans (plain vectors take the un-interpreted kernel) and an
    exclusive PLUS scan over a transformed view (the interpreted one), several tiles
    and a ragged tail, against the definition."""
    n = 3 * 8192 + 77
    x = inputs.uniform_int64(63, n, -500, 500).astype(dt)
    lens = [5, n - 10, 5]
    tdt = torch.int32 if dt == np.int32 else torch.float64
    out = G.empty_like_vec(lens, tdt)
    init = 3
    api.exclusive_scan(G.segvec(x, lens), out, init=init, op=op)
    api.sync_status()
    assert np.array_equal(G.to_np(out), oracle.scan(x, op, exclusive=True, init=init).astype(dt))
    # exclusive PLUS over view = transform(x, scale 2) | add 1 (the view's values
    # 2x + 1 are small integers in either type: exact)
    v = G.segvec(x, lens).view().transform("scale", 2).transform("add", 1)
    api.exclusive_scan(v, out, init=0)
    api.sync_status()
    y = (2 * x.astype(np.int64) + 1).astype(dt)
    assert np.array_equal(G.to_np(out), oracle.scan(y, "plus", exclusive=True, init=0).astype(dt))


def test_scan_over_zip_view_float_within_bound(api):
    """inclusive_scan(zip(x, y) | multiply) in fp32 through the interpreted view path:
    within the scan bound of the FP64 prefix of x_i * y_i."""
    from tests import tolerances as T
    n = 5 * 8192 + 3
    x = inputs.uniform_pm1_f32(65, n)
    y = inputs.uniform_pm1_f32(66, n)
    lens_x, lens_y = [4000, n - 4000], [n // 3, n - n // 3]
    out = G.empty_like_vec([n], torch.float32)
    api.inclusive_scan(api.dot_view(G.segvec(x, lens_x), G.segvec(y, lens_y)), out)
    api.sync_status()
    prod = x.astype(np.float64) * y.astype(np.float64)   # exact products of fp32 values
    ref = oracle.inclusive_scan_f64(prod)
    absref = oracle.inclusive_scan_f64(np.abs(prod))
    pieces = [4000, n // 3 - 4000, n - n // 3]
    tiles = G.tile_index(pieces, G.scan_tile(torch.float32, view=True))
    # each product is rounded once to fp32 before the scan: one more rounding per term
    bound = T.scan_bound(absref, tiles) + 2.0 ** -24 * absref
    assert np.all(np.abs(G.to_np(out).astype(np.float64) - ref) <= bound)


@pytest.mark.parametrize("n", [3 * 8192 + 5, 700 * 8192 + 3])
def test_scan_with_carry_inclusive_and_exclusive(api, n):
    """dr_scan_with_carry: the chain starts from a device value (inclusive), or the
    value is the exclusive scan's init; a small range (the one-wave kernel) and a
    range of more tiles than one wave (the pipeline), integer-valued, exact."""
    xi = inputs.uniform_int64(2406 + 600, n, -1, 2)
    lens = [n // 3, 0, n - n // 3]
    vx = G.segvec(xi.astype(np.float32), lens)
    out = G.empty_like_vec([n], torch.float32)
    carry = torch.tensor([17.0], device="cuda")
    api.scan_with_carry(vx, out, carry)
    api.sync_status()
    assert np.array_equal(G.to_np(out), (17 + oracle.inclusive_scan_i64(xi)).astype(np.float32))
    api.scan_with_carry(vx, out, carry, exclusive=True)
    api.sync_status()
    assert np.array_equal(G.to_np(out), oracle.scan(xi, "plus", exclusive=True, init=17).astype(np.float32))
    vi = G.segvec(xi * 1000, lens)
    o64 = G.empty_like_vec([n], torch.int64)
    api.scan_with_carry(vi, o64, torch.tensor([-5], dtype=torch.int64, device="cuda"), op="max")
    api.sync_status()
    assert np.array_equal(G.to_np(o64), oracle.scan(xi * 1000, "max", init=-5))
