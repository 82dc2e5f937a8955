"""transform_reduce (Algorithm 3) and the dot product of Algorithm 1 on the GPU,
through the C ABI, against the CPU oracle."""
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


def run_dot(api, x, y, lx, ly, offset=0):
    vx, vy = G.segvec(x, lx, offset_elems=offset), G.segvec(y, ly, offset_elems=offset)
    out = torch.full((1,), float("nan"), dtype=torch.float32, device="cuda")
    api.transform_reduce(api.dot_view(vx, vy), out)
    api.sync_status()
    return float(out.item())


@pytest.mark.parametrize("n,lx,ly,offset", [
    (3 * 4096 + 17, None, None, 0),                  # several tiles + ragged tail, one segment
    (50_003, [10_000, 0, 25_001, 15_002], None, 0),  # uneven, with an empty segment
    (50_003, [10_000, 40_003], [7, 29_996, 20_000], 0),  # non-aligned zip (re-segmented)
    (20_000, [5_001, 14_999], None, 1),              # unaligned pointers: scalar path
    (1, None, None, 0), (0, None, None, 0),
])
def test_dot_small_vs_oracle(api, n, lx, ly, offset):
    x = inputs.uniform_pm1_f32(inputs.SEED_DOT_X, n)
    y = inputs.uniform_pm1_f32(inputs.SEED_DOT_Y, n)
    lx = lx or [n]
    ly = ly or lx
    got = run_dot(api, x, y, lx, ly, offset)
    d, ad = oracle.dot_f64(x, y)
    assert abs(got - d) <= T.dot_bound(n, ad, G.sms()) + 1e-30, (got, d)


def test_dot_closed_forms(api):
    n = 1 << 22
    lens = inputs.block_segments(n, 8)
    for a, b in [(0.5, 0.25), (-2.0, 0.125)]:
        got = run_dot(api, np.full(n, a, np.float32), np.full(n, b, np.float32), lens, lens)
        assert got == n * a * b  # every partial is k * 2^m with few bits: exact
    m = 4096
    assert run_dot(api, np.arange(m, dtype=np.float32), np.ones(m, np.float32), [m], [m]) == m * (m - 1) // 2


def test_dot_full_size_8_segments(api):
    """fp32 dot over 2^28 elements in 8 equal segments (the headline workload)."""
    n = 1 << 28
    x = inputs.uniform_pm1_f32(inputs.SEED_DOT_X, n)
    y = inputs.uniform_pm1_f32(inputs.SEED_DOT_Y, n)
    lens = inputs.block_segments(n, 8)
    got = run_dot(api, x, y, lens, lens)
    again = run_dot(api, x, y, lens, lens)
    d, ad = oracle.dot_f64(x, y)
    assert abs(got - d) <= T.dot_bound(n, ad, G.sms()), (got, d, ad)
    assert got == again  # fixed reduction tree: run-to-run reproducible
    print(f"dot n=2^28: got {got!r} oracle {d!r} normalized err {abs(got - d) / ad:.3e} "
          f"bound {T.dot_bound(n, ad, G.sms()) / ad:.3e}")


@pytest.mark.parametrize("dtype,op", [(np.int64, "plus"), (np.int32, "plus"), (np.int64, "max"),
                                      (np.int64, "min"), (np.int32, "mul"), (np.float64, "plus"),
                                      (np.float32, "plus"), (np.float32, "max"), (np.float64, "min")])
def test_reduce_ops_and_dtypes(api, dtype, op):
    """Every operator and element type against the oracle's reduce: integers and
    MIN / MAX exactly; float PLUS within the derived bound of the EXACT sum."""
    import math
    from fractions import Fraction
    n = 70_001
    lens = inputs.random_cut_segments(5, n, 5)
    if op == "mul":
        x = inputs.uniform_int64(17, n, -1, 2).astype(dtype)       # products stay small: +-1, 0
        x[x == 0] = 1
    elif np.issubdtype(dtype, np.integer):
        x = inputs.uniform_int64(17, n, -1000, 1000).astype(dtype)
    else:
        x = inputs.uniform_pm1_f32(17, n).astype(dtype)
    vx = G.segvec(x, lens)
    out = torch.zeros(1, dtype=torch.from_numpy(x[:1]).dtype, device="cuda")
    init = {"plus": 3, "max": -(10**6), "min": 10**6, "mul": -1}[op]
    api.transform_reduce(vx, out, op=op, init=init)
    api.sync_status()
    got = out.item()
    exp = oracle.reduce(x, op, init=init)
    if np.issubdtype(dtype, np.floating) and op == "plus":
        esz = np.dtype(dtype).itemsize
        scale = math.fsum(np.abs(x.astype(np.float64))) + abs(init)
        err = abs(Fraction(got) - exp)
        assert err <= Fraction(T.reduce_bound(n, scale, G.sms(), esz)), (got, float(exp))
    else:
        assert got == exp


def test_reduce_fused_transform_view(api):
    """sum of (2*x + 1)^2 over a transformed view, computed in one kernel."""
    n = 40_000
    xi = inputs.uniform_int64(23, n, -50, 50)
    vx = G.segvec(xi, [12_000, 28_000])
    v = vx.view().transform("scale", 2).transform("add", 1).transform("square")
    out = torch.zeros(1, dtype=torch.int64, device="cuda")
    api.transform_reduce(v, out)
    api.sync_status()
    assert out.item() == oracle.reduce((2 * xi + 1) ** 2, "plus")


def test_reduce_take_drop(api):
    n = 30_000
    xi = inputs.uniform_int64(29, n, 0, 1000)
    vx = G.segvec(xi, [10_000, 10_000, 10_000])
    out = torch.zeros(1, dtype=torch.int64, device="cuda")
    api.transform_reduce(vx.view().drop(9_999).take(10_003), out)
    api.sync_status()
    lens = [10_000, 10_000, 10_000]
    kept = oracle.gather_segments(xi, lens, oracle.trim_segments(lens, 9_999, 9_999 + 10_003))
    assert out.item() == oracle.reduce(kept, "plus")
    # a scan over take / drop as well, into an output of another segmentation
    o = G.empty_like_vec([3, 10_000], torch.int64)
    api.inclusive_scan(vx.view().take(25_000).drop(14_997), o)
    api.sync_status()
    kept = oracle.gather_segments(xi, lens, oracle.trim_segments(lens, 14_997, 25_000))
    assert np.array_equal(G.to_np(o), oracle.inclusive_scan_i64(kept))
