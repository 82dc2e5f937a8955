"""Batched execution: thousands of independent segmented vectors, y_v =
inclusive_scan(x_v) and dots[v] = <x_v, p_v> in one persistent launch (and its
CUDA-graph replay), against the oracle per vector and against the
one-launch-per-range baseline; the autotuner and its cache."""
import os

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


def build(api, shapes, pshapes=None, seed=0):
    tot = sum(map(sum, shapes))
    x = inputs.uniform_pm1_f32(inputs.SEED_BATCH_X + seed, tot)
    p = inputs.uniform_pm1_f32(inputs.SEED_BATCH_P + seed, tot)
    xs = api.packed_vectors(x, shapes)
    ps = api.packed_vectors(p, pshapes or shapes)
    ys = api.packed_vectors(None, shapes)
    dots = torch.full((len(shapes),), float("nan"), dtype=torch.float32, device="cuda")
    return x, p, xs, ps, ys, dots


def check(x, p, shapes, ys, dots, tile=4096):
    off = 0
    dh = dots.cpu().numpy()
    for v, sh in enumerate(shapes):
        n = sum(sh)
        xv, pv = x[off:off + n], p[off:off + n]
        off += n
        y = ys[v].to_tensor().cpu().numpy()
        yr, s = oracle.inclusive_scan_f32_f64(xv)
        assert np.all(np.abs(y - yr) <= T.scan_bound(s, G.tile_index(sh, tile))), v
        d, ad = oracle.dot_f64(xv, pv)
        assert abs(dh[v] - d) <= T.gamma(-(-n // tile) + 64) * ad, (v, dh[v], d)


def small_shapes():
    shapes = [[1000], [1], [3, 5], [4096], [4097, 1], [10_000, 7, 1, 20_000], [8191, 8193],
              [2] * 8, [123_457], [0, 5000, 0], [0]]
    return shapes + inputs.batch_shapes(inputs.SEED_BATCH + 7, 40, lo=1e3, hi=2e5)


@pytest.mark.parametrize("tune", [None, (128, 16, 4, 0), (256, 8, 2, 0), (512, 16, 1, 0), (256, 16, 3, 1),
                                  (256, 32, 1, 1), (256, 16, 1, 1), (256, 12, 4, 1)])
def test_batch_small_vs_oracle_repeat_graph_per_range(api, tune):
    shapes = small_shapes()
    x, p, xs, ps, ys, dots = build(api, shapes)
    b = api.Batch(xs, ps, ys, dots, tune=tune)
    for _ in range(2):  # self-cleaning workspace: a second launch is right too
        dots.fill_(float("nan"))
        b.run()
        api.sync_status()
        check(x, p, shapes, ys, dots, tile=b.tune[0] * b.tune[1])
    dots.fill_(float("nan"))
    b.run_graph()
    b.run_graph()
    api.sync_status()
    check(x, p, shapes, ys, dots, tile=b.tune[0] * b.tune[1])
    dots.fill_(float("nan"))
    b.run_per_range()
    api.sync_status()
    check(x, p, shapes, ys, dots, tile=G.scan_tile(torch.float32))
    for _ in range(2):          # captured once, replayed
        dots.fill_(float("nan"))
        b.run_per_range_graph()
        api.sync_status()
        check(x, p, shapes, ys, dots, tile=G.scan_tile(torch.float32))


def test_batch_non_aligned_partner(api):
    shapes = small_shapes()
    pshapes = [inputs.random_cut_segments(900 + v, sum(sh), 1 + v % 5) for v, sh in enumerate(shapes)]
    x, p, xs, ps, ys, dots = build(api, shapes, pshapes, seed=1)
    b = api.Batch(xs, ps, ys, dots)
    b.run()
    api.sync_status()
    check(x, p, shapes, ys, dots)


def test_batch_full_config_4096_vectors(api):
    """4096 vectors, lengths log-uniform in [1e3, 1e6], 1-8 segments each."""
    shapes = inputs.batch_shapes(inputs.SEED_BATCH, 4096)
    x, p, xs, ps, ys, dots = build(api, shapes)
    b = api.Batch(xs, ps, ys, dots)
    b.run_graph()
    api.sync_status()
    check(x, p, shapes, ys, dots, tile=b.tune[0] * b.tune[1])


def test_batch_full_config_exact_integer_valued(api):
    """The 4096-vector batch with x and p integer-valued in {-1, 0, 1}: a vector
    has at most 10^6 elements, so every partial sum of its scan and of its dot is
    an integer below 2^24 in magnitude and exact in fp32.  The one-launch run
    (graph replay) and the per-range baseline must both equal the oracle bit for
    bit: the int64 scan per vector and the FP64 (here exact) dot."""
    shapes = inputs.batch_shapes(inputs.SEED_BATCH, 4096)
    tot = sum(map(sum, shapes))
    x = inputs.uniform_int64(inputs.SEED_BATCH_X + 50, tot, -1, 2).astype(np.float32)
    p = inputs.uniform_int64(inputs.SEED_BATCH_P + 50, tot, -1, 2).astype(np.float32)
    xs, ps, ys = api.packed_vectors(x, shapes), api.packed_vectors(p, shapes), api.packed_vectors(None, shapes)
    dots = torch.full((len(shapes),), float("nan"), dtype=torch.float32, device="cuda")
    b = api.Batch(xs, ps, ys, dots)
    starts = np.concatenate([[0], np.cumsum([sum(sh) for sh in shapes])])
    for run in (b.run_graph, b.run_per_range, b.run_per_range_graph):
        dots.fill_(float("nan"))
        run()
        api.sync_status()
        dh = dots.cpu().numpy()
        yall = torch.cat([torch.cat(v.segments) for v in ys]).cpu().numpy()
        for v in range(len(shapes)):
            lo, hi = starts[v], starts[v + 1]
            xv = x[lo:hi].astype(np.int64)
            yref = oracle.inclusive_scan_i64(xv)
            assert np.array_equal(yall[lo:hi], yref.astype(np.float32)), (run.__name__, v)
            assert dh[v] == oracle.dot_f64(x[lo:hi], p[lo:hi])[0], (run.__name__, v)


def test_autotune_and_cache(api, tmp_path):
    shapes = inputs.batch_shapes(inputs.SEED_BATCH + 99, 256, lo=1e3, hi=1e5)
    x, p, xs, ps, ys, dots = build(api, shapes, seed=2)
    b = api.Batch(xs, ps, ys, dots)
    cache = str(tmp_path / "tune.json")
    chosen = b.autotune(retune=True, cache_path=cache)
    assert chosen[3] in (0, 1) and chosen[0] in (128, 256, 512) and chosen[1] in (8, 16, 32)
    assert 1 <= chosen[2] <= 8
    assert b.tune == chosen
    text = open(cache).read()
    assert '"threads": %d' % chosen[0] in text and '"variant": %d' % chosen[3] in text
    b.tune = (256, 8, 1, 0)
    assert b.autotune(retune=False, cache_path=cache) == chosen  # served from the cache
    dots.fill_(float("nan"))
    b.run()
    api.sync_status()
    check(x, p, shapes, ys, dots, tile=chosen[0] * chosen[1])
