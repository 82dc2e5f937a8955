"""The seeded input recipe (CPU): the generators produce the ranges, distributions
and segmentations the design notes state, deterministically."""
import math

import numpy as np

from paper_2406_00158_gb300 import inputs


def test_value_maps_are_exact_and_in_range():
    u = inputs.uniform01_f32(1, 1 << 16)
    assert u.dtype == np.float32 and u.min() >= 0 and u.max() < 1
    assert np.all(u * np.float32(2 ** 24) == np.round(u * np.float32(2 ** 24)))   # k * 2^-24
    v = inputs.uniform_pm1_f32(1, 1 << 16)
    assert v.min() >= -1 and v.max() < 1
    d = inputs.uniform01_f64(1, 1 << 16)
    assert d.dtype == np.float64 and d.min() >= 0 and d.max() < 1
    i = inputs.uniform_int64(1, 1 << 16, -5, 7)
    assert i.min() == -5 and i.max() == 6 and set(np.unique(i)) == set(range(-5, 7))
    assert np.array_equal(inputs.uniform01_f32(1, 1000), inputs.uniform01_f32(1, 1000))  # seeded


def test_chunked_generation_matches_one_piece():
    n = (1 << 21) + 12345           # more than one internal chunk
    a = inputs.raw_u64(9, n)
    b = np.concatenate([inputs.raw_u64(9, 1000), inputs.raw_u64(9, n - 1000, start=1000)])
    assert np.array_equal(a, b)


def test_segmentations():
    assert inputs.proportional_segments(1 << 20, [1, 2, 3, 2]) == [131072, 262144, 393216, 262144]
    assert inputs.block_segments(10, 4) == [3, 3, 3, 1]
    assert inputs.block_segments(8, 5) == [2, 2, 2, 2, 0]
    for trial in range(20):
        cuts = inputs.random_cut_segments(100 + trial, 50, 1 + trial % 9)
        assert sum(cuts) == 50 and all(c >= 1 for c in cuts) and len(cuts) == 1 + trial % 9
    assert inputs.random_cut_segments(5, 3, 8) == [1, 1, 1]   # fewer cuts when n is small


def test_batch_shapes_follow_the_recipe():
    shapes = inputs.batch_shapes(inputs.SEED_BATCH, 4096)
    lens = np.array([sum(s) for s in shapes], dtype=np.float64)
    nseg = np.array([len(s) for s in shapes])
    assert lens.min() >= 1e3 - 1 and lens.max() <= 1e6 + 1
    # log-uniform on [1e3, 1e6]: mean (1e6 - 1e3) / ln(1e3) = 144,613; log-mean at ln(31,623)
    assert abs(lens.mean() / ((1e6 - 1e3) / math.log(1e3)) - 1) < 0.05
    assert abs(np.log(lens).mean() - math.log(math.sqrt(1e9))) < 0.05
    assert nseg.min() == 1 and nseg.max() == 8 and abs(nseg.mean() - 4.5) < 0.15
    assert all(min(s) >= 1 for s in shapes)


def test_black_scholes_and_stream_recipes():
    S, X, T = inputs.black_scholes_inputs(1 << 16)
    for a, (lo, hi) in zip((S, X, T), (inputs.BS_S_RANGE, inputs.BS_X_RANGE, inputs.BS_T_RANGE)):
        assert a.dtype == np.float32 and a.min() >= lo and a.max() < hi + 1e-5
        assert abs(a.mean() - (lo + hi) / 2) < 0.01 * (hi - lo)
    a, b, c = inputs.stream_inputs(1 << 16)
    assert a.dtype == np.float64 and min(a.min(), b.min(), c.min()) >= -1 and max(a.max(), b.max(), c.max()) < 1
    assert not np.array_equal(a, b) and not np.array_equal(b, c)   # one stream per array
    f = inputs.stream_inputs(1 << 10, np.float32)
    assert all(v.dtype == np.float32 for v in f)
