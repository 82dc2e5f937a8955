"""Halo-exchanging 5-point Jacobi for_each over a row-block segmented array on
the GPU, against the CPU oracle: bit-exact against the fixed-order fp32
oracle, within the contraction bound of the FP64 oracle."""
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


def run(api, u0, seg_rows, steps, wc=0.0, wn=0.25, transpose=False):
    u = torch.from_numpy(u0).cuda()
    a = G.md_from(u, seg_rows)                  # guarded blocks, sentinel outer ghost rows
    b = G.md_empty(seg_rows, u0.shape[1])
    t = G.md_empty(seg_rows, u0.shape[1]) if steps > 1 else None
    (api.stencil5_T if transpose else api.stencil5)(a, b, t, steps, wc, wn)
    api.sync_status()
    return b.to_tensor().cpu().numpy()


@pytest.mark.parametrize("R,C,seg_rows,steps", [
    (150, 1040, [64, 40, 46], 1),        # several CTAs per block, ragged row blocks, 3 column blocks
    (150, 1040, [64, 40, 46], 7),
    (97, 33, [1, 50, 46], 5),            # cols % 4 != 0: scalar path; a 1-row block
    (64, 64, [64], 3),
    (200, 516, [7] * 20 + [60], 4),      # many thin blocks
])
def test_stencil_bit_exact_small(api, R, C, seg_rows, steps):
    u0 = inputs.uniform01_f32(inputs.SEED_STENCIL, R * C).reshape(R, C)
    got = run(api, u0, seg_rows, steps)
    ref = oracle.stencil5_f32(u0, steps)
    assert np.array_equal(got.view(np.int32), ref.view(np.int32))
    ref64 = oracle.stencil5_f64(u0, steps)
    assert np.abs(got - ref64).max() <= T.stencil_f64_bound(steps, np.abs(u0).max())


def test_stencil_weights_and_transpose(api):
    R, C = 80, 128
    u0 = inputs.uniform_pm1_f32(91, R * C).reshape(R, C)
    got = run(api, u0, [30, 50], 3, wc=0.3, wn=0.15)
    assert np.array_equal(got.view(np.int32), oracle.stencil5_f32(u0, 3, 0.3, 0.15).view(np.int32))
    gotT = run(api, u0, [30, 50], 3, wc=0.3, wn=0.15, transpose=True)
    refT = oracle.stencil5_T_f64(u0.astype(np.float64), 3, 0.3, 0.15)
    assert np.abs(gotT - refT).max() <= 3 * 3 * T.U32 * 2.0


def test_stencil_segment_count_invariance(api):
    R, C = 256, 512
    u0 = inputs.uniform01_f32(93, R * C).reshape(R, C)
    base = run(api, u0, [R], 6)
    for seg_rows in ([128, 128], [1] * 64 + [192], inputs.random_cut_segments(3, R, 8)):
        assert np.array_equal(run(api, u0, seg_rows, 6).view(np.int32), base.view(np.int32))


def test_stencil_linear_field_harmonic(api):
    R, C, t = 128, 256, 9
    i = np.arange(R)[:, None].astype(np.float32)
    j = np.arange(C)[None, :].astype(np.float32)
    u0 = (3 * i - 2 * j + 5).astype(np.float32)
    got = run(api, u0, [40, 88], t)
    far = np.minimum(np.minimum(i, R - 1 - i), np.minimum(j, C - 1 - j)) >= t
    assert np.array_equal(got[far], u0[far])


def test_stencil_full_size_1_and_100_steps(api):
    """16384 x 16384 fp32, 8 row blocks of 2048, 1-row halos, zero boundary:
    full comparison after 1 step, sampled cells (corners, edges, block
    boundaries, random) after 100 steps."""
    R = C = 16384
    seg_rows = [2048] * 8
    u0 = inputs.uniform01_f32(inputs.SEED_STENCIL, R * C).reshape(R, C)
    got1 = run(api, u0, seg_rows, 1)
    ref1 = oracle.stencil5_f32(u0, 1)
    assert np.array_equal(got1.view(np.int32), ref1.view(np.int32))
    del got1, ref1
    got = run(api, u0, seg_rows, 100)
    cells = [(0, 0), (0, C - 1), (R - 1, 0), (R - 1, C - 1), (0, 5000), (R - 1, 77), (9, C - 1)]
    for b in range(1, 8):
        r = 2048 * b
        cells += [(r - 1, 1000 + b), (r, 3000 + b), (r - 2, C - 1), (r + 1, 0)]
    rnd = inputs.uniform_int64(95, 2 * 40, 0, R)
    cells += [(int(rnd[2 * k]), int(rnd[2 * k + 1])) for k in range(40)]
    cells = np.array(cells, np.int64)
    at32 = oracle.stencil5_f32_at(u0, 100, cells)
    assert np.array_equal(got[cells[:, 0], cells[:, 1]].view(np.int32), at32.view(np.int32))
    at64 = oracle.stencil5_f64_at(u0, 100, cells)
    assert np.abs(got[cells[:, 0], cells[:, 1]] - at64).max() <= T.stencil_f64_bound(100, 1.0)
