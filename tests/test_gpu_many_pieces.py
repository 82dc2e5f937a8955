"""Ranges of more segments than a launch carries inline (128 pieces after
re-segmentation): scan, reduce, transform and for_each keep the piece table in
device memory and must give the same results, against the oracle -- the
paper's model has one segment per memory locale, so the segment count grows
with the machine."""
import numpy as np
import pytest

import oracle
from paper_2406_00158_gb300 import inputs
from tests import gpu_util as G

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def api():
    G.dev()
    from paper_2406_00158_gb300 import api
    return api


def test_scan_reduce_transform_over_300_segments(api):
    n = 300 * 1000 + 4321
    lens = inputs.random_cut_segments(2406 + 500, n, 300)
    lens = lens[:10] + [0, 0] + lens[10:]                   # empty segments among them
    assert len(lens) > 128
    xi = inputs.uniform_int64(2406 + 501, n, -1000, 1000)
    vx = G.segvec(xi, lens)
    out = G.empty_like_vec(inputs.random_cut_segments(2406 + 502, n, 7), torch.int64)  # 300+ pieces zipped
    api.inclusive_scan(vx, out)
    api.sync_status()
    assert np.array_equal(G.to_np(out), oracle.inclusive_scan_i64(xi))
    api.exclusive_scan(vx, out, init=-4, op="max")
    api.sync_status()
    assert np.array_equal(G.to_np(out), oracle.scan(xi, "max", exclusive=True, init=-4))
    r = torch.zeros(1, dtype=torch.int64, device="cuda")
    api.transform_reduce(vx, r)
    api.sync_status()
    assert r.item() == oracle.reduce(xi, "plus")
    api.transform(vx.view().transform("scale", 2), out)
    api.sync_status()
    assert np.array_equal(G.to_np(out), 2 * xi)
    # a zip of two vectors cut differently: 129 + 129 boundaries
    yi = inputs.uniform_int64(2406 + 503, n, -1000, 1000)
    vy = G.segvec(yi, inputs.block_segments(n, 129))
    api.transform_reduce(api.dot_view(vx, vy), r)
    api.sync_status()
    assert r.item() == oracle.reduce(xi * yi, "plus")


def test_for_each_over_200_segments(api):
    n = 200 * 777 + 5
    a, b, c = inputs.stream_inputs(n, np.float64)
    la = inputs.block_segments(n, 200)
    va, vb, vc = G.segvec(a, la), G.segvec(b, inputs.block_segments(n, 3)), G.segvec(c, [n])
    api.for_each(api.View.zipn(va, vb, vc), "triad", 3.0)
    api.sync_status()
    assert np.array_equal(G.to_np(va), oracle.stream("triad", a, b, c, 3.0)[0])
