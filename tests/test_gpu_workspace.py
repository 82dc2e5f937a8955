"""Workspaces of views come from the library's stream-ordered pool and are freed
behind their last use: many short-lived views stay correct and keep device
memory bounded; views used on different streams do not interfere."""
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


def test_short_lived_views_are_correct_and_memory_bounded(api):
    n = 1 << 24  # sort scratch ~ 2 x 64 MiB + counts per view
    dev = torch.device("cuda:0")
    x = inputs.uniform_pm1_f32(91, n)
    vx = api.SegmentedVector.from_tensor(torch.from_numpy(x).to(dev), [n // 4] * 4)
    out = api.SegmentedVector.empty([n], torch.float32, dev)
    ref_sort = oracle.sort(x)
    ref_scan, absx = oracle.inclusive_scan_f32_f64(x)
    api.sort(vx, out)          # warm the pool
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for it in range(20):       # every call builds a new view (and workspace) and drops it
        api.sort(vx, out)
        if it % 5 == 4:
            api.sync_status()
            assert np.array_equal(G.to_np(out), ref_sort)
        api.inclusive_scan(vx, out)
        if it % 5 == 4:
            api.sync_status()
            assert np.all(np.abs(G.to_np(out) - ref_scan) <= 1e-5 * absx + 1e-30)
    torch.cuda.synchronize()
    drop = free0 - torch.cuda.mem_get_info()[0]
    assert drop < (1 << 30), f"device memory fell by {drop / 2**20:.0f} MiB over 20 sorts"


def test_views_on_two_streams(api):
    n = 1 << 22
    dev = torch.device("cuda:0")
    xs = [inputs.uniform_int64(93 + k, n, -1000, 1000) for k in range(2)]
    vs = [api.SegmentedVector.from_tensor(torch.from_numpy(x).to(dev), [n // 2, n // 2]) for x in xs]
    outs = [api.SegmentedVector.empty([n], torch.int64, dev) for _ in range(2)]
    views = [v.view() for v in vs]
    streams = [torch.cuda.Stream() for _ in range(2)]
    torch.cuda.synchronize()
    for _ in range(5):
        for k in range(2):
            api.inclusive_scan(views[k], outs[k], stream=streams[k])
    torch.cuda.synchronize()
    api.sync_status()
    for k in range(2):
        assert np.array_equal(G.to_np(outs[k]), oracle.inclusive_scan_i64(xs[k]))
    del views  # released behind each stream's last use
    torch.cuda.synchronize()
