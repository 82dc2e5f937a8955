"""The usage example of the design notes, run as written and checked against the
oracle (so the example cannot drift from the API)."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_usage_example():
    from tests import gpu_util as G
    G.dev()
    from paper_2406_00158_gb300 import api, autograd as AG

    dev = torch.device("cuda:0")
    g = torch.Generator(device=dev)
    g.manual_seed(7)
    xt = torch.rand(1 << 20, device=dev, generator=g)
    yt = torch.rand(1 << 20, device=dev, generator=g)
    x = api.SegmentedVector.from_tensor(xt.clone(), [1 << 18] * 4)
    y = api.SegmentedVector.from_tensor(yt.clone(), [1 << 19] * 2)
    out = api.SegmentedVector.empty([1 << 20], torch.float32, dev)
    d = torch.zeros(1, device=dev)
    xn, yn = xt.cpu().numpy(), yt.cpu().numpy()

    api.transform_reduce(api.dot_view(x, y), d)
    api.sync_status()
    dref, aref = oracle.dot_f64(xn, yn)
    assert abs(d.item() - dref) <= 1e-5 * aref

    api.inclusive_scan(x, out)
    api.sync_status()
    sref, absref = oracle.inclusive_scan_f32_f64(xn)
    assert np.all(np.abs(G.to_np(out) - sref) <= 1e-5 * absref + 1e-30)

    api.exclusive_scan(x.view().transform("scale", 2.0), out, init=0.0, op="plus")
    api.sync_status()
    eref, eabs = oracle.inclusive_scan_f32_f64(2 * xn)
    got = G.to_np(out)
    assert got[0] == 0.0 and np.all(np.abs(got[1:] - eref[:-1]) <= 1e-5 * eabs[:-1] + 1e-30)

    api.transform(x.view().zip(y.view()).zip_transform("max"), out)
    api.sync_status()
    assert np.array_equal(G.to_np(out), np.maximum(xn, yn))

    api.for_each(api.View.zipn(x, y, out), "triad", 3.0)  # x = y + 3 * out
    api.sync_status()
    a_ref, _, _ = oracle.stream("triad", xn, yn, np.maximum(xn, yn), 3.0)
    assert np.array_equal(G.to_np(x), a_ref)

    api.sort(x, out)
    api.sync_status()
    assert np.array_equal(G.to_np(out), oracle.sort(a_ref))

    segs = [t.clone().requires_grad_(True) for t in torch.rand(1024, device=dev, generator=g).split(256)]
    ys = AG.inclusive_scan(segs)
    torch.autograd.backward(list(ys), [torch.ones(256, device=dev)] * 4)
    gx = torch.cat([s.grad for s in segs]).cpu().numpy()
    assert np.array_equal(gx, np.arange(1024, 0, -1, dtype=np.float32))  # reverse scan of ones
