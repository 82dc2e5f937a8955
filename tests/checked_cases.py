"""Small cases of every kernel family, run against whichever build of the
library DR_GB300_LIB names (tests/test_gpu_checked.py points it at the
range-checked build).  Every case must leave the device status word clean
(dr_sync_status: no DR_E_BOUNDS from a failed address check) and match the
oracle.  Prints "checked cases ok" at the end."""
import os
import sys

import numpy as np
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2406_00158_gb300 import api, inputs  # noqa: E402
from tests import gpu_util as G  # noqa: E402


def main():
    assert os.environ.get("DR_GB300_LIB"), "DR_GB300_LIB must name the build under test"
    dev = torch.device("cuda:0")
    n = 5 * 8192 + 77
    lens = [100, 0, 20_000, n - 20_100]
    x = inputs.uniform_pm1_f32(901, n)
    y = inputs.uniform_pm1_f32(902, n)
    xi = inputs.uniform_int64(903, n, -1000, 1000)
    # scans: fp32 integer-valued (exact), int64, exclusive, reverse, a zip view, unaligned
    w = inputs.uniform_int64(904, n, -1, 2).astype(np.float32)
    o = G.empty_like_vec(lens, torch.float32)
    api.inclusive_scan(G.segvec(w, lens), o)
    api.sync_status()
    assert np.array_equal(G.to_np(o), oracle.inclusive_scan_i64(w.astype(np.int64)).astype(np.float32))
    o64 = G.empty_like_vec([n], torch.int64)
    api.exclusive_scan(G.segvec(xi, lens, offset_elems=1), o64, init=3)
    api.sync_status()
    assert np.array_equal(G.to_np(o64), oracle.scan(xi, "plus", exclusive=True, init=3))
    api.reverse_inclusive_scan(G.segvec(w, lens), o)
    api.sync_status()
    assert np.array_equal(G.to_np(o), oracle.reverse_inclusive_scan_f64(w.astype(np.float64)).astype(np.float32))
    api.inclusive_scan(api.dot_view(G.segvec(xi, lens), G.segvec(xi, [n])), o64)
    api.sync_status()
    assert np.array_equal(G.to_np(o64), oracle.inclusive_scan_i64(xi * xi))
    # reduce: dot, int64 max, a fused chain
    d = torch.zeros(1, device=dev)
    api.transform_reduce(api.dot_view(G.segvec(w, lens), G.segvec(w, [7, n - 7])), d)
    api.sync_status()
    assert d.item() == float(np.abs(w).sum())
    r = torch.zeros(1, dtype=torch.int64, device=dev)
    api.transform_reduce(G.segvec(xi, lens, offset_elems=1), r, op="max", init=-10**9)
    api.sync_status()
    assert r.item() == oracle.reduce(xi, "max")
    # transform and for_each (STREAM triad bit-exact)
    api.transform(G.segvec(xi, lens).view().transform("scale", 3).transform("add", 1), o64)
    api.sync_status()
    assert np.array_equal(G.to_np(o64), 3 * xi + 1)
    a, b, c = inputs.stream_inputs(n, np.float64)
    va, vb, vc = G.segvec(a, lens), G.segvec(b, [n]), G.segvec(c, [9, n - 9])
    api.for_each(api.View.zipn(va, vb, vc), "triad", 3.0)
    api.sync_status()
    assert np.array_equal(G.to_np(va), oracle.stream("triad", a, b, c, 3.0)[0])
    # sort (fp32 and int64)
    so = G.empty_like_vec([n // 3, n - n // 3], torch.float32)
    api.sort(G.segvec(x, lens), so)
    api.sync_status()
    assert np.array_equal(G.to_np(so).view(np.uint32), oracle.sort(x).view(np.uint32))
    so64 = G.empty_like_vec([n], torch.int64)
    api.sort(G.segvec(xi, lens), so64)
    api.sync_status()
    assert np.array_equal(G.to_np(so64), oracle.sort(xi))
    # stencil: several steps, a 1-row block, the scalar path, and the inner / outer split
    for R, C, rows in ((150, 1040, [64, 40, 1, 45]), (97, 33, [50, 47])):
        u0 = inputs.uniform01_f32(905, R * C).reshape(R, C)
        A = G.md_from(torch.from_numpy(u0).to(dev), rows)
        B, T = G.md_empty(rows, C), G.md_empty(rows, C)
        api.stencil5(A, B, T, 3)
        api.sync_status()
        assert np.array_equal(B.to_tensor().cpu().numpy(), oracle.stencil5_f32(u0, 3))
        api.stencil5_part(A, B, "inner")
        api.stencil5_part(A, B, "outer")
        api.sync_status()
        assert np.array_equal(B.to_tensor().cpu().numpy(), oracle.stencil5_f32(u0, 1))
    # batched, both kernel variants
    shapes = [[1000], [3, 5], [4096], [4097, 1], [10_000, 7, 1, 20_000], [0]]
    tot = sum(map(sum, shapes))
    bx = inputs.uniform_int64(906, tot, -1, 2).astype(np.float32)
    xs, ps, ys = api.packed_vectors(bx, shapes), api.packed_vectors(bx, shapes), api.packed_vectors(None, shapes)
    dots = torch.zeros(len(shapes), device=dev)
    bt = api.Batch(xs, ps, ys, dots)
    for tune in ((256, 16, 2, 0), (256, 16, 3, 1)):
        bt.tune = tune
        bt.run()
        api.sync_status()
        off = 0
        for v, sh in enumerate(shapes):
            m = sum(sh)
            ref = oracle.inclusive_scan_i64(bx[off:off + m].astype(np.int64)).astype(np.float32)
            assert np.array_equal(ys[v].to_tensor().cpu().numpy(), ref), (tune, v)
            assert dots[v].item() == float(np.abs(bx[off:off + m]).sum()), (tune, v)
            off += m
    bad = G.check_guards()
    assert not bad, bad
    print("checked cases ok", flush=True)


if __name__ == "__main__":
    main()
