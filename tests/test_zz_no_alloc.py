"""The allocation-free dot product (dr_dot_f32_noalloc) against the regular
transform_reduce entry point and the oracle, through the C ABI.

It exists for callers that cannot allocate device memory at the call (a
framework owning all device memory through its pool, or a latency-critical loop
that cannot pay for cudaMalloc / cudaFree): its scratch is a fixed device array
of the library.  It runs the same reduce kernel on the same grid as
dr_transform_reduce, so the two results must be bit-identical.  Two calls in a
row must both be right, since every call reuses the array left by the previous
one.  This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2406_00158_gb300 import inputs
from tests import gpu_util as G
from tests import tolerances as T

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _call(lib, vx, vy, lens, out, init=0.0):
    k = len(lens)
    lens_c = (ctypes.c_int64 * k)(*lens)
    xs = (ctypes.c_void_p * k)(*[s.data_ptr() for s in vx.segments])
    ys = (ctypes.c_void_p * k)(*[s.data_ptr() for s in vy.segments])
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return lib.dr_dot_f32_noalloc(k, lens_c, xs, ys, ctypes.c_float(init), ctypes.c_void_p(out.data_ptr()),
                                  stream)


@pytest.mark.parametrize("init", [0.0, 2.5])
def test_noalloc_dot_matches_transform_reduce_twice(init):
    G.dev()
    from paper_2406_00158_gb300 import _lib as L
    from paper_2406_00158_gb300 import api
    lib = L.lib()
    n = 7 * 4096 + 1234
    lens = [3000, 0, 20_000, n - 23_000]
    x = inputs.uniform_pm1_f32(inputs.SEED_DOT_X, n)
    y = inputs.uniform_pm1_f32(inputs.SEED_DOT_Y, n)
    vx, vy = G.segvec(x, lens), G.segvec(y, lens)
    ref = torch.zeros(1, dtype=torch.float32, device="cuda")
    api.transform_reduce(api.dot_view(vx, vy), ref, init=init)
    api.sync_status()
    d, ad = oracle.dot_f64(x, y)
    tol = T.dot_bound(n, ad + abs(init), G.sms())
    for _ in range(2):
        out = torch.full((1,), float("nan"), dtype=torch.float32, device="cuda")
        assert _call(lib, vx, vy, lens, out, init) == L.DR_OK, L.last_error()
        assert L.last_error() == ""
        api.sync_status()
        got = float(out.item())
        assert got == float(ref.item())          # same kernel, same grid: same bits
        assert abs(got - (d + init)) <= tol


def test_noalloc_dot_all_segments_empty():
    G.dev()
    from paper_2406_00158_gb300 import _lib as L
    from paper_2406_00158_gb300 import api
    lib = L.lib()
    lens = [0, 0, 0]
    vx, vy = G.segvec(np.zeros(0, np.float32), lens), G.segvec(np.zeros(0, np.float32), lens)
    for _ in range(2):
        out = torch.full((1,), float("nan"), dtype=torch.float32, device="cuda")
        assert _call(lib, vx, vy, lens, out, 1.75) == L.DR_OK, L.last_error()
        api.sync_status()
        assert float(out.item()) == 1.75         # the empty sum is init


def test_noalloc_dot_rejects_too_many_segments():
    G.dev()
    from paper_2406_00158_gb300 import _lib as L
    lib = L.lib()
    k = 129
    lens = (ctypes.c_int64 * k)(*([1] * k))
    ptrs = (ctypes.c_void_p * k)(*([1 << 20] * k))
    out = torch.zeros(1, dtype=torch.float32, device="cuda")
    rc = lib.dr_dot_f32_noalloc(k, lens, ptrs, ptrs, ctypes.c_float(0.0), ctypes.c_void_p(out.data_ptr()), None)
    assert rc == L.DR_E_UNSUPPORTED
    assert "at most 128" in L.last_error()
