"""for_each over k-ary zips (STREAM kernels, Black-Scholes) and transform (a
fused view written to a vector) on the GPU, through the C ABI, against the CPU
oracle: bit-exact for STREAM and integer views, the derived first-order bound
for Black-Scholes."""
import numpy as np
import pytest

import oracle
from paper_2406_00158_gb300 import inputs
from tests import gpu_util as G
from tests import tolerances as T

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

R32 = float(np.float32(inputs.BS_R))
SIG32 = float(np.float32(inputs.BS_SIGMA))


@pytest.fixture(scope="module")
def api():
    G.dev()
    from paper_2406_00158_gb300 import api
    return api


def _tdt(dt):
    return torch.float32 if dt == np.float32 else torch.float64


# ----------------------------------------------------------------------------------
# STREAM: bit-exact against the oracle in the element type
# ----------------------------------------------------------------------------------

# several 4096-element tiles, ragged tails, an empty segment, operands cut differently
STREAM_CASES = [
    (3 * 4096 + 123, [[1000, 0, 11_411], [6000, 6411], [3, 4000, 8408]], 0),
    (50_001, [[50_001], [50_001], [50_001]], 0),
    (20_000, [[7, 19_993], [10_000, 10_000], [20_000]], 1),   # unaligned segment starts
    (1, [[1], [1], [1]], 0),
]


@pytest.mark.parametrize("dt", [np.float32, np.float64])
@pytest.mark.parametrize("fn", ["copy", "scale", "add", "triad"])
@pytest.mark.parametrize("case", range(len(STREAM_CASES)))
def test_stream_bit_exact(api, dt, fn, case):
    n, lens, off = STREAM_CASES[case]
    a, b, c = inputs.stream_inputs(n, dt, key=inputs.SEED_STREAM + 10 * case)
    q = 3.0 if dt == np.float64 else float(np.float32(0.7))
    va, vb, vc = (G.segvec(x, l, offset_elems=off) for x, l in zip((a, b, c), lens))
    ops = {"copy": (va, vc), "scale": (vb, vc), "add": (va, vb, vc), "triad": (va, vb, vc)}[fn]
    z = api.View.zipn(*ops)
    args = (q,) if fn in ("scale", "triad") else ()
    api.for_each(z, fn, *args)
    api.sync_status()
    ea, eb, ec = oracle.stream(fn, a, b, c, q)
    for got, exp in zip((va, vb, vc), (ea, eb, ec)):
        assert np.array_equal(G.to_np(got), exp)


def test_stream_in_place_and_views(api):
    n = 30_000
    a, b, c = inputs.stream_inputs(n, np.float32, key=77)
    vb = G.segvec(b, [12_000, 18_000])
    # b = 2 * b in place (zip(b, b)): the written operand is the read one
    api.for_each(api.View.zipn(vb, vb), "scale", 2.0)
    api.sync_status()
    assert np.array_equal(G.to_np(vb), 2 * b)
    # operands trimmed by drop / take: c[5:] = a[100:] on the first n-100 elements
    va, vc = G.segvec(a, [n]), G.segvec(c, [4000, n - 4000])
    z = api.View.zipn(va.view().drop(100), vc.view().drop(5))
    assert z.size == n - 100
    api.for_each(z, "copy")
    api.sync_status()
    exp = c.copy()
    exp[5:5 + n - 100] = a[100:]
    assert np.array_equal(G.to_np(vc), exp)


def test_stream_overlap_rejected(api):
    from paper_2406_00158_gb300._lib import DRError
    base = torch.zeros(1000, dtype=torch.float32, device="cuda")
    va = api.SegmentedVector([base[0:500]])
    vb = api.SegmentedVector([base[8:508]])
    with pytest.raises(DRError):
        api.for_each(api.View.zipn(va, vb), "copy")


# ----------------------------------------------------------------------------------
# Black-Scholes: within the first-order bound of the FP64 oracle
# ----------------------------------------------------------------------------------

def _bs_run(api, S, X, Tm, lens, dt=np.float32, offset=0):
    vs = [G.segvec(v.astype(dt), l, offset_elems=offset) for v, l in zip((S, X, Tm), lens[:3])]
    vc = G.empty_like_vec(lens[3], _tdt(dt))
    vp = G.empty_like_vec(lens[4], _tdt(dt))
    api.for_each(api.View.zipn(*vs, vc, vp), "black_scholes", R32, SIG32)
    api.sync_status()
    return G.to_np(vc), G.to_np(vp)


@pytest.mark.parametrize("dt,u", [(np.float32, 2.0 ** -24), (np.float64, 2.0 ** -53)])
@pytest.mark.parametrize("offset", [0, 1])
def test_black_scholes_within_bound(api, dt, u, offset):
    n = 5 * 4096 + 77
    S, X, Tm = inputs.black_scholes_inputs(n)
    lens = [[n], [3000, n - 3000], [n - 1, 1], [n // 2, n - n // 2], [10, 0, n - 10]]
    call, put = _bs_run(api, S, X, Tm, lens, dt, offset)
    ec, ep, aux = oracle.black_scholes_f64(S, X, Tm, R32, SIG32, aux=True)
    bound = T.black_scholes_bound(S, X, Tm, R32, SIG32, aux, u)
    assert np.all(np.abs(call.astype(np.float64) - ec) <= bound)
    assert np.all(np.abs(put.astype(np.float64) - ep) <= bound)
    # the bound is not vacuous: prices are resolved far below their own size
    assert np.median(bound / (S + aux[:, 3])) < 2e-5 if dt == np.float32 else True


def test_black_scholes_extremes(api):
    # deep in / out of the money, short and long expiries, at the money
    S = np.array([30, 5, 20, 20, 10, 29.9, 5.1, 17.5], np.float32)
    X = np.array([1, 100, 20, 20.5, 10, 1.2, 99.5, 17.5], np.float32)
    Tm = np.array([0.25, 0.25, 10, 0.25, 1, 10, 10, 5], np.float32)
    lens = [[len(S)]] * 5
    call, put = _bs_run(api, S, X, Tm, lens)
    ec, ep, aux = oracle.black_scholes_f64(S, X, Tm, R32, SIG32, aux=True)
    bound = T.black_scholes_bound(S, X, Tm, R32, SIG32, aux)
    assert np.all(np.abs(call - ec) <= bound) and np.all(np.abs(put - ep) <= bound)
    assert np.all(call >= 0) and np.all(put >= 0)


def test_black_scholes_segmentation_invariant(api):
    # the same options under different cuts give identical bits (vector and
    # scalar paths evaluate one element function)
    n = 3 * 4096 + 5
    S, X, Tm = inputs.black_scholes_inputs(n, key=123)
    one = _bs_run(api, S, X, Tm, [[n]] * 5)
    cut = _bs_run(api, S, X, Tm, [[1, n - 1], [4097, n - 4097], [n], [3, 3, n - 6], [n]])
    assert np.array_equal(one[0], cut[0]) and np.array_equal(one[1], cut[1])


def test_black_scholes_full_size_sampled(api):
    """The benchmark's workload (2^28 options in 8 segments, the bench's launch):
    put-call parity everywhere, and the oracle on 2^16 sampled options."""
    n = 1 << 28
    S, X, Tm = inputs.black_scholes_inputs(n)
    lens = [n // 8] * 8
    dev = torch.device("cuda:0")
    vs = [api.SegmentedVector.from_tensor(torch.from_numpy(v).to(dev), lens) for v in (S, X, Tm)]
    vc = api.SegmentedVector.empty(lens, torch.float32, dev)
    vp = api.SegmentedVector.empty(lens, torch.float32, dev)
    api.for_each(api.View.zipn(*vs, vc, vp), "black_scholes", R32, SIG32)
    api.sync_status()
    c, p = vc.to_tensor(), vp.to_tensor()
    St, Xt, Tt = (v.to_tensor().double() for v in vs)
    par = (c.double() - p.double()) - (St - Xt * torch.exp(-R32 * Tt))
    assert float((par.abs() / (St + Xt)).max()) < 1e-5
    idx = np.sort(inputs.uniform_int64(5, 1 << 16, 0, n))
    ec, ep, aux = oracle.black_scholes_f64(S[idx], X[idx], Tm[idx], R32, SIG32, aux=True)
    bound = T.black_scholes_bound(S[idx], X[idx], Tm[idx], R32, SIG32, aux)
    it = torch.from_numpy(idx).to(dev)
    assert np.all(np.abs(c[it].cpu().numpy() - ec) <= bound)
    assert np.all(np.abs(p[it].cpu().numpy() - ep) <= bound)


def test_stream_triad_full_size_sampled(api):
    """STREAM triad at the benchmark's size (2^28 fp64 in 8 segments): sampled
    elements bit-exact against the oracle."""
    n = 1 << 28
    a, b, c = inputs.stream_inputs(n, np.float64)
    lens = [n // 8] * 8
    dev = torch.device("cuda:0")
    va, vb, vc = (api.SegmentedVector.from_tensor(torch.from_numpy(v).to(dev), lens) for v in (a, b, c))
    api.for_each(api.View.zipn(va, vb, vc), "triad", 3.0)
    api.sync_status()
    idx = np.sort(inputs.uniform_int64(6, 1 << 16, 0, n))
    ea, _, _ = oracle.stream("triad", a[idx], b[idx], c[idx], 3.0)
    got = va.to_tensor()[torch.from_numpy(idx).to(dev)].cpu().numpy()
    assert np.array_equal(got, ea)


# ----------------------------------------------------------------------------------
# transform: a fused view written out
# ----------------------------------------------------------------------------------

@pytest.mark.parametrize("dtype", [np.int64, np.int32])
def test_transform_integer_views_exact(api, dtype):
    n = 4 * 4096 + 9
    x = inputs.uniform_int64(31, n, -1000, 1000).astype(dtype)
    y = inputs.uniform_int64(37, n, -1000, 1000).astype(dtype)
    vx, vy = G.segvec(x, [100, n - 100]), G.segvec(y, [n // 3, n - n // 3])
    tdt = torch.int64 if dtype == np.int64 else torch.int32
    out = G.empty_like_vec([5000, n - 5000], tdt)
    api.transform(vx.view().transform("scale", 3).transform("add", -7), out)
    api.sync_status()
    assert np.array_equal(G.to_np(out), 3 * x - 7)
    api.transform(api.dot_view(vx, vy), out)
    api.sync_status()
    assert np.array_equal(G.to_np(out), x * y)
    api.transform(vx.view().zip(vy.view().transform("neg")).zip_transform("max"), out)
    api.sync_status()
    assert np.array_equal(G.to_np(out), np.maximum(x, -y))


def test_transform_float_single_rounding_and_in_place(api):
    n = 70_001
    x = inputs.uniform_pm1_f32(41, n)
    vx = G.segvec(x, [n - 3, 3], offset_elems=1)
    out = G.empty_like_vec([n], torch.float32)
    api.transform(vx.view().transform("scale", 0.3), out)
    api.sync_status()
    assert np.array_equal(G.to_np(out), x * np.float32(0.3))
    api.transform(vx.view().transform("square"), vx)   # in place
    api.sync_status()
    assert np.array_equal(G.to_np(vx), x * x)


def test_for_each_follows_a_rebound_vector():
    """for_each over a zip whose vectors were rebound to new storage writes the new storage."""
    G.dev()
    from paper_2406_00158_gb300 import api
    n = 4 * 1024 + 3
    a, b, c = inputs.stream_inputs(n, np.float64)
    va, vb, vc = G.segvec(a, [n]), G.segvec(b, [n]), G.segvec(c, [n])
    z = api.View.zipn(va, vb, vc)
    a2, b2, c2 = inputs.stream_inputs(n, np.float64, key=inputs.SEED_STREAM + 10)
    new = [G.guarded_segment(n, torch.float64) for _ in range(3)]
    for t, v in zip(new, (a2, b2, c2)):
        t.copy_(torch.from_numpy(v))
    va.rebind([new[0]]), vb.rebind([new[1]]), vc.rebind([new[2]])
    api.for_each(z, "triad", 3.0)
    api.sync_status()
    assert np.array_equal(new[0].cpu().numpy(), oracle.stream("triad", a2, b2, c2, 3.0)[0])
    assert np.array_equal(va._bases[0].cpu().numpy(), a)     # the old storage was not written
