"""Adjoint kernels behind torch.autograd.Function (reverse scan, scale-by-partner,
transposed stencil with checkpointed weight gradients): checked against FP64
central finite differences of the oracle on small inputs and against FP64
reference adjoints at full size."""
import math

import numpy as np
import pytest

import oracle
from paper_2406_00158_gb300 import inputs
from tests import gpu_util as G
from tests import tolerances as T

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ag():
    G.dev()
    from paper_2406_00158_gb300 import autograd
    return autograd


def split(t, lens):
    out, off = [], 0
    for n in lens:
        out.append(t[off:off + n].clone().requires_grad_(True))
        off += n
    return out


def test_scan_grad_vs_fd_n256(ag):
    n = 256
    lens = inputs.block_segments(n, 8)
    x = inputs.uniform_pm1_f32(inputs.SEED_GRAD, n)
    w = inputs.uniform_pm1_f32(inputs.SEED_GRAD + 1, n)
    segs = split(torch.from_numpy(x).cuda(), lens)
    ys = ag.inclusive_scan(segs)
    loss = (torch.cat(ys) * torch.from_numpy(w).cuda()).sum()
    loss.backward()
    g = torch.cat([s.grad for s in segs]).cpu().numpy().astype(np.float64)
    wd = w.astype(np.float64)
    fd = oracle.fd_gradient(lambda v: float(np.dot(wd, oracle.inclusive_scan_f64(v))), x.astype(np.float64))
    absw = oracle.reverse_inclusive_scan_f64(np.abs(wd))
    assert np.all(np.abs(g - fd) <= T.scan_bound(absw, np.zeros(n)) + 1e-10)


def test_scan_grad_full_size_vs_fp64_adjoint(ag):
    """n = 2^26 in 8 segments: x_bar = reverse inclusive scan of y_bar."""
    n = 1 << 26
    lens = inputs.block_segments(n, 8)
    x = inputs.uniform_pm1_f32(inputs.SEED_GRAD, n)
    w = inputs.uniform_pm1_f32(inputs.SEED_GRAD + 1, n)
    segs = split(torch.from_numpy(x).cuda(), lens)
    ys = ag.inclusive_scan(segs)
    wt = torch.from_numpy(w).cuda()
    torch.autograd.backward(list(ys), list(wt.split(lens)))
    g = torch.cat([s.grad for s in segs]).cpu().numpy()
    ref = oracle.reverse_inclusive_scan_f64(w.astype(np.float64))
    absref = oracle.reverse_inclusive_scan_f64(np.abs(w).astype(np.float64))
    tiles = G.tile_index(lens, G.scan_tile(torch.float32))
    err = np.abs(g.astype(np.float64) - ref)
    assert np.all(err <= T.scan_bound(absref, tiles.max() - tiles))
    # forward values too
    y = torch.cat([t.detach() for t in ys]).cpu().numpy()
    yref, s = oracle.inclusive_scan_f32_f64(x)
    assert np.all(np.abs(y - yref) <= T.scan_bound(s, tiles))


def test_scan_grad_full_size_exact_integer_valued(ag):
    """n = 2^26 in 8 segments with x and y_bar integer-valued in {-1, 0, 1}: every
    partial sum either kernel forms is a range sum of a walk whose prefixes span
    less than 2^24 (checked), so the forward values and the gradient are exact
    and must equal the oracle bit for bit."""
    n = 1 << 26
    lens = inputs.block_segments(n, 8)
    xi = inputs.uniform_int64(inputs.SEED_GRAD + 7, n, -1, 2)
    wi = inputs.uniform_int64(inputs.SEED_GRAD + 8, n, -1, 2)
    fwd = oracle.inclusive_scan_i64(xi)
    bwd = oracle.reverse_inclusive_scan_f64(wi.astype(np.float64))
    for walk in (fwd, oracle.inclusive_scan_i64(wi)):
        assert max(int(walk.max()), 0) - min(int(walk.min()), 0) < (1 << 24)
    segs = split(torch.from_numpy(xi.astype(np.float32)).cuda(), lens)
    ys = ag.inclusive_scan(segs)
    wt = torch.from_numpy(wi.astype(np.float32)).cuda()
    torch.autograd.backward(list(ys), list(wt.split(lens)))
    y = torch.cat([t.detach() for t in ys]).cpu().numpy()
    g = torch.cat([s.grad for s in segs]).cpu().numpy()
    assert np.array_equal(y, fwd.astype(np.float32))
    assert np.array_equal(g, bwd.astype(np.float32))


def test_scan_grad_repeated_calls_reuse_one_plan(ag):
    """The autograd scan keeps one vector / view per shape and rebinds it to each
    call's tensors: successive calls on new data must each be right."""
    n = 3 * 8192 + 100
    lens = [5000, 0, n - 5000]
    for seed in range(3):
        xi = inputs.uniform_int64(inputs.SEED_GRAD + 20 + seed, n, -1, 2)
        wi = inputs.uniform_int64(inputs.SEED_GRAD + 30 + seed, n, -1, 2)
        segs = split(torch.from_numpy(xi.astype(np.float32)).cuda(), lens)
        ys = ag.inclusive_scan(segs)
        torch.autograd.backward(list(ys), list(torch.from_numpy(wi.astype(np.float32)).cuda().split(lens)))
        y = torch.cat([t.detach() for t in ys]).cpu().numpy()
        g = torch.cat([s.grad for s in segs]).cpu().numpy()
        assert np.array_equal(y, oracle.inclusive_scan_i64(xi).astype(np.float32))
        assert np.array_equal(g, oracle.reverse_inclusive_scan_f64(wi.astype(np.float64)).astype(np.float32))


def test_scan_flat_full_size_exact_integer_valued(ag):
    """The one-tensor variant (segments = consecutive pieces of one flat tensor):
    2^26 in 8 segments, integer-valued walks, bit-exact forward and gradient."""
    n = 1 << 26
    lens = inputs.block_segments(n, 8)
    xi = inputs.uniform_int64(inputs.SEED_GRAD + 9, n, -1, 2)
    wi = inputs.uniform_int64(inputs.SEED_GRAD + 10, n, -1, 2)
    fwd = oracle.inclusive_scan_i64(xi)
    for walk in (fwd, oracle.inclusive_scan_i64(wi)):
        assert max(int(walk.max()), 0) - min(int(walk.min()), 0) < (1 << 24)
    x = torch.from_numpy(xi.astype(np.float32)).cuda().requires_grad_(True)
    y = ag.inclusive_scan_flat(x, lens)
    y.backward(torch.from_numpy(wi.astype(np.float32)).cuda())
    assert np.array_equal(y.detach().cpu().numpy(), fwd.astype(np.float32))
    assert np.array_equal(x.grad.cpu().numpy(),
                          oracle.reverse_inclusive_scan_f64(wi.astype(np.float64)).astype(np.float32))


def test_scan_flat_ragged_segments_repeated(ag):
    """Segment lengths that leave later segments off the 16-byte grid (the
    kernels' scalar path for those pieces), an empty segment, and two calls on
    new data through the same cached plan."""
    n = 5 * 8192 + 333
    lens = [1001, 0, 4099, 7, n - 1001 - 4099 - 7]
    for seed in range(2):
        xi = inputs.uniform_int64(inputs.SEED_GRAD + 40 + seed, n, -1, 2)
        wi = inputs.uniform_int64(inputs.SEED_GRAD + 50 + seed, n, -1, 2)
        x = torch.from_numpy(xi.astype(np.float32)).cuda().requires_grad_(True)
        y = ag.inclusive_scan_flat(x, lens)
        y.backward(torch.from_numpy(wi.astype(np.float32)).cuda())
        assert np.array_equal(y.detach().cpu().numpy(), oracle.inclusive_scan_i64(xi).astype(np.float32))
        assert np.array_equal(x.grad.cpu().numpy(),
                              oracle.reverse_inclusive_scan_f64(wi.astype(np.float64)).astype(np.float32))


def test_scan_flat_fwd_bwd_captured_in_a_cuda_graph(ag):
    """Forward and backward of the one-tensor scan captured into one CUDA graph
    (no host work per step) and replayed on new data copied into the static
    input and gradient: every replay bit-exact against the oracle."""
    n = 8 * (3 * 8192 + 100)
    lens = [n // 8] * 8
    x = torch.zeros(n, device="cuda", requires_grad=True)
    g = torch.zeros(n, device="cuda")
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):          # warm-up: plans, workspaces, allocations
        for _ in range(3):
            x.grad = None
            ag.inclusive_scan_flat(x, lens).backward(g)
    torch.cuda.current_stream().wait_stream(side)
    graph = torch.cuda.CUDAGraph()
    x.grad = None
    with torch.cuda.graph(graph):
        y = ag.inclusive_scan_flat(x, lens)
        y.backward(g)
    for seed in range(2):
        xi = inputs.uniform_int64(inputs.SEED_GRAD + 60 + seed, n, -1, 2)
        wi = inputs.uniform_int64(inputs.SEED_GRAD + 70 + seed, n, -1, 2)
        with torch.no_grad():
            x.copy_(torch.from_numpy(xi.astype(np.float32)))
            g.copy_(torch.from_numpy(wi.astype(np.float32)))
        graph.replay()
        torch.cuda.synchronize()
        assert np.array_equal(y.detach().cpu().numpy(), oracle.inclusive_scan_i64(xi).astype(np.float32))
        assert np.array_equal(x.grad.cpu().numpy(),
                              oracle.reverse_inclusive_scan_f64(wi.astype(np.float64)).astype(np.float32))


@pytest.mark.parametrize("n,lx,ly", [(300, [100, 200], [300]), (1 << 22, None, None)])
def test_dot_grad(ag, n, lx, ly):
    x = inputs.uniform_pm1_f32(51, n)
    y = inputs.uniform_pm1_f32(52, n)
    lx = lx or inputs.block_segments(n, 8)
    ly = ly or lx
    xs, ys = split(torch.from_numpy(x).cuda(), lx), split(torch.from_numpy(y).cuda(), ly)
    d = ag.dot(xs, ys)
    (0.75 * d).backward()
    gx = torch.cat([s.grad for s in xs]).cpu().numpy().astype(np.float64)
    gy = torch.cat([s.grad for s in ys]).cpu().numpy().astype(np.float64)
    rx, ry = oracle.dot_adjoint_f64(x, y, 0.75)
    # one fp32 multiply per element: |err| <= u |g y|
    assert np.all(np.abs(gx - rx) <= T.U32 * np.abs(rx) + 1e-30)
    assert np.all(np.abs(gy - ry) <= T.U32 * np.abs(ry) + 1e-30)
    if n <= 300:
        fdx = oracle.fd_gradient(lambda v: 0.75 * oracle.dot_f64(v.astype(np.float32), y)[0], x)
        assert np.allclose(gx, fdx, rtol=0, atol=1e-6)
    dref, ad = oracle.dot_f64(x, y)
    assert abs(float(d.detach()) - dref) <= T.dot_bound(n, ad, G.sms())


def stencil_loss_grads(ag, u0, seg_rows, steps, every, wc, wn, w):
    blocks = []
    r = 0
    for k in seg_rows:
        blocks.append(torch.from_numpy(u0[r:r + k]).cuda().requires_grad_(True))
        r += k
    wct = torch.tensor(wc, dtype=torch.float32, requires_grad=True)
    wnt = torch.tensor(wn, dtype=torch.float32, requires_grad=True)
    outs = ag.stencil(blocks, steps, wct, wnt, checkpoint_every=every)
    loss = (torch.cat(outs) * torch.from_numpy(w).cuda()).sum()
    loss.backward()
    g0 = torch.cat([b.grad for b in blocks]).cpu().numpy()
    return g0, float(wct.grad), float(wnt.grad), torch.cat(outs).detach().cpu().numpy()


def fp64_stencil_grads(u0, steps, wc, wn, w):
    """FP64 reference: forward states, adjoint states, and the weight gradients, plus
    the error-bound scales of the two weight gradients (in .bounds)."""
    states = [u0.astype(np.float64)]
    for _ in range(steps):
        states.append(oracle.stencil5_f64(states[-1], 1, wc, wn))
    ub = w.astype(np.float64)
    gwc = gwn = 0.0
    bwc = bwn = 0.0
    wmax = float(np.abs(w).max())
    for t in range(steps, 0, -1):
        p = states[t - 1]
        nb = oracle.stencil5_f64(ub, 1, 0.0, 1.0)  # N(u_bar_t); N is symmetric
        gwc += float((ub * p).sum())
        gwn += float((nb * p).sum())
        # fp32 kernel: 256-term per-thread chains + tree (<= 300 roundings of the |terms|),
        # plus the fp32 error of u_bar_t itself (<= 3 (steps - t + 1) u max|w| per cell, x4 in N)
        sp = float(np.abs(p).sum())
        bwc += 300 * T.U32 * float(np.abs(ub * p).sum()) + 3 * (steps - t + 1) * T.U32 * wmax * sp
        bwn += 300 * T.U32 * float(np.abs(nb * p).sum()) + 12 * (steps - t + 1) * T.U32 * wmax * sp
        ub = oracle.stencil5_T_f64(ub, 1, wc, wn)
    fp64_stencil_grads.bounds = (bwc, bwn)
    return ub, gwc, gwn, states[-1]


def test_stencil_grad_vs_fd_64x64(ag):
    R = C = 64
    steps, every = 50, 10
    wc, wn = 0.2, 0.2
    u0 = inputs.uniform01_f32(inputs.SEED_GRAD + 2, R * C).reshape(R, C)
    w = inputs.uniform_pm1_f32(inputs.SEED_GRAD + 3, R * C).reshape(R, C)
    g0, gwc, gwn, out = stencil_loss_grads(ag, u0, [16, 16, 32], steps, every, wc, wn, w)
    assert np.array_equal(out.view(np.int32), oracle.stencil5_f32(u0, steps, wc, wn).view(np.int32))
    wd = w.astype(np.float64)
    fd = oracle.fd_gradient(lambda v: float((oracle.stencil5_f64(v, steps, wc, wn) * wd).sum()),
                            u0.astype(np.float64))
    assert np.abs(g0 - fd).max() <= 3 * steps * T.U32 * np.abs(wd).max() + 1e-9
    h = 2.0 ** -12
    L = lambda a, b: float((oracle.stencil5_f64(u0.astype(np.float64), steps, a, b) * wd).sum())
    fd_wc = (L(wc + h, wn) - L(wc - h, wn)) / (2 * h)
    fd_wn = (L(wc, wn + h) - L(wc, wn - h)) / (2 * h)
    _, rwc, rwn, _ = fp64_stencil_grads(u0, steps, wc, wn, w)
    bwc, bwn = fp64_stencil_grads.bounds
    # the FD in the weights pins the FP64 adjoint sums (its truncation is O(h^2))
    assert fd_wc == pytest.approx(rwc, rel=1e-3, abs=1e-6) and fd_wn == pytest.approx(rwn, rel=1e-3, abs=1e-6)
    assert abs(gwc - rwc) <= bwc and abs(gwn - rwn) <= bwn


def test_stencil_weight_grads_512(ag):
    R, C = 512, 520
    steps, every = 50, 10
    wc, wn = 0.1, 0.22
    u0 = inputs.uniform01_f32(inputs.SEED_GRAD + 4, R * C).reshape(R, C)
    w = inputs.uniform_pm1_f32(inputs.SEED_GRAD + 5, R * C).reshape(R, C)
    g0, gwc, gwn, out = stencil_loss_grads(ag, u0, [100, 300, 112], steps, every, wc, wn, w)
    rg0, rwc, rwn, rout = fp64_stencil_grads(u0, steps, wc, wn, w)
    bwc, bwn = fp64_stencil_grads.bounds
    assert np.abs(g0 - rg0).max() <= 3 * steps * T.U32 * np.abs(w).max()
    assert abs(gwc - rwc) <= bwc and abs(gwn - rwn) <= bwn
    print(f"weight grads 512x520x50: wc {gwc:.6e} vs {rwc:.6e} (bound {bwc:.1e}); "
          f"wn {gwn:.6e} vs {rwn:.6e} (bound {bwn:.1e})")


def test_stencil_grad_full_size_sampled(ag):
    """16384^2, 50 steps, checkpoint every 10 (u0 gradient only): u_bar_0 = (A^T)^50 w,
    checked at sampled cells against the FP64 adjoint (A^T = A, pinned on the CPU)."""
    R = C = 16384
    steps = 50
    u0 = inputs.uniform01_f32(inputs.SEED_GRAD + 6, R * C).reshape(R, C)
    w = inputs.uniform_pm1_f32(inputs.SEED_GRAD + 7, R * C).reshape(R, C)
    seg_rows = [2048] * 8
    blocks = []
    for k in range(8):
        blocks.append(torch.from_numpy(u0[2048 * k:2048 * (k + 1)]).cuda().requires_grad_(True))
    outs = ag.stencil(blocks, steps, 0.0, 0.25, checkpoint_every=10)
    torch.autograd.backward(list(outs), list(torch.from_numpy(w).cuda().split(2048)))
    g0 = torch.cat([b.grad for b in blocks]).cpu().numpy()
    cells = [(0, 0), (R - 1, C - 1), (2047, 5), (2048, 9000), (8191, C - 1), (12000, 0)]
    rnd = inputs.uniform_int64(97, 40, 0, R)
    cells += [(int(rnd[2 * k]), int(rnd[2 * k + 1])) for k in range(20)]
    cells = np.array(cells, np.int64)
    ref = oracle.stencil5_f64_at(w.astype(np.float64), steps, cells, 0.0, 0.25)
    assert np.abs(g0[cells[:, 0], cells[:, 1]] - ref).max() <= 3 * steps * T.U32 * 1.0
