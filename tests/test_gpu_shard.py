"""The sharded path with the real kernels on one GPU: N ranks emulated by N
host threads, each with its own CUDA stream and its own share of the segments.
Exchanges happen on the host between launches (a rank's data is complete
before another rank reads it), so no kernel ever waits on another rank's
kernel.  Checked bit for bit against the oracle on integer-valued data (every
partial sum exact in fp32) and, for the stencil, against the fixed-order fp32
oracle."""
import threading

import numpy as np
import pytest

import oracle
from paper_2406_00158_gb300 import inputs
from tests import gpu_util as G

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


class _Hub:
    def __init__(self, world):
        self.world = world
        self.bar = threading.Barrier(world, timeout=120)
        self.slots = [None] * world
        self.msgs = {}


class ThreadComm:
    """Collectives between threads of one process (one GPU)."""

    def __init__(self, hub, rank):
        self.hub, self.rank, self.world = hub, rank, hub.world

    def all_gather(self, t, out=None):
        torch.cuda.current_stream().synchronize()
        self.hub.slots[self.rank] = t
        self.hub.bar.wait()
        if out is None:
            out = torch.empty(self.world * t.numel(), dtype=t.dtype, device=t.device)
        for r, s in enumerate(self.hub.slots):
            out[r * t.numel():(r + 1) * t.numel()].copy_(s)
        torch.cuda.current_stream().synchronize()
        self.hub.bar.wait()
        return out

    def start_exchange(self, sends, recvs):
        torch.cuda.current_stream().synchronize()
        for peer, t, tag in sends:
            self.hub.msgs[(self.rank, peer, tag)] = t
        self.hub.bar.wait()
        for peer, t, tag in recvs:
            t.copy_(self.hub.msgs[(peer, self.rank, tag)])
        torch.cuda.current_stream().synchronize()
        self.hub.bar.wait()
        if self.rank == 0:
            self.hub.msgs.clear()
        self.hub.bar.wait()
        return []

    @staticmethod
    def finish_exchange(reqs):
        pass


def run_ranks(world, fn):
    hub = _Hub(world)
    errs = [None] * world
    res = [None] * world

    def body(r):
        try:
            torch.cuda.set_device(0)
            s = torch.cuda.Stream()
            with torch.cuda.stream(s):
                res[r] = fn(ThreadComm(hub, r))
                s.synchronize()
        except BaseException as e:  # noqa: BLE001 (reported below)
            errs[r] = e
            hub.bar.abort()

    th = [threading.Thread(target=body, args=(r,)) for r in range(world)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    for e in errs:
        if e is not None and not isinstance(e, threading.BrokenBarrierError):
            raise e
    assert all(e is None for e in errs), errs
    return res


@pytest.fixture(scope="module")
def sh():
    G.dev()
    from paper_2406_00158_gb300 import shard
    return shard


def _owners(shard, kind, n, world):
    return shard.block_owners(n, world) if kind == "block" else [k % world for k in range(n)]


@pytest.mark.parametrize("world,kind", [(2, "block"), (3, "cyclic"), (4, "block")])
def test_sharded_dot_and_scans_exact(sh, world, kind):
    n = 1 << 22
    lens = inputs.random_cut_segments(2406 + 300, n, 8)
    lens = lens[:3] + [0] + lens[3:]                     # an empty segment
    xi = inputs.uniform_int64(2406 + 301, n, -1, 2)
    yi = inputs.uniform_int64(2406 + 302, n, -1, 2)
    x, y = xi.astype(np.float32), yi.astype(np.float32)
    owners = _owners(sh, kind, len(lens), world)
    starts = np.concatenate([[0], np.cumsum(lens)])
    inc = oracle.inclusive_scan_i64(xi).astype(np.float32)
    exc = oracle.scan(xi, "plus", exclusive=True, init=5).astype(np.float32)
    dref = oracle.dot_f64(x, y)[0]
    sl = lambda a, k: a[starts[k]:starts[k + 1]]

    def rank_fn(comm):
        mine = [k for k in range(len(lens)) if owners[k] == comm.rank]
        dev = torch.device("cuda:0")
        X = sh.ShardedVector(comm, lens, owners, [torch.from_numpy(sl(x, k).copy()).to(dev) for k in mine])
        Y = sh.ShardedVector(comm, lens, owners, [torch.from_numpy(sl(y, k).copy()).to(dev) for k in mine])
        O = sh.ShardedVector.empty_like(X)
        d = torch.zeros(1, dtype=torch.float32, device=dev)
        sh.dot(X, Y, d)
        got = {"dot": float(d.item())}
        sh.scan(X, O)
        got["inc"] = {k: O.seg[k].cpu().numpy() for k in mine}
        sh.scan(X, O, exclusive=True, init=5.0)
        got["exc"] = {k: O.seg[k].cpu().numpy() for k in mine}
        return got

    for got in run_ranks(world, rank_fn):
        assert got["dot"] == dref
        for k, v in got["inc"].items():
            assert np.array_equal(v, sl(inc, k)), k
        for k, v in got["exc"].items():
            assert np.array_equal(v, sl(exc, k)), k


@pytest.mark.parametrize("world,kind", [(2, "block"), (3, "cyclic")])
def test_sharded_stencil_exact(sh, world, kind):
    R, C, steps = 700, 516, 6
    seg_rows = [100, 64, 1, 135, 200, 70, 130]
    u0 = inputs.uniform01_f32(2406 + 303, R * C).reshape(R, C)
    owners = _owners(sh, kind, len(seg_rows), world)
    starts = np.concatenate([[0], np.cumsum(seg_rows)])
    ref = oracle.stencil5_f32(u0, steps)

    def rank_fn(comm):
        dev = torch.device("cuda:0")
        blocks = []
        for k, r in enumerate(seg_rows):
            if owners[k] == comm.rank:
                b = torch.zeros(r + 2, C, device=dev)
                b[1:r + 1] = torch.from_numpy(u0[starts[k]:starts[k + 1]]).to(dev)
                blocks.append(b)
        A = sh.ShardedMdArray(comm, seg_rows, C, owners, blocks)
        B = sh.ShardedMdArray.empty_like(A)
        res = sh.stencil5(A, B, steps)
        return {k: res.blk[k][1:seg_rows[k] + 1].cpu().numpy() for k in res.mine}

    for got in run_ranks(world, rank_fn):
        for k, v in got.items():
            assert np.array_equal(v.view(np.int32), ref[starts[k]:starts[k + 1]].view(np.int32)), k


def test_one_rank_is_the_plain_path(sh):
    """world 1: no collective; the sharded calls are the single-range kernels."""
    n = 3 * 8192 + 11
    xi = inputs.uniform_int64(2406 + 304, n, -1, 2)
    x = xi.astype(np.float32)
    lens = [5000, n - 5000]
    comm = sh.LocalComm()
    dev = torch.device("cuda:0")
    X = sh.ShardedVector(comm, lens, [0, 0], [torch.from_numpy(x[:5000].copy()).to(dev),
                                              torch.from_numpy(x[5000:].copy()).to(dev)])
    O = sh.ShardedVector.empty_like(X)
    sh.scan(X, O)
    got = torch.cat([O.seg[0], O.seg[1]]).cpu().numpy()
    assert np.array_equal(got, oracle.inclusive_scan_i64(xi).astype(np.float32))
    d = torch.zeros(1, device=dev)
    sh.dot(X, X, d)
    assert d.item() == float(np.abs(xi).sum())
