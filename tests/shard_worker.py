"""One gloo rank of the sharded-path tests (run as a process by
tests/test_dist_shard.py): builds its share of seeded global inputs, runs the
sharded algorithms of paper_2406_00158_gb300.shard with the CPU stand-in
backend, and checks its own output segments against the oracle applied to the
whole global input.  Prints one JSON line."""
import json
import os
import sys

import numpy as np
import torch
import torch.distributed as dist

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2406_00158_gb300 import inputs, shard  # noqa: E402
from tests.shard_cpu import CpuBackend  # noqa: E402


def owners_for(kind, n, world):
    if kind == "block":
        return shard.block_owners(n, world)
    if kind == "cyclic":
        return [k % world for k in range(n)]
    if kind == "last_rank_empty":          # rank world-1 owns nothing
        return [k % max(1, world - 1) for k in range(n)]
    raise ValueError(kind)


def local_of(x, lens, owners, rank):
    starts = np.concatenate([[0], np.cumsum(lens)])
    return [torch.from_numpy(x[starts[k]:starts[k + 1]].copy()) for k in range(len(lens)) if owners[k] == rank]


def check_local(out, exp, lens, owners, rank):
    starts = np.concatenate([[0], np.cumsum(lens)])
    mine = [k for k in range(len(lens)) if owners[k] == rank]
    for k in mine:
        got = out.seg[k].numpy()
        assert np.array_equal(got, exp[starts[k]:starts[k + 1]]), (k, got[:5], exp[starts[k]:starts[k] + 5])


def vector_case(comm, rank, world, kind, lens):
    be = CpuBackend()
    n = sum(lens)
    owners = owners_for(kind, len(lens), world)
    x = inputs.uniform_int64(71, n, -1000, 1000)
    y = inputs.uniform_int64(72, n, -1000, 1000)
    X = shard.ShardedVector(comm, lens, owners, local_of(x, lens, owners, rank), be, torch.int64)
    Y = shard.ShardedVector(comm, lens, owners, local_of(y, lens, owners, rank), be, torch.int64)
    out = torch.zeros(1, dtype=torch.int64)
    shard.dot(X, Y, out)
    assert int(out.item()) == oracle.reduce(x * y, "plus"), (int(out.item()), oracle.reduce(x * y, "plus"))
    shard.reduce(X, out, "max")
    assert int(out.item()) == oracle.reduce(x, "max")
    O = shard.ShardedVector.empty_like(X)
    shard.scan(X, O)
    check_local(O, oracle.inclusive_scan_i64(x), lens, owners, rank)
    shard.scan(X, O, exclusive=True, init=11)
    check_local(O, oracle.scan(x, "plus", exclusive=True, init=11), lens, owners, rank)
    shard.scan(X, O, op="min")
    check_local(O, oracle.scan(x, "min"), lens, owners, rank)
    shard.scan(X, O, op="max", exclusive=True, init=-5)
    check_local(O, oracle.scan(x, "max", exclusive=True, init=-5), lens, owners, rank)
    # a non-aligned partner is refused (the distributed runtime's rule)
    other = [lens[-1]] + lens[:-1] if len(lens) > 1 else lens
    if other != lens:
        Z = shard.ShardedVector(comm, other, owners, local_of(y, other, owners, rank), be, torch.int64)
        try:
            shard.dot(X, Z, out)
            raise AssertionError("non-aligned dot accepted")
        except ValueError:
            pass


def stencil_case(comm, rank, world, kind, seg_rows, cols, steps):
    be = CpuBackend()
    R = sum(seg_rows)
    owners = owners_for(kind, len(seg_rows), world)
    u0 = inputs.uniform01_f32(73, R * cols).reshape(R, cols)
    starts = np.concatenate([[0], np.cumsum(seg_rows)])
    blocks = []
    for k, r in enumerate(seg_rows):
        if owners[k] == rank:
            b = torch.zeros(r + 2, cols)
            b[1:r + 1] = torch.from_numpy(u0[starts[k]:starts[k + 1]])
            blocks.append(b)
    A = shard.ShardedMdArray(comm, seg_rows, cols, owners, blocks, be)
    B = shard.ShardedMdArray.empty_like(A)
    res = shard.stencil5(A, B, steps)
    exp = oracle.stencil5_f32(u0, steps)
    for k in res.mine:
        got = res.blk[k][1:seg_rows[k] + 1].numpy()
        assert np.array_equal(got.view(np.int32), exp[starts[k]:starts[k + 1]].view(np.int32)), k


def main():
    dist.init_process_group("gloo")
    comm = shard.TorchComm()
    rank, world = comm.rank, comm.world
    cases = json.loads(sys.argv[1])
    done = []
    for c in cases:
        if c[0] == "vector":
            vector_case(comm, rank, world, c[1], c[2])
        else:
            stencil_case(comm, rank, world, c[1], c[2], c[3], c[4])
        done.append(c[:2])
    print(json.dumps({"rank": rank, "world": world, "done": done}), flush=True)
    dist.destroy_process_group()


if __name__ == "__main__":
    main()
