"""The sharded path (one range over N ranks, its segments placed on the ranks) on
CPU gloo ranks, world sizes 2 and 3: the placement and exchange logic of
paper_2406_00158_gb300.shard -- all-gather of partials and run totals, carries,
point-to-point halo rows -- with a CPU stand-in for the local kernels, checked
against the oracle on the whole input.  Owner maps: contiguous blocks,
block-cyclic (several runs per rank), and a rank that owns nothing; uneven and
empty segments."""
import json
import os

import pytest

from paper_2406_00158_gb300 import shard
from tests.test_dist_gloo import ROOT, _run_ranks

VECTOR_LENS = [1000, 0, 3333, 17, 2048, 5000, 1]
CASES = [["vector", "block", VECTOR_LENS], ["vector", "cyclic", VECTOR_LENS],
         ["vector", "last_rank_empty", VECTOR_LENS],
         ["stencil", "block", [70, 5, 130, 64, 1], 48, 5], ["stencil", "cyclic", [70, 5, 130, 64, 1], 48, 3],
         ["stencil", "block", [200, 129], 36, 4]]


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_algorithms_on_gloo_ranks(world):
    outs = _run_ranks(["-m", "tests.shard_worker", json.dumps(CASES)], world=world, timeout=600)
    res = [json.loads(o.strip().splitlines()[-1]) for o in outs]
    assert sorted(r["rank"] for r in res) == list(range(world))
    for r in res:
        assert r["world"] == world and len(r["done"]) == len(CASES)


def test_placement_helpers():
    assert shard.block_owners(8, 8) == list(range(8))
    assert shard.block_owners(8, 2) == [0] * 4 + [1] * 4
    assert shard.block_owners(5, 3) == [0, 0, 1, 1, 2]
    assert shard.runs([0, 1, 0, 0, 1], 0) == [(0, 1), (2, 4)]
    assert shard.runs([0, 1, 0, 0, 1], 1) == [(1, 2), (4, 5)]
    assert shard.runs([0, 0], 1) == []
    assert shard.run_heads([0, 1, 0, 0, 1]) == [(0, 0, 0), (1, 1, 0), (2, 0, 1), (4, 1, 1)]
    own = shard.balanced_owners([10, 10, 10, 10, 40], 2)
    assert own == [0, 0, 0, 0, 1]
    own = shard.balanced_owners([5] * 12, 4)
    assert own == [0, 0, 0, 1, 1, 1, 2, 2, 2, 3, 3, 3]
    assert shard.balanced_owners([0, 0], 3) == [0, 0]
