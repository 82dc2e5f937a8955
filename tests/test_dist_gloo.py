"""The N > 1 path of bench.py on the CPU: two gloo ranks (one process each, as
torchrun launches them) use bench.Dist for the barrier, the max-over-ranks
time and the whole-job sum; the reference arm prints on rank 0 only."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


WORKER = r'''
import json, os, sys, time
sys.path.insert(0, sys.argv[1])
import bench
d = bench.Dist("gloo")
rank = d.rank
time.sleep(0.05 * rank)
d.barrier()
mx = d.max(10.0 + rank)          # per-rank "ms"
tot = d.sum(100.0 * (rank + 1))  # per-rank "bytes"
print(json.dumps({"rank": rank, "world": d.world, "max": mx, "sum": tot}), flush=True)
d.close()
'''


def _run_ranks(code_args, world=2, timeout=120):
    port = _free_port()
    procs = []
    for r in range(world):
        env = dict(os.environ, RANK=str(r), LOCAL_RANK=str(r), WORLD_SIZE=str(world),
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), CUDA_VISIBLE_DEVICES="")
        procs.append(subprocess.Popen([sys.executable] + code_args, env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True, cwd=ROOT))
    outs = []
    for p in procs:
        try:
            o, e = p.communicate(timeout=timeout)
        except subprocess.TimeoutExpired:
            p.kill()
            raise
        assert p.returncode == 0, e[-2000:]
        outs.append(o)
    return outs


def test_dist_barrier_max_sum_two_gloo_ranks():
    outs = _run_ranks(["-c", WORKER, ROOT])
    res = [json.loads(o.strip().splitlines()[-1]) for o in outs]
    for r in res:
        assert r["world"] == 2
        assert r["max"] == 11.0        # max over ranks
        assert r["sum"] == 300.0       # whole-job aggregate
    assert sorted(r["rank"] for r in res) == [0, 1]


def test_reference_arm_prints_on_rank0_only():
    outs = _run_ranks([os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2", "--steps", "1",
                       "--warmup", "0"], timeout=300)
    lines = [[l for l in o.splitlines() if l.startswith("{")] for o in outs]
    assert len(lines[0]) == 1 and len(lines[1]) == 0
    j = json.loads(lines[0][0])
    assert j["impl"] == "reference" and j["unit"] == "GB/s" and j["value"] > 0
    assert j["e2e"]["h2d_bytes_per_step"] == 0 and j["cpu_baseline"]["kind"] == "oracle"


def test_all_cores_oracle_baseline_spawns_and_times_every_slice(tmp_path):
    """bench.cpu_oracle_all_cores: spawned processes (no fork after any device
    work), each timing the oracle on its own slice; the bytes are the whole
    sample's and the wall time spans every process's run."""
    code = r'''
import json, sys
sys.path.insert(0, sys.argv[1])
import bench
from paper_2406_00158_gb300 import inputs
if __name__ == "__main__":
    n = 1 << 16
    x = inputs.uniform_pm1_f32(inputs.SEED_DOT_X, n)
    y = inputs.uniform_pm1_f32(inputs.SEED_DOT_Y, n)
    dt, nb = bench.cpu_oracle_all_cores(x, y, 2, 3)
    print(json.dumps({"dt": dt, "nb": nb, "expect": 2 * n * (bench.BYTES_DOT + bench.BYTES_SCAN)}))
'''
    path = tmp_path / "allcores_main.py"   # spawned children re-import the main script
    path.write_text(code)
    r = subprocess.run([sys.executable, str(path), ROOT], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    out = json.loads(r.stdout.strip().splitlines()[-1])
    assert out["nb"] == out["expect"] and out["dt"] > 0
