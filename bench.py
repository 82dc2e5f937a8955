"""Benchmark of the segmented-range hot path on GB300.

One step = one pass of the headline workload: transform_reduce(zip(x, y) |
multiply, plus) (the dot product of Algorithm 1) and inclusive_scan(x), fp32,
n = 2^28 in 8 equal segments (one allocation each), inputs resident in HBM
(3 GiB touched per step > 129 MB L2, so no flush is needed between steps).
Metric: achieved HBM GB/s = algorithmic bytes / time (8 B/element for the dot,
8 B/element for the scan).  The other hot-path rows (int64 scan, stencil,
adjoints, batched vs one launch per range) are measured in the same run and
reported under "rows".

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun the one 2^28 range is sharded over the ranks (segment k of 8 on
rank k*N//8; strong scaling): the dot all-gathers the per-rank partials, the scan
all-gathers the run totals and starts each rank's local scan from its carry
(NCCL); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2406_00158_gb300 import inputs  # noqa: E402

N_ELEMS = 1 << 28
NSEG = 8
BYTES_DOT = 8   # per element: x and y read
BYTES_SCAN = 8  # per element: x read, y written
METRIC = "HBM GB/s (% of GB300 peak) for scan/dot/stencil; batched vs one-launch-per-range"
WORKLOAD = "fp32 dot (transform_reduce over zip|multiply) + fp32 inclusive_scan, n=2^28, 8 equal segments"


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ------------------------------------------------------------------------------------------
# clocks sampled during the timed region
# ------------------------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: str):
        self.gpu = gpu_index
        self.proc = None
        self.lines: list[str] = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-i", self.gpu,
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            f = [x.strip() for x in l.split(",")]
            if len(f) < 6:
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
            except ValueError:
                continue
            for name, v in zip(names, f[2:6]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def gpu_index_for_smi(local_rank: int) -> str:
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    if vis:
        ids = [v.strip() for v in vis.split(",") if v.strip()]
        if local_rank < len(ids):
            return ids[local_rank]
    return str(local_rank)


# ------------------------------------------------------------------------------------------
# distributed plumbing (barrier + max over ranks); one process per GPU
# ------------------------------------------------------------------------------------------
class Dist:
    def __init__(self, backend: str):
        import torch
        import torch.distributed as dist
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        self.dist = dist if self.world > 1 else None
        self.backend = backend
        if self.dist is not None:
            dist.init_process_group(backend=backend)
        self.torch = torch

    def barrier(self):
        if self.dist is not None:
            self.dist.barrier()

    def max(self, v: float) -> float:
        if self.dist is None:
            return v
        dev = "cuda" if self.backend == "nccl" else "cpu"
        t = self.torch.tensor([v], dtype=self.torch.float64, device=dev)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX)
        return float(t.item())

    def sum(self, v: float) -> float:
        if self.dist is None:
            return v
        dev = "cuda" if self.backend == "nccl" else "cpu"
        t = self.torch.tensor([v], dtype=self.torch.float64, device=dev)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.SUM)
        return float(t.item())

    def close(self):
        if self.dist is not None:
            self.dist.destroy_process_group()


# ------------------------------------------------------------------------------------------
# the oracle as a CPU baseline / the reference arm
# ------------------------------------------------------------------------------------------
def cpu_oracle_run(x: np.ndarray, y: np.ndarray, reps: int) -> tuple[float, int]:
    import oracle
    oracle.lib()
    t0 = time.perf_counter()
    for _ in range(reps):
        oracle.dot_f64(x, y)
        oracle.inclusive_scan_f32_f64(x)
    dt = time.perf_counter() - t0
    return dt, reps * x.size * (BYTES_DOT + BYTES_SCAN)


def _oracle_core(x: np.ndarray, y: np.ndarray, reps: int, barrier, q) -> None:
    """One host core's share of the all-cores baseline (a spawned process): the oracle
    as it stands on its own slice of the sample, timed after every process is ready."""
    import oracle
    oracle.lib()
    cpu_oracle_run(x[:1 << 16], y[:1 << 16], 1)
    barrier.wait(timeout=600)
    t0 = time.perf_counter()
    dt, nb = cpu_oracle_run(x, y, reps)
    q.put((t0, t0 + dt, nb))


def cpu_oracle_all_cores(x: np.ndarray, y: np.ndarray, reps: int, procs: int) -> tuple[float, int]:
    """The oracle on every host core at once: `procs` spawned processes, each over an
    independent slice of the sample (one dot + one scan per slice), so the figure is
    the host's aggregate oracle throughput.  Returns (wall seconds from the first start
    to the last finish, bytes)."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    barrier, q = ctx.Barrier(procs), ctx.Queue()
    cut = np.linspace(0, x.size, procs + 1).astype(np.int64)
    ps = [ctx.Process(target=_oracle_core, args=(x[cut[k]:cut[k + 1]], y[cut[k]:cut[k + 1]], reps, barrier, q))
          for k in range(procs)]
    for p in ps:
        p.start()
    import queue
    res, deadline = [], time.monotonic() + 900
    try:
        while len(res) < procs:
            try:
                res.append(q.get(timeout=2))
            except queue.Empty:
                if time.monotonic() > deadline or any(p.exitcode not in (None, 0) for p in ps):
                    raise RuntimeError("all-cores oracle baseline: a worker failed or timed out")
    finally:
        for p in ps:
            p.join(timeout=5)
            if p.is_alive():
                p.kill()
    return max(r[1] for r in res) - min(r[0] for r in res), sum(r[2] for r in res)


def cpu_stencil_f64(steps: int) -> float:
    """Seconds for `steps` steps of the oracle's FP64 5-point stencil on the 16384^2 grid."""
    import oracle
    u0 = inputs.uniform01_f32(inputs.SEED_STENCIL, 16384 * 16384).reshape(16384, 16384).astype(np.float64)
    oracle.stencil5_f64(u0[:64, :64], 1)
    t0 = time.perf_counter()
    oracle.stencil5_f64(u0, steps)
    return time.perf_counter() - t0


def run_reference(args) -> None:
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    sample = 1 << 26  # a quarter of the workload per step keeps the run within minutes
    x = inputs.uniform_pm1_f32(inputs.SEED_DOT_X, sample)
    y = inputs.uniform_pm1_f32(inputs.SEED_DOT_Y, sample)
    # the oracle as it stands on every host core: one process per core, each over
    # its own slice of the sample, every step (warm-up calls inside each process)
    procs = os.cpu_count() or 1
    if procs > 1:
        dt, nbytes = cpu_oracle_all_cores(x, y, args.steps, procs)
    else:
        cpu_oracle_run(x[:1 << 20], y[:1 << 20], max(0, args.warmup))
        dt, nbytes = cpu_oracle_run(x, y, args.steps)
    gbs = nbytes / dt / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": gbs, "unit": "GB/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded SplitMix64, U[-1,1))",
        "config": {"workload": WORKLOAD, "sample": f"n=2^26 of the 2^28 workload per step",
                   "parallelism": f"CPU oracle, {procs} processes (one per host core)"},
        "cpu_baseline": {"value": gbs, "unit": "GB/s", "cores": procs, "kind": "oracle",
                         "sample": f"oracle dot (FP64) + inclusive_scan (FP64) over 2^26 elements per step, cut into "
                                   f"{procs} independent slices (one process each), {args.steps} steps"},
        "e2e": {"value": gbs, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "gpu_launches": 0,
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------------------------------
# the other hot-path rows (each timed with CUDA events on the launching stream)
# ------------------------------------------------------------------------------------------
def _time(fn, s, reps, flush=None, warmup=2):
    """Mean ms per call over `reps` calls after `warmup` untimed calls, CUDA events on
    stream s (flush between calls if given, outside the measured interval)."""
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    tot = 0.0
    for _ in range(reps):
        if flush is not None:
            flush()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(s)
        fn()
        b.record(s)
        b.synchronize()
        tot += a.elapsed_time(b)
    return tot / reps


def _row(ms, nbytes, peak, **kw):
    gbs = nbytes / (ms / 1e3) / 1e9
    d = {"ms": ms, "GB/s": gbs, "frac_of_peak": gbs / peak, "bytes": nbytes}
    d.update(kw)
    return d


def measure_rows(api, dev, s, peak) -> dict:
    """The other hot-path rows, each on its own workload."""
    import torch
    from paper_2406_00158_gb300 import autograd as AG
    rows = {}
    l2 = torch.cuda.get_device_properties(dev).L2_cache_size
    flushbuf = torch.empty(4 * l2 // 4, dtype=torch.float32, device=dev)
    flush = lambda: flushbuf.zero_()

    # int64 inclusive_scan, 2^20 in 4 segments 1:2:3:2 (16.8 MB: L2-resident), and 2^28
    for n, name in ((1 << 20, "int64_scan_2^20_1:2:3:2"), (1 << 28, "int64_scan_2^28_1:2:3:2")):
        lens = inputs.proportional_segments(n, [1, 2, 3, 2])
        x = inputs.uniform_int64(inputs.SEED_SCAN_I64, n)
        vx = api.SegmentedVector.from_tensor(torch.from_numpy(x).to(dev), lens)
        vo = api.SegmentedVector.empty(lens, torch.int64, dev)
        v = vx.view()
        fn = lambda: api.inclusive_scan(v, vo, stream=s)
        if n < (1 << 24):
            # kernel time without the host's per-call launch cost: 20 back-to-back calls
            # captured into one CUDA graph, replayed (L2-resident)
            side = torch.cuda.Stream()
            side.wait_stream(s)
            with torch.cuda.stream(side):
                for _ in range(3):
                    api.inclusive_scan(v, vo, stream=side)
            s.wait_stream(side)
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g):
                for _ in range(20):
                    api.inclusive_scan(v, vo)
            ms_graph = _time(g.replay, s, 20) / 20
            rows[name] = _row(_time(fn, s, 50, flush), n * 16, peak, l2="flushed between calls",
                              l2_resident=_row(_time(fn, s, 200), n * 16, peak),
                              graph_replay=_row(ms_graph, n * 16, peak, note="20 calls per graph, L2-resident"))
            del g
        else:
            rows[name] = _row(_time(fn, s, 20), n * 16, peak, l2="4 GiB per array > L2")
        api.sync_status(s)
        del vx, vo, v, x

    # stencil: 16384^2 fp32, 8 row blocks of 2048 (+2 ghost rows), 100 steps
    R = C = 16384
    seg_rows = [2048] * 8
    u0 = torch.from_numpy(inputs.uniform01_f32(inputs.SEED_STENCIL, R * C).reshape(R, C)).to(dev)
    a = api.MdArray.from_tensor(u0, seg_rows)
    b = api.MdArray.empty(seg_rows, C, dev)
    t = api.MdArray.empty(seg_rows, C, dev)
    ms = _time(lambda: api.stencil5(a, b, t, 100, stream=s), s, 3)
    try:
        st_traffic = json.load(open(os.path.join(ROOT, "profiles", "traffic.json"))).get("stencil")
    except (OSError, ValueError):
        st_traffic = None
    rows["stencil_16384^2_8blocks_100steps"] = _row(ms, 8 * R * C * 100, peak, ms_per_step=ms / 100,
                                                    launches=101, traffic_per_step=st_traffic)
    api.sync_status(s)

    # autograd: stencil 50 steps, checkpoint every 10 (u0 gradient), fwd + bwd
    blocks = [u0[2048 * k:2048 * (k + 1)].clone().requires_grad_(True) for k in range(8)]
    gw = torch.ones(R, C, device=dev).split(2048)

    def stencil_fb():
        for q in blocks:
            q.grad = None
        outs = AG.stencil(blocks, 50, 0.0, 0.25, checkpoint_every=10)
        torch.autograd.backward(list(outs), list(gw))

    torch.cuda.empty_cache()
    ms = _time(stencil_fb, s, 3)
    rows["autograd_stencil_16384^2_50steps_ckpt10_fwd+bwd"] = _row(
        ms, 8 * R * C * 100, peak, note="100 stencil steps (50 fwd + 50 A^T); includes checkpoint copies")
    del a, b, t, blocks, gw, u0

    # for_each over k-ary zips: STREAM (fp64, 2^28 per array, 8 segments) and
    # Black-Scholes (fp32, 2^28 options, 8 segments).  Arrays > L2: no flush needed.
    n = 1 << 28
    lens = [n // 8] * 8
    sa, sb, sc = (api.SegmentedVector.from_tensor(torch.from_numpy(v).to(dev), lens)
                  for v in inputs.stream_inputs(n, np.float64))
    stream_bytes = {"copy": 16, "scale": 16, "add": 24, "triad": 24}
    zips = {"copy": api.View.zipn(sa, sc), "scale": api.View.zipn(sb, sc),
            "add": api.View.zipn(sa, sb, sc), "triad": api.View.zipn(sa, sb, sc)}
    for fn, z in zips.items():
        args = (3.0,) if fn in ("scale", "triad") else ()
        ms = _time(lambda: api.for_each(z, fn, *args, stream=s), s, 20)
        rows[f"stream_{fn}_f64_2^28_8segs"] = _row(ms, stream_bytes[fn] * n, peak,
                                                   note="STREAM byte counting (no write-allocate)")
    api.sync_status(s)
    del zips, sa, sb, sc
    S, X, Tm = inputs.black_scholes_inputs(n)
    bs = [api.SegmentedVector.from_tensor(torch.from_numpy(v).to(dev), lens) for v in (S, X, Tm)]
    bs += [api.SegmentedVector.empty(lens, torch.float32, dev) for _ in range(2)]
    zbs = api.View.zipn(*bs)
    r32, sig32 = float(np.float32(inputs.BS_R)), float(np.float32(inputs.BS_SIGMA))
    ms = _time(lambda: api.for_each(zbs, "black_scholes", r32, sig32, stream=s), s, 20)
    api.sync_status(s)
    try:
        bs_traffic = json.load(open(os.path.join(ROOT, "profiles", "traffic.json"))).get("black_scholes")
    except (OSError, ValueError):
        bs_traffic = None
    rows["black_scholes_f32_2^28_8segs"] = _row(ms, 20 * n, peak, options_per_s=n / (ms / 1e3),
                                                traffic=bs_traffic,
                                                note="S, X, T read; call, put written: 20 B/option")
    del zbs, bs, S, X, Tm

    # sort: 2^28 fp32 keys U[-1, 1) in 8 segments, into another 8-segment vector.
    # Radix sort traffic: one histogram read + 4 passes of read + write = 36 B/key
    # (the minimum any sort needs is 8 B/key: one read, one write).
    x = torch.from_numpy(inputs.uniform_pm1_f32(inputs.SEED_SORT, n)).to(dev)
    vin = api.SegmentedVector.from_tensor(x, lens)
    vout = api.SegmentedVector.empty(lens, torch.float32, dev)
    ms = _time(lambda: api.sort(vin, vout, stream=s), s, 10)
    api.sync_status(s)
    rows["sort_f32_2^28_8segs"] = _row(ms, 36 * n, peak, keys_per_s=n / (ms / 1e3),
                                       note="GB/s over the radix sort's 36 B/key (histogram + 4 passes)")
    del vin, vout, x
    xi = torch.from_numpy(inputs.raw_u64(inputs.SEED_SORT + 1, n // 2).view(np.int64)).to(dev)
    vin = api.SegmentedVector.from_tensor(xi, [n // 16] * 8)
    vout = api.SegmentedVector.empty([n // 16] * 8, torch.int64, dev)
    ms = _time(lambda: api.sort(vin, vout, stream=s), s, 5)
    api.sync_status(s)
    rows["sort_i64_2^27_8segs"] = _row(ms, 136 * (n // 2), peak, keys_per_s=(n // 2) / (ms / 1e3),
                                       note="GB/s over 136 B/key (histogram + 8 passes of 16 B)")
    del vin, vout, xi

    # fused views (Sec. 4.4): the view is evaluated in the kernel's loads, no intermediate
    # array; 2^26 fp32 in 8 segments, bytes = what the fused kernel must move
    m = 1 << 26
    fx = api.SegmentedVector.from_tensor(torch.from_numpy(inputs.uniform_pm1_f32(inputs.SEED_DOT_X, m)).to(dev), [m // 8] * 8)
    fy = api.SegmentedVector.from_tensor(torch.from_numpy(inputs.uniform_pm1_f32(inputs.SEED_DOT_Y, m)).to(dev), [m // 8] * 8)
    fo = api.SegmentedVector.empty([m // 8] * 8, torch.float32, dev)
    fr = torch.zeros(1, dtype=torch.float32, device=dev)
    chain = fx.view().transform("scale", 2.0).transform("add", 1.0).transform("abs")
    dv = api.dot_view(fx, fy)
    for name, fn, nb in [("view_scan_plain_f32_2^26", lambda: api.inclusive_scan(fx, fo, stream=s), 8),
                         ("view_scan_zip*mul_f32_2^26", lambda: api.inclusive_scan(dv, fo, stream=s), 12),
                         ("view_reduce_chain3_f32_2^26", lambda: api.transform_reduce(chain, fr, stream=s), 4),
                         ("view_transform_chain3_f32_2^26", lambda: api.transform(chain, fo, stream=s), 8),
                         ("view_scan_min_f32_2^26", lambda: api.inclusive_scan(fx, fo, op="min", stream=s), 8)]:
        ms = _time(fn, s, 20, flush=lambda: flushbuf.zero_())
        rows[name] = _row(ms, nb * m, peak, l2="flushed between calls")
    api.sync_status(s)
    del fx, fy, fo, chain, dv

    # autograd: scan n = 2^26 in 8 segments, fwd + bwd (reverse scan)
    n = 1 << 26
    xs = [q.clone().requires_grad_(True) for q in
          torch.from_numpy(inputs.uniform_pm1_f32(inputs.SEED_GRAD, n)).to(dev).split(n // 8)]
    gy = list(torch.from_numpy(inputs.uniform_pm1_f32(inputs.SEED_GRAD + 1, n)).to(dev).split(n // 8))

    def scan_fb():
        for q in xs:            # a training step's zero_grad(set_to_none=True)
            q.grad = None
        ys = AG.inclusive_scan(xs)
        torch.autograd.backward(list(ys), gy)

    ms = _time(scan_fb, s, 10)
    rows["autograd_scan_2^26_8segs_fwd+bwd"] = _row(ms, 16 * n, peak)
    # the same through the one-tensor variant (one autograd node: less host work)
    xf = torch.cat([q.detach() for q in xs]).requires_grad_(True)
    gf = torch.cat(gy)

    def scan_flat_fb():
        xf.grad = None
        AG.inclusive_scan_flat(xf, [n // 8] * 8).backward(gf)

    ms = _time(scan_flat_fb, s, 10)
    rows["autograd_scan_flat_2^26_8segs_fwd+bwd"] = _row(ms, 16 * n, peak)
    # and with forward + backward captured into one CUDA graph (no host work per step)
    side = torch.cuda.Stream()
    side.wait_stream(s)
    with torch.cuda.stream(side):
        for _ in range(3):
            scan_flat_fb()
    s.wait_stream(side)
    graph = torch.cuda.CUDAGraph()
    xf.grad = None
    with torch.cuda.graph(graph):
        AG.inclusive_scan_flat(xf, [n // 8] * 8).backward(gf)
    ms = _time(graph.replay, s, 10)
    rows["autograd_scan_flat_graph_2^26_8segs_fwd+bwd"] = _row(ms, 16 * n, peak,
                                                              note="forward + backward replayed as one CUDA graph")
    del xs, gy, xf, gf, graph

    # batched: 4096 vectors, log-uniform [1e3, 1e6], 1-8 segments; one launch vs one per range
    shapes = inputs.batch_shapes(inputs.SEED_BATCH, 4096)
    tot = sum(map(sum, shapes))
    X = api.packed_vectors(inputs.uniform_pm1_f32(inputs.SEED_BATCH_X, tot), shapes, device=dev)
    P = api.packed_vectors(inputs.uniform_pm1_f32(inputs.SEED_BATCH_P, tot), shapes, device=dev)
    Y = api.packed_vectors(None, shapes, device=dev)
    dots = torch.zeros(len(shapes), dtype=torch.float32, device=dev)
    batch = api.Batch(X, P, Y, dots)
    # autotune on a calibration batch of the same distribution (other seeds), not the timed data
    cshapes = inputs.batch_shapes(inputs.SEED_BATCH + 1, 4096)
    ctot = sum(map(sum, cshapes))
    CX = api.packed_vectors(inputs.uniform_pm1_f32(inputs.SEED_BATCH_X + 1, ctot), cshapes, device=dev)
    CP = api.packed_vectors(inputs.uniform_pm1_f32(inputs.SEED_BATCH_P + 1, ctot), cshapes, device=dev)
    CY = api.packed_vectors(None, cshapes, device=dev)
    cal = api.Batch(CX, CP, CY, torch.zeros(len(cshapes), dtype=torch.float32, device=dev))
    default_tune = batch.tune
    chosen = cal.autotune(retune=True)
    del cal, CX, CP, CY
    ms_default = _time(lambda: batch.run(stream=s), s, 20)
    batch.tune = chosen
    ms_batch = _time(lambda: batch.run_graph(stream=s), s, 20)
    ms_plain = _time(lambda: batch.run(stream=s), s, 20)
    ms_per = _time(lambda: batch.run_per_range(stream=s), s, 3)
    ms_per_graph = _time(lambda: batch.run_per_range_graph(stream=s), s, 5)
    api.sync_status(s)
    rows["batched_4096_vectors"] = _row(
        ms_batch, 12 * tot, peak, elements=tot, tune=list(chosen), default_tune=list(default_tune),
        ms_default_tune=ms_default, ms_one_launch_no_graph=ms_plain, ms_one_launch_per_range=ms_per,
        ms_one_launch_per_range_graph=ms_per_graph,
        speedup_vs_per_range=ms_per / ms_batch, speedup_vs_per_range_graph=ms_per_graph / ms_batch,
        launches=1, per_range_launches=2 * len(shapes))
    return rows


# ------------------------------------------------------------------------------------------
# the headline step: one GPU, or the one range sharded over the ranks
# ------------------------------------------------------------------------------------------
class Headline:
    """dot + inclusive_scan of the 2^28 fp32 range in 8 segments.  One rank: the
    single-range kernels on persistent views.  N ranks: segment k lives on rank
    k*N//8 and the step is the sharded dot and scan (paper_2406_00158_gb300.shard):
    per rank 2 + 3 of the library's launches plus two NCCL all-gathers."""

    def __init__(self, api, D, dev, s, x, y):
        import torch
        self.api, self.s, self.D, self.torch = api, s, D, torch
        self.x, self.y = x, y
        lens = inputs.block_segments(N_ELEMS, NSEG)
        starts = np.concatenate([[0], np.cumsum(lens)])
        self.dotbuf = torch.zeros(1, dtype=torch.float32, device=dev)
        if D.world == 1:
            self.vx = api.SegmentedVector.from_tensor(torch.from_numpy(x).to(dev), lens)
            self.vy = api.SegmentedVector.from_tensor(torch.from_numpy(y).to(dev), lens)
            self.out = api.SegmentedVector.empty(lens, torch.float32, dev)
            self.dview = api.dot_view(self.vx, self.vy)
            self.xview = self.vx.view()
            self.ranges = [(0, N_ELEMS)]
            self.local_elems = N_ELEMS
            self.launches_per_step = 2
            self.sharded = False
        else:
            from paper_2406_00158_gb300 import shard
            self.shard = shard
            comm = shard.TorchComm()
            owners = shard.block_owners(NSEG, D.world)
            mine = [k for k in range(NSEG) if owners[k] == D.rank]
            seg = lambda a, k: torch.from_numpy(a[starts[k]:starts[k + 1]]).to(dev)
            self.X = shard.ShardedVector(comm, lens, owners, [seg(x, k) for k in mine])
            self.Y = shard.ShardedVector(comm, lens, owners, [seg(y, k) for k in mine])
            self.O = shard.ShardedVector.empty_like(self.X)
            self.ranges = [(int(starts[k]), int(starts[k + 1])) for k in mine]
            self.local_elems = sum(b - a for a, b in self.ranges)
            self.launches_per_step = 5
            self.sharded = True

    def dot(self):
        if self.sharded:
            self.shard.dot(self.X, self.Y, self.dotbuf)
        else:
            self.api.transform_reduce(self.dview, self.dotbuf, stream=self.s)

    def scan(self):
        if self.sharded:
            self.shard.scan(self.X, self.O)
        else:
            self.api.inclusive_scan(self.xview, self.out, stream=self.s)

    def step(self):
        self.dot()
        self.scan()

    def pin_host(self):
        t = self.torch
        self.hx = [t.from_numpy(self.x[a:b]).pin_memory() for a, b in self.ranges]
        self.hy = [t.from_numpy(self.y[a:b]).pin_memory() for a, b in self.ranges]
        self.hout = [t.empty(b - a, dtype=t.float32).pin_memory() for a, b in self.ranges]
        self.hdot = t.empty(1, dtype=t.float32).pin_memory()

    def e2e_begin(self, start_event):
        """Streams for the end-to-end loop: host->device copies, the step, and
        device->host copies each on their own stream, so that one step's result
        read-back overlaps the next step's input upload (opposite directions of
        the link).  Every step still uploads its inputs and reads its result."""
        t = self.torch
        if not hasattr(self, "s_in"):
            self.s_in, self.s_out = t.cuda.Stream(), t.cuda.Stream()
            self.ev_in, self.ev_kern, self.ev_out = t.cuda.Event(), t.cuda.Event(), t.cuda.Event()
        for st in (self.s_in, self.s_out):
            st.wait_event(start_event)
        self.ev_kern.record(self.s)
        self.ev_out.record(self.s)

    def e2e_end(self):
        """The launching stream waits for the last read-back (before the closing event)."""
        if not self.sharded:
            self.s.wait_event(self.ev_out)

    def e2e_step(self):
        """This rank's inputs from pinned host memory, the step, its results back."""
        if not self.sharded:
            t = self.torch
            self.s_in.wait_event(self.ev_kern)      # the previous step's kernels read x, y
            self.vx.copy_from_host(self.hx[0], self.s_in)
            self.vy.copy_from_host(self.hy[0], self.s_in)
            self.ev_in.record(self.s_in)
            self.s.wait_event(self.ev_in)
            self.s.wait_event(self.ev_out)          # the previous result has been read back
            self.step()
            self.ev_kern.record(self.s)
            self.s_out.wait_event(self.ev_kern)
            self.out.copy_to_host(self.hout[0], self.s_out)
            with t.cuda.stream(self.s_out):
                self.hdot.copy_(self.dotbuf, non_blocking=True)
            self.ev_out.record(self.s_out)
            return
        if self.sharded:
            for k, hx, hy in zip(self.X.mine, self.hx, self.hy):
                self.X.seg[k].copy_(hx, non_blocking=True)
                self.Y.seg[k].copy_(hy, non_blocking=True)
            self.step()
            for k, ho in zip(self.O.mine, self.hout):
                ho.copy_(self.O.seg[k], non_blocking=True)
        self.hdot.copy_(self.dotbuf, non_blocking=True)


# ------------------------------------------------------------------------------------------
# our arm
# ------------------------------------------------------------------------------------------
def main() -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-rows", action="store_true", help="only the headline workload")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--log2n", type=int, default=28, help="headline size 2^log2n (profiling captures use less)")
    ap.add_argument("--stencil-only", type=int, default=0, metavar="N",
                    help="profiling helper: only run the stencil on an N x N grid (8 row blocks), 5 steps")
    ap.add_argument("--scan-only", default="", metavar="DTYPE",
                    help="profiling helper: only the inclusive scan of 2^log2n int64 (i64) or fp32 (f32) "
                         "elements in 4 segments 1:2:3:2, or of zip(x, y) | multiply (zip: fp32, 8 "
                         "segments), 5 times")
    ap.add_argument("--batched-only", type=int, default=0, metavar="NVEC",
                    help="profiling helper: only the batched scan + dot over NVEC vectors of the batch "
                         "recipe, one launch, 5 times")
    ap.add_argument("--link-only", action="store_true",
                    help="measurement helper: host<->device copy bandwidth of 1 GiB pinned buffers "
                         "(the link that bounds the end-to-end number)")
    ap.add_argument("--sort-only", action="store_true",
                    help="profiling helper: only sort 2^log2n fp32 keys in 8 segments, 5 times")
    ap.add_argument("--foreach-only", default="", metavar="FN",
                    help="profiling helper: only run for_each FN (copy, scale, add, triad: fp64; "
                         "black_scholes: fp32) over 2^log2n elements in 8 segments, 5 times")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    if args.impl == "reference":
        run_reference(args)
        return

    import torch
    from paper_2406_00158_gb300 import api, build

    global N_ELEMS
    N_ELEMS = 1 << args.log2n
    build.build()
    if args.link_only:
        dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
        nb = 1 << 30
        h = torch.empty(nb // 4, dtype=torch.float32).pin_memory()
        d = torch.empty(nb // 4, dtype=torch.float32, device=dev)
        s = torch.cuda.current_stream()
        h2d = _time(lambda: d.copy_(h, non_blocking=True), s, 5)
        d2h = _time(lambda: h.copy_(d, non_blocking=True), s, 5)
        print(json.dumps({"link": "pinned host <-> HBM, 1 GiB, cudaMemcpyAsync",
                          "h2d_GB/s": nb / (h2d / 1e3) / 1e9, "d2h_GB/s": nb / (d2h / 1e3) / 1e9}))
        return
    if args.scan_only:
        n = N_ELEMS
        dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
        lens = inputs.proportional_segments(n, [1, 2, 3, 2])
        if args.scan_only == "i64":
            x = torch.from_numpy(inputs.uniform_int64(inputs.SEED_SCAN_I64, n)).to(dev)
        else:
            x = torch.from_numpy(inputs.uniform_pm1_f32(inputs.SEED_DOT_X, n)).to(dev)
        vx = api.SegmentedVector.from_tensor(x, lens)
        vo = api.SegmentedVector.empty(lens, x.dtype, dev)
        v = vx.view()
        nb = 2 * x.element_size() * n
        if args.scan_only == "zip":  # the fused zip(x, y) | multiply view, 8 equal segments each
            segs = [n // 8] * 8
            vx = api.SegmentedVector.from_tensor(x, segs)
            vy = api.SegmentedVector.from_tensor(
                torch.from_numpy(inputs.uniform_pm1_f32(inputs.SEED_DOT_Y, n)).to(dev), segs)
            vo = api.SegmentedVector.empty(segs, x.dtype, dev)
            v = api.dot_view(vx, vy)
            nb = 3 * x.element_size() * n
        s = torch.cuda.current_stream()
        ms = _time(lambda: api.inclusive_scan(v, vo, stream=s), s, 5)
        api.sync_status(s)
        print(json.dumps({"scan": args.scan_only, "n": n, "ms": ms, "GB/s": nb / (ms / 1e3) / 1e9}))
        return
    if args.batched_only:
        dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
        shapes = inputs.batch_shapes(inputs.SEED_BATCH, args.batched_only)
        tot = sum(map(sum, shapes))
        X = api.packed_vectors(inputs.uniform_pm1_f32(inputs.SEED_BATCH_X, tot), shapes, device=dev)
        Pv = api.packed_vectors(inputs.uniform_pm1_f32(inputs.SEED_BATCH_P, tot), shapes, device=dev)
        Y = api.packed_vectors(None, shapes, device=dev)
        batch = api.Batch(X, Pv, Y, torch.zeros(len(shapes), dtype=torch.float32, device=dev))
        s = torch.cuda.current_stream()
        ms = _time(lambda: batch.run(stream=s), s, 5)
        api.sync_status(s)
        print(json.dumps({"batched": len(shapes), "elements": tot, "tune": list(batch.tune), "ms": ms,
                          "GB/s": 12 * tot / (ms / 1e3) / 1e9}))
        return
    if args.sort_only:
        n = N_ELEMS
        dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
        lens = [n // 8] * 8
        x = torch.from_numpy(inputs.uniform_pm1_f32(inputs.SEED_SORT, n)).to(dev)
        vin = api.SegmentedVector.from_tensor(x, lens)
        vout = api.SegmentedVector.empty(lens, torch.float32, dev)
        s = torch.cuda.current_stream()
        ms = _time(lambda: api.sort(vin, vout, stream=s), s, 5)
        api.sync_status(s)
        print(json.dumps({"sort": "f32", "n": n, "ms": ms, "Gkeys/s": n / (ms / 1e3) / 1e9,
                          "GB/s_36B": 36 * n / (ms / 1e3) / 1e9}))
        return
    if args.foreach_only:
        fn, n = args.foreach_only, N_ELEMS
        dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
        lens = [n // 8] * 8
        if fn == "black_scholes":
            vs = [api.SegmentedVector.from_tensor(torch.from_numpy(v).to(dev), lens)
                  for v in inputs.black_scholes_inputs(n)]
            vs += [api.SegmentedVector.empty(lens, torch.float32, dev) for _ in range(2)]
            fargs, nbytes = (float(np.float32(inputs.BS_R)), float(np.float32(inputs.BS_SIGMA))), 20 * n
        else:
            vs = [api.SegmentedVector.from_tensor(torch.from_numpy(v).to(dev), lens)
                  for v in inputs.stream_inputs(n, np.float64)]
            sel = {"copy": (0, 2), "scale": (1, 2), "add": (0, 1, 2), "triad": (0, 1, 2)}[fn]
            vs = [vs[i] for i in sel]
            fargs = (3.0,) if fn in ("scale", "triad") else ()
            nbytes = {"copy": 16, "scale": 16, "add": 24, "triad": 24}[fn] * n
        z = api.View.zipn(*vs)
        s = torch.cuda.current_stream()
        ms = _time(lambda: api.for_each(z, fn, *fargs, stream=s), s, 5)
        api.sync_status(s)
        print(json.dumps({"for_each": fn, "n": n, "ms": ms, "GB/s": nbytes / (ms / 1e3) / 1e9}))
        return
    if args.stencil_only:
        n = args.stencil_only
        dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
        u0 = torch.from_numpy(inputs.uniform01_f32(inputs.SEED_STENCIL, n * n).reshape(n, n)).to(dev)
        rows = [n // 8] * 8
        a = api.MdArray.from_tensor(u0, rows)
        b = api.MdArray.empty(rows, n, dev)
        t = api.MdArray.empty(rows, n, dev)
        s = torch.cuda.current_stream()
        ms = _time(lambda: api.stencil5(a, b, t, 5, stream=s), s, 3) / 5
        api.sync_status(s)
        print(json.dumps({"stencil_n": n, "ms_per_step": ms, "GB/s": 8 * n * n / (ms / 1e3) / 1e9}))
        return
    D = Dist("nccl")
    torch.cuda.set_device(D.local)
    dev = torch.device("cuda", D.local)
    s = torch.cuda.current_stream()

    # ---- inputs: x, y fp32 U[-1,1), 8 equal segments, one allocation each; with N > 1
    # ranks the segments are sharded over the GPUs (segment k on rank k*N//8) and the
    # one 2^28 range is strong-scaled
    x = inputs.uniform_pm1_f32(inputs.SEED_DOT_X, N_ELEMS)
    y = inputs.uniform_pm1_f32(inputs.SEED_DOT_Y, N_ELEMS)
    H = Headline(api, D, dev, s, x, y)
    for _ in range(args.warmup):
        H.step()
    api.sync_status(s)

    # ---- timed region: K steps, events around each part on the launching stream
    K = args.steps
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * K + 1)]
    clocks = ClockSampler(gpu_index_for_smi(D.local))
    D.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.15)
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(s)
    ev[0].record(s)
    for k in range(K):
        H.dot()
        ev[2 * k + 1].record(s)
        H.scan()
        ev[2 * k + 2].record(s)
    t1.record(s)
    torch.cuda.synchronize()
    clk = clocks.stop()
    D.barrier()
    api.sync_status(s)
    ms_local = t0.elapsed_time(t1)
    ms = D.max(ms_local)
    dot_ms = [ev[2 * k].elapsed_time(ev[2 * k + 1]) for k in range(K)]
    scan_ms = [ev[2 * k + 1].elapsed_time(ev[2 * k + 2]) for k in range(K)]
    bytes_step = N_ELEMS * (BYTES_DOT + BYTES_SCAN)          # the whole range, all ranks together
    value = bytes_step * K / (ms / 1e3) / 1e9

    peak, peak_kind = peaks()
    kern = {
        "dot": (statistics.mean(dot_ms), H.local_elems * BYTES_DOT),
        "scan": (statistics.mean(scan_ms), H.local_elems * BYTES_SCAN),
    }
    dom = max(kern, key=lambda k: kern[k][0])
    dom_ms, dom_bytes = kern[dom]
    achieved = dom_bytes / (dom_ms / 1e3) / 1e9
    traffic = None
    tr_path = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(tr_path) and D.world == 1:
        traffic = json.load(open(tr_path)).get(dom)

    # ---- end to end through the C ABI with host buffers (pinned), copies inside the timed region
    e2e_val = None
    if not args.no_e2e:
        H.pin_host()
        e2e_steps = max(3, min(10, K))
        w0 = torch.cuda.Event()
        w0.record(s)
        H.e2e_begin(w0)
        H.e2e_step()
        H.e2e_end()
        torch.cuda.synchronize()
        D.barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(s)
        H.e2e_begin(e0)
        for _ in range(e2e_steps):
            H.e2e_step()
        H.e2e_end()
        e1.record(s)
        torch.cuda.synchronize()
        e2e_ms = D.max(e0.elapsed_time(e1))
        e2e_val = bytes_step * e2e_steps / (e2e_ms / 1e3) / 1e9
        api.sync_status(s)

    # ---- CPU baseline: the oracle on the host cores, bounded sample (rank 0, N = 1)
    cpu = None
    if D.rank == 0 and D.world == 1 and not args.no_cpu_baseline:
        sample = 1 << 26
        dt, nb = cpu_oracle_run(x[:sample], y[:sample], 2)
        import platform
        cpu = {"value": nb / dt / 1e9, "unit": "GB/s", "cores": 1, "kind": "oracle",
               "sample": "oracle FP64 dot + FP64 inclusive_scan over the first 2^26 elements, 2 repetitions",
               "host": {"machine": platform.machine(), "logical_cpus": os.cpu_count()}}
        procs = os.cpu_count() or 1
        dt, nb = cpu_oracle_all_cores(x[:sample], y[:sample], 2, procs)
        cpu["all_cores"] = {"value": nb / dt / 1e9, "unit": "GB/s", "cores": procs, "kind": "oracle",
                            "sample": f"the same 2^26 elements cut into {procs} independent slices, one process "
                                      "per core, each an oracle dot + scan of its slice, 2 repetitions"}
        st = cpu_stencil_f64(2)
        cpu["stencil"] = {"ms_100_steps": st / 2 * 100 * 1e3, "extrapolated_from_steps": 2, "cores": 1,
                          "kind": "oracle", "sample": "oracle FP64 5-point stencil on 16384^2, 2 timed steps, "
                          "extrapolated linearly to 100 steps"}

    rows = {}
    if not args.no_rows and D.world == 1:      # the other rows are single-GPU workloads
        rows = measure_rows(api, dev, s, peak)

    line = {
        "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": D.world, "steps": K,
        "warmup": args.warmup, "ms_per_step": ms / K, "higher_is_better": True, "scaling": "strong",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded SplitMix64, U[-1,1))",
        "config": {"workload": WORKLOAD if args.log2n == 28 else WORKLOAD.replace("2^28", f"2^{args.log2n}"),
                   "n": N_ELEMS, "segments": NSEG,
                   "l2": "no flush: 3 GiB touched per step > 129 MB L2",
                   "parallelism": (f"one range sharded over {D.world} GPUs: segment k on rank k*{D.world}//8; "
                                   "dot: all-gather of partials; scan: all-gather of run totals + carry-in")
                   if D.world > 1 else "1 GPU"},
        "frac_of_peak": value / D.world / peak,
        "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "peak_kind": peak_kind, "traffic": traffic,
                     "per_kernel": {k: {"ms": v[0], "GB/s": v[1] / (v[0] / 1e3) / 1e9,
                                        "frac": v[1] / (v[0] / 1e3) / 1e9 / peak} for k, v in kern.items()}},
        "clocks": clk,
        "device": {"name": torch.cuda.get_device_name(dev),
                   "sms": torch.cuda.get_device_properties(dev).multi_processor_count,
                   "l2_bytes": torch.cuda.get_device_properties(dev).L2_cache_size},
        "e2e": {"value": e2e_val, "unit": "GB/s", "h2d_bytes_per_step": 2 * N_ELEMS * 4,
                "d2h_bytes_per_step": N_ELEMS * 4 + 4 * D.world,
                "copies": ("uploads, step and read-back on three streams: step k's read-back overlaps "
                           "step k+1's upload" if D.world == 1 else "in order on the launching stream")}
        if e2e_val is not None else None,
        "gpu_launches": H.launches_per_step * K,
        "cpu_baseline": cpu,
        "rows": rows,
    }
    if D.rank == 0:
        print(json.dumps(line), flush=True)
    D.close()


if __name__ == "__main__":
    main()
