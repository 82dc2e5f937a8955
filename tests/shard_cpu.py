"""A CPU stand-in for the sharded path's local steps, so that the placement and
exchange logic of paper_2406_00158_gb300.shard runs on gloo ranks without a
GPU.  Each local step is the oracle's definition of that step on CPU tensors;
the stencil's inner / outer row-block split follows the library's 64-row
blocks, and the inner part reads no outer ghost row (it may still be in
flight)."""
import numpy as np
import torch

import oracle

ROWS_PER_BLOCK = 64


class _Md:
    def __init__(self, blocks, top, bottom):
        self.blocks, self.top, self.bottom = list(blocks), top, bottom


class CpuBackend:
    def vector(self, tensors):
        return list(tensors)

    @staticmethod
    def default_device():
        return torch.device("cpu")

    def scratch(self, k, dtype, device):
        return torch.zeros(k, dtype=dtype)

    @staticmethod
    def _cat(v):
        return torch.cat(list(v)).numpy() if v else np.zeros(0, np.int64)

    def reduce(self, v, op, out1):
        x = self._cat(v)
        r = oracle.reduce(x, op)
        out1[0] = float(r) if x.dtype.kind == "f" else int(r)

    def dot(self, x, y, out1):
        a, b = self._cat(x), self._cat(y)
        out1[0] = oracle.reduce(a.astype(np.int64) * b.astype(np.int64), "plus")

    def fold(self, parts, op, out1):
        vals = np.array([p.item() for p in parts], dtype=np.int64 if not out1.is_floating_point() else np.float64)
        out1[0] = oracle.reduce(vals, op) if vals.size else oracle.identity(op, vals.dtype)

    def scan(self, x, out, op, carry1, exclusive):
        a = self._cat(x)
        init = None if carry1 is None else carry1.item()
        y = oracle.scan(a, op, exclusive=exclusive, init=init)
        off = 0
        for t in out:
            t.copy_(torch.from_numpy(np.ascontiguousarray(y[off:off + t.numel()])).to(t.dtype))
            off += t.numel()

    def md(self, blocks, top, bottom):
        return _Md(blocks, top, bottom)

    def stencil_part(self, a, b, part, wc, wn):
        """One step over the run's rows of the given part (oracle fixed-order fp32
        arithmetic on the run extended by its outer ghost rows, zero where the
        run ends at the grid's edge)."""
        rows = [blk.shape[0] - 2 for blk in a.blocks]
        C = a.blocks[0].shape[1]
        own = torch.cat([blk[1:r + 1] for blk, r in zip(a.blocks, rows)]).numpy()
        R = own.shape[0]
        # global row-block ranges (per block, 64 rows each)
        rbs, s = [], 0
        for r in rows:
            for lo in range(0, r, ROWS_PER_BLOCK):
                rbs.append((s + lo, s + min(r, lo + ROWS_PER_BLOCK)))
            s += r
        if part == "inner":
            sel = rbs[1:-1]
            top = bot = np.zeros(C, np.float32)      # the inner rows do not read the outer ghosts
        else:
            sel = [rbs[0], rbs[-1]] if len(rbs) > 1 else rbs[:1]
            top = a.blocks[0][0].numpy() if a.top else np.zeros(C, np.float32)
            bot = a.blocks[-1][rows[-1] + 1].numpy() if a.bottom else np.zeros(C, np.float32)
        ext = np.concatenate([top[None], own, bot[None]])
        new = oracle.stencil5_f32(ext, 1, wc, wn)[1:R + 1]
        off = 0
        starts = []
        for blk, r in zip(b.blocks, rows):
            starts.append(off)
            off += r
        for lo, hi in sel:
            for k, (blk, r) in enumerate(zip(b.blocks, rows)):
                s0 = starts[k]
                a0, a1 = max(lo, s0), min(hi, s0 + r)
                if a1 > a0:
                    blk[1 + a0 - s0:1 + a1 - s0] = torch.from_numpy(new[a0:a1])
