"""torch.autograd.Function wrappers over the C ABI: every forward and backward
pass is the library's kernels (the tensors are only plumbing).

* scan:    y = inclusive_scan(x) over a segmented fp32 vector; the gradient is the
           reverse inclusive scan of y_bar (x_bar_j = sum_{i >= j} y_bar_i).
* dot:     d = transform_reduce(zip(x, y) | multiply, plus) (Algorithm 1); the
           gradient is scale-by-partner (x_bar = d_bar * y, y_bar = d_bar * x).
* stencil: u_T = A^steps u_0 with the 5-point Jacobi operator A u = wc*u + wn*N(u) on a row-block array; u_bar_0 =
           (A^T)^steps u_bar_T.  The forward pass keeps a checkpoint of the state
           every k steps; when wc or wn need gradients the backward pass walks the
           chain back one k-step window at a time, recomputing the window's states
           from its checkpoint, and each backward step (one fused kernel) also
           accumulates <u_bar_t, u_{t-1}> and <N(u_bar_t), u_{t-1}>.
"""
from __future__ import annotations

import threading
from typing import Sequence

import torch

from . import api


def _contig(ts):
    return [t.contiguous() for t in ts]


_ESZ = {torch.float32: 4, torch.float64: 8, torch.int32: 4, torch.int64: 8}


def _segments_like(lens, dtype, device):
    """Output segments in one allocation, each starting on a 16-byte boundary
    (so the kernels keep their 128-bit path)."""
    a = 16 // _ESZ.get(dtype, 16)
    if a and all(n % a == 0 for n in lens) and sum(lens) > 0:
        # every length keeps the next segment aligned: one split, no padding
        return list(torch.empty(sum(lens), dtype=dtype, device=device).split_with_sizes(lens))
    a = max(a, 1)
    offs, pos = [], 0
    for n in lens:
        offs.append(pos)
        pos += (int(n) + a - 1) // a * a
    buf = torch.empty(max(pos, 1), dtype=dtype, device=device)
    return [buf[o:o + int(n)] for o, n in zip(offs, lens)]


class _Plan:
    """An input vector, its view and an output vector for one shape (segment
    lengths, dtype, device), rebound to each call's tensors: the view's device
    workspace is allocated on the first call only.  One per thread, so that
    calls on different threads never share a workspace."""

    def __init__(self, xs, ys):
        self.x = api.SegmentedVector(xs)
        self.view = self.x.view()
        self.y = api.SegmentedVector(ys)

    def bind(self, xs, ys):
        # xs are contiguous 1-D tensors of the plan's lengths (the key guarantees
        # lengths, dtype and device), ys come from _segments_like
        self.x._rebind_unchecked(xs)
        self.y._rebind_unchecked(ys)

    def release(self):
        # drop this call's tensors (launches already made keep their storage)
        self.x.segments = []
        self.y.segments = []


_plans = threading.local()


def _plan(kind, xs, ys):
    cache = getattr(_plans, "d", None)
    if cache is None:
        cache = _plans.d = {}
    key = (kind, tuple(t.numel() for t in xs), xs[0].dtype, xs[0].device)
    p = cache.get(key)
    if p is None:
        if len(cache) >= 32:
            cache.clear()
        p = cache[key] = _Plan(xs, ys)
    else:
        p.bind(xs, ys)
    return p


class _ScanFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, *segs):
        xs = _contig(segs)
        lens = [s.numel() for s in xs]
        ys = _segments_like(lens, xs[0].dtype, xs[0].device)
        p = _plan("scan", xs, ys)
        api.inclusive_scan(p.view, p.y)
        p.release()
        ctx.lens = lens
        return tuple(ys)

    @staticmethod
    def backward(ctx, *gys):
        dev = next(g for g in gys if g is not None).device
        gys = [g.contiguous() if g is not None else torch.zeros(n, device=dev) for g, n in zip(gys, ctx.lens)]
        gxs = _segments_like(ctx.lens, gys[0].dtype, dev)
        p = _plan("reverse_scan", gys, gxs)
        api.reverse_inclusive_scan(p.view, p.y)
        p.release()
        return tuple(gxs)


def inclusive_scan(segments: Sequence[torch.Tensor]) -> tuple:
    """Differentiable segmented inclusive scan: one output tensor per segment."""
    return _ScanFn.apply(*segments)


class _ScanFlatFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, lens):
        x = x.contiguous()
        y = torch.empty_like(x)
        p = _plan("scan_flat", list(x.split_with_sizes(lens)), list(y.split_with_sizes(lens)))
        api.inclusive_scan(p.view, p.y)
        p.release()
        ctx.lens = lens
        return y

    @staticmethod
    def backward(ctx, gy):
        gy = gy.contiguous()
        gx = torch.empty_like(gy)
        p = _plan("reverse_scan_flat", list(gy.split_with_sizes(ctx.lens)), list(gx.split_with_sizes(ctx.lens)))
        api.reverse_inclusive_scan(p.view, p.y)
        p.release()
        return gx, None


def inclusive_scan_flat(x: torch.Tensor, lens: Sequence[int]) -> torch.Tensor:
    """The same scan over one flat tensor whose consecutive pieces of the given
    lengths are the segments (one autograd node with one input and one output,
    instead of one tensor per segment)."""
    lens = [int(n) for n in lens]
    if x.dim() != 1 or sum(lens) != x.numel():
        raise ValueError("inclusive_scan_flat: x must be 1-D with sum(lens) elements")
    return _ScanFlatFn.apply(x, lens)


class _DotFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, nx: int, *segs):
        xs, ys = _contig(segs[:nx]), _contig(segs[nx:])
        x, y = api.SegmentedVector(xs), api.SegmentedVector(ys)
        out = torch.zeros(1, dtype=torch.float32, device=xs[0].device)
        api.transform_reduce(api.dot_view(x, y), out)
        ctx.save_for_backward(*xs, *ys)
        ctx.nx = nx
        return out.reshape(())

    @staticmethod
    def backward(ctx, gd):
        saved = ctx.saved_tensors
        xs, ys = list(saved[:ctx.nx]), list(saved[ctx.nx:])
        x, y = api.SegmentedVector(xs), api.SegmentedVector(ys)
        need_y = any(ctx.needs_input_grad[1 + ctx.nx:])
        need_x = any(ctx.needs_input_grad[1:1 + ctx.nx])
        g = gd.reshape(1).to(torch.float32).contiguous()
        gx = api.SegmentedVector.empty([t.numel() for t in xs], torch.float32, g.device) if need_x else None
        gy = api.SegmentedVector.empty([t.numel() for t in ys], torch.float32, g.device) if need_y else None
        api.scale_by_partner(x, y, g, gx, gy)
        gxs = list(gx.segments) if gx is not None else [None] * len(xs)
        gys = list(gy.segments) if gy is not None else [None] * len(ys)
        return (None, *gxs, *gys)


def dot(x_segments: Sequence[torch.Tensor], y_segments: Sequence[torch.Tensor]) -> torch.Tensor:
    """Differentiable <x, y> over segmented fp32 vectors (segmentations may differ)."""
    return _DotFn.apply(len(x_segments), *x_segments, *y_segments)


class _StencilFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, wc, wn, steps: int, every: int, *blocks):
        seg_rows = [b.shape[0] for b in blocks]
        cols = blocks[0].shape[1]
        dev = blocks[0].device
        wcf, wnf = float(wc), float(wn)
        u = api.MdArray.empty(seg_rows, cols, dev)
        u.load(torch.cat(blocks) if len(blocks) > 1 else blocks[0])
        tmp = api.MdArray.empty(seg_rows, cols, dev)
        ckpts = [u]  # state at steps 0, every, 2*every, ...
        cur = u
        done = 0
        while done < steps:
            n = min(every, steps - done)
            nxt = api.MdArray.empty(seg_rows, cols, dev)
            api.stencil5(cur, nxt, tmp if n > 1 else None, n, wcf, wnf)
            done += n
            if done < steps:
                ckpts.append(nxt)
            cur = nxt
        ctx.ckpts = ckpts
        ctx.meta = (seg_rows, cols, steps, every, wcf, wnf)
        ctx.wmeta = ((wc.device, wc.dtype), (wn.device, wn.dtype))
        return tuple(b[1:r + 1] for b, r in zip(cur.blocks, seg_rows))

    @staticmethod
    def backward(ctx, *gouts):
        seg_rows, cols, steps, every, wcf, wnf = ctx.meta
        dev = next(g for g in gouts if g is not None).device
        g = api.MdArray.empty(seg_rows, cols, dev)
        g.load(torch.cat([gg if gg is not None else torch.zeros(r, cols, device=dev)
                          for gg, r in zip(gouts, seg_rows)]))
        need_w = ctx.needs_input_grad[0] or ctx.needs_input_grad[1]
        other = api.MdArray.empty(seg_rows, cols, dev)
        acc = torch.zeros(2, dtype=torch.float64, device=dev)
        if not need_w:
            tmp = api.MdArray.empty(seg_rows, cols, dev) if steps > 1 else None
            api.stencil5_T(g, other, tmp, steps, wcf, wnf)
            g = other
        else:
            # windows in reverse: states u_{c*every} .. u_{c*every + n - 1} recomputed from checkpoint c
            nwin = len(ctx.ckpts)
            states = [api.MdArray.empty(seg_rows, cols, dev) for _ in range(max(0, every - 1))]
            for c in reversed(range(nwin)):
                n = min(every, steps - c * every)
                window = [ctx.ckpts[c]]
                for j in range(1, n):
                    api.stencil5(window[-1], states[j - 1], None, 1, wcf, wnf)
                    window.append(states[j - 1])
                for j in reversed(range(n)):  # step t = c*every + j + 1 reads u_{t-1} = window[j]
                    api.stencil5_T_wgrad(g, other, window[j], acc, wcf, wnf)
                    g, other = other, g
        (dc, tc), (dn, tn) = ctx.wmeta
        gwc = acc[0].to(device=dc, dtype=tc) if ctx.needs_input_grad[0] else None
        gwn = acc[1].to(device=dn, dtype=tn) if ctx.needs_input_grad[1] else None
        grads_blocks = tuple(b[1:r + 1].clone() for b, r in zip(g.blocks, seg_rows))
        ctx.ckpts = None
        return (gwc, gwn, None, None, *grads_blocks)


def stencil(blocks: Sequence[torch.Tensor], steps: int, wc=0.0, wn=0.25, checkpoint_every: int = 10) -> tuple:
    """Differentiable `steps` steps of the 5-point Jacobi for_each over a row-block
    array (one (rows_k, cols) fp32 tensor per block).  wc / wn may be 0-dim
    tensors that require grad."""
    wc_t = wc if isinstance(wc, torch.Tensor) else torch.tensor(float(wc))
    wn_t = wn if isinstance(wn, torch.Tensor) else torch.tensor(float(wn))
    return _StencilFn.apply(wc_t, wn_t, int(steps), int(checkpoint_every), *blocks)
