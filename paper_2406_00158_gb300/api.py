"""Thin Python layer over the C ABI: PyTorch supplies device memory and streams,
every step of every algorithm runs in the library's CUDA kernels.

Objects mirror the handles of ``dr.h``: ``SegmentedVector`` (dr_vec),
``View`` (dr_view), ``MdArray`` (dr_md2), ``Batch`` (dr_batch).  Python
objects keep references to the tensors and handles they were built from, so a
view never outlives its base (Sec. 4.4: views are non-owning).
"""
from __future__ import annotations

import ctypes
from typing import Optional, Sequence

import torch

from . import _lib as L
from ._lib import call

_DT = {torch.float32: L.DR_F32, torch.float64: L.DR_F64, torch.int64: L.DR_I64, torch.int32: L.DR_I32}
_TORCH = {v: k for k, v in _DT.items()}
_OPS = {"plus": L.DR_PLUS, "mul": L.DR_MUL, "min": L.DR_MIN, "max": L.DR_MAX}
_UOPS = {"scale": L.DR_U_SCALE, "add": L.DR_U_ADD, "neg": L.DR_U_NEG, "abs": L.DR_U_ABS,
         "square": L.DR_U_SQUARE}


def _op(op) -> int:
    return _OPS[op] if isinstance(op, str) else int(op)


def stream_handle(stream: Optional[torch.cuda.Stream] = None) -> ctypes.c_void_p:
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _handle_out():
    return ctypes.c_void_p()


def _ptr_array(ptrs) -> ctypes.Array:
    return (ctypes.c_void_p * len(ptrs))(*[ctypes.c_void_p(int(p)) for p in ptrs])


def _scalar_bytes(value, dtype_code: int) -> ctypes.Array:
    t = {L.DR_F32: ctypes.c_float, L.DR_F64: ctypes.c_double, L.DR_I64: ctypes.c_int64,
         L.DR_I32: ctypes.c_int32}[dtype_code]
    return t(value)


def sync_status(stream: Optional[torch.cuda.Stream] = None) -> None:
    """Synchronizes the stream and raises DRError if a device-side wait expired."""
    call("dr_sync_status", stream_handle(stream))


def set_spin_limit(polls: int) -> None:
    call("dr_set_spin_limit", int(polls))


def debug_skip_publish(tile: int) -> None:
    call("dr_debug_skip_publish", int(tile))


def block_lengths(n: int, p: int) -> list[int]:
    out = (ctypes.c_int64 * p)()
    call("dr_block_lengths", int(n), int(p), out)
    return list(out)


class SegmentedVector:
    """A distributed vector (Sec. 4.2.1) over caller-owned device segments."""

    def __init__(self, segments: Sequence[torch.Tensor]):
        segs = list(segments)
        if not segs:
            raise ValueError("a segmented vector needs at least one segment")
        dt = segs[0].dtype
        for s in segs:
            if s.dtype != dt or s.dim() != 1 or not s.is_contiguous():
                raise ValueError("segments must be 1-D contiguous tensors of one dtype")
        self.segments = segs
        self.dtype = dt
        self._lens = [s.numel() for s in segs]
        lens = (ctypes.c_int64 * len(segs))(*self._lens)
        ptrs = _ptr_array([s.data_ptr() for s in segs])
        h = _handle_out()
        call("dr_vec_create", _DT[dt], len(segs), lens, ptrs, ctypes.byref(h))
        self.handle = h

    @classmethod
    def empty(cls, lens: Sequence[int], dtype=torch.float32, device="cuda"):
        """One separate allocation per segment (one memory locale each)."""
        return cls([torch.empty(int(n), dtype=dtype, device=device) for n in lens])

    @classmethod
    def from_tensor(cls, t: torch.Tensor, lens: Sequence[int]):
        """Copies a flat tensor into a new vector with the given segment sizes."""
        v = cls.empty(lens, t.dtype, t.device)
        off = 0
        for s in v.segments:
            s.copy_(t[off:off + s.numel()])
            off += s.numel()
        return v

    def rebind(self, segments: Sequence[torch.Tensor]) -> "SegmentedVector":
        """Points this vector at new tensors of the same segment lengths and
        dtype; its views follow and keep their device workspaces."""
        segs = list(segments)
        if len(segs) != len(self._lens):
            raise ValueError("rebind needs one tensor per segment")
        for s, n in zip(segs, self._lens):
            if s.dtype != self.dtype or s.dim() != 1 or not s.is_contiguous() or s.numel() != n:
                raise ValueError("rebind: segments must match in dtype, length and be 1-D contiguous")
        call("dr_vec_rebind", self.handle, _ptr_array([s.data_ptr() for s in segs]))
        self.segments = segs
        return self

    def _rebind_unchecked(self, segs: list) -> None:
        """rebind() for tensors the caller already made 1-D, contiguous and of
        this vector's lengths and dtype (the autograd plans): one pointer array
        reused, no Python-side checks (the library still checks the pointers)."""
        arr = getattr(self, "_ptrs", None)
        if arr is None:
            arr = self._ptrs = (ctypes.c_void_p * len(self._lens))()
        for i, t in enumerate(segs):
            arr[i] = t.data_ptr()
        call("dr_vec_rebind", self.handle, arr)
        self.segments = segs

    @property
    def n(self) -> int:
        return sum(s.numel() for s in self.segments)

    @property
    def lens(self) -> list[int]:
        return [s.numel() for s in self.segments]

    def locate(self, i: int) -> tuple[int, int]:
        seg, off = ctypes.c_int(), ctypes.c_int64()
        call("dr_vec_locate", self.handle, int(i), ctypes.byref(seg), ctypes.byref(off))
        return seg.value, off.value

    def to_tensor(self) -> torch.Tensor:
        return torch.cat(self.segments) if self.segments else torch.empty(0)

    def copy_from_host(self, host: torch.Tensor, stream=None) -> None:
        assert host.device.type == "cpu" and host.is_contiguous() and host.numel() == self.n
        call("dr_vec_copy_from_host", self.handle, ctypes.c_void_p(host.data_ptr()), stream_handle(stream))

    def copy_to_host(self, host: torch.Tensor, stream=None) -> None:
        assert host.device.type == "cpu" and host.is_contiguous() and host.numel() == self.n
        call("dr_vec_copy_to_host", self.handle, ctypes.c_void_p(host.data_ptr()), stream_handle(stream))

    def view(self) -> "View":
        return View.of(self)

    def __del__(self):
        h = getattr(self, "handle", None)
        if h and L._lib is not None:
            L._lib.dr_vec_destroy(h)


def packed_vectors(flat, shapes: Sequence[Sequence[int]], device="cuda", dtype=torch.float32):
    """Many segmented vectors in one device buffer: vector v has segments
    shapes[v] (element counts) taken in order from the flat host array `flat`
    (None: uninitialized).  Every segment starts on a 16-byte boundary of the
    buffer (128-bit access); the buffer is filled with one host-to-device copy.
    Returns the list of SegmentedVector (each keeps the buffer alive)."""
    esz = torch.empty((), dtype=dtype).element_size()
    align = 16 // esz
    offs, pos = [], 0
    for sh in shapes:
        o = []
        for n in sh:
            o.append(pos)
            pos += (int(n) + align - 1) // align * align
        offs.append(o)
    buf = torch.empty(max(pos, 1), dtype=dtype, device=device)
    if flat is not None:
        src = torch.as_tensor(flat).reshape(-1)
        host = torch.zeros(max(pos, 1), dtype=dtype)
        k = 0
        for sh, o in zip(shapes, offs):
            for n, p0 in zip(sh, o):
                host[p0:p0 + n] = src[k:k + n]
                k += n
        buf.copy_(host.pin_memory() if device != "cpu" else host)
    vecs = []
    for sh, o in zip(shapes, offs):
        v = SegmentedVector([buf[p0:p0 + int(n)] for n, p0 in zip(sh, o)])
        v._buffer = buf
        vecs.append(v)
    return vecs


class View:
    """A lazy view (Sec. 4.4); its kernels fuse it into their loads."""

    def __init__(self, handle, keep):
        self.handle = handle
        self._keep = keep

    @classmethod
    def of(cls, v: SegmentedVector) -> "View":
        h = _handle_out()
        call("dr_view_of", v.handle, ctypes.byref(h))
        return cls(h, [v])

    def transform(self, op, arg: float = 0.0) -> "View":
        h = _handle_out()
        call("dr_view_transform", self.handle, _UOPS[op] if isinstance(op, str) else int(op), float(arg),
             ctypes.byref(h))
        return View(h, [self])

    def zip(self, other: "View", strict_align: bool = False) -> "View":
        """zip(self, other); with strict_align=True, operands that are not
        aligned are refused (DR_E_ALIGN) instead of re-cut."""
        h = _handle_out()
        if strict_align:
            call("dr_view_zip_ex", self.handle, other.handle, L.DR_ZIP_STRICT_ALIGN, ctypes.byref(h))
        else:
            call("dr_view_zip", self.handle, other.handle, ctypes.byref(h))
        return View(h, [self, other])

    @classmethod
    def zipn(cls, *leaves) -> "View":
        """k-ary zip (2 <= k <= 6) of untransformed views or vectors; for_each
        writes through its elements."""
        vs = [_as_view(v) for v in leaves]
        arr = (ctypes.c_void_p * len(vs))(*[v.handle for v in vs])
        h = _handle_out()
        call("dr_view_zipn", len(vs), arr, ctypes.byref(h))
        return cls(h, vs)

    def zip_transform(self, op) -> "View":
        h = _handle_out()
        call("dr_view_zip_transform", self.handle, _op(op), ctypes.byref(h))
        return View(h, [self])

    def take(self, l: int) -> "View":
        h = _handle_out()
        call("dr_view_take", self.handle, int(l), ctypes.byref(h))
        return View(h, [self])

    def drop(self, f: int) -> "View":
        h = _handle_out()
        call("dr_view_drop", self.handle, int(f), ctypes.byref(h))
        return View(h, [self])

    def info(self) -> dict:
        size, arity, dtype, np_ = ctypes.c_int64(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        call("dr_view_info", self.handle, ctypes.byref(size), ctypes.byref(arity), ctypes.byref(dtype),
             ctypes.byref(np_))
        return {"size": size.value, "arity": arity.value, "dtype": dtype.value, "npieces": np_.value}

    @property
    def size(self) -> int:
        return self.info()["size"]

    def segments(self) -> list[tuple]:
        """(start, len, seg_a, off_a, seg_b, off_b) per piece of the segmentation."""
        n = self.info()["npieces"]
        arr = (L.dr_piece * max(1, n))()
        call("dr_view_segments", self.handle, n, arr)
        return [(p.start, p.len, p.seg[0], p.off[0], p.seg[1], p.off[1]) for p in arr[:n]]

    def __del__(self):
        h = getattr(self, "handle", None)
        if h and L._lib is not None:
            L._lib.dr_view_destroy(h)


def _as_view(v) -> View:
    return v if isinstance(v, View) else View.of(v)


def dot_view(x: SegmentedVector, y: SegmentedVector) -> View:
    """zip(x, y) | transform(multiply): the view of Algorithm 1."""
    return View.of(x).zip(View.of(y)).zip_transform("mul")


def inclusive_scan(inp, out: SegmentedVector, op="plus", stream=None) -> SegmentedVector:
    v = _as_view(inp)  # held for the duration of the call (its handle is freed with it)
    call("dr_inclusive_scan", v.handle, out.handle, _op(op), stream_handle(stream))
    return out


def exclusive_scan(inp, out: SegmentedVector, init, op="plus", stream=None) -> SegmentedVector:
    v = _as_view(inp)
    init_c = _scalar_bytes(init, _DT[out.dtype])
    call("dr_exclusive_scan", v.handle, out.handle, _op(op), ctypes.byref(init_c), stream_handle(stream))
    return out


def scan_with_carry(inp, out: SegmentedVector, carry: torch.Tensor, op="plus", exclusive: bool = False,
                    stream=None) -> SegmentedVector:
    """Scan whose chain starts from a device value: inclusive out_i = carry op
    in_0 op ... op in_i; exclusive out_0 = carry, ... (carry: a 1-element device
    tensor of the vector's dtype)."""
    v = _as_view(inp)
    assert carry.is_cuda and carry.dtype == out.dtype and carry.numel() >= 1
    call("dr_scan_with_carry", v.handle, out.handle, _op(op), 1 if exclusive else 0,
         ctypes.c_void_p(carry.data_ptr()), stream_handle(stream))
    return out


def reverse_inclusive_scan(inp, out: SegmentedVector, stream=None) -> SegmentedVector:
    v = _as_view(inp)
    call("dr_reverse_inclusive_scan", v.handle, out.handle, stream_handle(stream))
    return out


def transform_reduce(inp, out: torch.Tensor, op="plus", init=0, stream=None) -> torch.Tensor:
    """out[0] = init op v_0 op ... op v_{n-1}; `out` is a 1-element device tensor."""
    v = _as_view(inp)
    init_c = _scalar_bytes(init, _DT[out.dtype])
    call("dr_transform_reduce", v.handle, _op(op), ctypes.byref(init_c), ctypes.c_void_p(out.data_ptr()),
         stream_handle(stream))
    return out


FOR_EACH_FNS = {"copy": 0, "scale": 1, "add": 2, "triad": 3, "black_scholes": 4}


def for_each(zip_view: View, fn, *args: float, stream=None) -> None:
    """for_each over a k-ary zip with a built-in element function (operand roles
    in dr.h): copy zip(a, c); scale zip(b, c), q; add zip(a, b, c);
    triad zip(a, b, c), q; black_scholes zip(S, X, T, C, P), r, sigma."""
    code = FOR_EACH_FNS[fn] if isinstance(fn, str) else int(fn)
    arr = (ctypes.c_double * max(1, len(args)))(*[float(a) for a in args])
    call("dr_for_each", zip_view.handle, code, arr, len(args), stream_handle(stream))


def transform(inp, out: SegmentedVector, stream=None) -> SegmentedVector:
    """out_i = inp_i: a (fused) view written out to a vector."""
    v = _as_view(inp)
    call("dr_transform", v.handle, out.handle, stream_handle(stream))
    return out


def sort(inp, out: SegmentedVector, stream=None) -> SegmentedVector:
    """out = the elements of inp in ascending order (floats in IEEE totalOrder);
    out may be inp's own vector (in place)."""
    v = _as_view(inp)
    call("dr_sort", v.handle, out.handle, stream_handle(stream))
    return out


def scale_by_partner(x: SegmentedVector, y: SegmentedVector, g: torch.Tensor, gx: Optional[SegmentedVector],
                     gy: Optional[SegmentedVector], stream=None) -> None:
    call("dr_scale_by_partner", x.handle, y.handle, ctypes.c_void_p(g.data_ptr()),
         gx.handle if gx is not None else None, gy.handle if gy is not None else None, stream_handle(stream))


class MdArray:
    """Row-block segmented 2-D fp32 array with one ghost row above and below
    each block (block k: tensor of shape (rows_k + 2, cols))."""

    def __init__(self, blocks: Sequence[torch.Tensor]):
        blocks = list(blocks)
        cols = blocks[0].shape[1]
        for b in blocks:
            if b.dtype != torch.float32 or b.dim() != 2 or b.shape[1] != cols or not b.is_contiguous():
                raise ValueError("blocks must be contiguous fp32 (rows_k + 2, cols) tensors")
        self.blocks = blocks
        self.cols = cols
        self.seg_rows = [b.shape[0] - 2 for b in blocks]
        self.rows = sum(self.seg_rows)
        srows = (ctypes.c_int64 * len(blocks))(*self.seg_rows)
        h = _handle_out()
        call("dr_md2_create", L.DR_F32, self.rows, cols, len(blocks), srows,
             _ptr_array([b.data_ptr() for b in blocks]), ctypes.byref(h))
        self.handle = h

    @classmethod
    def empty(cls, seg_rows: Sequence[int], cols: int, device="cuda"):
        return cls([torch.zeros(int(r) + 2, cols, dtype=torch.float32, device=device) for r in seg_rows])

    @classmethod
    def from_tensor(cls, u: torch.Tensor, seg_rows: Sequence[int]):
        m = cls.empty(seg_rows, u.shape[1], u.device)
        m.load(u)
        return m

    def load(self, u: torch.Tensor) -> None:
        r = 0
        for b, k in zip(self.blocks, self.seg_rows):
            b[1:k + 1].copy_(u[r:r + k])
            r += k

    def to_tensor(self) -> torch.Tensor:
        return torch.cat([b[1:k + 1] for b, k in zip(self.blocks, self.seg_rows)])

    def exchange_halos(self, stream=None) -> None:
        call("dr_md2_exchange_halos", self.handle, stream_handle(stream))

    def set_external_halos(self, top: bool, bottom: bool) -> None:
        """This array is one rank's share of a taller grid: its outer ghost rows
        hold the neighbouring shares' rows (written by the caller)."""
        call("dr_md2_set_external_halos", self.handle, 1 if top else 0, 1 if bottom else 0)
        self.ext = (bool(top), bool(bottom))

    def __del__(self):
        h = getattr(self, "handle", None)
        if h and L._lib is not None:
            L._lib.dr_md2_destroy(h)


def stencil5(inp: MdArray, out: MdArray, tmp: Optional[MdArray], steps: int, wc: float = 0.0,
             wn: float = 0.25, stream=None) -> MdArray:
    call("dr_stencil5", inp.handle, out.handle, tmp.handle if tmp is not None else None, int(steps),
         float(wc), float(wn), stream_handle(stream))
    return out


ROWS = {"all": L.DR_ROWS_ALL, "inner": L.DR_ROWS_INNER, "outer": L.DR_ROWS_OUTER}


def stencil5_part(inp: MdArray, out: MdArray, part="all", wc: float = 0.0, wn: float = 0.25,
                  stream=None) -> MdArray:
    """One stencil step over the inner or outer row blocks only (see dr.h)."""
    call("dr_stencil5_part", inp.handle, out.handle, ROWS[part] if isinstance(part, str) else int(part),
         float(wc), float(wn), stream_handle(stream))
    return out


def stencil5_T(inp: MdArray, out: MdArray, tmp: Optional[MdArray], steps: int, wc: float = 0.0,
               wn: float = 0.25, stream=None) -> MdArray:
    call("dr_stencil5_T", inp.handle, out.handle, tmp.handle if tmp is not None else None, int(steps),
         float(wc), float(wn), stream_handle(stream))
    return out


def stencil5_T_wgrad(inp: MdArray, out: MdArray, prev: MdArray, acc: torch.Tensor, wc: float = 0.0,
                     wn: float = 0.25, stream=None) -> MdArray:
    """out = A^T inp; acc[0] += <inp, prev>, acc[1] += <N(inp), prev> (acc: 2 fp64 on device)."""
    assert acc.dtype == torch.float64 and acc.numel() >= 2 and acc.is_contiguous()
    call("dr_stencil5_T_wgrad", inp.handle, out.handle, prev.handle, float(wc), float(wn),
         ctypes.c_void_p(acc.data_ptr()), stream_handle(stream))
    return out


class Batch:
    """y_v = inclusive_scan(x_v), dots[v] = <x_v, p_v> for many vectors in one launch."""

    def __init__(self, xs: Sequence[SegmentedVector], ps: Sequence[SegmentedVector],
                 ys: Sequence[SegmentedVector], dots: torch.Tensor, tune: Optional[tuple] = None):
        n = len(xs)
        assert len(ps) == n and len(ys) == n and dots.numel() >= n and dots.dtype == torch.float32
        self._keep = (list(xs), list(ps), list(ys), dots)
        arr = lambda vs: (ctypes.c_void_p * n)(*[v.handle.value for v in vs])
        t = L.dr_tune(*tune) if tune else None
        h = _handle_out()
        call("dr_batch_plan", n, arr(xs), arr(ps), arr(ys), ctypes.c_void_p(dots.data_ptr()),
             ctypes.byref(t) if t is not None else None, ctypes.byref(h))
        self.handle = h
        self.nvec = n

    def run(self, stream=None) -> None:
        call("dr_batch_run", self.handle, stream_handle(stream))

    def run_graph(self, stream=None) -> None:
        call("dr_batch_run_graph", self.handle, stream_handle(stream))

    def run_per_range(self, stream=None) -> None:
        call("dr_batch_run_per_range", self.handle, stream_handle(stream))

    def run_per_range_graph(self, stream=None) -> None:
        """The per-range baseline's launches captured once in a CUDA graph, replayed."""
        call("dr_batch_run_per_range_graph", self.handle, stream_handle(stream))

    @property
    def tune(self) -> tuple:
        """(threads, items, ctas_per_sm, variant) of the batched kernel."""
        t = L.dr_tune()
        call("dr_batch_get_tune", self.handle, ctypes.byref(t))
        return (t.threads, t.items, t.ctas_per_sm, t.variant)

    @tune.setter
    def tune(self, value) -> None:
        t = L.dr_tune(*value)
        call("dr_batch_set_tune", self.handle, ctypes.byref(t))

    def autotune(self, retune: bool = False, cache_path: Optional[str] = None) -> tuple:
        t = L.dr_tune()
        call("dr_batch_autotune", self.handle, 1 if retune else 0,
             cache_path.encode() if cache_path else None, ctypes.byref(t))
        return (t.threads, t.items, t.ctas_per_sm, t.variant)

    def __del__(self):
        h = getattr(self, "handle", None)
        if h and L._lib is not None:
            L._lib.dr_batch_destroy(h)
