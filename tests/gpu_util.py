"""Helpers for the GPU parity tests: build / load the library once, move seeded
numpy inputs into segmented device containers and back.

Every segment these helpers allocate sits inside a larger allocation with a
guard band of sentinel bytes on both sides (and the two outer ghost rows of a
row-block array, which no kernel may touch, hold sentinels too).  The bands of
every live allocation are checked after each GPU test (tests/conftest.py), so
a kernel that writes past the end of a segment -- into slack that the caching
allocator would otherwise hide -- fails the test that did it."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

GUARD_BYTES = 64          # per side; a multiple of 16 keeps segments 16-byte aligned
SENTINEL = 0xA5
_guarded = []             # (base tensor, [(lo, hi) byte ranges], label), until the next check


def dev():
    from paper_2406_00158_gb300 import build
    build.build()
    from paper_2406_00158_gb300 import _lib
    _lib.lib()
    return torch.device("cuda:0")


def sms() -> int:
    return torch.cuda.get_device_properties(0).multi_processor_count


def _dt_code(dtype) -> int:
    from paper_2406_00158_gb300 import _lib as L
    return {torch.float32: L.DR_F32, torch.float64: L.DR_F64, torch.int64: L.DR_I64,
            torch.int32: L.DR_I32}[dtype]


def scan_tile(dtype=torch.float32, view=False) -> int:
    """Elements per tile of the scan kernel (the unit of its carry chain); view:
    the kernel for a fused view (ops or a zip)."""
    from paper_2406_00158_gb300 import _lib as L
    return L.kernel_geometry(L.DR_K_SCAN_VIEW if view else L.DR_K_SCAN, _dt_code(dtype))[0]


def reduce_geometry(dtype=torch.float32):
    """(tile elements, CTAs per SM) of the reduce kernel."""
    from paper_2406_00158_gb300 import _lib as L
    return L.kernel_geometry(L.DR_K_REDUCE, _dt_code(dtype))


def _guard(base: torch.Tensor, ranges, label: str) -> None:
    b = base.view(torch.uint8)
    for lo, hi in ranges:
        b[lo:hi].fill_(SENTINEL)
    _guarded.append((base, list(ranges), label))


def guarded_segment(n: int, dtype, device=None, offset_elems: int = 0, label: str = "segment"):
    """An n-element device tensor at GUARD_BYTES (+ offset_elems elements) into a
    larger allocation whose first and last GUARD_BYTES hold the sentinel."""
    device = device or torch.device("cuda:0")
    esz = torch.empty((), dtype=dtype).element_size()
    g = GUARD_BYTES // esz
    base = torch.empty(n + offset_elems + 2 * g, dtype=dtype, device=device)
    nb = base.numel() * esz
    _guard(base, [(0, (g + offset_elems) * esz), (nb - GUARD_BYTES, nb)], label)
    seg = base[g + offset_elems:g + offset_elems + n]
    seg._guard_base = base
    return seg


def check_guards() -> list:
    """Sentinel bands that were overwritten since they were set.  The bands are
    held (with their allocations) until this check, then forgotten."""
    bad = []
    if _guarded:
        torch.cuda.synchronize()
    for base, ranges, label in _guarded:
        b = base.view(torch.uint8)
        for lo, hi in ranges:
            if not bool((b[lo:hi] == SENTINEL).all()):
                bad.append(f"{label}: bytes [{lo}, {hi}) of a {b.numel()}-byte allocation")
    _guarded.clear()
    return bad


def segvec(arr: np.ndarray, lens, device=None, offset_elems: int = 0):
    """A SegmentedVector holding `arr` split into `lens`; each segment is its own
    guarded allocation.  offset_elems > 0 shifts every segment's start inside
    its allocation (to exercise unaligned pointers)."""
    from paper_2406_00158_gb300 import api
    device = device or torch.device("cuda:0")
    t = torch.from_numpy(np.ascontiguousarray(arr))
    segs, off = [], 0
    for k, n in enumerate(lens):
        s = guarded_segment(n, t.dtype, device, offset_elems, label=f"input segment {k}")
        s.copy_(t[off:off + n].to(device, non_blocking=False))
        segs.append(s)
        off += n
    v = api.SegmentedVector(segs)
    v._bases = segs
    return v


def empty_like_vec(lens, dtype, device=None):
    """An output vector of guarded segments (contents uninitialized)."""
    from paper_2406_00158_gb300 import api
    device = device or torch.device("cuda:0")
    segs = [guarded_segment(n, dtype, device, label=f"output segment {k}") for k, n in enumerate(lens)]
    v = api.SegmentedVector(segs)
    v._bases = segs
    return v


def md_empty(seg_rows, cols: int, device=None):
    """A row-block array (block k: (rows_k + 2) x cols fp32, zero-filled) with
    guard bands around every block and sentinels in the grid's two outer ghost
    rows (row 0 of the first block, the last row of the last block), which the
    stencil never reads or writes."""
    from paper_2406_00158_gb300 import api
    device = device or torch.device("cuda:0")
    blocks = []
    last = len(seg_rows) - 1
    for k, r in enumerate(seg_rows):
        n = (int(r) + 2) * cols
        flat = guarded_segment(n, torch.float32, device, label=f"row block {k}")
        flat.zero_()
        base = flat._guard_base
        lo = GUARD_BYTES
        if k == 0:                       # outer top ghost row
            _guard(base, [(lo, lo + cols * 4)], "outer top ghost row")
        if k == last:                    # outer bottom ghost row
            _guard(base, [(lo + (n - cols) * 4, lo + n * 4)], "outer bottom ghost row")
        b = flat.view(int(r) + 2, cols)
        b._guard_base = base
        blocks.append(b)
    m = api.MdArray(blocks)
    m._bases = blocks
    return m


def md_from(u: torch.Tensor, seg_rows):
    m = md_empty(seg_rows, u.shape[1], u.device)
    m.load(u)
    return m


def to_np(v) -> np.ndarray:
    return v.to_tensor().cpu().numpy()


def tile_index(lens, tile: int) -> np.ndarray:
    """Global tile index of every element under per-segment tiling."""
    out, t = [], 0
    for n in lens:
        k = np.arange(n) // tile + t
        out.append(k)
        t += -(-n // tile)
    return np.concatenate(out) if out else np.zeros(0, np.int64)
