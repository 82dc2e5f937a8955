"""Helpers for the GPU parity tests: build / load the library once, move seeded
numpy inputs into segmented device containers and back."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


def dev():
    from paper_2406_00158_gb300 import build
    build.build()
    from paper_2406_00158_gb300 import _lib
    _lib.lib()
    return torch.device("cuda:0")


def sms() -> int:
    return torch.cuda.get_device_properties(0).multi_processor_count


def segvec(arr: np.ndarray, lens, device=None, offset_elems: int = 0):
    """A SegmentedVector holding `arr` split into `lens`; each segment is its own
    allocation.  offset_elems > 0 shifts every segment's start inside a larger
    allocation (to exercise unaligned pointers)."""
    from paper_2406_00158_gb300 import api
    device = device or torch.device("cuda:0")
    t = torch.from_numpy(np.ascontiguousarray(arr))
    segs, off = [], 0
    for n in lens:
        base = torch.empty(n + offset_elems, dtype=t.dtype, device=device)
        s = base[offset_elems:offset_elems + n]
        s.copy_(t[off:off + n].to(device, non_blocking=False))
        segs.append(s)
        off += n
    v = api.SegmentedVector(segs)
    v._bases = segs
    return v


def empty_like_vec(lens, dtype, device=None):
    from paper_2406_00158_gb300 import api
    return api.SegmentedVector.empty(lens, dtype, device or torch.device("cuda:0"))


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
