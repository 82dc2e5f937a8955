"""GB300-native (sm_103a) hot path of the Distributed Ranges model (arXiv 2406.00158):
segmented vectors and row-block arrays over one GPU's HBM, lazy zip / transform
views fused into hand-written CUDA kernels (inclusive / exclusive / reverse scan
with decoupled lookback, transform_reduce, transform, for_each over k-ary zips
(STREAM, Black-Scholes), a halo-exchanging 5-point stencil, the dot-product
adjoint), autograd wrappers, and a batched persistent launch
with an autotuner -- all behind the C ABI in include/dr.h.

Submodules load lazily so that ``paper_2406_00158_gb300.inputs`` (the seeded
generator) imports without torch or the CUDA library.
"""
import importlib

_API = ("SegmentedVector", "View", "MdArray", "Batch", "inclusive_scan", "exclusive_scan", "scan_with_carry",
        "reverse_inclusive_scan", "transform_reduce", "scale_by_partner", "stencil5", "stencil5_part", "stencil5_T", "stencil5_T_wgrad",
        "sync_status", "set_spin_limit", "debug_skip_publish", "block_lengths", "dot_view", "stream_handle",
        "for_each", "transform", "FOR_EACH_FNS", "sort")


def __getattr__(name):
    if name in _API:
        return getattr(importlib.import_module(".api", __name__), name)
    if name in ("autograd", "api", "inputs", "build", "_lib"):
        return importlib.import_module("." + name, __name__)
    raise AttributeError(name)
