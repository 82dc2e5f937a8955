"""ctypes binding of the C ABI in ``include/dr.h`` (argument marshalling only).

Every function of the header is declared here under its C name.  ``call``
raises ``DRError`` (with ``dr_last_error()``) on a non-zero status.  Loading
fails loudly if the library has not been built: there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
# DR_GB300_LIB selects another build of this library (e.g. the range-checked one)
LIB_PATH = os.environ.get("DR_GB300_LIB") or os.path.join(_HERE, "libdr_gb300.so")

# enum dr_status
DR_OK, DR_E_INVAL, DR_E_DTYPE, DR_E_ALIGN, DR_E_CUDA, DR_E_TIMEOUT, DR_E_BOUNDS, DR_E_NOMEM, \
    DR_E_UNSUPPORTED = range(9)
STATUS_NAMES = {0: "DR_OK", 1: "DR_E_INVAL", 2: "DR_E_DTYPE", 3: "DR_E_ALIGN", 4: "DR_E_CUDA",
                5: "DR_E_TIMEOUT", 6: "DR_E_BOUNDS", 7: "DR_E_NOMEM", 8: "DR_E_UNSUPPORTED"}
# enum dr_dtype
DR_F32, DR_F64, DR_I64, DR_I32 = range(4)
# enum dr_binop
DR_PLUS, DR_MUL, DR_MIN, DR_MAX = range(4)
# enum dr_unop
DR_U_SCALE, DR_U_ADD, DR_U_NEG, DR_U_ABS, DR_U_SQUARE = range(5)
# enum dr_kernel_family
DR_K_SCAN, DR_K_REDUCE, DR_K_FOREACH, DR_K_SORT, DR_K_SCAN_VIEW = range(5)
DR_ZIP_STRICT_ALIGN = 1
# enum dr_rows_part
DR_ROWS_ALL, DR_ROWS_INNER, DR_ROWS_OUTER = range(3)


class dr_piece(ctypes.Structure):
    _fields_ = [("start", ctypes.c_int64), ("len", ctypes.c_int64),
                ("seg", ctypes.c_int32 * 2), ("off", ctypes.c_int64 * 2)]


class dr_tune(ctypes.Structure):
    _fields_ = [("threads", ctypes.c_int32), ("items", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32),
                ("variant", ctypes.c_int32)]


class DRError(RuntimeError):
    def __init__(self, name: str, status: int, msg: str):
        super().__init__(f"{name} -> {STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_P = ctypes.c_void_p
_PP = ctypes.POINTER(ctypes.c_void_p)
_I = ctypes.c_int
_I64 = ctypes.c_int64
_PI64 = ctypes.POINTER(ctypes.c_int64)
_PI = ctypes.POINTER(ctypes.c_int)
_D = ctypes.c_double

# name -> (restype, argtypes); opaque handles and streams are void*.
PROTOTYPES = {
    "dr_last_error": (ctypes.c_char_p, []),
    "dr_version": (_I, []),
    "dr_sync_status": (_I, [_P]),
    "dr_kernel_geometry": (_I, [_I, _I, _PI64, _PI]),
    "dr_set_spin_limit": (_I, [_I64]),
    "dr_debug_skip_publish": (_I, [_I64]),
    "dr_block_lengths": (_I, [_I64, _I, _PI64]),
    "dr_vec_create": (_I, [_I, _I, _PI64, _PP, _PP]),
    "dr_vec_destroy": (_I, [_P]),
    "dr_vec_rebind": (_I, [_P, _PP]),
    "dr_vec_info": (_I, [_P, _PI, _PI, _PI64]),
    "dr_vec_segment": (_I, [_P, _I, _PP, _PI64, _PI64]),
    "dr_vec_locate": (_I, [_P, _I64, _PI, _PI64]),
    "dr_vec_copy_from_host": (_I, [_P, _P, _P]),
    "dr_vec_copy_to_host": (_I, [_P, _P, _P]),
    "dr_md2_create": (_I, [_I, _I64, _I64, _I, _PI64, _PP, _PP]),
    "dr_md2_destroy": (_I, [_P]),
    "dr_md2_exchange_halos": (_I, [_P, _P]),
    "dr_view_of": (_I, [_P, _PP]),
    "dr_view_transform": (_I, [_P, _I, _D, _PP]),
    "dr_view_zip": (_I, [_P, _P, _PP]),
    "dr_view_zip_ex": (_I, [_P, _P, _I, _PP]),
    "dr_view_zip_transform": (_I, [_P, _I, _PP]),
    "dr_view_zipn": (_I, [_I, _PP, _PP]),
    "dr_view_take": (_I, [_P, _I64, _PP]),
    "dr_view_drop": (_I, [_P, _I64, _PP]),
    "dr_view_destroy": (_I, [_P]),
    "dr_view_info": (_I, [_P, _PI64, _PI, _PI, _PI]),
    "dr_view_segments": (_I, [_P, _I, ctypes.POINTER(dr_piece)]),
    "dr_inclusive_scan": (_I, [_P, _P, _I, _P]),
    "dr_exclusive_scan": (_I, [_P, _P, _I, _P, _P]),
    "dr_scan_with_carry": (_I, [_P, _P, _I, _I, _P, _P]),
    "dr_reverse_inclusive_scan": (_I, [_P, _P, _P]),
    "dr_transform_reduce": (_I, [_P, _I, _P, _P, _P]),
    "dr_scale_by_partner": (_I, [_P, _P, _P, _P, _P, _P]),
    "dr_for_each": (_I, [_P, _I, ctypes.POINTER(_D), _I, _P]),
    "dr_transform": (_I, [_P, _P, _P]),
    "dr_sort": (_I, [_P, _P, _P]),
    "dr_dot_f32_noalloc": (_I, [_I, _PI64, _PP, _PP, ctypes.c_float, _P, _P]),
    "dr_stencil5": (_I, [_P, _P, _P, _I, _D, _D, _P]),
    "dr_stencil5_part": (_I, [_P, _P, _I, _D, _D, _P]),
    "dr_md2_set_external_halos": (_I, [_P, _I, _I]),
    "dr_stencil5_T": (_I, [_P, _P, _P, _I, _D, _D, _P]),
    "dr_stencil5_T_wgrad": (_I, [_P, _P, _P, _D, _D, _P, _P]),
    "dr_batch_plan": (_I, [_I, _PP, _PP, _PP, _P, ctypes.POINTER(dr_tune), _PP]),
    "dr_batch_destroy": (_I, [_P]),
    "dr_batch_set_tune": (_I, [_P, ctypes.POINTER(dr_tune)]),
    "dr_batch_get_tune": (_I, [_P, ctypes.POINTER(dr_tune)]),
    "dr_batch_run": (_I, [_P, _P]),
    "dr_batch_run_graph": (_I, [_P, _P]),
    "dr_batch_run_per_range": (_I, [_P, _P]),
    "dr_batch_run_per_range_graph": (_I, [_P, _P]),
    "dr_batch_autotune": (_I, [_P, _I, ctypes.c_char_p, ctypes.POINTER(dr_tune)]),
}

_lock = threading.Lock()
_lib = None


def lib():
    """The loaded library.  Raises if it was never built."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(
                    f"CUDA library {LIB_PATH} is missing: build it first "
                    "(python -m paper_2406_00158_gb300.build); there is no CPU fallback")
            l = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in PROTOTYPES.items():
                f = getattr(l, name)
                f.restype = res
                f.argtypes = args
            _lib = l
    return _lib


def last_error() -> str:
    return (lib().dr_last_error() or b"").decode()


def kernel_geometry(kernel: int, dtype: int) -> tuple[int, int]:
    """(tile elements, fixed CTAs per SM or 0) of a kernel family for a dtype."""
    t, c = ctypes.c_int64(), ctypes.c_int()
    call("dr_kernel_geometry", int(kernel), int(dtype), ctypes.byref(t), ctypes.byref(c))
    return t.value, c.value


def call(name: str, *args) -> None:
    rc = getattr(lib(), name)(*args)
    if rc != DR_OK:
        raise DRError(name, rc, last_error())
