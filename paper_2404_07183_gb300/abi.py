"""ctypes view of the C ABI in ``include/pcf.h`` (argument marshalling only).

Loading is lazy; there is no fallback: if the CUDA library has not been built
(``paper_2404_07183_gb300.build``) every call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

PCF_OK, PCF_EINVAL, PCF_ENOWS, PCF_ECUDA, PCF_ETIMEOUT, PCF_EUNSUPPORTED = range(6)
PCF_F32, PCF_F64 = 0, 1
PCF_L1, PCF_L2, PCF_LP, PCF_GRAM = 0, 1, 2, 3
PCF_PREC_F64, PCF_PREC_F32_COMP, PCF_PREC_F32, PCF_PREC_F32_BLOCK = 0, 1, 2, 3
PCF_PREC_ROUND_TIMES = 0x100
PCF_PREC_AUTO64 = 0x200
PCF_OUT_FULL, PCF_OUT_UPPER_PACKED, PCF_OUT_FULL_SORTED = 0, 1, 2
PCF_WS_FORWARD, PCF_WS_BACKWARD = 0, 1
PCF_CROSS_REUSE_B = 1
PCF_PAIRWISE_PREPARED = 1
PCF_MAX_INTEGRALS = 4

ERR_DETAIL = {
    1: "offsets not increasing / out of range",
    2: "first breakpoint time is not 0",
    3: "breakpoint times not strictly increasing",
    4: "breakpoint time not finite",
    5: "value not finite",
    6: "time or value outside float32 range for a float32 walk",
    7: "more coincident float32 breakpoints than one window holds",
    8: "result or intermediate larger than the output capacity or the workspace",
    9: "a bounded device wait gave up",
    10: "weight PCF invalid (negative or non-finite value, t_0 != 0, times not increasing)",
}

SYMBOLS = ("pcf_workspace_size", "pcf_prepare", "pcf_pairwise", "pcf_cross", "pcf_pairwise_backward",
           "pcf_check", "pcf_status_string", "pcf_version", "pcf_pairwise_noalloc",
           "pcf_walk_promoted", "pcf_weighted_workspace_size", "pcf_pairwise_weighted",
           "pcf_cross_weighted_workspace_size", "pcf_cross_weighted",
           "pcf_pairwise_ex", "pcf_cross_ex", "pcf_sort_order", "pcf_segment_integrals",
           "pcf_reduce_workspace_size", "pcf_reduce", "pcf_combine_workspace_size",
           "pcf_combine", "pcf_reduce_counters", "pcf_selftest_wait_timeout",
           "pcf_pairwise_backward_ex", "pcf_pairwise_to_host")
PCF_RED_SUM, PCF_RED_MEAN, PCF_RED_MAX, PCF_RED_MIN, PCF_RED_STD = range(5)
PCF_OP_ADD, PCF_OP_SUB, PCF_OP_MUL, PCF_OP_MAX, PCF_OP_MIN, PCF_OP_SQDIFF = range(6)
PCF_FN_INTEGRAL, PCF_FN_LP = 0, 1
PCF_SCHED_AUTO, PCF_SCHED_TILE_1024, PCF_SCHED_TILE_512X2, PCF_SCHED_MERGEPATH = 0, 1, 2, 3
PCF_SCHED_TILE_512X3 = 4
PCF_NOALLOC_SCRATCH_BYTES = 16 << 20


class PcfCsr(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("nnz", ctypes.c_int64),
                ("offsets", ctypes.c_void_p), ("times", ctypes.c_void_p),
                ("values", ctypes.c_void_p), ("dtype", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class PcfSchedule(ctypes.Structure):
    _fields_ = [("kernel", ctypes.c_int32), ("window", ctypes.c_int32),
                ("shard_index", ctypes.c_int32), ("shard_count", ctypes.c_int32),
                ("reserved", ctypes.c_int32 * 4)]


class PcfWindow(ctypes.Structure):
    _fields_ = [("a", ctypes.c_double), ("b", ctypes.c_double), ("lam", ctypes.c_double),
                ("reserved", ctypes.c_int32 * 4)]


class PcfCsrOut(ctypes.Structure):
    _fields_ = [("capacity", ctypes.c_int64), ("offsets", ctypes.c_void_p),
                ("times", ctypes.c_void_p), ("values", ctypes.c_void_p)]


class PcfIntegral(ctypes.Structure):
    _fields_ = [("metric", ctypes.c_int32), ("apply_root", ctypes.c_int32),
                ("p", ctypes.c_double), ("out", ctypes.c_void_p)]


_lib = None
_lock = threading.Lock()


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False):
    """Load (and optionally build) the CUDA library; raises if unavailable."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if not os.path.exists(path):
            if not build_if_missing:
                raise RuntimeError(
                    f"CUDA library {path} is not built; run "
                    "`python -m paper_2404_07183_gb300.build` (no CPU fallback exists)")
            _build.build()
        lib = ctypes.CDLL(path)
        P, I, I64, D, SZ = (ctypes.c_void_p, ctypes.c_int, ctypes.c_int64,
                            ctypes.c_double, ctypes.c_size_t)
        CSR = ctypes.POINTER(PcfCsr)
        INT = ctypes.POINTER(PcfIntegral)
        lib.pcf_workspace_size.restype = I
        lib.pcf_workspace_size.argtypes = [CSR, CSR, I, I, ctypes.POINTER(SZ)]
        lib.pcf_pairwise.restype = I
        lib.pcf_pairwise.argtypes = [CSR, INT, I, I, I, I, I, P, SZ, P]
        SCH = ctypes.POINTER(PcfSchedule)
        lib.pcf_pairwise_ex.restype = I
        WIN = ctypes.POINTER(PcfWindow)
        lib.pcf_pairwise_ex.argtypes = [CSR, INT, I, I, I, I, I, SCH, WIN, P, SZ, P]
        lib.pcf_pairwise_to_host.restype = I
        lib.pcf_pairwise_to_host.argtypes = [CSR, INT, I, I, I, SCH, P, I, P, SZ, P, P]
        lib.pcf_cross_ex.restype = I
        lib.pcf_cross_ex.argtypes = [CSR, CSR, I64, I64, INT, I, I, I64, I, I, SCH, WIN, P, SZ, P]
        lib.pcf_segment_integrals.restype = I
        lib.pcf_segment_integrals.argtypes = [CSR, I, D, I, D, D, I, P, I, P, SZ, P]
        lib.pcf_sort_order.restype = I
        lib.pcf_sort_order.argtypes = [CSR, I, P, SZ, P, P]
        lib.pcf_prepare.restype = I
        lib.pcf_prepare.argtypes = [CSR, I, P, SZ, P]
        lib.pcf_cross.restype = I
        lib.pcf_cross.argtypes = [CSR, CSR, I64, I64, INT, I, I, I64, I, I, P, SZ, P]
        lib.pcf_pairwise_backward.restype = I
        lib.pcf_pairwise_backward.argtypes = [CSR, I, D, I, P, P, I, P, P, P, SZ, P]
        lib.pcf_pairwise_backward_ex.restype = I
        lib.pcf_pairwise_backward_ex.argtypes = [CSR, I, D, I, P, P, I, P, P, SCH, P, SZ, P]
        lib.pcf_check.restype = I
        lib.pcf_check.argtypes = [P, P, ctypes.POINTER(I), ctypes.POINTER(I64)]
        lib.pcf_walk_promoted.restype = I
        lib.pcf_walk_promoted.argtypes = [P, P, ctypes.POINTER(I)]
        lib.pcf_weighted_workspace_size.restype = I
        lib.pcf_weighted_workspace_size.argtypes = [CSR, CSR, I, ctypes.POINTER(SZ)]
        lib.pcf_pairwise_weighted.restype = I
        lib.pcf_pairwise_weighted.argtypes = [CSR, CSR, INT, I, I, I, I, P, P, SZ, P]
        lib.pcf_cross_weighted_workspace_size.restype = I
        lib.pcf_cross_weighted_workspace_size.argtypes = [CSR, CSR, CSR, I, ctypes.POINTER(SZ)]
        lib.pcf_cross_weighted.restype = I
        lib.pcf_cross_weighted.argtypes = [CSR, CSR, I64, I64, CSR, INT, I, I, I64, I, P, P, SZ, P]
        lib.pcf_status_string.restype = ctypes.c_char_p
        lib.pcf_status_string.argtypes = [I]
        lib.pcf_pairwise_noalloc.restype = I
        lib.pcf_pairwise_noalloc.argtypes = [CSR, INT, I, I, I, I, P]
        OUT = ctypes.POINTER(PcfCsrOut)
        lib.pcf_reduce_workspace_size.restype = I
        lib.pcf_reduce_workspace_size.argtypes = [CSR, I64, I, I64, ctypes.POINTER(SZ)]
        lib.pcf_reduce.restype = I
        lib.pcf_reduce.argtypes = [CSR, I64, I, OUT, P, SZ, P]
        lib.pcf_combine_workspace_size.restype = I
        lib.pcf_combine_workspace_size.argtypes = [CSR, CSR, ctypes.POINTER(SZ)]
        lib.pcf_combine.restype = I
        lib.pcf_combine.argtypes = [CSR, CSR, I, OUT, P, SZ, P]
        lib.pcf_reduce_counters.restype = I
        lib.pcf_reduce_counters.argtypes = [P, P, ctypes.POINTER(I64), ctypes.POINTER(I64)]
        lib.pcf_selftest_wait_timeout.restype = I
        lib.pcf_selftest_wait_timeout.argtypes = [I64, P, SZ, P]
        lib.pcf_version.restype = ctypes.c_char_p
        lib.pcf_version.argtypes = []
        _lib = lib
        return lib


def status_string(code: int) -> str:
    return load().pcf_status_string(int(code)).decode()
