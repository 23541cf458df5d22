"""ctypes binding of libspmv_gb300.so: the C ABI of include/spmv_gb300.h, same names.

Argument marshalling only; every step of the products runs in the CUDA library.
The library is built in-tree by ``paper_1812_00904_gb300.build``; if it is
missing, loading raises instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libspmv_gb300.so")

# enums of the header
SPMV_OK, SPMV_ERR_INVALID_ARG, SPMV_ERR_BAD_MATRIX, SPMV_ERR_OOM, SPMV_ERR_CUDA = 0, 1, 2, 3, 4
SPMV_ERR_DEVICE, SPMV_ERR_TIMEOUT, SPMV_ERR_BUSY, SPMV_ERR_UNSUPPORTED, SPMV_ERR_NOT_FOUND = 5, 6, 7, 8, 9
STATUS_NAMES = {0: "SPMV_OK", 1: "SPMV_ERR_INVALID_ARG", 2: "SPMV_ERR_BAD_MATRIX", 3: "SPMV_ERR_OOM",
                4: "SPMV_ERR_CUDA", 5: "SPMV_ERR_DEVICE", 6: "SPMV_ERR_TIMEOUT", 7: "SPMV_ERR_BUSY",
                8: "SPMV_ERR_UNSUPPORTED", 9: "SPMV_ERR_NOT_FOUND"}
SPMV_CSC_WIDE, SPMV_CSR_TALL = 0, 1
SPMV_F64, SPMV_F32, SPMV_BF16, SPMV_F16 = 0, 1, 2, 3
SPMV_OP_AX, SPMV_OP_VTA = 0, 1
SPMV_PLAN_NO_VALIDATE, SPMV_PLAN_PROFILE, SPMV_PLAN_SHORT_IN_GLOBAL, SPMV_PLAN_BANK_ORDER = 0x1, 0x2, 0x4, 0x8
SPMV_PLAN_COO_UNSORTED = 0x10
SPMV_PLAN_ROW_BLOCKS = 0x20

KERNEL_SCATTER, KERNEL_COMBINE, KERNEL_SEGDOT, KERNEL_FIXUP, KERNEL_DVALUES = 0, 1, 2, 3, 4
KERNEL_ROWBLOCK_DOT, KERNEL_ROWBLOCK_FIXUP = 5, 6


class SpmvError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        self.status = status
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {msg}")


class spmv_plan_opts(ctypes.Structure):
    _fields_ = [("chunks", ctypes.c_int32), ("warps_per_cta", ctypes.c_int32), ("tile_items", ctypes.c_int32),
                ("stages", ctypes.c_int32), ("chunk_tiles", ctypes.c_int32)]


class spmv_plan_info_t(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int64), ("n", ctypes.c_int64), ("nnz", ctypes.c_int64),
                ("layout", ctypes.c_int32), ("val_dtype", ctypes.c_int32), ("vec_dtype", ctypes.c_int32),
                ("chunks", ctypes.c_int32), ("ctas", ctypes.c_int32), ("warps_per_cta", ctypes.c_int32),
                ("tile_items", ctypes.c_int32), ("stages", ctypes.c_int32), ("tiles", ctypes.c_int32),
                ("zones", ctypes.c_int32), ("max_zone_size", ctypes.c_int32), ("short_on_chip", ctypes.c_int32),
                ("batch_width", ctypes.c_int32), ("max_chunk_nnz", ctypes.c_int64), ("min_chunk_nnz", ctypes.c_int64),
                ("imbalance", ctypes.c_double), ("workspace_bytes", ctypes.c_int64), ("setup_ms", ctypes.c_double),
                ("row_blocks", ctypes.c_int32), ("row_block_window", ctypes.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class spmv_chunk_t(ctypes.Structure):
    _fields_ = [("nz_begin", ctypes.c_int64), ("nz_end", ctypes.c_int64), ("jf", ctypes.c_int32), ("jl", ctypes.c_int32),
                ("needLeft", ctypes.c_int32), ("needRight", ctypes.c_int32), ("leftGroupEnd", ctypes.c_int32),
                ("rightGroup", ctypes.c_int32), ("leftGroup", ctypes.c_int32), ("procsOnLeft", ctypes.c_int32),
                ("procsOnRight", ctypes.c_int32)]


class serve_stats_t(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64), ("failed", ctypes.c_int64),
                ("vectors", ctypes.c_int64), ("launches", ctypes.c_int64), ("admissions", ctypes.c_int64),
                ("evictions", ctypes.c_int64), ("resident_matrices", ctypes.c_int64),
                ("resident_bytes", ctypes.c_uint64), ("max_inflight_launches", ctypes.c_int32),
                ("tracked_requests", ctypes.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_P = ctypes.c_void_p
_I32, _I64, _U32, _U64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32, ctypes.c_uint64

# name -> (restype, argtypes); every function of include/spmv_gb300.h
SIGNATURES = {
    "spmv_plan": (_I32, [ctypes.POINTER(_P), _I64, _I64, _I64, _I32, _P, _P, _P, _I32, _I32, _P, _U32]),
    "spmv_plan_ex": (_I32, [ctypes.POINTER(_P), _I64, _I64, _I64, _I32, _P, _P, _P, _I32, _I32, _P, _U32,
                            ctypes.POINTER(spmv_plan_opts)]),
    "spmv_plan_coo": (_I32, [ctypes.POINTER(_P), _I64, _I64, _I64, _I32, _P, _P, _P, _I32, _I32, _P, _U32,
                             ctypes.POINTER(spmv_plan_opts)]),
    "spmv_plan_destroy": (_I32, [_P]),
    "spmv_plan_info": (_I32, [_P, ctypes.POINTER(spmv_plan_info_t)]),
    "spmv_plan_chunks": (_I32, [_P, ctypes.POINTER(spmv_chunk_t), _I32]),
    "spmv": (_I32, [_P, _P, _P, _P]),
    "spvtm": (_I32, [_P, _P, _P, _P]),
    "spmv_pair": (_I32, [_P, _P, _P, _P, _P, _P]),
    "spmv_batch": (_I32, [_P, _I32, _I32, _P, _I64, _P, _I64, _P]),
    "spmv_dvalues": (_I32, [_P, _P, _P, _P, _P]),
    "spmv_check": (_I32, [_P, _P]),
    "spmv_plan_export": (_I32, [_P, _P, _P, _P]),
    "spmv_profile_enable": (_I32, [_P, _I32]),
    "spmv_profile_read": (_I32, [_P, _I32, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(_I64)]),
    "spmv_profile_reset": (_I32, [_P]),
    "spmv_noalloc": (_I32, [_I64, _I64, _I64, _P, _P, _P, _P, _P, _P]),
    "spmv_normal": (_I32, [_P, _P, _P, _P, _P]),
    "spmv_cgls": (_I32, [_P, _P, _P, _I32, ctypes.c_double, _P, ctypes.POINTER(_I32), ctypes.POINTER(ctypes.c_double)]),
    "spmv_last_error": (ctypes.c_char_p, []),
    "spmv_version": (ctypes.c_char_p, []),
    "serve_create": (_I32, [ctypes.POINTER(_P), _U64, _I32, _I32]),
    "serve_register": (_I32, [_P, _P, ctypes.POINTER(_I32)]),
    "serve_register_host": (_I32, [_P, _I64, _I64, _I64, _I32, _P, _P, _P, _I32, _I32, ctypes.POINTER(_I32)]),
    "serve_submit": (_I32, [_P, _I32, _I32, _I32, _P, _P, ctypes.POINTER(_U64)]),
    "serve_poll": (_I32, [_P, _U64, ctypes.POINTER(_I32), ctypes.POINTER(ctypes.c_double)]),
    "serve_wait": (_I32, [_P, _U64, _I32]),
    "serve_stats": (_I32, [_P, ctypes.POINTER(serve_stats_t)]),
    "serve_destroy": (_I32, [_P]),
}

_lock = threading.Lock()
_lib = None


def load(path: str = LIB_PATH):
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(path):
                raise RuntimeError(f"{path} is missing: build it with `python -m paper_1812_00904_gb300.build` "
                                   "(there is no fallback implementation)")
            lib = ctypes.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                f = getattr(lib, name)
                f.restype = res
                f.argtypes = args
            _lib = lib
        return _lib


def check(status: int, where: str):
    if status != SPMV_OK:
        raise SpmvError(status, where, load().spmv_last_error().decode())
    return status


def call(name: str, *args):
    """Call a C ABI function by name and raise SpmvError on a failing status."""
    return check(getattr(load(), name)(*args), name)
