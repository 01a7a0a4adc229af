"""ctypes declarations of the C ABI in include/spd.h (argument marshalling only).

The shared library is built in-tree by ``paper_2207_13901_gb300.build`` into
``paper_2207_13901_gb300/_build/libspd.so``. There is no fallback: if the library
cannot be built or loaded, every call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

SPD_OK = 0
SPD_ERR_SHAPE = 2
SPD_ERR_TIMEOUT = 9
SPD_MAX_INDEX = 2**31 - 2**17 - 1  # largest dimension, entry or fiber count of a descriptor
SPD_F64, SPD_F32, SPD_BF16 = 0, 1, 2
SPD_SPLIT_ROW, SPD_SPLIT_NNZ, SPD_SPLIT_AUTO = 0, 1, 2
SPD_OP_SPMV, SPD_OP_SPMM, SPD_OP_SPMM_T, SPD_OP_SDDMM, SPD_OP_SPTTV, SPD_OP_SPMTTKRP = range(6)

STATUS_NAMES = {
    0: "SPD_OK", 1: "SPD_ERR_NULL", 2: "SPD_ERR_SHAPE", 3: "SPD_ERR_DTYPE", 4: "SPD_ERR_ALIGN",
    5: "SPD_ERR_STRUCTURE", 6: "SPD_ERR_WORKSPACE", 7: "SPD_ERR_CUDA", 8: "SPD_ERR_OOM",
    9: "SPD_ERR_TIMEOUT", 10: "SPD_ERR_ARG",
}


class spd_csr(ctypes.Structure):
    _fields_ = [
        ("nrows", ctypes.c_int64), ("ncols", ctypes.c_int64), ("nnz", ctypes.c_int64),
        ("pos", ctypes.c_void_p), ("crd", ctypes.c_void_p), ("vals", ctypes.c_void_p),
        ("vtype", ctypes.c_int32), ("reserved", ctypes.c_int32),
    ]


class spd_csf3(ctypes.Structure):
    _fields_ = [
        ("dim0", ctypes.c_int64), ("dim1", ctypes.c_int64), ("dim2", ctypes.c_int64),
        ("nfib", ctypes.c_int64), ("nnz", ctypes.c_int64),
        ("pos1", ctypes.c_void_p), ("crd1", ctypes.c_void_p), ("pos2", ctypes.c_void_p),
        ("crd2", ctypes.c_void_p), ("vals", ctypes.c_void_p),
        ("vtype", ctypes.c_int32), ("reserved", ctypes.c_int32),
    ]


class spd_tune(ctypes.Structure):
    _fields_ = [
        ("unit_items", ctypes.c_int32), ("row_pieces", ctypes.c_int32),
        ("block_threads", ctypes.c_int32), ("inflight", ctypes.c_int32), ("lane_groups", ctypes.c_int32),
        ("form", ctypes.c_int32),
    ]


class spd_batch_item(ctypes.Structure):
    _fields_ = [
        ("A", spd_csr), ("X", ctypes.c_void_p), ("ldx", ctypes.c_int64), ("Y", ctypes.c_void_p),
        ("ldy", ctypes.c_int64), ("split", ctypes.c_int32), ("unit_items", ctypes.c_int32),
    ]


class spd_batch_plan(ctypes.Structure):
    _fields_ = [
        ("count", ctypes.c_int64), ("total_pieces", ctypes.c_int64), ("L", ctypes.c_int64),
        ("vtype", ctypes.c_int32), ("epl", ctypes.c_int32), ("group", ctypes.c_int32),
        ("block_threads", ctypes.c_int32),
        ("grid", ctypes.c_int32), ("fulltile", ctypes.c_int32), ("has_nnz", ctypes.c_int32),
        ("ws", ctypes.c_void_p),
        ("off_desc", ctypes.c_size_t), ("off_pstart", ctypes.c_size_t), ("off_prow", ctypes.c_size_t),
        ("off_ppos", ctypes.c_size_t), ("off_crow", ctypes.c_size_t), ("off_cval", ctypes.c_size_t),
        ("off_pmat", ctypes.c_size_t),
    ]


_P = ctypes.c_void_p
_I = ctypes.c_int
_I64 = ctypes.c_int64
_SZ = ctypes.c_size_t
_CSR = ctypes.POINTER(spd_csr)
_CSF = ctypes.POINTER(spd_csf3)
_TUNE = ctypes.POINTER(spd_tune)

# name -> (restype, argtypes); kept in the order of include/spd.h
SIGNATURES = {
    "spd_abi_version": (ctypes.c_int, []),
    "spd_status_str": (ctypes.c_char_p, [_I]),
    "spd_last_error": (ctypes.c_char_p, []),
    "spd_set_checked": (_I, [_I]),
    "spd_checked": (ctypes.c_int, []),
    "spd_fault_status": (_I, [ctypes.POINTER(ctypes.c_uint32), _P]),
    "spd_probe_bounded_wait": (_I, [_P]),
    "spd_csr_workspace_size": (_I, [_I, _CSR, _I, _I64, _TUNE, ctypes.POINTER(ctypes.c_size_t)]),
    "spd_csf3_workspace_size": (_I, [_I, _CSF, _I, _I64, _TUNE, ctypes.POINTER(ctypes.c_size_t)]),
    "spd_csr_validate": (_I, [_CSR, _P, _SZ, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64), _P]),
    "spd_csf3_validate": (_I, [_CSF, _P, _SZ, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64), _P]),
    "spd_csr_partition": (_I, [_CSR, _I, _I64, _I64, _P, _P, _P]),
    "spd_spmv": (_I, [_CSR, _P, _I, _P, _I, _I, _TUNE, _P, _SZ, _P]),
    "spd_spmm": (_I, [_CSR, _P, _I64, _I64, _I, _P, _I64, _I, _I, _TUNE, _P, _SZ, _P]),
    "spd_spmm_accumulate": (_I, [_CSR, _P, _I64, _I64, _I, _P, _I64, _I, _I, _TUNE, _P, _SZ, _P]),
    "spd_spmm_t": (_I, [_CSR, _P, _I64, _I64, _I, _P, _I64, _I, _I, _TUNE, _P, _SZ, _P]),
    "spd_csr_transpose_workspace_size": (_I, [_CSR, ctypes.POINTER(ctypes.c_size_t)]),
    "spd_csr_transpose": (_I, [_CSR, _P, _P, _P, _P, _SZ, _P]),
    "spd_gather_vals": (_I, [_I64, _P, _P, _P, _I, _P]),
    "spd_csr_column_blocks_workspace_size": (_I, [_CSR, _I64, ctypes.POINTER(ctypes.c_size_t)]),
    "spd_csr_column_blocks": (_I, [_CSR, _I64, _P, _P, _P, _P, _P, _P, _SZ, _P]),
    "spd_spadd3_workspace_size": (_I, [_CSR, _CSR, _CSR, _I, _TUNE, ctypes.POINTER(ctypes.c_size_t)]),
    "spd_spadd3_symbolic": (_I, [_CSR, _CSR, _CSR, _I, _TUNE, _P, ctypes.POINTER(ctypes.c_int64), _P, _SZ, _P]),
    "spd_spadd3_numeric": (_I, [_CSR, _CSR, _CSR, _I, _TUNE, _P, _I64, _P, _P, _I, _P, _SZ, _P]),
    "spd_sddmm": (_I, [_CSR, _P, _I64, _I64, _P, _I64, _I, _P, _I, _I, _TUNE, _P, _SZ, _P]),
    "spd_spttv": (_I, [_CSF, _P, _I, _P, _I, _I, _TUNE, _P, _SZ, _P]),
    "spd_spmttkrp": (_I, [_CSF, _P, _I64, _P, _I64, _I64, _I, _P, _I64, _I, _I, _TUNE, _P, _SZ, _P]),
    "spd_spmm_batched_workspace_size": (_I, [_I64, ctypes.POINTER(spd_batch_item), _I64, _I, _TUNE,
                                             ctypes.POINTER(ctypes.c_size_t)]),
    "spd_spmm_batched_plan": (_I, [_I64, ctypes.POINTER(spd_batch_item), _I64, _I, _TUNE, _P, _SZ,
                                   ctypes.POINTER(spd_batch_plan), _P]),
    "spd_spmm_batched_run": (_I, [ctypes.POINTER(spd_batch_plan), _P]),
    "spd_spmv_noalloc": (_I, [_CSR, _P, _I, _P, _I, _P]),
}

_lock = threading.Lock()
_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_needed: bool = True):
    """Load libspd.so (building it first when it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if build_if_needed and not _build.up_to_date():
            _build.build()
        path = _build.LIB
        if not os.path.exists(path):
            raise RuntimeError("libspd.so is not built (%s); run paper_2207_13901_gb300.build" % path)
        lib = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        if lib.spd_abi_version() != 2:
            raise RuntimeError("libspd ABI version mismatch")
        _lib = lib
        return lib


class SpdError(RuntimeError):
    def __init__(self, call: str, status: int, detail: str):
        self.status = status
        super().__init__("%s failed: %s (%s)%s" % (call, STATUS_NAMES.get(status, status),
                                                    load().spd_status_str(status).decode(),
                                                    (": " + detail) if detail else ""))


def check(call: str, status: int) -> None:
    if status != SPD_OK:
        raise SpdError(call, status, load().spd_last_error().decode())
