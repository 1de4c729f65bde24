"""ctypes mirror of include/fv.h and the loader for libfv.so.

Argument marshalling only: every step of decoding runs inside libfv's CUDA
kernels.  Importing this module never falls back to anything else: if the
library is missing it raises.
"""
from __future__ import annotations

import ctypes
import os
import re

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libfv.so")
HEADER = os.path.join(os.path.dirname(PKG), "include", "fv.h")

FV_OK, FV_EINVAL, FV_ENOMEM, FV_ECUDA, FV_ETIMEOUT, FV_EUNSUPPORTED, FV_EINFEASIBLE = range(7)
STATUS_NAMES = {0: "FV_OK", 1: "FV_EINVAL", 2: "FV_ENOMEM", 3: "FV_ECUDA", 4: "FV_ETIMEOUT",
                5: "FV_EUNSUPPORTED", 6: "FV_EINFEASIBLE"}
FV_VANILLA, FV_FLASH, FV_BEAM, FV_CHECKPOINT = 0, 1, 2, 3
FV_TRANS_DENSE, FV_TRANS_CSR = 0, 1
FV_EMIT_DENSE, FV_EMIT_DISCRETE = 0, 1
FV_COMPLETE_PRUNING = 0x1
FV_NO_SORT = 0x2
FV_CHECKED = 0x4
FV_NO_TUNE = 0x8
FV_STATIC_BEAM = 0x10
FV_SHARED_GPU = 0x20
FV_TEST_WITHHOLD_STEP = 0x80000000

P = ctypes.c_void_p


class fv_model(ctypes.Structure):
    _fields_ = [
        ("K", ctypes.c_int32),
        ("log_pi", P),
        ("trans", ctypes.c_int32),
        ("logA", P),
        ("row_ptr", P),
        ("col", P),
        ("val", P),
        ("nnz", ctypes.c_int64),
        ("emit", ctypes.c_int32),
        ("V", ctypes.c_int32),
        ("logB", P),
    ]


class fv_batch(ctypes.Structure):
    _fields_ = [
        ("n_seq", ctypes.c_int32),
        ("T_host", P),
        ("model_host", P),
        ("T", P),
        ("model_idx", P),
        ("e_off", P),
        ("E", P),
        ("obs", P),
        ("path_off", P),
    ]


class fv_params(ctypes.Structure):
    _fields_ = [
        ("mode", ctypes.c_int32),
        ("P", ctypes.c_int32),
        ("B", ctypes.c_int32),
        ("mem_budget_bytes", ctypes.c_uint64),
        ("flags", ctypes.c_uint32),
    ]


class FVError(RuntimeError):
    def __init__(self, status, where=""):
        self.status = int(status)
        super().__init__(f"{where}: {STATUS_NAMES.get(self.status, self.status)}")


def declared_functions():
    """Names of the functions include/fv.h declares (for export checks)."""
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fv_[a-z_]+)\s*\(", src)))


_lib = None


def load(build_if_missing: bool = False):
    """Load libfv.so.  Raises if it is missing (no fallback of any kind)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        if build_if_missing:
            from . import build as _b
            _b.build()
        else:
            raise ImportError(f"libfv.so not built ({LIB_PATH}); run __graft_entry__.build()")
    lib = ctypes.CDLL(LIB_PATH)
    sz = ctypes.c_size_t
    i32 = ctypes.c_int32
    MP, BP, PP = ctypes.POINTER(fv_model), ctypes.POINTER(fv_batch), ctypes.POINTER(fv_params)
    lib.fv_workspace_size.argtypes = [MP, i32, BP, PP]
    lib.fv_workspace_size.restype = sz
    lib.fv_decode.argtypes = [MP, i32, BP, PP, P, sz, P, P, P]
    lib.fv_decode.restype = ctypes.c_int
    lib.fv_backward.argtypes = [MP, i32, BP, P, P, P, P, P, P, sz, P]
    lib.fv_backward.restype = ctypes.c_int
    lib.fv_backward_workspace_size.argtypes = [MP, i32, BP]
    lib.fv_backward_workspace_size.restype = sz
    lib.fv_last_device_status.argtypes = [P, P]
    lib.fv_last_device_status.restype = ctypes.c_int
    lib.fv_status_str.argtypes = [ctypes.c_int]
    lib.fv_status_str.restype = ctypes.c_char_p
    lib.fv_path_score.argtypes = [MP, i32, BP, P, P, P]
    lib.fv_path_score.restype = ctypes.c_int
    lib.fv_timing_enable.argtypes = [i32]
    lib.fv_timing_enable.restype = ctypes.c_int
    lib.fv_timing_reset.argtypes = []
    lib.fv_timing_reset.restype = ctypes.c_int
    lib.fv_timing_pairs.argtypes = [P, i32, P]
    lib.fv_timing_pairs.restype = ctypes.c_int
    lib.fv_timing_read.argtypes = [P, P]
    lib.fv_timing_read.restype = ctypes.c_int
    lib.fv_decode_noalloc.argtypes = [MP, i32, BP, P, P, P]
    lib.fv_decode_noalloc.restype = ctypes.c_int
    lib.fv_decode_noalloc_status.argtypes = [P]
    lib.fv_decode_noalloc_status.restype = ctypes.c_int
    lib.fv_autotune.argtypes = [MP, i32, BP, PP, P, sz, P, P, P, P]
    lib.fv_autotune.restype = ctypes.c_int
    lib.fv_set_engine_variant.argtypes = [i32, i32]
    lib.fv_set_engine_variant.restype = i32
    lib.fv_maxplus_peak.argtypes = [i32, P, P, P, P]
    lib.fv_maxplus_peak.restype = ctypes.c_int
    lib.fv_version.argtypes = []
    lib.fv_version.restype = ctypes.c_char_p
    _lib = lib
    return lib
