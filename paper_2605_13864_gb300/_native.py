"""ctypes view of ``liboptigpu.so`` (declared in ``include/optigpu.h``).

Argument marshalling only: every step of the transpose and the sum runs in
the library's CUDA kernels.  The library is loaded from the in-tree build
directory; if it is missing it is built with nvcc, and if that is impossible
the import of any operation raises -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import build_lib

_lock = threading.Lock()
_lib = None

# optigpu_status
OK = 0
ERR_INVALID_ARG = 1
ERR_UNSUPPORTED_DTYPE = 2
ERR_OVERLAP = 3
ERR_CUDA = 4
ERR_OOM = 5
ERR_TIMEOUT = 6
ERR_BUSY = 7
ERR_NOT_FOUND = 8

# optigpu_dtype
INT32, FLOAT32, BFLOAT16, FLOAT16 = 0, 1, 2, 3

# optigpu_transpose_kernel
TRANSPOSE_AUTO, TRANSPOSE_TILE32, TRANSPOSE_TMA = 0, 1, 2

OP_TRANSPOSE, OP_REDUCE = 0, 1

REDUCE_PLAIN = 0
REDUCE_COMPENSATED = 1
REDUCE_CHUNK = 16384

# Every symbol include/optigpu.h declares, with (restype, argtypes).
_i64, _u32, _u64, _vp, _ci = ctypes.c_int64, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_void_p, ctypes.c_int
SIGNATURES = {
    "optigpu_transpose": (_ci, [_vp, _vp, _i64, _i64, _ci, _vp]),
    "optigpu_transpose_ex": (_ci, [_vp, _vp, _i64, _i64, _ci, _ci, _vp]),
    "optigpu_transpose_tma_eligible": (_ci, [_vp, _vp, _i64, _i64, _ci]),
    "optigpu_transpose_config_for": (_ci, [_i64, _i64, _ci]),
    "optigpu_transpose_strided": (_ci, [_vp, _i64, _vp, _i64, _i64, _i64, _ci, _vp]),
    "optigpu_transpose_batched": (_ci, [_vp, _i64, _vp, _i64, _i64, _i64, _i64, _ci, _vp]),
    "optigpu_transpose_inplace": (_ci, [_vp, _i64, _ci, _vp]),
    "optigpu_reduce_sum": (_ci, [_vp, _i64, _ci, _vp, _vp]),
    "optigpu_reduce_sum_ex": (_ci, [_vp, _i64, _ci, _vp, _u32, _vp]),
    "optigpu_reduce_sum_noalloc": (_ci, [_vp, _i64, _ci, _vp, _u32, _vp]),
    "optigpu_reduce_reserve": (_ci, [_i64, _vp]),
    "optigpu_reduce_segmented": (_ci, [_vp, _vp, ctypes.c_int32, _ci, _vp, _u32, _vp]),
    "optigpu_scan_inclusive": (_ci, [_vp, _vp, _i64, _ci, _vp]),
    "optigpu_histogram_i32": (_ci, [_vp, _i64, _i64, _i64, ctypes.c_int32, _vp, _vp]),
    "optigpu_transpose_host": (_ci, [_vp, _vp, _i64, _i64, _ci, _vp]),
    "optigpu_reduce_sum_host": (_ci, [_vp, _i64, _ci, _vp, _u32, _vp]),
    "optigpu_batch_plan_create": (_ci, [_vp, ctypes.c_int32, _u32, ctypes.POINTER(_vp)]),
    "optigpu_batch_run": (_ci, [_vp, _vp]),
    "optigpu_batch_plan_info": (_ci, [_vp, ctypes.POINTER(_i64), ctypes.POINTER(_i64),
                                      ctypes.POINTER(ctypes.c_int32)]),
    "optigpu_batch_autotune": (_ci, [_vp, _ci, _vp, ctypes.POINTER(_ci), ctypes.POINTER(ctypes.c_float)]),
    "optigpu_batch_plan_destroy": (None, [_vp]),
    "optigpu_server_create": (_ci, [ctypes.c_size_t, ctypes.c_int32, ctypes.c_int32, _u32,
                                    ctypes.POINTER(_vp)]),
    "optigpu_server_submit": (_ci, [_vp, _vp, ctypes.POINTER(ctypes.c_uint64)]),
    "optigpu_server_step": (_ci, [_vp, ctypes.POINTER(ctypes.c_int32)]),
    "optigpu_server_poll": (_ci, [_vp, ctypes.c_uint64, ctypes.POINTER(ctypes.c_int32)]),
    "optigpu_server_drain": (_ci, [_vp]),
    "optigpu_server_get_stats": (_ci, [_vp, _vp]),
    "optigpu_server_replay": (_ci, [_vp, _vp, _vp, _i64, _vp]),
    "optigpu_server_inject_step_failure": (_ci, [_vp, ctypes.c_int32]),
    "optigpu_server_destroy": (None, [_vp]),
    "optigpu_tune_num_configs": (_ci, [_ci, _ci]),
    "optigpu_tune_config_name": (ctypes.c_char_p, [_ci, _ci, _ci]),
    "optigpu_tune_select": (_ci, [_ci, _ci, _ci]),
    "optigpu_tune_selected": (_ci, [_ci, _ci]),
    "optigpu_tune_set_param": (_ci, [ctypes.c_char_p, _i64]),
    "optigpu_tune_get_param": (_i64, [ctypes.c_char_p]),
    "optigpu_autotune": (_ci, [_ci, _ci, _i64, _i64, _ci, _vp, ctypes.POINTER(_ci),
                              ctypes.POINTER(ctypes.c_float)]),
    "optigpu_tune_save": (_ci, [ctypes.c_char_p]),
    "optigpu_tune_load": (_ci, [ctypes.c_char_p]),
    "optigpu_stream_status": (_ci, [_vp]),
    "optigpu_selftest_wait_timeout": (_ci, [_u64, _vp]),
    "optigpu_status_string": (ctypes.c_char_p, [_ci]),
    "optigpu_last_error": (ctypes.c_char_p, []),
    "optigpu_set_wait_limit_ns": (None, [_u64]),
    "optigpu_release_workspaces": (_ci, []),
    "optigpu_version": (_ci, []),
}


class Desc(ctypes.Structure):
    """optigpu_desc: one instance of a batch."""
    _fields_ = [("op", ctypes.c_int32), ("dtype", ctypes.c_int32), ("src", ctypes.c_void_p),
                ("dst", ctypes.c_void_p), ("rows", ctypes.c_int64), ("cols", ctypes.c_int64)]


class Request(ctypes.Structure):
    """optigpu_request: one served request with host buffers."""
    _fields_ = [("op", ctypes.c_int32), ("dtype", ctypes.c_int32), ("rows", ctypes.c_int64),
                ("cols", ctypes.c_int64), ("host_src", ctypes.c_void_p), ("host_dst", ctypes.c_void_p)]


class ServerStats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in ("submitted", "completed", "pending", "in_flight",
                                               "max_in_flight", "steps", "launches", "bytes_in_use",
                                               "peak_bytes", "replay_max_loop_gap_ns")]


SERVER_PER_CALL = 4
SERVER_COPY_ENGINES = 8
SERVER_COPY_KERNELS = 16
BATCH_NO_GRAPH = 2
OP_BATCH = 2
OP_SCAN = 3


class OptigpuError(RuntimeError):
    """A non-OK optigpu_status, with the library's message."""

    def __init__(self, status: int, where: str, message: str):
        self.status = status
        super().__init__(f"{where}: status {status} ({message})")


def load(build: bool = True):
    """Loads the library (building it first if needed and allowed)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = build_lib.LIB
        if build:
            path = build_lib.build()
        if not os.path.exists(path):
            raise RuntimeError(f"liboptigpu.so is not built ({path}); run "
                               "`python -c 'import __graft_entry__ as g; g.build()'`")
        lib = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def lib():
    return _lib if _lib is not None else load()


def check(status: int, where: str) -> None:
    if status != OK:
        L = lib()
        msg = L.optigpu_last_error().decode() or L.optigpu_status_string(status).decode()
        raise OptigpuError(status, where, msg)
