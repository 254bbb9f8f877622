"""The C-ABI library builds, loads and exports every symbol include/optigpu.h
declares; host-side argument validation answers without touching a GPU.

No compute call is made here: every call below is rejected (or answered) by
the host before any CUDA API is reached.
"""
import ctypes
import os
import re

import pytest

from paper_2605_13864_gb300 import _native as N
from paper_2605_13864_gb300 import build_lib

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "optigpu.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(optigpu_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    return N.load(build=True)


def test_header_declares_the_core_calls():
    names = declared_functions()
    for must in ("optigpu_transpose", "optigpu_reduce_sum", "optigpu_reduce_sum_ex",
                 "optigpu_stream_status", "optigpu_status_string"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    raw = ctypes.CDLL(build_lib.LIB)
    missing = [n for n in declared_functions() if not hasattr(raw, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    assert set(declared_functions()) <= set(N.SIGNATURES)


def test_library_is_built_for_sm_103a_only():
    assert build_lib.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_version_and_status_strings(lib):
    assert lib.optigpu_version() == 100
    for code in range(0, 9):
        assert lib.optigpu_status_string(code)
    assert lib.optigpu_status_string(0) == b"ok"


FAKE = 0x7F0000000000  # never dereferenced: validation rejects first


@pytest.mark.parametrize("args,status", [
    ((None, None, -1, 4, N.FLOAT32), N.ERR_INVALID_ARG),
    ((None, None, 4, -1, N.FLOAT32), N.ERR_INVALID_ARG),
    ((None, None, 4, 4, N.FLOAT32), N.ERR_INVALID_ARG),
    ((FAKE, FAKE + (1 << 20), 4, 4, 9), N.ERR_UNSUPPORTED_DTYPE),
    ((FAKE, FAKE + 8, 4, 4, N.FLOAT32), N.ERR_OVERLAP),
    ((FAKE + 8, FAKE, 4, 4, N.BFLOAT16), N.ERR_OVERLAP),
    ((FAKE, FAKE + 64, 1 << 40, 1 << 40, N.FLOAT32), N.ERR_INVALID_ARG),
    ((FAKE + 2, FAKE + (1 << 20), 4, 4, N.FLOAT32), N.ERR_INVALID_ARG),  # not element-aligned
    ((FAKE, FAKE + (1 << 20) + 1, 4, 4, N.FLOAT16), N.ERR_INVALID_ARG),
    ((None, None, 0, 5, N.FLOAT32), N.OK),   # empty: a no-op
    ((None, None, 7, 0, N.INT32), N.OK),
])
def test_transpose_validation(lib, args, status):
    src, dst, rows, cols, dt = args
    assert lib.optigpu_transpose(src, dst, rows, cols, dt, None) == status


def test_transpose_ex_rejects_unknown_kernel(lib):
    assert lib.optigpu_transpose_ex(FAKE, FAKE + (1 << 20), 4, 4, N.FLOAT32, 7, None) == N.ERR_INVALID_ARG


def test_transpose_ex_rejects_tma_on_ineligible_shape(lib):
    # cols = 3 floats is not a multiple of 16 bytes
    assert lib.optigpu_transpose_ex(FAKE, FAKE + (1 << 20), 4, 3, N.FLOAT32, N.TRANSPOSE_TMA,
                                    None) == N.ERR_INVALID_ARG
    assert b"TMA" in lib.optigpu_last_error()


@pytest.mark.parametrize("rows,cols,dt,align,ok", [
    (64, 64, N.FLOAT32, 0, 1), (4, 8, N.INT32, 0, 1), (8, 16, N.BFLOAT16, 0, 1),
    (4, 4, N.BFLOAT16, 0, 0), (3, 64, N.FLOAT32, 0, 0), (64, 64, N.FLOAT32, 4, 0),
    (0, 64, N.FLOAT32, 0, 0),
])
def test_tma_eligibility(lib, rows, cols, dt, align, ok):
    assert lib.optigpu_transpose_tma_eligible(FAKE + align, FAKE + (1 << 30), rows, cols, dt) == ok


@pytest.mark.parametrize("args,status", [
    ((FAKE, -1, N.FLOAT32, FAKE, 0), N.ERR_INVALID_ARG),
    ((FAKE, 10, 17, FAKE, 0), N.ERR_UNSUPPORTED_DTYPE),
    ((FAKE, 10, N.FLOAT32, None, 0), N.ERR_INVALID_ARG),
    ((None, 10, N.FLOAT32, FAKE, 0), N.ERR_INVALID_ARG),
    ((FAKE, 10, N.FLOAT32, FAKE, 6), N.ERR_INVALID_ARG),
    ((FAKE, (1 << 62) + 1, N.INT32, FAKE, 0), N.ERR_INVALID_ARG),
    ((FAKE + 2, 10, N.FLOAT32, FAKE, 0), N.ERR_INVALID_ARG),   # src not element-aligned
    ((FAKE + 1, 10, N.BFLOAT16, FAKE, 0), N.ERR_INVALID_ARG),
    ((FAKE, 10, N.FLOAT32, FAKE + 4, 0), N.ERR_INVALID_ARG),   # out not 8-byte aligned
])
def test_reduce_validation(lib, args, status):
    src, n, dt, out, flags = args
    assert lib.optigpu_reduce_sum_ex(src, n, dt, out, flags, None) == status


def test_errors_carry_a_message(lib):
    lib.optigpu_reduce_sum_ex(FAKE, 10, 17, FAKE, 0, None)
    assert b"dtype" in lib.optigpu_last_error()


def _desc_array(rows):
    arr = (N.Desc * len(rows))()
    for k, (op, dt, src, dst, r, c) in enumerate(rows):
        arr[k].op, arr[k].dtype, arr[k].src, arr[k].dst, arr[k].rows, arr[k].cols = op, dt, src, dst, r, c
    return arr


@pytest.mark.parametrize("rows,status", [
    ([(5, N.FLOAT32, FAKE, FAKE + (1 << 20), 4, 4)], N.ERR_INVALID_ARG),            # unknown op
    ([(N.OP_TRANSPOSE, 9, FAKE, FAKE + (1 << 20), 4, 4)], N.ERR_UNSUPPORTED_DTYPE),
    ([(N.OP_TRANSPOSE, N.FLOAT32, FAKE, FAKE + 8, 4, 4)], N.ERR_OVERLAP),
    ([(N.OP_TRANSPOSE, N.FLOAT32, None, FAKE, 4, 4)], N.ERR_INVALID_ARG),
    ([(N.OP_REDUCE, N.FLOAT32, FAKE, FAKE + 4, 10, 1)], N.ERR_INVALID_ARG),          # out not 8-aligned
    ([(N.OP_REDUCE, N.FLOAT32, FAKE, FAKE + 64, -1, 1)], N.ERR_INVALID_ARG),
    ([(N.OP_TRANSPOSE, N.FLOAT32, FAKE, FAKE + (1 << 30), 4, 4),
      (N.OP_REDUCE, N.BFLOAT16, FAKE + 1, FAKE + 64, 10, 1)], N.ERR_INVALID_ARG),  # 2nd bad
])
def test_batch_plan_validation(lib, rows, status):
    plan = ctypes.c_void_p()
    arr = _desc_array(rows)
    assert lib.optigpu_batch_plan_create(arr, len(rows), 0, ctypes.byref(plan)) == status
    assert not plan.value


def test_batch_plan_rejects_bad_flags_and_tables(lib):
    plan = ctypes.c_void_p()
    assert lib.optigpu_batch_plan_create(None, 3, 0, ctypes.byref(plan)) == N.ERR_INVALID_ARG
    assert lib.optigpu_batch_plan_create(None, -1, 0, ctypes.byref(plan)) == N.ERR_INVALID_ARG
    arr = _desc_array([(N.OP_REDUCE, N.FLOAT32, FAKE, FAKE + 64, 10, 1)])
    assert lib.optigpu_batch_plan_create(arr, 1, 1 << 7, ctypes.byref(plan)) == N.ERR_INVALID_ARG
    assert lib.optigpu_batch_run(None, None) == N.ERR_INVALID_ARG


def test_tune_tables_are_host_only(lib):
    for op, dt in ((N.OP_TRANSPOSE, N.FLOAT32), (N.OP_TRANSPOSE, N.BFLOAT16), (N.OP_REDUCE, N.FLOAT32),
                   (N.OP_BATCH, 0), (N.OP_SCAN, 0)):
        n = lib.optigpu_tune_num_configs(op, dt)
        assert n >= 2
        names = [lib.optigpu_tune_config_name(op, dt, i) for i in range(n)]
        assert all(names) and len(set(names)) == n
        assert lib.optigpu_tune_config_name(op, dt, n) is None
    assert lib.optigpu_tune_select(N.OP_REDUCE, N.FLOAT32, 99) == N.ERR_INVALID_ARG
    assert lib.optigpu_tune_set_param(b"no.such.param", 1) == N.ERR_NOT_FOUND
    assert lib.optigpu_tune_set_param(b"transpose.group_rows", 0) == N.ERR_INVALID_ARG
    assert lib.optigpu_tune_get_param(b"transpose.group_rows") >= 1


def test_tune_cache_round_trip(lib, tmp_path):
    path = str(tmp_path / "tune.txt").encode()
    assert lib.optigpu_tune_select(N.OP_TRANSPOSE, N.FLOAT32, 1) == N.OK
    assert lib.optigpu_tune_set_param(b"transpose.group_rows", 8) == N.OK
    assert lib.optigpu_tune_save(path) == N.OK
    assert lib.optigpu_tune_select(N.OP_TRANSPOSE, N.FLOAT32, 0) == N.OK
    assert lib.optigpu_tune_set_param(b"transpose.group_rows", 16) == N.OK
    assert lib.optigpu_tune_load(path) == N.OK
    assert lib.optigpu_tune_selected(N.OP_TRANSPOSE, N.FLOAT32) == 1
    assert lib.optigpu_tune_get_param(b"transpose.group_rows") == 8
    assert lib.optigpu_tune_load(b"/nonexistent/tune.txt") == N.ERR_NOT_FOUND
    lib.optigpu_tune_select(N.OP_TRANSPOSE, N.FLOAT32, 0)
    lib.optigpu_tune_set_param(b"transpose.group_rows", 16)


def test_tune_cache_keeps_the_scan_form(lib, tmp_path):
    path = str(tmp_path / "tune_scan.txt").encode()
    I, F, B = N.INT32, N.FLOAT32, N.BFLOAT16
    assert lib.optigpu_tune_selected(N.OP_SCAN, I) == 0          # radix single pass for int32
    assert lib.optigpu_tune_selected(N.OP_SCAN, F) == 3          # windowed single pass for floats
    assert lib.optigpu_tune_selected(N.OP_SCAN, B) == 3          # one choice for every float type
    assert lib.optigpu_tune_select(N.OP_SCAN, I, 1) == N.OK
    assert lib.optigpu_tune_select(N.OP_SCAN, F, 2) == N.OK
    assert lib.optigpu_tune_selected(N.OP_SCAN, B) == 2
    assert lib.optigpu_tune_save(path) == N.OK
    text = open(path, "rb").read()
    assert b"scan int32 " in text and b"scan float " in text
    assert lib.optigpu_tune_select(N.OP_SCAN, I, 0) == N.OK
    assert lib.optigpu_tune_select(N.OP_SCAN, F, 3) == N.OK
    assert lib.optigpu_tune_load(path) == N.OK
    assert lib.optigpu_tune_selected(N.OP_SCAN, I) == 1
    assert lib.optigpu_tune_selected(N.OP_SCAN, F) == 2
    # A line without the input class sets both classes.
    name = lib.optigpu_tune_config_name(N.OP_SCAN, F, 3)
    with open(path, "wb") as fh:
        fh.write(b"scan " + name + b"\n")
    assert lib.optigpu_tune_load(path) == N.OK
    assert lib.optigpu_tune_selected(N.OP_SCAN, I) == 3 and lib.optigpu_tune_selected(N.OP_SCAN, F) == 3
    assert lib.optigpu_tune_select(N.OP_SCAN, F, lib.optigpu_tune_num_configs(N.OP_SCAN, F)) == N.ERR_INVALID_ARG
    assert lib.optigpu_tune_select(N.OP_SCAN, I, 0) == N.OK
    assert lib.optigpu_tune_select(N.OP_SCAN, F, 3) == N.OK


def test_server_validation_is_host_side(lib):
    sv = ctypes.c_void_p()
    assert lib.optigpu_server_create(1 << 10, 4, 2, 0, ctypes.byref(sv)) == N.ERR_INVALID_ARG   # budget < 1 MiB
    assert lib.optigpu_server_create(1 << 30, 0, 2, 0, ctypes.byref(sv)) == N.ERR_INVALID_ARG
    assert lib.optigpu_server_create(1 << 30, 4, 0, 0, ctypes.byref(sv)) == N.ERR_INVALID_ARG
    assert lib.optigpu_server_create(1 << 30, 4, 2, 1 << 9, ctypes.byref(sv)) == N.ERR_INVALID_ARG
    assert lib.optigpu_server_create(1 << 30, 4, 2, 0, None) == N.ERR_INVALID_ARG
    assert not sv.value
    assert lib.optigpu_server_submit(None, None, None) == N.ERR_INVALID_ARG
    assert lib.optigpu_server_step(None, None) == N.ERR_INVALID_ARG
    assert lib.optigpu_server_drain(None) == N.ERR_INVALID_ARG
    assert lib.optigpu_server_replay(None, None, None, 1, None) == N.ERR_INVALID_ARG
    lib.optigpu_server_destroy(None)


def test_host_entry_points_validate_on_the_host(lib):
    assert lib.optigpu_transpose_host(None, None, -1, 3, N.FLOAT32, None) == N.ERR_INVALID_ARG
    assert lib.optigpu_transpose_host(FAKE, FAKE + 8, 4, 4, N.FLOAT32, None) == N.ERR_OVERLAP
    assert lib.optigpu_transpose_host(None, None, 0, 3, N.FLOAT32, None) == N.OK
    assert lib.optigpu_transpose_host(FAKE, FAKE + (1 << 20), 4, 4, 11, None) == N.ERR_UNSUPPORTED_DTYPE
    assert lib.optigpu_reduce_sum_host(None, 5, N.FLOAT32, FAKE, 0, None) == N.ERR_INVALID_ARG
    assert lib.optigpu_reduce_sum_host(FAKE, 5, N.FLOAT32, None, 0, None) == N.ERR_INVALID_ARG
    assert lib.optigpu_reduce_sum_host(FAKE + 2, 5, N.FLOAT32, FAKE, 0, None) == N.ERR_INVALID_ARG
    assert lib.optigpu_reduce_sum_host(FAKE, 5, N.FLOAT32, FAKE, 8, None) == N.ERR_INVALID_ARG


def test_strided_transpose_validation(lib):
    f = lib.optigpu_transpose_strided
    assert f(FAKE, 3, FAKE + (1 << 20), 4, 4, 4, N.FLOAT32, None) == N.ERR_INVALID_ARG   # lds < cols
    assert f(FAKE, 4, FAKE + (1 << 20), 3, 4, 4, N.FLOAT32, None) == N.ERR_INVALID_ARG   # ldd < rows
    assert f(FAKE, 100, FAKE + 64, 4, 4, 4, N.FLOAT32, None) == N.ERR_OVERLAP           # src span reaches dst
    assert f(None, 4, None, 4, 0, 4, N.FLOAT32, None) == N.OK


def test_batched_transpose_validation(lib):
    f = lib.optigpu_transpose_batched
    assert f(FAKE, 15, FAKE + (1 << 30), 16, 2, 4, 4, N.FLOAT32, None) == N.ERR_INVALID_ARG   # stride < n
    assert f(FAKE, 16, FAKE + 64, 16, 2, 4, 4, N.FLOAT32, None) == N.ERR_OVERLAP
    assert f(FAKE, 16, FAKE + (1 << 30), 16, -1, 4, 4, N.FLOAT32, None) == N.ERR_INVALID_ARG
    assert f(None, 16, None, 16, 0, 4, 4, N.FLOAT32, None) == N.OK
    assert f(FAKE, 16, FAKE + (1 << 30), 16, 2, 4, 4, 12, None) == N.ERR_UNSUPPORTED_DTYPE


def test_segmented_validation(lib):
    import numpy as np
    f = lib.optigpu_reduce_segmented
    bad = np.array([0, 5, 3], dtype=np.int64)          # decreasing
    assert f(FAKE, bad.ctypes.data, 2, N.FLOAT32, FAKE, 0, None) == N.ERR_INVALID_ARG
    neg = np.array([-1, 5], dtype=np.int64)
    assert f(FAKE, neg.ctypes.data, 1, N.FLOAT32, FAKE, 0, None) == N.ERR_INVALID_ARG
    ok = np.array([0, 5], dtype=np.int64)
    assert f(FAKE, ok.ctypes.data, 1, N.FLOAT32, FAKE + 4, 0, None) == N.ERR_INVALID_ARG   # out misaligned
    assert f(FAKE, ok.ctypes.data, 1, 19, FAKE, 0, None) == N.ERR_UNSUPPORTED_DTYPE
    assert f(None, None, 0, N.FLOAT32, None, 0, None) == N.OK


def test_inplace_validation(lib):
    f = lib.optigpu_transpose_inplace
    assert f(None, -1, N.FLOAT32, None) == N.ERR_INVALID_ARG
    assert f(None, 5, N.FLOAT32, None) == N.ERR_INVALID_ARG
    assert f(FAKE + 2, 5, N.FLOAT32, None) == N.ERR_INVALID_ARG
    assert f(None, 1, N.FLOAT32, None) == N.OK
    assert f(FAKE, 5, 33, None) == N.ERR_UNSUPPORTED_DTYPE


def test_scan_validation(lib):
    f = lib.optigpu_scan_inclusive
    assert f(FAKE, FAKE + 16, 100, N.FLOAT32, None) == N.ERR_OVERLAP
    assert f(FAKE, FAKE + (1 << 20) + 4, 100, N.INT32, None) == N.ERR_INVALID_ARG   # int64 out misaligned
    assert f(None, None, 0, N.FLOAT32, None) == N.OK
    assert f(FAKE, FAKE + (1 << 20), -1, N.FLOAT32, None) == N.ERR_INVALID_ARG
    assert f(FAKE, FAKE + (1 << 20), 5, 9, None) == N.ERR_UNSUPPORTED_DTYPE


def test_histogram_validation(lib):
    f = lib.optigpu_histogram_i32
    assert f(FAKE, 10, 0, 0, 4, FAKE, None) == N.ERR_INVALID_ARG        # width 0
    assert f(FAKE, 10, 0, 1, 0, FAKE, None) == N.ERR_INVALID_ARG        # no bins
    assert f(FAKE, 10, 0, 1, 4, FAKE + 4, None) == N.ERR_INVALID_ARG    # counts misaligned
    assert f(FAKE + 2, 10, 0, 1, 4, FAKE, None) == N.ERR_INVALID_ARG    # src misaligned
    assert f(FAKE, 10, 1 << 41, 1, 4, FAKE, None) == N.ERR_INVALID_ARG


def test_transpose_default_configuration_is_chosen_by_size(lib):
    """Configuration 0 (the default) launches the four-stage ring below 1 GiB
    moved and the six-stage ring from 1 GiB up; an explicit selection is
    launched as selected."""
    names = [lib.optigpu_tune_config_name(N.OP_TRANSPOSE, N.FLOAT32, i).decode() for i in range(3)]
    assert "by size" in names[0] and names[1].endswith("s6 o2") and names[2].endswith("s4 o2")
    prev = lib.optigpu_tune_selected(N.OP_TRANSPOSE, N.FLOAT32)
    try:
        assert lib.optigpu_tune_select(N.OP_TRANSPOSE, N.FLOAT32, 0) == N.OK
        assert lib.optigpu_transpose_config_for(16384, 16384, N.FLOAT32) == 1   # 2 GiB moved
        assert lib.optigpu_transpose_config_for(8192, 16384, N.FLOAT32) == 1    # exactly 1 GiB
        assert lib.optigpu_transpose_config_for(8192, 8192, N.FLOAT32) == 2     # 512 MiB
        assert lib.optigpu_transpose_config_for(16384, 16384, N.BFLOAT16) == 1  # 1 GiB of bf16
        assert lib.optigpu_transpose_config_for(12288, 12288, N.BFLOAT16) == 2
        n = lib.optigpu_tune_num_configs(N.OP_TRANSPOSE, N.FLOAT32)
        assert lib.optigpu_transpose_config_for(30, 16384, N.FLOAT32) == n - 1   # rows not a multiple of 4: tile32
        assert lib.optigpu_tune_select(N.OP_TRANSPOSE, N.FLOAT32, 3) == N.OK
        assert lib.optigpu_transpose_config_for(8192, 8192, N.FLOAT32) == 3
        assert lib.optigpu_transpose_config_for(-1, 8, N.FLOAT32) == -1
    finally:
        lib.optigpu_tune_select(N.OP_TRANSPOSE, N.FLOAT32, prev)
