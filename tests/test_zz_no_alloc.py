"""The allocation-free sum, optigpu_reduce_sum_noalloc, called through the C ABI.

It exists for callers that must not have the library allocate device memory
(an application whose own pool owns all device memory, a loop that must not
reach the driver's allocator after start-up, a process held to a hard memory
budget).  It runs the same kernel with the same chunk partition and
combine order as optigpu_reduce_sum_ex, so its result must equal that
entry point's bit for bit, on two calls in a row (every call reuses the same
fixed device array); both must also match the oracle -- exactly for int32,
within the 1e-6 * sum|x| tolerance the other sum tests use for floats.
This file is named to be collected last.
"""
import ctypes

import numpy as np
import pytest

import oracle
from gpu_util import require_gpu, to_device, torch
from paper_2605_13864_gb300 import _native as N
from paper_2605_13864_gb300 import workloads

pytestmark = pytest.mark.gpu

DT = {"int32": N.INT32, "float32": N.FLOAT32, "bfloat16": N.BFLOAT16, "float16": N.FLOAT16}
LIMIT = 32768 * 16384


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def _sum(fn, d, dtype, flags, stream):
    odt = torch.int64 if dtype == "int32" else torch.float64
    out = torch.full((), -1, dtype=odt, device="cuda")
    st = fn(d.data_ptr() if d.numel() else None, d.numel(), DT[dtype], out.data_ptr(), flags,
            stream.cuda_stream)
    assert st == N.OK, N.lib().optigpu_last_error()
    stream.synchronize()
    return out.item()


@pytest.mark.parametrize("dtype,flags", [("int32", 0), ("float32", 0), ("float32", 1),
                                         ("bfloat16", 0), ("bfloat16", 1), ("float16", 1)])
def test_noalloc_matches_the_allocating_entry_point(dtype, flags):
    L = N.lib()
    stream = torch.cuda.Stream()
    for n in (0, 1, 16385, 3 * 16384 + 77, 1 << 20):
        a = workloads.vector(n, dtype, seed=n + 5)
        d = to_device(a, dtype)
        want = _sum(L.optigpu_reduce_sum_ex, d, dtype, flags, stream)
        first = _sum(L.optigpu_reduce_sum_noalloc, d, dtype, flags, stream)
        second = _sum(L.optigpu_reduce_sum_noalloc, d, dtype, flags, stream)
        assert first == want == second, (n, first, second, want)
        if dtype == "int32":
            assert want == oracle.sum_i64(a)
        else:
            ref = oracle.reduce_reference(a, dtype)
            assert abs(want - ref["f64"]) <= 1e-6 * ref["abs"] + 1e-300, (n, want, ref["f64"])


def test_noalloc_rejects_sizes_beyond_its_limit():
    L = N.lib()
    out = torch.zeros((), dtype=torch.float64, device="cuda")
    src = torch.zeros(16, dtype=torch.float32, device="cuda")
    st = L.optigpu_reduce_sum_noalloc(src.data_ptr(), LIMIT + 1, N.FLOAT32, out.data_ptr(), 0, None)
    assert st == N.ERR_INVALID_ARG
    assert b"limit" in L.optigpu_last_error()


def test_noalloc_leaves_device_memory_untouched():
    L = N.lib()
    a = workloads.vector(5 * 16384 + 3, "float32", seed=99)
    d = to_device(a, "float32")
    out = torch.zeros((), dtype=torch.float64, device="cuda")
    stream = torch.cuda.Stream()
    # The first call on a device may load the library's module (the runtime
    # maps the fixed array then) and looks up the array's address.
    assert L.optigpu_reduce_sum_noalloc(d.data_ptr(), d.numel(), N.FLOAT32, out.data_ptr(), 0,
                                        stream.cuda_stream) == N.OK
    torch.cuda.synchronize()
    free_before, _ = torch.cuda.mem_get_info()
    for _ in range(2):
        assert L.optigpu_reduce_sum_noalloc(d.data_ptr(), d.numel(), N.FLOAT32, out.data_ptr(), 0,
                                            stream.cuda_stream) == N.OK
    stream.synchronize()
    free_after, _ = torch.cuda.mem_get_info()
    assert free_after == free_before
    ref = oracle.reduce_reference(a)
    assert abs(out.item() - ref["f64"]) <= 1e-6 * ref["abs"]


def test_noalloc_at_its_exact_limit():
    # 2^29 ones: the largest n the fixed array serves; every partial is exact.
    L = N.lib()
    d = torch.ones(LIMIT, dtype=torch.float32, device="cuda")
    stream = torch.cuda.Stream()
    want = _sum(L.optigpu_reduce_sum_ex, d, "float32", 0, stream)
    got = _sum(L.optigpu_reduce_sum_noalloc, d, "float32", 0, stream)
    assert got == want == float(LIMIT)
    del d
    torch.cuda.empty_cache()
