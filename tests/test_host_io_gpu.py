"""The host-buffer entry points (copies pipelined against the kernels in row
or chunk bands over two internal streams) give the same results as the
device-buffer calls: transposes bit-exact against the oracle, sums
bit-identical to optigpu_reduce_sum_ex and within 1e-6 * sum|x| of the
oracle.  Sizes span several bands and ragged last bands.
"""
import numpy as np
import pytest

import oracle
from gpu_util import TORCH_DT, require_gpu, to_device, torch
from paper_2605_13864_gb300 import api, workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def host(a, dtype, pin=True):
    if dtype in ("bfloat16", "float16"):
        t = torch.from_numpy(np.ascontiguousarray(a).view(np.int16)).view(TORCH_DT[dtype])
    else:
        t = torch.from_numpy(np.ascontiguousarray(a))
    return t.pin_memory() if pin else t


def raw(t):
    return t.contiguous().view(-1).view(torch.uint8).numpy()


@pytest.mark.parametrize("rows,cols,dtype", [
    (1, 1, "float32"), (67, 45, "int32"), (16384, 4096, "float32"), (5000, 3001, "float32"),
    (100000, 7, "bfloat16"), (3, 300000, "float32"), (8192, 8200, "bfloat16"),
])
def test_transpose_host_matches_oracle(rows, cols, dtype):
    a = workloads.matrix(rows, cols, dtype, seed=rows + cols)
    out = api.transpose(host(a, dtype))
    assert not out.is_cuda
    want = oracle.transpose(a)
    assert np.array_equal(raw(out), want.view(np.uint8).reshape(-1))


def test_transpose_host_pageable_memory():
    a = workloads.matrix(3000, 1000, "float32", seed=3)
    out = torch.empty((1000, 3000), dtype=torch.float32)  # pageable
    api.transpose(host(a, "float32", pin=False), out=out)
    assert np.array_equal(out.numpy(), oracle.transpose(a))


@pytest.mark.parametrize("n,dtype,comp", [
    (0, "float32", False), (1, "int32", False), (16385, "float32", True),
    ((1 << 24) * 2 + 12345, "float32", False), ((1 << 24) * 2 + 12345, "float32", True),
    ((1 << 25) + 7, "bfloat16", True), ((1 << 24) + 1, "int32", False), (3 << 22, "float16", False),
])
def test_reduce_host_bit_identical_to_device(n, dtype, comp):
    a = workloads.vector(n, dtype, seed=n % 1000)
    got = api.reduce_sum(host(a, dtype), compensated=comp).item()
    dev = api.reduce_sum(to_device(a, dtype), compensated=comp).item() if n else 0
    assert got == dev
    if dtype == "int32":
        assert got == oracle.sum_i64(a)
    else:
        ref = oracle.reduce_reference(a, dtype)
        assert abs(got - ref["f64"]) <= 1e-6 * ref["abs"] + 1e-300


def test_back_to_back_host_calls_on_two_streams():
    """Consecutive calls from different caller streams reuse the staging
    buffers and partials safely."""
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    v1 = workloads.vector((1 << 24) + 99, "float32", seed=1)
    v2 = workloads.vector((1 << 25) + 5, "float32", seed=2)
    h1, h2 = host(v1, "float32"), host(v2, "float32")
    o1 = torch.empty((), dtype=torch.float64, pin_memory=True)
    o2 = torch.empty((), dtype=torch.float64, pin_memory=True)
    for _ in range(3):
        api.reduce_sum(h1, out=o1, stream=s1)
        api.reduce_sum(h2, out=o2, stream=s2)
    torch.cuda.synchronize()
    assert o1.item() == api.reduce_sum(to_device(v1, "float32")).item()
    assert o2.item() == api.reduce_sum(to_device(v2, "float32")).item()


@pytest.mark.parametrize("n,dtype", [((1 << 24) * 2 + 12345, "float32"), ((1 << 22) + 3, "int32")])
def test_reduce_host_pageable_staged_path(n, dtype):
    """Pageable input goes through the banded staging path; the result is the
    same bits as the device call."""
    a = workloads.vector(n, dtype, seed=77)
    got = api.reduce_sum(host(a, dtype, pin=False)).item()
    assert got == api.reduce_sum(to_device(a, dtype)).item()


def test_transpose_host_pinned_and_pageable_agree():
    a = workloads.matrix(4100, 2050, "float32", seed=9)
    pinned = api.transpose(host(a, "float32", pin=True))
    out = torch.empty((2050, 4100), dtype=torch.float32)
    api.transpose(host(a, "float32", pin=False), out=out)
    assert torch.equal(pinned.view(torch.int32), out.view(torch.int32))


@pytest.mark.parametrize("pin", [True, False])
def test_concurrent_non_blocking_transpose_and_sum(pin):
    """A host-buffer transpose and a host-buffer sum issued without waiting on
    two streams (the benchmark's end-to-end step) both give the oracle's
    result once the streams are synchronized."""
    s_t, s_r = torch.cuda.Stream(), torch.cuda.Stream()
    m = workloads.matrix(1031, 2053, "float32", seed=31)
    v = workloads.vector((1 << 23) + 17, "float32", seed=32)
    hm, hv = host(m, "float32", pin=pin), host(v, "float32", pin=pin)
    out_t = torch.empty((2053, 1031), dtype=torch.float32)
    out_r = torch.empty((), dtype=torch.float64)
    if pin:
        out_t, out_r = out_t.pin_memory(), out_r.pin_memory()
    for _ in range(2):
        api.transpose(hm, out=out_t, stream=s_t, blocking=False)
        api.reduce_sum(hv, out=out_r, stream=s_r, blocking=False)
        s_t.synchronize()
        s_r.synchronize()
        assert np.array_equal(out_t.numpy().view(np.uint32), oracle.transpose(m).view(np.uint32))
        ref = oracle.reduce_reference(v)
        assert abs(out_r.item() - ref["f64"]) <= 1e-6 * ref["abs"]
        assert out_r.item() == api.reduce_sum(to_device(v, "float32")).item()
