"""Sizes past 32-bit element counts, checked against closed forms.

The other parity tests stop at 2^28 elements.  These cover the index
arithmetic past 2^31 and 2^32 elements with inputs built on the device (tens
of GB; a GB300 holds 288 GB) and results fixed by their definition, so no
host copy is needed: a sum of ones is n, an inclusive scan of ones is
i + 1 (exactly as int64, or rounded once to fp32), a histogram of zeros is
n in bin 0, and the transpose of the matrix whose entries are their own
linear index has dst[c, r] = r * cols + c.
"""
import numpy as np
import pytest

from gpu_util import require_gpu, torch
from paper_2605_13864_gb300 import api

pytestmark = pytest.mark.gpu

N_BIG = (1 << 32) + 12345  # past 2^32 elements, ragged last chunk


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()
    yield
    torch.cuda.empty_cache()


@pytest.mark.parametrize("dtype", [torch.int32, torch.float32])
def test_sum_of_ones_past_2p32_elements(dtype):
    x = torch.ones(N_BIG, dtype=dtype, device="cuda")
    for comp in ((False, True) if dtype == torch.float32 else (False,)):
        # Every per-thread, per-chunk and final sum of ones is an exact integer.
        assert api.reduce_sum(x, compensated=comp).item() == N_BIG
    # An unaligned start (one element in) takes the gather path on every chunk.
    assert api.reduce_sum(x[1:]).item() == N_BIG - 1
    api.stream_status()
    del x
    torch.cuda.empty_cache()


def test_histogram_past_2p32_values():
    x = torch.zeros(N_BIG, dtype=torch.int32, device="cuda")
    x[-7:] = 5
    counts = api.histogram(x, 0, 1, 8).cpu().numpy()
    assert counts.tolist() == [N_BIG - 7, 0, 0, 0, 0, 7, 0, 0]
    del x
    torch.cuda.empty_cache()


def test_scan_of_ones_past_2p32_elements():
    x = torch.ones(N_BIG, dtype=torch.int32, device="cuda")
    out = api.scan(x)  # int64, 34 GB
    torch.cuda.synchronize()
    api.stream_status()
    idx = torch.cat([torch.arange(0, 4096, device="cuda"),
                     torch.randint(0, N_BIG, (1 << 20,), device="cuda", generator=torch.Generator("cuda").manual_seed(1)),
                     torch.arange(N_BIG - 4096, N_BIG, device="cuda")])
    assert torch.equal(out[idx], idx + 1)  # inclusive prefix of ones
    del x, out, idx
    torch.cuda.empty_cache()


@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16])
def test_float_scan_of_ones_past_2p32_elements(dtype):
    # The windowed pass (the float default) past 2^32 elements: 2^20 chunks,
    # a ragged last slice.  Every carry is an integer below 2^33, exact in its
    # FP32 hi + lo pair, and every in-chunk prefix is exact, so each output is
    # the single rounding of i + 1 to fp32.
    assert api.tune_selected("scan", dtype) == 3
    x = torch.ones(N_BIG, dtype=dtype, device="cuda")
    out = api.scan(x)  # fp32, 17 GB
    del x
    torch.cuda.synchronize()
    api.stream_status()
    idx = torch.cat([torch.arange(0, 4096, device="cuda"),
                     torch.randint(0, N_BIG, (1 << 20,), device="cuda", generator=torch.Generator("cuda").manual_seed(3)),
                     torch.arange(N_BIG - 12288, N_BIG, device="cuda")])
    assert torch.equal(out[idx], (idx + 1).to(torch.float32))
    del out, idx
    torch.cuda.empty_cache()


@pytest.mark.parametrize("rows,cols", [(46344, 46340),   # TMA kernel (multiples of 4), ragged 64-tiles
                                       (46341, 46344)])  # odd rows: the padded tile32 kernel
def test_transpose_past_2p31_elements(rows, cols):
    n = rows * cols
    assert n > (1 << 31)
    # Entry (r, c) holds its linear index r * cols + c as an int32 bit pattern.
    src = torch.empty(n, dtype=torch.int32, device="cuda")
    step = 1 << 28
    for s0 in range(0, n, step):
        e = min(n, s0 + step)
        src[s0:e] = torch.arange(s0, e, dtype=torch.int64, device="cuda").to(torch.int32)
    src = src.view(rows, cols)
    dst = api.transpose(src)
    torch.cuda.synchronize()
    api.stream_status()
    g = torch.Generator("cuda").manual_seed(2)
    r = torch.cat([torch.randint(0, rows, (1 << 20,), device="cuda", generator=g),
                   torch.tensor([0, rows - 1, rows - 1, 0], device="cuda")])
    c = torch.cat([torch.randint(0, cols, (1 << 20,), device="cuda", generator=g),
                   torch.tensor([0, cols - 1, 0, cols - 1], device="cuda")])
    want = (r * cols + c).to(torch.int32)  # the same int64 -> int32 wrap as the fill
    assert torch.equal(dst[c, r], want)
    del src, dst
    torch.cuda.empty_cache()
