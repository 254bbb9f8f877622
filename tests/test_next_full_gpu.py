"""GPU parity of the neighbouring problems at the benchmark's full sizes.

Each case runs the CUDA path on seeded synthetic inputs of the size the
benchmark times, and compares with the CPU oracle:
- the stack of 64 2048 x 2048 float32 transposes: three whole matrices bit-exact,
  plus 2^20 sampled elements spread over every matrix;
- the in-place 16384 x 16384 float32 transpose: bit-exact in full;
- 2^28 float32 in 16384 segments: every segment sum within 1e-6 of the segment's
  sum of |x|, and sampled segments bit-identical to their single calls;
- the 2^28-element inclusive scans: every element of int32 -> int64 exact,
  float32 within 1e-6 of the running sum of |x|;
- the 2^28-value histogram in 4096 bins: exact;
- two windowed scans on concurrent streams: the same bits as alone.
"""
import numpy as np
import pytest

import oracle
from gpu_util import require_gpu, to_device, to_host_bits, torch
from paper_2605_13864_gb300 import api, workloads

pytestmark = pytest.mark.gpu
N28 = 1 << 28


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()
    yield
    torch.cuda.empty_cache()


def test_transpose_stack_64x2048x2048():
    b, r, c = 64, 2048, 2048
    a = workloads.matrix(b * r, c, "float32", seed=71).reshape(b, r, c)
    d = to_device(a.reshape(b * r, c), "float32").view(b, r, c)
    out = api.transpose_batched(d)
    torch.cuda.synchronize()
    api.stream_status()
    del d
    got = out.cpu().numpy()
    del out
    for k in (0, 31, 63):
        assert np.array_equal(got[k].view(np.uint32), oracle.transpose(a[k]).view(np.uint32)), k
    rng = np.random.default_rng(72)
    bi, ri, ci = rng.integers(0, b, 1 << 20), rng.integers(0, r, 1 << 20), rng.integers(0, c, 1 << 20)
    assert np.array_equal(got[bi, ci, ri].view(np.uint32), a[bi, ri, ci].view(np.uint32))


def test_transpose_inplace_16384_float32():
    n = 16384
    a = workloads.roofline_matrix(n, n)
    d = to_device(a, "float32")
    api.transpose_inplace(d)
    torch.cuda.synchronize()
    api.stream_status()
    got = d.cpu().numpy()
    del d
    assert np.array_equal(got.view(np.uint32), oracle.transpose(a).view(np.uint32))


def test_transpose_inplace_16384_bfloat16():
    """The 16-bit in-place path (128 x 128 tile pairs) on the full square."""
    n = 16384
    a = workloads.matrix(n, n, "bfloat16", seed=74)
    d = to_device(a, "bfloat16")
    api.transpose_inplace(d)
    torch.cuda.synchronize()
    api.stream_status()
    got = to_host_bits(d)
    del d
    assert np.array_equal(got, oracle.transpose(a))


def test_segmented_2p28_float32_16384_segments():
    a = workloads.roofline_vector(N28)
    offs = workloads.segment_offsets(N28, 16384)
    d = to_device(a, "float32")
    got = api.reduce_segmented(d, offs).cpu().numpy()
    want = oracle.segmented_sums(a, offs, "float32")
    absums = oracle.segmented_sums(np.abs(a), offs, "float32")
    for s in range(len(offs) - 1):
        assert abs(float(got[s]) - want[s]) <= 1e-6 * absums[s] + 1e-300, s
    for s in np.random.default_rng(73).integers(0, len(offs) - 1, 16):
        lo, hi = int(offs[s]), int(offs[s + 1])
        if hi > lo:
            assert api.reduce_sum(d[lo:hi]).item() == got[s], s


@pytest.mark.parametrize("form", [0, 2, 3], ids=["single_pass", "single_pass_carries_at_once",
                                                 "single_pass_windowed"])
@pytest.mark.parametrize("dtype", ["int32", "float32"])
def test_scan_2p28(dtype, form):
    a = workloads.roofline_vector(N28) if dtype == "float32" else workloads.histogram_values(N28, 1 << 20)
    d = to_device(a, dtype)
    tdt = torch.int32 if dtype == "int32" else torch.float32
    prev = api.tune_selected("scan", tdt)
    api.tune_select("scan", tdt, form)
    try:
        got = api.scan(d)
    finally:
        api.tune_select("scan", tdt, prev)
    torch.cuda.synchronize()
    api.stream_status()
    del d
    g = got.cpu().numpy()
    del got
    want = oracle.scan(a, dtype)
    if dtype == "int32":
        assert np.array_equal(g, want)
    else:
        scale = oracle.scan(np.abs(a), dtype)
        assert (np.abs(g.astype(np.float64) - want) <= 1e-6 * scale + 1e-30).all()


def test_scan_2p28_repeatable():
    # The default pass for fp32 (windowed) under full HBM load: slice totals
    # are fetched by asynchronous copies while other CTAs are still
    # publishing, and still every run gives the same bits.
    d = to_device(workloads.roofline_vector(N28), "float32")
    out = torch.empty(N28, dtype=torch.float32, device="cuda")
    api.scan(d, out=out)
    first = out.view(torch.int32).clone()
    for _ in range(4):
        api.scan(d, out=out)
        assert torch.equal(out.view(torch.int32), first)
    api.stream_status()


def test_windowed_scans_on_concurrent_streams():
    # The windowed pass's CTAs wait for one another's slice totals, which is
    # safe because its launch is cooperative (every CTA resident at once).
    # Two 2^26 scans issued on two streams with no sync between them, and a
    # 2^28 sum on a third, give the same bits as the scans run alone, and no
    # bounded wait gives up.
    n = 1 << 26
    xs = [to_device(workloads.vector(n, "float32", seed=90 + k), "float32") for k in range(2)]
    alone = [api.scan(x) for x in xs]
    torch.cuda.synchronize()
    v = to_device(workloads.roofline_vector(N28), "float32")
    want_sum = api.reduce_sum(v).item()
    outs = [torch.empty_like(a) for a in alone]
    s_sum = torch.empty((), dtype=torch.float64, device="cuda")
    streams = [torch.cuda.Stream() for _ in range(3)]
    torch.cuda.synchronize()
    for rep in range(3):
        api.scan(xs[0], out=outs[0], stream=streams[0])
        api.scan(xs[1], out=outs[1], stream=streams[1])
        api.reduce_sum(v, out=s_sum, stream=streams[2])
        torch.cuda.synchronize()
        api.stream_status()
        for o, a in zip(outs, alone):
            assert torch.equal(o.view(torch.int32), a.view(torch.int32)), rep
        assert s_sum.item() == want_sum
    del xs, alone, outs, v


def test_histogram_2p28_4096_bins():
    a = workloads.histogram_values(N28, 4096)
    got = api.histogram(to_device(a, "int32"), 0, 1, 4096).cpu().numpy()
    want = oracle.histogram_i32(a, 0, 1, 4096)
    assert np.array_equal(got, want)
    assert got.sum() == N28
