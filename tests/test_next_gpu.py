"""GPU parity of the neighbouring problems against the CPU oracle: stacks of
transposes (3-D TMA or padded tiles), and the other variants as they land.
Bit-exact for transposes."""
import numpy as np
import pytest

import oracle
from gpu_util import require_gpu, to_device, to_host_bits, torch
from paper_2605_13864_gb300 import _native as N
from paper_2605_13864_gb300 import api, workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def bits(a):
    return a.view(np.uint32) if a.dtype == np.float32 else a


@pytest.mark.parametrize("dtype", ["float32", "bfloat16", "int32"])
@pytest.mark.parametrize("batch,rows,cols", [(1, 64, 64), (3, 128, 64), (5, 136, 264), (4, 33, 17),
                                             (7, 1, 300), (2, 1000, 8)])
def test_transpose_batched_dense(dtype, batch, rows, cols):
    a = workloads.matrix(batch * rows, cols, dtype, seed=batch + rows).reshape(batch, rows, cols)
    d = to_device(a.reshape(batch * rows, cols), dtype).view(batch, rows, cols)
    out = api.transpose_batched(d)
    torch.cuda.synchronize()
    api.stream_status()
    got = to_host_bits(out.reshape(batch * cols, rows)).reshape(batch, cols, rows)
    assert np.array_equal(got, bits(oracle.transpose_batched(a)))


@pytest.mark.parametrize("dtype", ["float32", "bfloat16"])
@pytest.mark.parametrize("batch,rows,cols,gap_s,gap_d", [(3, 64, 128, 64, 32), (4, 40, 24, 8, 16),
                                                         (5, 33, 17, 3, 5)])
def test_transpose_batched_with_gaps(dtype, batch, rows, cols, gap_s, gap_d):
    """Matrices stride_src / stride_dst elements apart; the gaps between
    output matrices keep their canary."""
    n = rows * cols
    ss, sd = n + gap_s, n + gap_d
    flat = workloads.vector(batch * ss, dtype, seed=9)
    src = to_device(flat, dtype)
    tdt = src.dtype
    wide = torch.int16 if tdt == torch.bfloat16 else torch.int32
    dst_raw = torch.full((batch * sd,), 0x2B2B, dtype=wide, device="cuda")
    dst = dst_raw.view(tdt)
    st = N.lib().optigpu_transpose_batched(src.data_ptr(), ss, dst.data_ptr(), sd, batch, rows, cols,
                                           api.dtype_code(tdt), torch.cuda.current_stream().cuda_stream)
    assert st == N.OK, N.lib().optigpu_last_error()
    torch.cuda.synchronize()
    got = to_host_bits(dst)
    for b in range(batch):
        m = flat[b * ss:b * ss + n].reshape(rows, cols)
        assert np.array_equal(got[b * sd:b * sd + n].reshape(cols, rows), bits(oracle.transpose(m)))
        tail = got[b * sd + n:(b + 1) * sd]
        assert (tail.view(np.uint16 if tail.dtype == np.uint16 else np.uint32) == 0x2B2B).all()


@pytest.mark.parametrize("compensated", [False, True])
@pytest.mark.parametrize("dtype", ["int32", "float32", "bfloat16"])
def test_reduce_segmented_matches_oracle_and_single_calls(dtype, compensated):
    rng = np.random.default_rng(51)
    lens = [0, 1, 7, 16384, 16385, 0, 50000, 3, 100000, 0]
    offs = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    a = workloads.vector(int(offs[-1]), dtype, seed=52)
    d = to_device(a, dtype)
    got = api.reduce_segmented(d, offs, compensated=compensated).cpu().numpy()
    want = oracle.segmented_sums(a, offs, dtype)
    for s in range(len(lens)):
        seg = a[offs[s]:offs[s + 1]]
        if dtype == "int32":
            assert int(got[s]) == want[s]
        else:
            tol = 1e-6 * oracle.sum_abs_f64(seg, dtype) + 1e-300 if seg.size else 0.0
            assert abs(float(got[s]) - want[s]) <= tol
        if seg.size:
            single = api.reduce_sum(d[offs[s]:offs[s + 1]], compensated=compensated).item()
            assert single == got[s]          # the same bits alone and segmented
        else:
            assert got[s] == 0


def test_reduce_segmented_many_small_segments():
    rng = np.random.default_rng(53)
    lens = rng.integers(0, 300, size=5000)
    offs = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    a = workloads.vector(int(offs[-1]), "int32", seed=54)
    got = api.reduce_segmented(to_device(a, "int32"), offs).cpu().numpy()
    assert got.tolist() == oracle.segmented_sums(a, offs)


def test_reduce_segmented_back_to_back_calls():
    # Several one-shot calls queued on one stream without a sync in between:
    # each call's tables go through the pinned staging pair, which must not
    # be overwritten before its copy has run.
    rng = np.random.default_rng(55)
    a = workloads.vector(3 << 20, "int32", seed=56)
    d = to_device(a, "int32")
    cases = []
    for _ in range(6):
        lens = rng.integers(0, 40000, size=int(rng.integers(1, 200)))
        offs = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
        offs = np.minimum(offs, a.size)
        cases.append((offs, api.reduce_segmented(d, offs)))
    torch.cuda.synchronize()
    api.stream_status()
    for offs, got in cases:
        assert got.cpu().numpy().tolist() == oracle.segmented_sums(a, offs)


@pytest.mark.parametrize("dtype", ["float32", "bfloat16", "int32"])
@pytest.mark.parametrize("n", [1, 2, 63, 64, 65, 127, 128, 200, 392, 1000, 2048, 4100])
def test_transpose_inplace(dtype, n):
    a = workloads.matrix(n, n, dtype, seed=n)
    d = to_device(a, dtype)
    api.transpose_inplace(d)
    torch.cuda.synchronize()
    api.stream_status()
    want = oracle.transpose_inplace(np.ascontiguousarray(a).copy())
    assert np.array_equal(to_host_bits(d), bits(want))
    api.transpose_inplace(d)  # twice is the identity
    assert np.array_equal(to_host_bits(d), bits(a))


def _abs_bits(a, dtype):
    if dtype in ("bfloat16", "float16"):
        return (a & np.uint16(0x7FFF)).astype(np.uint16)
    return np.abs(a)


@pytest.fixture(params=[0, 1, 2, 3], ids=["single_pass", "three_pass", "single_pass_carries_at_once",
                                         "single_pass_windowed"])
def scan_config(request):
    # The form is kept per input class: select it for int32 and for floats.
    prev = [api.tune_selected("scan", dt) for dt in (torch.int32, torch.float32)]
    for dt in (torch.int32, torch.float32):
        api.tune_select("scan", dt, request.param)
    yield request.param
    for dt, p in zip((torch.int32, torch.float32), prev):
        api.tune_select("scan", dt, p)


@pytest.mark.parametrize("dtype", ["int32", "float32", "bfloat16", "float16"])
@pytest.mark.parametrize("n", [1, 2, 15, 16, 17, 4095, 4096, 4097, 16384, 16385, 3 * 16384 + 77, 1 << 20,
                               (1 << 23) + 11])
def test_scan_matches_oracle(dtype, n, scan_config):
    a = workloads.vector(n, dtype, seed=n + 3)
    got = api.scan(to_device(a, dtype))
    torch.cuda.synchronize()
    api.stream_status()
    want = oracle.scan(a, dtype)
    g = got.cpu().numpy()
    if dtype == "int32":
        assert np.array_equal(g, want)
    else:
        scale = oracle.scan(_abs_bits(a, dtype), dtype)
        err = np.abs(g.astype(np.float64) - want)
        assert (err <= 1e-6 * scale + 1e-30).all(), (n, float(err.max()))


def test_scan_closed_form_and_repeatability(scan_config):
    n = (1 << 22) + 5
    a = np.arange(n, dtype=np.int64).astype(np.int32) % 1000
    d = to_device(np.ascontiguousarray(a), "int32")
    g1 = api.scan(d).cpu().numpy()
    assert np.array_equal(g1, oracle.scan(a))
    assert g1[-1] == oracle.sum_i64(a)
    f = workloads.vector(3 << 20, "float32", seed=8)
    df = to_device(f, "float32")
    r1 = api.scan(df).cpu().numpy()
    r2 = api.scan(df).cpu().numpy()
    assert np.array_equal(r1.view(np.uint32), r2.view(np.uint32))   # bit-identical runs


@pytest.mark.parametrize("dtype", ["int32", "float32", "bfloat16"])
@pytest.mark.parametrize("n", [5000, 3 * 4096, 70001])
def test_scan_unaligned_pointers(dtype, n, scan_config):
    # Source and destination off the 16-byte grid: the single pass takes its
    # plain-load / plain-store path for every chunk.
    a = workloads.vector(n, dtype, seed=n + 11)
    d = to_device(a, dtype, offset_elems=1)
    odt = torch.int64 if dtype == "int32" else torch.float32
    out = torch.empty(n + 1, dtype=odt, device="cuda")[1:]
    api.scan(d, out=out)
    torch.cuda.synchronize()
    api.stream_status()
    want = oracle.scan(a, dtype)
    g = out.cpu().numpy()
    if dtype == "int32":
        assert np.array_equal(g, want)
    else:
        scale = oracle.scan(_abs_bits(a, dtype), dtype)
        assert (np.abs(g.astype(np.float64) - want) <= 1e-6 * scale + 1e-30).all()


@pytest.mark.parametrize("dtype", ["int32", "float32", "bfloat16"])
@pytest.mark.parametrize("src_off,dst_off", [(0, 1), (1, 0)])
def test_scan_mixed_alignment(dtype, src_off, dst_off, scan_config):
    # One pointer on the 16-byte grid and the other off it: TMA loads with
    # plain stores, and plain loads with TMA stores; the bits equal the
    # aligned call's (the expression of each output depends on its index
    # only, not on how the chunk moved).
    n = 3 * 8192 * 5 + 77
    a = workloads.vector(n, dtype, seed=n + src_off + 2 * dst_off)
    aligned = api.scan(to_device(a, dtype))
    d = to_device(a, dtype, offset_elems=src_off)
    odt = torch.int64 if dtype == "int32" else torch.float32
    out = torch.empty(n + dst_off, dtype=odt, device="cuda")[dst_off:]
    api.scan(d, out=out)
    torch.cuda.synchronize()
    api.stream_status()
    assert torch.equal(out.view(torch.int32) if odt == torch.float32 else out,
                       aligned.view(torch.int32) if odt == torch.float32 else aligned)


@pytest.mark.parametrize("n", [4096 * 5 + 3, 1 << 20])
def test_scan_infinities_and_nan(n, scan_config):
    # IEEE semantics of the running sum: +inf from the first +inf on, NaN
    # from the first point where both infinities (or a NaN) are included.
    a = workloads.vector(n, "float32", seed=n + 21)
    i1, i2, i3 = n // 7, n // 3, (2 * n) // 3
    a[i1] = np.float32(np.inf)
    a[i2 + 1] = np.float32(np.inf)
    a[i3] = np.float32(-np.inf)
    got = api.scan(to_device(a, "float32")).cpu().numpy().astype(np.float64)
    want = oracle.scan(a, "float32")
    assert np.array_equal(np.isnan(got), np.isnan(want))
    assert np.array_equal(np.isposinf(got), np.isposinf(want))
    fin = np.isfinite(want)
    assert np.isfinite(got[fin]).all()
    scale = oracle.scan(np.abs(np.where(np.isfinite(a), a, 0)).astype(np.float32), "float32")
    assert (np.abs(got[fin] - want[fin]) <= 1e-6 * scale[fin] + 1e-30).all()


def test_scan_autotune_selects_a_form():
    best, name, ms = api.autotune("scan", torch.float32, 1 << 12, 1 << 12, reps=3)
    forms = api.tune_configs("scan", torch.float32)
    assert 0 <= best < len(forms) and ms > 0 and name == forms[best]
    assert api.tune_selected("scan", torch.float32) == best
    a = workloads.vector(100003, "float32", seed=12)
    got = api.scan(to_device(a, "float32")).cpu().numpy().astype(np.float64)
    scale = oracle.scan(np.abs(a), "float32")
    assert (np.abs(got - oracle.scan(a, "float32")) <= 1e-6 * scale + 1e-30).all()
    api.tune_select("scan", torch.float32, 3)


def test_scan_default_forms_per_input_class():
    # The windowed pass for float input, the radix pass for int32 input.
    assert api.tune_selected("scan", torch.float32) == 3
    assert api.tune_selected("scan", torch.bfloat16) == 3
    assert api.tune_selected("scan", torch.int32) == 0


@pytest.mark.parametrize("dtype,n", [("float32", (1 << 24) + 77), ("int32", (1 << 23) + 5),
                                     ("bfloat16", 1 << 22), ("float16", 4096 * 40 + 1)])
def test_scan_single_pass_forms_give_the_same_bits(dtype, n):
    # The two single-pass forms (configurations 0 and 2) form every output by
    # the same operations in the same order; only the moment the carry is
    # read differs.
    a = workloads.vector(n, dtype, seed=n + 31)
    d = to_device(a, dtype)
    tdt = torch.int32 if dtype == "int32" else torch.float32
    prev = api.tune_selected("scan", tdt)
    try:
        api.tune_select("scan", tdt, 0)
        first = api.scan(d).cpu().numpy()
        api.tune_select("scan", tdt, 2)
        second = api.scan(d).cpu().numpy()
    finally:
        api.tune_select("scan", tdt, prev)
    assert first.tobytes() == second.tobytes()


def test_scan_repeatable_many_chunks(scan_config):
    # 2^24 fp32 = 4096 single-pass chunks: bit-identical over repeated runs.
    f = workloads.vector(1 << 24, "float32", seed=9)
    df = to_device(f, "float32")
    first = api.scan(df).cpu().numpy().view(np.uint32)
    for _ in range(3):
        assert np.array_equal(api.scan(df).cpu().numpy().view(np.uint32), first)


@pytest.mark.parametrize("lo,width,nbins", [(0, 1, 100), (-50, 7, 29), (-1000, 1, 2001), (0, 16, 4096),
                                            (-2**31, 2**24, 256), (5, 3, 20000), (0, 1, 1),
                                            # 64-bit bin rule: lo outside int32, or width >= 2^32
                                            (-2**35, 2**24, 4096), (-2**33, 3 * 2**30 + 7, 8),
                                            (-2**32, 2**32, 3), (2**31, 1, 64), (-2**34, 2**20, 20000)])
@pytest.mark.parametrize("n", [0, 1, 1000, 123457, 1 << 22])
def test_histogram_matches_oracle(lo, width, nbins, n):
    rng = np.random.default_rng(n + nbins)
    a = rng.integers(-1200, 1200, size=n, dtype=np.int32)
    got = api.histogram(to_device(a, "int32"), lo, width, nbins).cpu().numpy()
    assert np.array_equal(got, oracle.histogram_i32(a, lo, width, nbins))


@pytest.mark.parametrize("width,nbins", [(3 * 2**29 + 5, 3), (1000003, 4295), (2**31 + 1, 2), (7, 1 << 20),
                                         (3, 12288)])
def test_histogram_full_range_widths_not_powers_of_two(width, nbins):
    # 32-bit bins by a multiply-high with a precomputed constant: values over
    # the whole int32 range, widths up to 2^31 + 1 (ceil(log2 width) = 32).
    a = np.random.default_rng(width).integers(-2**31, 2**31 - 1, size=300007, dtype=np.int64).astype(np.int32)
    a[:4] = [-2**31, 2**31 - 1, -2**31 + width - 1, -2**31 + width]
    got = api.histogram(to_device(a, "int32"), -2**31, width, nbins).cpu().numpy()
    assert np.array_equal(got, oracle.histogram_i32(a, -2**31, width, nbins))


def test_histogram_unaligned_source_and_full_range():
    a = np.random.default_rng(3).integers(-2**31, 2**31 - 1, size=100003, dtype=np.int64).astype(np.int32)
    d = to_device(a, "int32", offset_elems=1)
    got = api.histogram(d, -2**31, 2**28, 16).cpu().numpy()
    assert np.array_equal(got, oracle.histogram_i32(a, -2**31, 2**28, 16))
    assert got.sum() == a.size
