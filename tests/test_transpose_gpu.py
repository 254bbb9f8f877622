"""GPU parity of the transpose (Listing 3.5, Sec. 3.1) against the CPU oracle.

Bit-exact comparison, element by element, through the C ABI (the Python
binding only marshals pointers).  Shapes cover every rows, cols in 1..67,
shapes around the 32 / 64 / 128 tile sizes, TMA-eligible shapes with ragged
last tiles, unaligned pointers, guard bands around the output, and the full
16384x16384 float32, 8192x8192 bfloat16 and 1024x1024 int32 matrices.
"""
import numpy as np
import pytest

import oracle
from gpu_util import require_gpu, to_device, to_host_bits, torch
from paper_2605_13864_gb300 import api, workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def gpu_transpose(a, dtype, kernel="auto", src_offset=0):
    d = to_device(a, dtype, src_offset)
    out = api.transpose(d, kernel=kernel)
    torch.cuda.synchronize()
    api.stream_status()
    return to_host_bits(out)


def bits(a):
    return a.view(np.uint32) if a.dtype == np.float32 else a


def check(a, dtype, kernel="auto", src_offset=0):
    got = gpu_transpose(a, dtype, kernel, src_offset)
    want = bits(oracle.transpose(a))
    assert got.shape == want.shape
    if not np.array_equal(got, want):
        bad = np.argwhere(got != want)
        raise AssertionError(f"{a.shape} {dtype} {kernel}: {len(bad)} mismatches, first at {bad[0]}")


def test_tile32_every_small_shape():
    rng = np.random.default_rng(100)
    for r in range(1, 68):
        for c in range(1, 68):
            a = rng.integers(-2**31, 2**31 - 1, size=(r, c), dtype=np.int64).astype(np.int32)
            check(a, "int32", "tile32")


@pytest.mark.parametrize("dtype", ["float32", "bfloat16", "float16", "int32"])
@pytest.mark.parametrize("kernel", ["tile32", "auto"])
def test_shapes_around_tiles(dtype, kernel):
    sizes = [1, 2, 31, 32, 33, 63, 64, 65, 127, 128, 129, 255, 256, 257, 1000]
    for r in sizes:
        for c in sizes:
            a = workloads.matrix(r, c, dtype, seed=r * 7919 + c)
            check(a, dtype, kernel)


def _tma_sizes(dtype):
    step = 16 // workloads.ESIZE[dtype]
    small = list(range(step, 8 * step + 1, step))
    return small + [120, 128, 136, 248, 256, 264, 1016, 1024, 1032]


@pytest.mark.parametrize("dtype", ["float32", "int32", "bfloat16", "float16"])
def test_tma_eligible_shapes_with_ragged_tiles(dtype):
    for r in _tma_sizes(dtype):
        for c in _tma_sizes(dtype):
            a = workloads.matrix(r, c, dtype, seed=r * 131 + c)
            check(a, dtype, "tma")


@pytest.mark.parametrize("dtype", ["float32", "bfloat16"])
def test_unaligned_pointers_take_the_general_kernel(dtype):
    a = workloads.matrix(100, 200, dtype, seed=5)
    check(a, dtype, "auto", src_offset=1)


@pytest.mark.parametrize("kernel,shape", [("tma", (264, 136)), ("tile32", (67, 33)), ("tma", (1024, 8))])
def test_guard_bands_untouched(kernel, shape):
    rows, cols = shape
    a = workloads.matrix(rows, cols, "float32", seed=9)
    src = to_device(a, "float32")
    guard = 4096
    buf = torch.full((rows * cols + 2 * guard,), float("nan"), dtype=torch.float32, device="cuda")
    buf.view(torch.int32).fill_(0x5A5A5A5A)
    dst = buf[guard:guard + rows * cols].view(cols, rows)
    api.transpose(src, out=dst, kernel=kernel)
    torch.cuda.synchronize()
    host = buf.view(torch.int32).cpu().numpy()
    assert (host[:guard] == 0x5A5A5A5A).all() and (host[-guard:] == 0x5A5A5A5A).all()
    assert np.array_equal(host[guard:-guard].view(np.uint32).reshape(cols, rows), bits(oracle.transpose(a)))


def test_nan_payloads_and_negative_zero_survive():
    a = workloads.matrix(64, 128, "float32", seed=3)
    b = a.view(np.uint32)
    b[0, 0] = 0x7FC01234
    b[5, 7] = 0x80000000
    b[63, 127] = 0xFF800001
    check(a, "float32", "tma")
    check(a, "float32", "tile32")


def test_repeated_calls_identical():
    a = workloads.matrix(640, 384, "float32", seed=4)
    first = gpu_transpose(a, "float32", "tma")
    for _ in range(3):
        assert np.array_equal(gpu_transpose(a, "float32", "tma"), first)


def test_small_workload_int32_1024():
    a = workloads.small()
    check(a, "int32", "auto")
    check(a, "int32", "tile32")


def test_roofline_workload_float32_16384():
    """The full 16384x16384 float32 transpose, bit-exact against the oracle,
    in the launch configuration the benchmark times (AUTO -> TMA kernel)."""
    mat = workloads.roofline_matrix()
    src = to_device(mat, "float32")
    assert api.tma_eligible(src, torch.empty_like(src))
    out = api.transpose(src)
    back = api.transpose(out)  # involution, on the device
    torch.cuda.synchronize()
    api.stream_status()
    assert torch.equal(back.view(torch.int32), src.view(torch.int32))
    del back, src
    got = to_host_bits(out)
    del out
    want = oracle.transpose(mat).view(np.uint32)
    assert np.array_equal(got, want)


def test_precision_workload_bfloat16_8192():
    check(workloads.precision_matrix(), "bfloat16", "auto")


@pytest.mark.parametrize("dtype", ["float32", "bfloat16"])
def test_every_compiled_configuration(dtype):
    """Every configuration the autotuner may select is bit-exact, on shapes
    with ragged last tiles in both directions."""
    tdt = {"float32": torch.float32, "bfloat16": torch.bfloat16}[dtype]
    names = api.tune_configs("transpose", tdt)
    prev = api.tune_selected("transpose", tdt)
    step = 16 // workloads.ESIZE[dtype]
    shapes = [(step, step), (264, 136), (136, 264), (1000, 1024), (72, 4096)]
    shapes = [(r - r % step or step, c - c % step or step) for r, c in shapes]
    try:
        for i, name in enumerate(names):
            api.tune_select("transpose", tdt, i)
            for r, c in shapes:
                a = workloads.matrix(r, c, dtype, seed=r + 17 * c + i)
                check(a, dtype, "auto")
            # A stack of matrices (3-D tensor maps) through the same configuration.
            r, c = shapes[1]
            stack = np.stack([workloads.matrix(r, c, dtype, seed=900 + i + k) for k in range(3)])
            got = api.transpose_batched(to_device(stack, dtype))
            want = oracle.transpose_batched(stack)
            assert np.array_equal(to_host_bits(got), bits(want)), (name, stack.shape)
    finally:
        api.tune_select("transpose", tdt, prev)


def test_autotune_selects_a_valid_configuration():
    idx, name, ms = api.autotune("transpose", torch.float32, 2048, 2048, reps=3)
    assert 0 <= idx < len(api.tune_configs("transpose", torch.float32)) and ms > 0
    a = workloads.matrix(2048, 2048, "float32", seed=8)
    check(a, "float32", "auto")
    api.tune_select("transpose", torch.float32, 0)


@pytest.mark.parametrize("dtype", ["float32", "bfloat16"])
@pytest.mark.parametrize("rows,cols,lds,ldd", [
    (64, 64, 64, 64), (100, 37, 50, 120), (256, 128, 384, 264), (33, 65, 65, 33), (512, 512, 520, 776),
])
def test_strided_transpose_sub_blocks(dtype, rows, cols, lds, ldd):
    """Pitched transpose: the source block is rows x cols inside a row pitch
    lds, the destination block cols x rows inside a row pitch ldd; elements
    outside the destination block keep their canary value."""
    from paper_2605_13864_gb300 import _native as N
    full = workloads.matrix(rows, lds, dtype, seed=rows * 3 + lds)
    src = to_device(full, dtype)
    tdt = src.dtype
    canary = torch.full((cols, ldd), 0, dtype=torch.int16 if tdt in (torch.bfloat16, torch.float16)
                        else torch.int32, device="cuda")
    canary.fill_(0x3A3A)
    dst = canary.view(tdt)
    st = N.lib().optigpu_transpose_strided(src.data_ptr(), lds, dst.data_ptr(), ldd, rows, cols,
                                           api.dtype_code(tdt), torch.cuda.current_stream().cuda_stream)
    assert st == N.OK, N.lib().optigpu_last_error()
    torch.cuda.synchronize()
    got = to_host_bits(dst)
    want = oracle.transpose(np.ascontiguousarray(full[:, :cols]))
    want = want.view(np.uint32) if want.dtype == np.float32 else want
    assert np.array_equal(got[:, :rows], want)
    pad = got[:, rows:]
    if pad.size:
        assert (pad.view(np.uint16 if pad.dtype == np.uint16 else np.uint32) ==
                (0x3A3A if pad.dtype == np.uint16 else 0x3A3A)).all()
