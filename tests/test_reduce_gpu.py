"""GPU parity of the sum reduction (Listing 2.1, Sec. 2.1) against the oracle.

int32 sums are compared bit-exactly with the oracle's int64 sum.  Float sums
(float32, bfloat16, float16; plain and compensated) must lie within
1e-6 * sum|x| of the oracle's FP64 sum, and every error is printed.  The
summation structure is fixed by (n, dtype, mode), so repeated calls and calls
on an unaligned copy of the same data must agree bit for bit.  Sizes span the
16384-element chunk, the 16-byte vector, ragged tails and the empty input, up
to the full 2^28-element vectors.
"""
import math

import numpy as np
import pytest

import oracle
from gpu_util import require_gpu, to_device, torch
from paper_2605_13864_gb300 import api, workloads

pytestmark = pytest.mark.gpu

REL_TOL = 1e-6
CHUNK = 16384
SIZES = [0, 1, 2, 3, 4, 5, 7, 8, 9, 15, 16, 17, 255, 256, 257, 4095, 4096, 4097,
         CHUNK - 1, CHUNK, CHUNK + 1, 2 * CHUNK + 7, 3 * CHUNK + 5, 100_000, 1 << 20, (1 << 20) + 3]


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def gpu_sum(a, dtype, compensated=False, offset=0):
    d = to_device(a, dtype, offset)
    out = api.reduce_sum(d, compensated=compensated)
    torch.cuda.synchronize()
    api.stream_status()
    return out.item()


def float_error(got, a, dtype):
    ref = oracle.reduce_reference(a, dtype)
    err = abs(got - ref["f64"])
    return err, ref["abs"]


@pytest.mark.parametrize("n", SIZES)
def test_int32_exact(n):
    rng = np.random.default_rng(n + 1)
    a = rng.integers(-2**31, 2**31 - 1, size=n, dtype=np.int64).astype(np.int32)
    assert gpu_sum(a, "int32") == oracle.sum_i64(a)


def test_int32_closed_forms():
    for n in (1, 1000, CHUNK + 3, 65536):
        assert gpu_sum(np.arange(n, dtype=np.int32), "int32") == n * (n - 1) // 2
    big = np.full(3 * CHUNK + 11, 2**31 - 1, dtype=np.int32)
    assert gpu_sum(big, "int32") == (2**31 - 1) * big.size


def test_small_workload_int32_1024():
    a = workloads.small()
    assert gpu_sum(a, "int32") == oracle.sum_i64(a)
    assert gpu_sum(a, "int32", offset=1) == oracle.sum_i64(a)


@pytest.mark.parametrize("compensated", [False, True])
@pytest.mark.parametrize("dtype", ["float32", "bfloat16", "float16"])
def test_float_sizes_within_bound(dtype, compensated):
    worst = 0.0
    for n in SIZES:
        a = workloads.vector(n, dtype, seed=1000 + n)
        got = gpu_sum(a, dtype, compensated)
        err, absum = float_error(got, a, dtype)
        assert err <= REL_TOL * absum + 1e-300, (n, got, err, absum)
        worst = max(worst, err / absum if absum else 0.0)
    print(f"{dtype} compensated={compensated}: worst relative error {worst:.3e}")


@pytest.mark.parametrize("compensated", [False, True])
@pytest.mark.parametrize("dtype", ["float32", "bfloat16", "float16", "int32"])
def test_unaligned_and_repeated_calls_bit_identical(dtype, compensated):
    n = 5 * CHUNK + 333
    a = workloads.vector(n, dtype, seed=77)
    first = gpu_sum(a, dtype, compensated)
    assert gpu_sum(a, dtype, compensated) == first
    assert gpu_sum(a, dtype, compensated, offset=1) == first
    assert gpu_sum(a, dtype, compensated, offset=3) == first


def test_float_special_values():
    assert gpu_sum(np.ones(1 << 20, dtype=np.float32), "float32") == float(1 << 20)
    a = np.ones(CHUNK * 3, dtype=np.float32)
    a[CHUNK + 5] = np.nan
    assert math.isnan(gpu_sum(a, "float32"))
    a[CHUNK + 5] = np.inf
    assert gpu_sum(a, "float32") == math.inf
    assert gpu_sum(np.zeros(0, dtype=np.float32), "float32") == 0.0


def test_compensated_recovers_small_terms():
    # 1 + many tiny terms: plain FP32 per-thread sums drop them, Neumaier keeps them.
    n = CHUNK
    a = np.full(n, 2.0 ** -24, dtype=np.float32)
    a[::256] = 1.0  # thread 0 of every 256-vector stride sees a 1 first
    want = oracle.sum_f64(a)
    got_c = gpu_sum(a, "float32", compensated=True)
    got_p = gpu_sum(a, "float32", compensated=False)
    assert abs(got_c - want) <= abs(got_p - want)
    assert abs(got_c - want) <= 1e-7 * oracle.sum_abs_f64(a)


def test_roofline_workload_float32_2p28():
    """The full 2^28-element float32 vector in the benchmark's configuration."""
    v = workloads.roofline_vector()
    d = to_device(v, "float32")
    ref = oracle.reduce_reference(v, "float32")
    for comp in (False, True):
        got = api.reduce_sum(d, compensated=comp).item()
        err = abs(got - ref["f64"])
        print(f"float32 2^28 compensated={comp}: sum {got!r} oracle {ref['f64']!r} "
              f"error {err:.3e} = {err / ref['abs']:.3e} * sum|x|")
        assert err <= REL_TOL * ref["abs"]
    api.stream_status()


@pytest.mark.parametrize("dtype", ["bfloat16", "float16"])
def test_precision_workload_2p28(dtype):
    vb, vh = workloads.precision_vectors()
    v = vb if dtype == "bfloat16" else vh
    del vb, vh
    d = to_device(v, dtype)
    ref = oracle.reduce_reference(v, dtype)
    # N(100,1) values rounded to 16 bits are multiples of 2^-4 (or coarser) and
    # their sum stays far below 2^53: the FP64 sequential oracle is exact.
    assert ref["f64"] == ref["f64_neumaier"]
    for comp in (False, True):
        got = api.reduce_sum(d, compensated=comp).item()
        err = abs(got - ref["f64"])
        print(f"{dtype} 2^28 N(100,1) compensated={comp}: error {err:.3e} = "
              f"{err / ref['abs']:.3e} * sum|x|")
        assert err <= REL_TOL * ref["abs"]
    api.stream_status()
