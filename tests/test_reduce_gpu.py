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
    # A 1.0 heads every chunk and 2^-27 fills the rest.  The thread that reads
    # the 1.0 keeps a running FP32 sum near 1; each of its later 16-byte
    # vectors of small values sums to 2^-25, under half an ulp of 1, so plain
    # mode drops all 15 of them (60 * 2^-27 per chunk), while Neumaier's term
    # keeps them.  Both modes lose the same 3 * 2^-27 per chunk inside the
    # first vector, whose pairwise tree is plain FP32 in either mode.
    chunks = 4
    t = 2.0 ** -27
    a = np.full(chunks * CHUNK, t, dtype=np.float32)
    a[::CHUNK] = 1.0
    want = oracle.sum_f64(a)
    assert want == chunks + (a.size - chunks) * t  # exact in FP64
    got_c = gpu_sum(a, "float32", compensated=True)
    got_p = gpu_sum(a, "float32", compensated=False)
    assert want - got_p == chunks * 63 * t
    assert want - got_c == chunks * 3 * t


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


def test_graph_replay_after_workspace_growth():
    """A sum captured into a CUDA graph stays correct after a larger sum on the
    same stream made the library grow that stream's workspace: the workspace
    the graph was captured with is retired, not freed, so replays still find
    their counter and partials there."""
    s = torch.cuda.Stream()
    small = workloads.vector(3 * CHUNK + 5, "float32", seed=91)
    # A new workspace holds at least 64 KiB (8160 partials); this sum needs more.
    big_n = 8200 * CHUNK + 1
    d_small = to_device(small, "float32")
    d_big = torch.ones(big_n, dtype=torch.float32, device="cuda")
    out_g = torch.full((), -1.0, dtype=torch.float64, device="cuda")
    out_b = torch.full((), -1.0, dtype=torch.float64, device="cuda")
    with torch.cuda.stream(s):
        api.reduce_reserve(small.size)
        api.reduce_sum(d_small, out=out_g)  # device facts and workspace ready before the capture
    torch.cuda.synchronize()
    direct = out_g.item()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        api.reduce_sum(d_small, out=out_g)
    with torch.cuda.stream(s):
        api.reduce_sum(d_big, out=out_b)  # needs a larger workspace on the same stream
    # Churn device memory so that a freed workspace would likely be handed out again.
    junk = [torch.full((1 << 20,), 7, dtype=torch.int32, device="cuda") for _ in range(8)]
    torch.cuda.synchronize()
    for _ in range(3):
        out_g.fill_(-1.0)
        g.replay()
        torch.cuda.synchronize()
        assert out_g.item() == direct
    ref = oracle.reduce_reference(small)
    assert abs(direct - ref["f64"]) <= REL_TOL * ref["abs"]
    assert out_b.item() == float(big_n)  # ones: every partial and the total are exact
    with torch.cuda.stream(s):
        api.stream_status()
    del junk, g
