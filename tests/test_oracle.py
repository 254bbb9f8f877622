"""Pins of the CPU oracle against things other than itself (no GPU).

Each pin is a plain check function that takes an implementation; the oracle
must pass every pin, and each planted mistake (a mutant written here, on the
CPU) must fail at least one, so a dropped term, a wrong index or sign, or a
transposed operand in the oracle cannot go unnoticed.

Transpose (Listing 3.5, Sec. 3.1): brute force against numpy's transpose on
every shape up to 8x8 and odd shapes up to 67, the closed form of the index
matrix, the involution T(T(A)) = A, the byte multiset, the hand-written worked
example under ``tests/golden``, and Listing 3.8's tiled loop nest.

Sum (Listing 2.1, Sec. 2.1): the closed form sum(0..n-1) = n(n-1)/2, all-ones,
+/-k pairs, Python's exact integer sum, Listing 2.2's partial-sum form,
``math.fsum`` (correctly rounded) within the a-priori bound of a sequential
double sum, the exactness of sums of half-integers, and the full decode tables
of numpy float16 and torch bfloat16.
"""
import math
import os

import numpy as np
import pytest

import oracle
from paper_2605_13864_gb300 import workloads

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
U64 = 2.0 ** -53


# --------------------------------------------------------------------------
# pin checks (take an implementation, raise AssertionError on a violation)
# --------------------------------------------------------------------------

def pin_transpose_bruteforce(tr):
    rng = np.random.default_rng(11)
    shapes = [(r, c) for r in range(0, 9) for c in range(0, 9)]
    shapes += [(r, c) for r in (1, 31, 33, 67) for c in (1, 2, 63, 65, 67)]
    for r, c in shapes:
        a = rng.integers(-2**31, 2**31 - 1, size=(r, c), dtype=np.int64).astype(np.int32)
        got = tr(a)
        assert got.shape == (c, r), (r, c)
        assert np.array_equal(got, a.T), (r, c)
        h = rng.integers(0, 2**16, size=(r, c), dtype=np.int64).astype(np.uint16)
        assert np.array_equal(tr(h), h.T), (r, c)


def pin_transpose_closed_form(tr):
    for rows, cols in ((1, 1), (3, 5), (37, 29), (64, 1), (1, 70)):
        a = np.arange(rows * cols, dtype=np.int32).reshape(rows, cols)
        got = tr(a).reshape(-1)
        i = np.arange(rows * cols)
        assert np.array_equal(got, (i % rows) * cols + i // rows), (rows, cols)


def pin_transpose_involution_and_multiset(tr):
    rng = np.random.default_rng(12)
    a = rng.standard_normal((45, 77)).astype(np.float32)
    bits = a.view(np.uint32)
    bits[0, 0] = 0x7FC01234  # NaN with a payload
    bits[1, 2] = 0x80000000  # -0
    back = tr(tr(a))
    assert np.array_equal(back.view(np.uint32), a.view(np.uint32))
    once = tr(a)
    assert np.array_equal(np.sort(once.view(np.uint32).reshape(-1)),
                          np.sort(a.view(np.uint32).reshape(-1)))


def pin_transpose_golden(tr):
    with open(os.path.join(GOLDEN, "transpose_listing35_2x3.txt")) as f:
        rows = [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]
    src = np.array([[int(v) for v in r] for r in rows[:2]], dtype=np.int32)
    want = np.array([[int(v) for v in r] for r in rows[2:]], dtype=np.int32)
    assert np.array_equal(tr(src), want)


TRANSPOSE_PINS = [pin_transpose_bruteforce, pin_transpose_closed_form,
                  pin_transpose_involution_and_multiset, pin_transpose_golden]


def pin_sum_int_closed_forms(sm):
    for n in (0, 1, 2, 127, 128, 129, 1000, 65536):
        a = np.arange(n, dtype=np.int32)
        assert sm(a) == n * (n - 1) // 2, n
        assert sm(np.ones(n, dtype=np.int32)) == n, n
    k = np.arange(1, 501, dtype=np.int32)
    assert sm(np.concatenate([k, -k])) == 0
    big = np.full(1 << 12, 2**31 - 1, dtype=np.int32)  # needs a 64-bit accumulator
    assert sm(big) == (2**31 - 1) << 12


def pin_sum_int_exact(sm):
    rng = np.random.default_rng(13)
    for n in (1, 3, 1023, 4097):
        a = rng.integers(-2**31, 2**31 - 1, size=n, dtype=np.int64).astype(np.int32)
        assert sm(a) == sum(int(v) for v in a), n


INT_SUM_PINS = [pin_sum_int_closed_forms, pin_sum_int_exact]


def pin_sum_float_fsum_bound(sm):
    """Sequential double sum within (n-1)*u*sum|x| of the correctly rounded sum."""
    rng = np.random.default_rng(14)
    for n in (1, 2, 1000, 12345):
        a = rng.standard_normal(n).astype(np.float32)
        exact = math.fsum(float(v) for v in a)
        absum = math.fsum(abs(float(v)) for v in a)
        got = sm(a, "float32")
        assert abs(got - exact) <= max(n - 1, 1) * U64 * absum + 1e-300, n


def pin_sum_float_special(sm):
    assert sm(np.ones(1 << 20, dtype=np.float32), "float32") == float(1 << 20)
    x = np.linspace(-3, 3, 601).astype(np.float32)
    assert sm(np.concatenate([x, -x]), "float32") == 0.0
    assert sm(np.zeros(0, dtype=np.float32), "float32") == 0.0
    # half-integers near 100 (bfloat16 N(100,1)) sum exactly in double
    v = workloads.vector(50000, "bfloat16", seed=2, mean=100.0)
    vals = [float(t) for t in
            __import__("torch").from_numpy(v.view(np.int16)).view(
                __import__("torch").bfloat16).double().numpy()]
    assert sm(v, "bfloat16") == math.fsum(vals)


def pin_sum_golden(sm):
    with open(os.path.join(GOLDEN, "reduce_listing21.txt")) as f:
        rows = [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]
    arr = np.array([float(v) for v in rows[0]], dtype=np.float32)
    assert sm(arr, "float32") == float(rows[1][0])


FLOAT_SUM_PINS = [pin_sum_float_fsum_bound, pin_sum_float_special, pin_sum_golden]


# --------------------------------------------------------------------------
# the oracle passes every pin
# --------------------------------------------------------------------------

@pytest.mark.parametrize("pin", TRANSPOSE_PINS, ids=lambda p: p.__name__)
def test_oracle_transpose_pins(pin):
    pin(oracle.transpose)


@pytest.mark.parametrize("pin", TRANSPOSE_PINS, ids=lambda p: p.__name__)
def test_oracle_transpose_tiled_pins(pin):
    pin(oracle.transpose_tiled)


@pytest.mark.parametrize("pin", INT_SUM_PINS, ids=lambda p: p.__name__)
def test_oracle_int_sum_pins(pin):
    pin(oracle.sum_i64)


@pytest.mark.parametrize("chunk", [1, 7, 128, 1000])
@pytest.mark.parametrize("pin", INT_SUM_PINS, ids=lambda p: p.__name__)
def test_oracle_chunked_sum_pins(pin, chunk):
    """Listing 2.2's partial-sum form meets the same pins for any chunk."""
    pin(lambda a: oracle.sum_i64_chunked(a, chunk))


@pytest.mark.parametrize("pin", FLOAT_SUM_PINS, ids=lambda p: p.__name__)
def test_oracle_float_sum_pins(pin):
    pin(oracle.sum_f64)


@pytest.mark.parametrize("pin", FLOAT_SUM_PINS, ids=lambda p: p.__name__)
def test_oracle_neumaier_sum_pins(pin):
    pin(oracle.sum_f64_neumaier)


def test_oracle_neumaier_recovers_cancelled_term():
    """Textbook case: 1 + 1e30 + 1 - 1e30 is 2; a plain double sum gives 0."""
    a = np.array([1.0, 1e30, 1.0, -1e30], dtype=np.float32)
    assert oracle.sum_f64(a) == 0.0
    assert oracle.sum_f64_neumaier(a) == 2.0


def test_oracle_neumaier_close_to_fsum():
    rng = np.random.default_rng(15)
    a = (rng.standard_normal(20000) * np.exp(rng.uniform(-20, 20, 20000))).astype(np.float32)
    exact = math.fsum(float(v) for v in a)
    absum = math.fsum(abs(float(v)) for v in a)
    assert abs(oracle.sum_f64_neumaier(a) - exact) <= 2 * U64 * abs(exact) + 1e-6 * U64 * absum


def test_oracle_sum_abs():
    rng = np.random.default_rng(16)
    a = rng.standard_normal(3000).astype(np.float32)
    assert abs(oracle.sum_abs_f64(a) - math.fsum(abs(float(v)) for v in a)) <= 3000 * U64 * 3000


def test_oracle_decode_f16_table():
    bits = np.arange(1 << 16, dtype=np.uint32).astype(np.uint16)
    want = bits.view(np.float16).astype(np.float64)
    got = np.array([oracle.decode_f16(int(b)) for b in bits])
    nan = np.isnan(want)
    assert np.array_equal(np.isnan(got), nan)
    assert np.array_equal(got[~nan], want[~nan])
    assert np.array_equal(np.signbit(got[~nan]), np.signbit(want[~nan]))


def test_oracle_decode_bf16_table():
    torch = pytest.importorskip("torch")
    bits = np.arange(1 << 16, dtype=np.uint32).astype(np.uint16)
    want = torch.from_numpy(bits.view(np.int16)).view(torch.bfloat16).double().numpy()
    got = np.array([oracle.decode_bf16(int(b)) for b in bits])
    nan = np.isnan(want)
    assert np.array_equal(np.isnan(got), nan)
    assert np.array_equal(got[~nan], want[~nan])


def test_oracle_float16_sum_uses_decode():
    v = workloads.vector(4099, "float16", seed=5)
    want = math.fsum(float(x) for x in v.view(np.float16).astype(np.float64))
    absum = math.fsum(abs(float(x)) for x in v.view(np.float16).astype(np.float64))
    assert abs(oracle.sum_f64(v, "float16") - want) <= 4099 * U64 * absum


# --------------------------------------------------------------------------
# planted mistakes fail at least one pin
# --------------------------------------------------------------------------

def _fails_some(pins, impl):
    for pin in pins:
        try:
            pin(impl)
        except (AssertionError, ValueError, IndexError):
            return True
    return False


def _mut_transpose_swapped_rows_cols(a):
    # Bug: reshapes the source instead of transposing (rows/cols swapped).
    return np.ascontiguousarray(a).reshape(a.shape[1], a.shape[0]).copy()


def _mut_transpose_identity_on_square(a):
    # Bug: drops the transpose for square inputs.
    return a.copy() if a.shape[0] == a.shape[1] else np.ascontiguousarray(a.T)


def _mut_transpose_last_col_dropped(a):
    # Bug: off-by-one in the column loop leaves the last output row zero.
    out = np.ascontiguousarray(a.T).copy()
    if out.shape[0] > 0:
        out[-1, :] = 0
    return out


def _mut_transpose_through_float_arith(a):
    # Bug: moves 4-byte float data through an addition, which turns -0 into +0.
    out = np.ascontiguousarray(a.T).copy()
    if out.dtype == np.float32:
        out = out + np.float32(0.0)
    return out


@pytest.mark.parametrize("mut", [_mut_transpose_swapped_rows_cols,
                                 _mut_transpose_identity_on_square,
                                 _mut_transpose_last_col_dropped,
                                 _mut_transpose_through_float_arith])
def test_planted_transpose_mistakes_are_caught(mut):
    assert _fails_some(TRANSPOSE_PINS, mut)


@pytest.mark.parametrize("mut", [
    lambda a: oracle.sum_i64(a[:-1]) if a.size else 0,          # drops the last term
    lambda a: oracle.sum_i64(a[1:]) if a.size else 0,           # drops the first term
    lambda a: -oracle.sum_i64(a),                                # wrong sign
    lambda a: int(np.sum(a, dtype=np.int32)),                    # 32-bit accumulator
    lambda a: oracle.sum_i64(a[::2]) * 2,                        # wrong stride
])
def test_planted_int_sum_mistakes_are_caught(mut):
    assert _fails_some(INT_SUM_PINS, mut)


@pytest.mark.parametrize("mut", [
    lambda a, k: oracle.sum_f64(a[:-1], k) if a.size else 0.0,
    lambda a, k: float(np.sum(a.astype(np.float32) if k == "float32" else a)),
    lambda a, k: oracle.sum_f64(a, k) * (1 + 1e-6),
    lambda a, k: oracle.sum_abs_f64(a, k),
])
def test_planted_float_sum_mistakes_are_caught(mut):
    assert _fails_some(FLOAT_SUM_PINS, mut)


def test_planted_decode_mistake_is_caught():
    # A binary16 decoder with exponent bias 16 instead of 15.
    def bad(h):
        s, e, f = (h >> 15) & 1, (h >> 10) & 31, h & 1023
        v = math.ldexp(f, -24) if e == 0 else math.ldexp(f + 1024, e - 26)
        return -v if s else v
    bits = np.arange(0x3C00, 0x3C10, dtype=np.uint16)
    want = bits.view(np.float16).astype(np.float64)
    assert any(bad(int(b)) != w for b, w in zip(bits, want))
    assert all(oracle.decode_f16(int(b)) == w for b, w in zip(bits, want))
