"""Pins of the oracle's neighbouring problems against things other than
itself (no GPU): pitched, batched and in-place transposes (numpy slicing and
transposes, the involution), inclusive prefix sums (closed forms, first
differences, numpy's cumulative sum in float64 within the sequential-sum
bound, the total against the sum oracle's pins), per-segment sums, and the
integer histogram (numpy's bincount, totals, closed forms).  Planted mistakes
fail at least one pin.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2605_13864_gb300 import workloads

U64 = 2.0 ** -53


# ---------------------------------------------------------------- transposes

def pin_strided(impl):
    rng = np.random.default_rng(31)
    for rows, cols, lds, ldd in ((1, 1, 1, 1), (3, 5, 7, 4), (37, 29, 40, 50), (8, 64, 64, 8)):
        full = rng.integers(-2**31, 2**31 - 1, size=(rows, lds), dtype=np.int64).astype(np.int32)
        dst = np.full(cols * ldd, 77, dtype=np.int32)
        impl(full.reshape(-1), lds, dst, ldd, rows, cols)
        d2 = dst.reshape(cols, ldd)
        assert np.array_equal(d2[:, :rows], full[:, :cols].T)
        assert (d2[:, rows:] == 77).all()


def pin_batched(impl):
    rng = np.random.default_rng(32)
    for b, r, c in ((1, 1, 1), (3, 4, 5), (5, 33, 17)):
        a = rng.integers(0, 2**16, size=(b, r, c), dtype=np.int64).astype(np.uint16)
        got = impl(a)
        assert np.array_equal(got, np.transpose(a, (0, 2, 1)))


def pin_inplace(impl):
    rng = np.random.default_rng(33)
    for n in (0, 1, 2, 3, 8, 31, 64):
        a = rng.standard_normal((n, n)).astype(np.float32)
        want = a.T.copy()
        got = impl(a.copy())
        assert np.array_equal(got.view(np.uint32), want.view(np.uint32))
        assert np.array_equal(impl(impl(a.copy())).view(np.uint32), a.view(np.uint32))


@pytest.mark.parametrize("pin,impl", [
    (pin_strided, lambda src, lds, dst, ldd, r, c: oracle.transpose_strided(src, lds, dst, ldd, r, c)),
    (pin_batched, oracle.transpose_batched),
    (pin_inplace, oracle.transpose_inplace),
])
def test_oracle_transpose_variants(pin, impl):
    pin(impl)


def test_planted_transpose_variant_mistakes():
    def bad_strided(src, lds, dst, ldd, r, c):   # uses cols as the source pitch
        oracle.transpose_strided(src, c, dst, ldd, r, c)

    def bad_batched(a):                          # forgets the batch stride
        return np.stack([a[0].T] * a.shape[0])

    def bad_inplace(a):                          # swaps only half the pairs
        n = a.shape[0]
        for i in range(n):
            for j in range(i + 1, n, 2):
                a[i, j], a[j, i] = a[j, i], a[i, j]
        return a
    for pin, bad in ((pin_strided, bad_strided), (pin_batched, bad_batched), (pin_inplace, bad_inplace)):
        with pytest.raises(AssertionError):
            pin(bad)


# -------------------------------------------------------------------- scans

def pin_scan_int(sc):
    for n in (0, 1, 2, 1000, 65537):
        a = np.arange(n, dtype=np.int32)
        i = np.arange(n, dtype=np.int64)
        assert np.array_equal(sc(a), i * (i + 1) // 2)
    rng = np.random.default_rng(34)
    a = rng.integers(-2**31, 2**31 - 1, size=5000, dtype=np.int64).astype(np.int32)
    out = sc(a)
    assert out[-1] == sum(int(v) for v in a)              # exact total
    assert np.array_equal(np.diff(out), a[1:].astype(np.int64))  # first differences
    assert out[0] == a[0]


def pin_scan_float(sc):
    rng = np.random.default_rng(35)
    a = rng.standard_normal(20000).astype(np.float32)
    got = sc(a, "float32")
    ref = np.cumsum(a.astype(np.float64))      # numpy's own float64 cumulative sum
    absum = np.cumsum(np.abs(a.astype(np.float64)))
    k = np.arange(1, a.size + 1)
    assert (np.abs(got - ref) <= 2 * k * U64 * absum).all()
    assert got[-1] == pytest.approx(math.fsum(float(v) for v in a), abs=a.size * U64 * absum[-1])
    h = workloads.vector(4096, "bfloat16", seed=2, mean=100.0)  # half-integers: exact
    hv = [float(x) for x in __import__("torch").from_numpy(h.view(np.int16)).view(
        __import__("torch").bfloat16).double().numpy()]
    assert np.array_equal(sc(h, "bfloat16"), np.cumsum(np.array(hv)))


def test_oracle_scan_pins():
    pin_scan_int(oracle.scan)
    pin_scan_float(oracle.scan)


def test_planted_scan_mistakes():
    with pytest.raises(AssertionError):          # exclusive instead of inclusive
        pin_scan_int(lambda a: np.concatenate([[0], oracle.scan(a)[:-1]]).astype(np.int64) if a.size else oracle.scan(a))
    with pytest.raises(AssertionError):          # 32-bit running sum
        pin_scan_int(lambda a: np.cumsum(a, dtype=np.int32).astype(np.int64))
    with pytest.raises(AssertionError):          # float32 running sum
        pin_scan_float(lambda a, k: np.cumsum(a.astype(np.float32) if k == "float32" else a, dtype=np.float32).astype(np.float64) * (1 + 1e-6))


# ----------------------------------------------------------- segmented sums

def test_oracle_segmented_sums():
    rng = np.random.default_rng(36)
    a = rng.integers(-1000, 1001, size=10000, dtype=np.int32)
    offs = [0, 0, 1, 17, 17, 4096, 9999, 10000]
    got = oracle.segmented_sums(a, offs)
    assert got == [int(a[offs[s]:offs[s + 1]].astype(np.int64).sum()) for s in range(len(offs) - 1)]
    assert sum(got) == oracle.sum_i64(a)
    f = rng.standard_normal(5000).astype(np.float32)
    fs = oracle.segmented_sums(f, [0, 100, 5000])
    for s, (lo, hi) in enumerate(((0, 100), (100, 5000))):
        seg = [float(v) for v in f[lo:hi]]
        assert abs(fs[s] - math.fsum(seg)) <= len(seg) * U64 * math.fsum(abs(v) for v in seg)


# ---------------------------------------------------------------- histogram

def pin_histogram(h):
    rng = np.random.default_rng(37)
    a = rng.integers(-50, 150, size=100000, dtype=np.int32)
    got = h(a, 0, 1, 100)
    assert np.array_equal(got, np.bincount(a[(a >= 0) & (a < 100)], minlength=100).astype(np.int64))
    got = h(a, -50, 7, 29)   # bins of 7 covering [-50, 153)
    want = np.bincount((a.astype(np.int64) + 50) // 7, minlength=29)[:29]
    assert np.array_equal(got, want)
    assert got.sum() == a.size
    r = np.arange(1000, dtype=np.int32)
    assert (h(r, 0, 10, 100) == 10).all()
    assert h(np.full(5, -1, dtype=np.int32), 0, 1, 3).sum() == 0
    assert h(np.array([2**31 - 1, -2**31], dtype=np.int32), -2**31, 2**31, 2).tolist() == [1, 1]
    # lo outside int32 and widths of 2^32 and more: the bin of x is (x - lo) // width in exact
    # integer arithmetic.
    full = rng.integers(-2**31, 2**31, size=20000, dtype=np.int64).astype(np.int32)
    for lo, w, nb in ((-2**35, 2**24, 4096), (-2**33, 3 * 2**30 + 7, 8), (-2**32, 2**32, 3),
                      (-2**34, 2**20, 20000)):
        d = full.astype(np.int64) - lo
        want = np.bincount(d // w, minlength=nb)[:nb]
        assert np.array_equal(h(full, lo, w, nb), want), (lo, w, nb)
    assert h(full, 2**31, 1, 64).sum() == 0                 # every int32 lies below lo
    # x - lo lies in [2^31, 3 * 2^31): negative values in bin 0, the rest in bin 1.
    assert h(full, -2**32, 2**32, 3).tolist() == [int((full < 0).sum()), int((full >= 0).sum()), 0]


def test_oracle_histogram_pins():
    pin_histogram(oracle.histogram_i32)


def test_planted_histogram_mistakes():
    with pytest.raises(AssertionError):          # off-by-one bin
        pin_histogram(lambda a, lo, w, n: np.roll(oracle.histogram_i32(a, lo, w, n), 1))
    with pytest.raises(AssertionError):          # counts values below lo into bin 0
        pin_histogram(lambda a, lo, w, n: oracle.histogram_i32(np.maximum(a, lo).astype(np.int32), lo, w, n))
