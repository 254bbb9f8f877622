"""CPU oracle for the transpose and the sum reduction -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The library never does, and the two
share no code: the oracle is plain C (``optigpu_oracle.c``) compiled with gcc
into ``oracle/_build/liboptigpu_oracle.so`` and called through ctypes with
numpy arrays.

Definitions followed (thesis arxiv 2605.13864):

* ``transpose`` -- Listing 3.5 (Sec. 3.1): ``out[x][y] = in[y][x]``; for a
  ``rows x cols`` row-major input this is ``dst[c, r] = src[r, c]``.
* ``transpose_tiled`` -- Listing 3.8 (Sec. 3.2): the same result through the
  32x32 tile loop nest.
* ``sum_i64`` / ``sum_f64`` -- Listing 2.1 (Sec. 2.1): ``reduce_sum(N, A)``
  as a sequential loop, in int64 for int32 input and in double for float
  input (each element widened exactly).
* ``sum_f64_neumaier`` / ``sum_abs_f64`` -- the compensated double sum and
  ``sum |x|`` used to report errors.
* ``sum_i64_chunked`` -- Listing 2.2 (Sec. 2.2.1): per-chunk partial sums,
  then a sequential sum of the partials.
* ``transpose_strided`` / ``transpose_batched`` / ``transpose_inplace`` --
  Listing 3.5 on pitched sub-blocks, on a batch of matrices, and in place
  (swap a[i][j] with a[j][i] for i < j).
* ``scan`` -- inclusive prefix sums (Sec. 9 future work): Listing 2.1's
  loop keeping every intermediate sum, int64 for int32 input, double for
  float input.
* ``segmented_sums`` -- ``sum_i64`` / ``sum_f64`` per segment.
* ``histogram_i32`` -- counts of int32 values in bins of an integer width
  (Sec. 9 future work).

Pins against things other than the oracle itself live in
``tests/test_oracle.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "optigpu_oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "liboptigpu_oracle.so")

_lock = threading.Lock()
_lib = None

# The oracle's own element-kind numbering (see optigpu_oracle.c).
_KIND = {"int32": 0, "float32": 1, "bfloat16": 2, "float16": 3}


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (``-O2``, no vector ISA flags)."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    stale = (not os.path.exists(_LIB_PATH)
             or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC))
    if force or stale:
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared",
               "-fno-fast-math", "-ffp-contract=off", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        i64, vp, dbl, ci = ctypes.c_int64, ctypes.c_void_p, ctypes.c_double, ctypes.c_int
        lib.oracle_transpose.argtypes = [vp, vp, i64, i64, i64]
        lib.oracle_transpose.restype = None
        lib.oracle_transpose_tiled.argtypes = [vp, vp, i64, i64, i64]
        lib.oracle_transpose_tiled.restype = None
        lib.oracle_sum_i32.argtypes = [vp, i64]
        lib.oracle_sum_i32.restype = i64
        lib.oracle_sum_i32_chunked.argtypes = [vp, i64, i64]
        lib.oracle_sum_i32_chunked.restype = i64
        for name in ("oracle_sum_f64", "oracle_sum_f64_neumaier", "oracle_sum_abs_f64"):
            fn = getattr(lib, name)
            fn.argtypes = [vp, i64, ci]
            fn.restype = dbl
        lib.oracle_transpose_strided.argtypes = [vp, i64, vp, i64, i64, i64, i64]
        lib.oracle_transpose_strided.restype = None
        lib.oracle_transpose_batched.argtypes = [vp, i64, vp, i64, i64, i64, i64, i64]
        lib.oracle_transpose_batched.restype = None
        lib.oracle_transpose_inplace.argtypes = [vp, i64, i64]
        lib.oracle_transpose_inplace.restype = None
        lib.oracle_scan_i32.argtypes = [vp, i64, vp]
        lib.oracle_scan_i32.restype = None
        lib.oracle_scan_f64.argtypes = [vp, i64, ci, vp]
        lib.oracle_scan_f64.restype = None
        lib.oracle_histogram_i32.argtypes = [vp, i64, i64, i64, i64, vp]
        lib.oracle_histogram_i32.restype = None
        lib.oracle_decode_f16.argtypes = [ctypes.c_uint16]
        lib.oracle_decode_f16.restype = dbl
        lib.oracle_decode_bf16.argtypes = [ctypes.c_uint16]
        lib.oracle_decode_bf16.restype = dbl
        _lib = lib
        return lib


def _as_c(a: np.ndarray) -> np.ndarray:
    return np.ascontiguousarray(a)


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def kind_of(a: np.ndarray, dtype: str | None = None) -> str:
    """Element kind of a numpy array; 16-bit arrays need ``dtype`` because
    numpy has no bfloat16 (bfloat16 data is carried as uint16 bit patterns)."""
    if dtype is not None:
        return dtype
    if a.dtype == np.int32:
        return "int32"
    if a.dtype == np.float32:
        return "float32"
    if a.dtype == np.float16:
        return "float16"
    raise TypeError(f"oracle: pass dtype= for arrays of {a.dtype}")


def transpose(src: np.ndarray) -> np.ndarray:
    """``dst[c, r] = src[r, c]`` for a 2-D array of any element size."""
    src = _as_c(src)
    if src.ndim != 2:
        raise ValueError("oracle.transpose expects a 2-D array")
    rows, cols = src.shape
    dst = np.empty((cols, rows), dtype=src.dtype)
    _load().oracle_transpose(_ptr(src), _ptr(dst), rows, cols, src.dtype.itemsize)
    return dst


def transpose_tiled(src: np.ndarray) -> np.ndarray:
    """Listing 3.8's 32x32 tiled loop nest; same result as ``transpose``."""
    src = _as_c(src)
    rows, cols = src.shape
    if src.dtype.itemsize > 8:
        raise ValueError("element size above 8 bytes")
    dst = np.empty((cols, rows), dtype=src.dtype)
    _load().oracle_transpose_tiled(_ptr(src), _ptr(dst), rows, cols, src.dtype.itemsize)
    return dst


def sum_i64(a: np.ndarray) -> int:
    """Exact int64 sum of int32 values (Listing 2.1 in integer arithmetic)."""
    a = _as_c(a).reshape(-1)
    if a.dtype != np.int32:
        raise TypeError("sum_i64 expects int32")
    return int(_load().oracle_sum_i32(_ptr(a), a.size))


def sum_i64_chunked(a: np.ndarray, chunk: int = 128) -> int:
    """Listing 2.2's partial-sum form with ``chunk``-element chunks."""
    a = _as_c(a).reshape(-1)
    if a.dtype != np.int32:
        raise TypeError("sum_i64_chunked expects int32")
    return int(_load().oracle_sum_i32_chunked(_ptr(a), a.size, chunk))


def _float_call(fn_name: str, a: np.ndarray, dtype: str | None) -> float:
    kind = kind_of(a, dtype)
    a = _as_c(a).reshape(-1)
    return float(getattr(_load(), fn_name)(_ptr(a), a.size, _KIND[kind]))


def sum_f64(a: np.ndarray, dtype: str | None = None) -> float:
    """Sequential double sum of the exactly widened elements."""
    return _float_call("oracle_sum_f64", a, dtype)


def sum_f64_neumaier(a: np.ndarray, dtype: str | None = None) -> float:
    """Neumaier-compensated double sum of the exactly widened elements."""
    return _float_call("oracle_sum_f64_neumaier", a, dtype)


def sum_abs_f64(a: np.ndarray, dtype: str | None = None) -> float:
    """Sequential double sum of |x|, the scale of the error bound."""
    return _float_call("oracle_sum_abs_f64", a, dtype)


def decode_f16(bits: int) -> float:
    return float(_load().oracle_decode_f16(bits))


def decode_bf16(bits: int) -> float:
    return float(_load().oracle_decode_bf16(bits))


def reduce_reference(a: np.ndarray, dtype: str | None = None) -> dict:
    """Everything a float or integer sum is checked against.

    int32 input: ``{"exact": int}``.  Float input: the sequential double sum,
    its Neumaier twin and ``sum |x|``.
    """
    kind = kind_of(a, dtype)
    if kind == "int32":
        return {"kind": kind, "exact": sum_i64(a)}
    return {"kind": kind,
            "f64": sum_f64(a, kind),
            "f64_neumaier": sum_f64_neumaier(a, kind),
            "abs": sum_abs_f64(a, kind)}


def transpose_strided(src: np.ndarray, lds: int, dst: np.ndarray, ldd: int, rows: int, cols: int) -> None:
    """In place into ``dst`` (flat, pitch ``ldd``): dst[x*ldd + y] = src[y*lds + x]."""
    src = _as_c(src)
    if not dst.flags.c_contiguous:
        raise ValueError("dst must be contiguous")
    _load().oracle_transpose_strided(_ptr(src), lds, _ptr(dst), ldd, rows, cols, src.dtype.itemsize)


def transpose_batched(src: np.ndarray) -> np.ndarray:
    """(batch, rows, cols) -> (batch, cols, rows), each matrix transposed."""
    src = _as_c(src)
    b, r, c = src.shape
    dst = np.empty((b, c, r), dtype=src.dtype)
    _load().oracle_transpose_batched(_ptr(src), r * c, _ptr(dst), r * c, b, r, c, src.dtype.itemsize)
    return dst


def transpose_inplace(a: np.ndarray) -> np.ndarray:
    """Transposes the square array ``a`` in place (and returns it)."""
    if a.ndim != 2 or a.shape[0] != a.shape[1] or not a.flags.c_contiguous:
        raise ValueError("transpose_inplace expects a contiguous square array")
    _load().oracle_transpose_inplace(_ptr(a), a.shape[0], a.dtype.itemsize)
    return a


def scan(a: np.ndarray, dtype: str | None = None) -> np.ndarray:
    """Inclusive prefix sums: int64 for int32 input, float64 for float input."""
    kind = kind_of(a, dtype)
    a = _as_c(a).reshape(-1)
    if kind == "int32":
        out = np.empty(a.size, dtype=np.int64)
        _load().oracle_scan_i32(_ptr(a), a.size, _ptr(out))
    else:
        out = np.empty(a.size, dtype=np.float64)
        _load().oracle_scan_f64(_ptr(a), a.size, _KIND[kind], _ptr(out))
    return out


def segmented_sums(a: np.ndarray, offsets, dtype: str | None = None) -> list:
    """Sum of every segment a[offsets[s]:offsets[s+1]] (ints exact, floats in
    double), each by the same sequential loop as sum_i64 / sum_f64."""
    kind = kind_of(a, dtype)
    a = _as_c(a).reshape(-1)
    out = []
    for s in range(len(offsets) - 1):
        seg = a[offsets[s]:offsets[s + 1]]
        out.append(sum_i64(seg) if kind == "int32" else sum_f64(seg, kind))
    return out


def histogram_i32(a: np.ndarray, lo: int, width: int, nbins: int) -> np.ndarray:
    """counts[b] = #{x : lo + b*width <= x < lo + (b+1)*width}, as int64."""
    a = _as_c(a).reshape(-1)
    if a.dtype != np.int32:
        raise TypeError("histogram_i32 expects int32")
    counts = np.empty(nbins, dtype=np.int64)
    _load().oracle_histogram_i32(_ptr(a), a.size, lo, width, nbins, _ptr(counts))
    return counts
