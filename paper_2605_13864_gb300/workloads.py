"""Seeded synthetic inputs for the transpose and the sum reduction.

This module holds random-number recipes only -- no part of the transpose or
the sum.  Both the CPU oracle's tests and the CUDA path draw their inputs from
here, so the two sides always see the same bytes.  Everything is numpy PCG64
(``numpy.random.default_rng``) on the host; 16-bit floats are produced by
round-to-nearest-even from float32 draws through torch's CPU casts and are
handed around as raw ``uint16`` bit patterns (numpy has no bfloat16).

Workloads (the thesis's case studies, arxiv 2605.13864, Sec. 7.1, scaled to
one GB300):

* ``small``      -- 1024x1024 int32 in [-1000, 1000], seed 0; the same matrix
  is transposed and summed.
* ``roofline``   -- 16384x16384 float32 N(0,1) transpose and a 2^28 float32
  N(0,1) vector, seed 1 (the vector from an independent sub-stream of the
  seed, so either can be drawn alone).
* ``precision``  -- 2^28 draws of N(100,1), seed 2, rounded to bfloat16 and,
  separately, to float16; an 8192x8192 bfloat16 N(0,1) matrix from an
  independent sub-stream of seed 2.
* ``batched``    -- 4096 instances, seed 3: transposes of float32 matrices
  with rows and cols log-uniform in [1, 2048] and float32 sums with lengths
  log-uniform in [1, 2^22], interleaved T, R, T, R, ...
* ``serving``    -- a Poisson request stream, seed 4: exponential
  inter-arrival times (mean 1/rate), op 50/50, dtype uniform over
  {int32, float32, bfloat16}, sizes as in ``batched``.

Log-uniform sizes: ``v = clip(rint(exp(U(0, ln hi))), 1, hi)``, drawn in the
order rows, cols, lengths.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

DTYPES = ("int32", "float32", "bfloat16", "float16")
ESIZE = {"int32": 4, "float32": 4, "bfloat16": 2, "float16": 2}


def _round_to_16(x32: np.ndarray, dtype: str) -> np.ndarray:
    """float32 -> bfloat16/float16 bit patterns, round to nearest even."""
    import torch  # CPU casts only

    t = torch.from_numpy(np.ascontiguousarray(x32, dtype=np.float32))
    tt = torch.bfloat16 if dtype == "bfloat16" else torch.float16
    return t.to(tt).view(torch.int16).numpy().view(np.uint16).copy()


def storage_dtype(dtype: str):
    """numpy dtype that carries elements of ``dtype`` (16-bit floats as uint16)."""
    return {"int32": np.int32, "float32": np.float32,
            "bfloat16": np.uint16, "float16": np.uint16}[dtype]


def draw(rng: np.random.Generator, shape, dtype: str, dist: str = "normal",
         mean: float = 0.0, lo: int = -1000, hi: int = 1000) -> np.ndarray:
    """Draw an array of ``dtype`` elements.

    ``dist`` is ``"normal"`` (N(mean, 1), rounded for 16-bit floats, truncated
    toward zero for int32) or ``"uniform_int"`` (integers in [lo, hi]).
    """
    if dist == "uniform_int":
        ints = rng.integers(lo, hi + 1, size=shape, dtype=np.int64)
        if dtype == "int32":
            return ints.astype(np.int32)
        if dtype == "float32":
            return ints.astype(np.float32)
        return _round_to_16(ints.astype(np.float32), dtype)
    x = rng.standard_normal(size=shape, dtype=np.float32)
    if mean != 0.0:
        x += np.float32(mean)
    if dtype == "float32":
        return x
    if dtype == "int32":
        return (x * np.float32(1000.0)).astype(np.int32)
    return _round_to_16(x, dtype)


def matrix(rows: int, cols: int, dtype: str = "float32", seed: int = 0,
           dist: str = "normal") -> np.ndarray:
    return draw(np.random.default_rng(seed), (rows, cols), dtype, dist)


def vector(n: int, dtype: str = "float32", seed: int = 0, dist: str = "normal",
           mean: float = 0.0) -> np.ndarray:
    return draw(np.random.default_rng(seed), (n,), dtype, dist, mean=mean)


# --------------------------------------------------------------------------
# The five workloads
# --------------------------------------------------------------------------

def small(rows: int = 1024, cols: int = 1024) -> np.ndarray:
    """1024x1024 int32, entries uniform in [-1000, 1000], seed 0."""
    rng = np.random.default_rng(0)
    return rng.integers(-1000, 1001, size=(rows, cols), dtype=np.int32)


def _substream(seed: int, k: int) -> np.random.Generator:
    """Independent generator number k of workload `seed` (PCG64 spawn key)."""
    return np.random.default_rng(np.random.SeedSequence(entropy=seed, spawn_key=(k,)))


def roofline_matrix(rows: int = 16384, cols: int = 16384) -> np.ndarray:
    """float32 N(0,1), seed 1."""
    return np.random.default_rng(1).standard_normal(size=(rows, cols), dtype=np.float32)


def roofline_vector(n: int = 1 << 28) -> np.ndarray:
    """float32 N(0,1), seed 1, sub-stream 1 (independent of the matrix)."""
    return _substream(1, 1).standard_normal(size=(n,), dtype=np.float32)


def precision_vectors(n: int = 1 << 28):
    """(bf16, fp16) bit patterns of the same n draws of N(100, 1), seed 2."""
    x = np.random.default_rng(2).standard_normal(size=(n,), dtype=np.float32)
    x += np.float32(100.0)
    return _round_to_16(x, "bfloat16"), _round_to_16(x, "float16")


def precision_matrix(side: int = 8192) -> np.ndarray:
    """bfloat16 N(0, 1) bit patterns, seed 2, sub-stream 1."""
    m = _substream(2, 1).standard_normal(size=(side, side), dtype=np.float32)
    return _round_to_16(m, "bfloat16").reshape(side, side)


def log_uniform(rng: np.random.Generator, hi: int, size: int) -> np.ndarray:
    """clip(rint(exp(U(0, ln hi))), 1, hi) as int64."""
    u = rng.uniform(0.0, math.log(hi), size=size)
    return np.clip(np.rint(np.exp(u)), 1, hi).astype(np.int64)


@dataclass
class Instance:
    """One problem of a batch: op 0 = transpose (rows x cols), op 1 = sum (n)."""
    op: int
    dtype: str
    rows: int       # transpose rows, or sum length
    cols: int       # transpose cols, 1 for sums

    @property
    def elems(self) -> int:
        return self.rows * self.cols

    @property
    def algorithmic_bytes(self) -> int:
        e = ESIZE[self.dtype] * self.elems
        return 2 * e if self.op == 0 else e


def batched_instances(count: int = 4096, seed: int = 3, max_side: int = 2048,
                      max_len: int = 1 << 22, dtype: str = "float32"):
    """``count`` instances, interleaved transpose / sum, sizes log-uniform."""
    rng = np.random.default_rng(seed)
    nt = (count + 1) // 2
    nr = count // 2
    rows = log_uniform(rng, max_side, nt)
    cols = log_uniform(rng, max_side, nt)
    lens = log_uniform(rng, max_len, nr)
    out = []
    for i in range(count):
        if i % 2 == 0:
            out.append(Instance(0, dtype, int(rows[i // 2]), int(cols[i // 2])))
        else:
            out.append(Instance(1, dtype, int(lens[i // 2]), 1))
    return out


def batched_data(instances, seed: int = 3):
    """Input arrays for ``instances`` (N(0,1), one generator, instance order).

    The generator is seeded with ``seed + 1000`` so the size draws of
    ``batched_instances`` stay independent of the value draws.
    """
    rng = np.random.default_rng(seed + 1000)
    data = []
    for inst in instances:
        shape = (inst.rows, inst.cols) if inst.op == 0 else (inst.rows,)
        data.append(draw(rng, shape, inst.dtype, "normal"))
    return data


def segment_offsets(n: int, nseg: int, seed: int = 6, max_len: int = 32768) -> np.ndarray:
    """nseg + 1 offsets of consecutive segments of a length-n array: lengths
    uniform in [1, max_len), clipped at n (trailing segments may be empty)."""
    lens = np.random.default_rng(seed).integers(1, max_len, size=nseg)
    return np.minimum(np.concatenate([[0], np.cumsum(lens)]), n).astype(np.int64)


def histogram_values(n: int, nbins: int = 4096, seed: int = 7) -> np.ndarray:
    """int32 values uniform in [0, nbins)."""
    return draw(np.random.default_rng(seed), (n,), "int32", "uniform_int", lo=0, hi=nbins - 1)


@dataclass
class Request:
    arrival_s: float
    inst: Instance


def serving_requests(count: int = 100_000, rate: float = 20_000.0, seed: int = 4,
                     max_side: int = 2048, max_len: int = 1 << 22):
    """Open-loop Poisson stream: arrival times, op, dtype and size per request."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate, size=count)
    arrivals = np.cumsum(gaps)
    ops = rng.integers(0, 2, size=count)
    dts = rng.integers(0, 3, size=count)
    rows = log_uniform(rng, max_side, count)
    cols = log_uniform(rng, max_side, count)
    lens = log_uniform(rng, max_len, count)
    names = ("int32", "float32", "bfloat16")
    reqs = []
    for i in range(count):
        dt = names[int(dts[i])]
        if ops[i] == 0:
            inst = Instance(0, dt, int(rows[i]), int(cols[i]))
        else:
            inst = Instance(1, dt, int(lens[i]), 1)
        reqs.append(Request(float(arrivals[i]), inst))
    return reqs
