"""Python API over the C ABI: torch tensors in, torch tensors out.

PyTorch supplies device memory and the current CUDA stream; the operations
themselves run in ``liboptigpu.so``.  Each function accepts CUDA tensors (the
result stays on the device, the call is asynchronous on the current stream)
or CPU tensors (the inputs are copied to the device, the library runs, and the
result is copied back -- the end-to-end path a host caller uses).
"""
from __future__ import annotations

import torch

from . import _native as N

_DTYPES = {torch.int32: N.INT32, torch.float32: N.FLOAT32,
           torch.bfloat16: N.BFLOAT16, torch.float16: N.FLOAT16}
_KERNELS = {"auto": N.TRANSPOSE_AUTO, "tile32": N.TRANSPOSE_TILE32, "tma": N.TRANSPOSE_TMA}


def dtype_code(dt: torch.dtype) -> int:
    try:
        return _DTYPES[dt]
    except KeyError:
        raise TypeError(f"optigpu: unsupported dtype {dt}") from None


def _stream_ptr(stream) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def transpose(src: torch.Tensor, out: torch.Tensor | None = None, kernel: str = "auto",
              stream=None) -> torch.Tensor:
    """``out[c, r] = src[r, c]`` (thesis Listing 3.5: out[x][y] = in[y][x])."""
    if src.dim() != 2:
        raise ValueError("transpose expects a 2-D tensor")
    if not src.is_cuda:
        dev = torch.device("cuda", torch.cuda.current_device())
        d_src = src.to(dev, non_blocking=True)
        d_out = transpose(d_src, kernel=kernel, stream=stream)
        host = out if out is not None else torch.empty(
            (src.shape[1], src.shape[0]), dtype=src.dtype, pin_memory=True)
        host.copy_(d_out, non_blocking=True)
        torch.cuda.current_stream().synchronize()
        return host
    if not src.is_contiguous():
        raise ValueError("transpose expects a contiguous (row-major) source")
    rows, cols = src.shape
    if out is None:
        out = torch.empty((cols, rows), dtype=src.dtype, device=src.device)
    elif out.shape != (cols, rows) or out.dtype != src.dtype or not out.is_contiguous():
        raise ValueError("out must be a contiguous (cols, rows) tensor of the source dtype")
    st = N.lib().optigpu_transpose_ex(src.data_ptr(), out.data_ptr(), rows, cols,
                                      dtype_code(src.dtype), _KERNELS[kernel], _stream_ptr(stream))
    N.check(st, "optigpu_transpose")
    return out


def reduce_sum(x: torch.Tensor, compensated: bool = False, out: torch.Tensor | None = None,
               stream=None) -> torch.Tensor:
    """Sum of all elements (thesis Listing 2.1: reduce_sum(N, A)).

    Returns a 0-d int64 tensor for int32 input and a 0-d float64 tensor for
    float input (the partials are combined in FP64 on the GPU).
    """
    if not x.is_cuda:
        dev = torch.device("cuda", torch.cuda.current_device())
        d = reduce_sum(x.to(dev, non_blocking=True), compensated=compensated, stream=stream)
        res = d.to("cpu")
        return res
    if not x.is_contiguous():
        raise ValueError("reduce_sum expects a contiguous tensor")
    odt = torch.int64 if x.dtype == torch.int32 else torch.float64
    if out is None:
        out = torch.empty((), dtype=odt, device=x.device)
    elif out.dtype != odt or out.numel() != 1:
        raise ValueError(f"out must hold one {odt} value")
    flags = N.REDUCE_COMPENSATED if compensated else N.REDUCE_PLAIN
    st = N.lib().optigpu_reduce_sum_ex(x.data_ptr() if x.numel() else None, x.numel(),
                                       dtype_code(x.dtype), out.data_ptr(), flags, _stream_ptr(stream))
    N.check(st, "optigpu_reduce_sum")
    return out


def tma_eligible(src: torch.Tensor, dst: torch.Tensor) -> bool:
    rows, cols = src.shape
    return bool(N.lib().optigpu_transpose_tma_eligible(src.data_ptr(), dst.data_ptr(), rows, cols,
                                                       dtype_code(src.dtype)))


def stream_status(stream=None) -> None:
    """Raises OptigpuError if queued work failed or a device wait timed out."""
    N.check(N.lib().optigpu_stream_status(_stream_ptr(stream)), "optigpu_stream_status")


def set_wait_limit_ns(ns: int) -> None:
    N.lib().optigpu_set_wait_limit_ns(int(ns))


def release_workspaces() -> None:
    N.check(N.lib().optigpu_release_workspaces(), "optigpu_release_workspaces")


# ---------------------------------------------------------------- autotuning

_OPS = {"transpose": N.OP_TRANSPOSE, "reduce": N.OP_REDUCE}


def tune_configs(op: str, dtype: torch.dtype) -> list[str]:
    """Names of the compiled configurations of ``op`` for ``dtype``."""
    L = N.lib()
    n = L.optigpu_tune_num_configs(_OPS[op], dtype_code(dtype))
    return [L.optigpu_tune_config_name(_OPS[op], dtype_code(dtype), i).decode() for i in range(n)]


def tune_select(op: str, dtype: torch.dtype, config: int) -> None:
    N.check(N.lib().optigpu_tune_select(_OPS[op], dtype_code(dtype), int(config)), "optigpu_tune_select")


def tune_selected(op: str, dtype: torch.dtype) -> int:
    return int(N.lib().optigpu_tune_selected(_OPS[op], dtype_code(dtype)))


def tune_set_param(name: str, value: int) -> None:
    N.check(N.lib().optigpu_tune_set_param(name.encode(), int(value)), "optigpu_tune_set_param")


def autotune(op: str, dtype: torch.dtype, rows: int, cols: int = 1, reps: int = 10, stream=None):
    """Times every configuration on a rows x cols problem; selects and returns
    ``(index, name, ms)`` of the fastest."""
    import ctypes
    best = ctypes.c_int(-1)
    ms = ctypes.c_float(0.0)
    N.check(N.lib().optigpu_autotune(_OPS[op], dtype_code(dtype), int(rows), int(cols), int(reps),
                                     _stream_ptr(stream), ctypes.byref(best), ctypes.byref(ms)),
            "optigpu_autotune")
    return best.value, tune_configs(op, dtype)[best.value], float(ms.value)


def tune_save(path: str) -> None:
    N.check(N.lib().optigpu_tune_save(path.encode()), "optigpu_tune_save")


def tune_load(path: str) -> None:
    N.check(N.lib().optigpu_tune_load(path.encode()), "optigpu_tune_load")
