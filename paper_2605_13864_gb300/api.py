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
              stream=None, blocking: bool = True) -> torch.Tensor:
    """``out[c, r] = src[r, c]`` (thesis Listing 3.5: out[x][y] = in[y][x]).

    For host tensors the call waits for the result unless ``blocking`` is
    False; then ``out`` is complete once ``stream`` (default: the current
    stream) has been synchronized, and both tensors must stay alive until
    then."""
    if src.dim() != 2:
        raise ValueError("transpose expects a 2-D tensor")
    if not src.is_cuda:
        # Host buffers: the library pipelines copy-in, kernel and copy-out.
        if not src.is_contiguous():
            raise ValueError("transpose expects a contiguous (row-major) source")
        rows, cols = src.shape
        host = out if out is not None else torch.empty((cols, rows), dtype=src.dtype, pin_memory=True)
        if host.is_cuda or tuple(host.shape) != (cols, rows) or not host.is_contiguous():
            raise ValueError("out must be a contiguous host (cols, rows) tensor")
        s = stream if stream is not None else torch.cuda.current_stream()
        st = N.lib().optigpu_transpose_host(src.data_ptr() if src.numel() else None,
                                            host.data_ptr() if host.numel() else None, rows, cols,
                                            dtype_code(src.dtype), int(s.cuda_stream))
        N.check(st, "optigpu_transpose_host")
        if blocking:
            s.synchronize()
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


def transpose_inplace(a: torch.Tensor, stream=None) -> torch.Tensor:
    """Transposes the square contiguous CUDA tensor ``a`` in place."""
    if a.dim() != 2 or a.shape[0] != a.shape[1] or not a.is_cuda or not a.is_contiguous():
        raise ValueError("transpose_inplace expects a square contiguous CUDA tensor")
    st = N.lib().optigpu_transpose_inplace(a.data_ptr() if a.numel() else None, int(a.shape[0]),
                                           dtype_code(a.dtype), _stream_ptr(stream))
    N.check(st, "optigpu_transpose_inplace")
    return a


def transpose_batched(src: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """(batch, rows, cols) CUDA tensor -> (batch, cols, rows): each matrix
    transposed, in one launch."""
    if src.dim() != 3 or not src.is_cuda:
        raise ValueError("transpose_batched expects a 3-D CUDA tensor")
    b, rows, cols = src.shape
    if src.stride(2) != 1 or src.stride(1) != cols:
        raise ValueError("each source matrix must be dense row-major")
    if out is None:
        out = torch.empty((b, cols, rows), dtype=src.dtype, device=src.device)
    elif tuple(out.shape) != (b, cols, rows) or out.stride(2) != 1 or out.stride(1) != rows:
        raise ValueError("out must be (batch, cols, rows) with dense matrices")
    st = N.lib().optigpu_transpose_batched(src.data_ptr(), src.stride(0) if b > 1 else rows * cols,
                                           out.data_ptr(), out.stride(0) if b > 1 else rows * cols,
                                           b, rows, cols, dtype_code(src.dtype), _stream_ptr(stream))
    N.check(st, "optigpu_transpose_batched")
    return out


def reduce_sum(x: torch.Tensor, compensated: bool = False, out: torch.Tensor | None = None,
               stream=None, blocking: bool = True) -> torch.Tensor:
    """Sum of all elements (thesis Listing 2.1: reduce_sum(N, A)).

    Returns a 0-d int64 tensor for int32 input and a 0-d float64 tensor for
    float input (the partials are combined in FP64 on the GPU).  For a host
    tensor the call waits for the result unless ``blocking`` is False (then
    synchronize ``stream`` before reading it).
    """
    if not x.is_cuda:
        # Host buffer: the library pipelines the copy-in against the partials.
        if not x.is_contiguous():
            raise ValueError("reduce_sum expects a contiguous tensor")
        odt = torch.int64 if x.dtype == torch.int32 else torch.float64
        res = out if out is not None else torch.empty((), dtype=odt, pin_memory=True)
        s = stream if stream is not None else torch.cuda.current_stream()
        flags = N.REDUCE_COMPENSATED if compensated else N.REDUCE_PLAIN
        st = N.lib().optigpu_reduce_sum_host(x.data_ptr() if x.numel() else None, x.numel(),
                                             dtype_code(x.dtype), res.data_ptr(), flags, int(s.cuda_stream))
        N.check(st, "optigpu_reduce_sum_host")
        if blocking:
            s.synchronize()
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


def reduce_reserve(n: int, stream=None) -> None:
    """Pre-allocates the sum workspace of ``stream`` for up to ``n`` elements
    (do this before capturing sums into a CUDA graph)."""
    N.check(N.lib().optigpu_reduce_reserve(int(n), _stream_ptr(stream)), "optigpu_reduce_reserve")


def scan(x: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Inclusive prefix sums of a contiguous CUDA tensor (flattened): int64
    for int32 input, float32 for float input."""
    if not x.is_cuda or not x.is_contiguous():
        raise ValueError("scan expects a contiguous CUDA tensor")
    odt = torch.int64 if x.dtype == torch.int32 else torch.float32
    if out is None:
        out = torch.empty(x.numel(), dtype=odt, device=x.device)
    elif out.dtype != odt or out.numel() != x.numel() or not out.is_contiguous():
        raise ValueError(f"out must be a contiguous {odt} tensor of x.numel() elements")
    st = N.lib().optigpu_scan_inclusive(x.data_ptr() if x.numel() else None, out.data_ptr() if x.numel() else None,
                                        x.numel(), dtype_code(x.dtype), _stream_ptr(stream))
    N.check(st, "optigpu_scan_inclusive")
    return out


def histogram(x: torch.Tensor, lo: int, width: int, nbins: int, stream=None) -> torch.Tensor:
    """int64 counts of the int32 values of ``x`` in ``nbins`` bins of
    ``width`` integers starting at ``lo`` (on the device)."""
    if not x.is_cuda or x.dtype != torch.int32 or not x.is_contiguous():
        raise ValueError("histogram expects a contiguous int32 CUDA tensor")
    counts = torch.empty(nbins, dtype=torch.int64, device=x.device)
    st = N.lib().optigpu_histogram_i32(x.data_ptr() if x.numel() else None, x.numel(), int(lo), int(width),
                                       int(nbins), counts.data_ptr(), _stream_ptr(stream))
    N.check(st, "optigpu_histogram_i32")
    return counts


def reduce_segmented(x: torch.Tensor, offsets, compensated: bool = False, stream=None) -> torch.Tensor:
    """Sums of x[offsets[s]:offsets[s+1]] for every segment, in one launch;
    int64 results for int32 input, float64 otherwise (on the device)."""
    import ctypes
    import numpy as np
    if not x.is_cuda or not x.is_contiguous():
        raise ValueError("reduce_segmented expects a contiguous CUDA tensor")
    offs = np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
    nseg = offs.size - 1
    odt = torch.int64 if x.dtype == torch.int32 else torch.float64
    out = torch.empty(max(nseg, 0), dtype=odt, device=x.device)
    flags = N.REDUCE_COMPENSATED if compensated else N.REDUCE_PLAIN
    st = N.lib().optigpu_reduce_segmented(x.data_ptr() if x.numel() else None, offs.ctypes.data,
                                          nseg, dtype_code(x.dtype), out.data_ptr() if nseg else None, flags,
                                          _stream_ptr(stream))
    N.check(st, "optigpu_reduce_segmented")
    return out


def transpose_config_for(rows: int, cols: int, dtype: torch.dtype = torch.float32) -> tuple[int, str]:
    """(index, name) of the configuration AUTO launches for an aligned
    rows x cols matrix of ``dtype``."""
    i = int(N.lib().optigpu_transpose_config_for(int(rows), int(cols), dtype_code(dtype)))
    return i, tune_configs("transpose", dtype)[i]


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

_OPS = {"transpose": N.OP_TRANSPOSE, "reduce": N.OP_REDUCE, "batch": N.OP_BATCH, "scan": N.OP_SCAN}


def tune_configs(op: str, dtype: torch.dtype = torch.float32) -> list[str]:
    """Names of the compiled configurations of ``op`` for ``dtype``."""
    L = N.lib()
    n = L.optigpu_tune_num_configs(_OPS[op], dtype_code(dtype))
    return [L.optigpu_tune_config_name(_OPS[op], dtype_code(dtype), i).decode() for i in range(n)]


def tune_select(op: str, dtype: torch.dtype, config: int) -> None:
    """Selects the configuration ``op`` uses from now on.  The transpose
    keeps one choice per element size; the scan one per input class (int32,
    and the float types together); the sum and the batch kernel one each."""
    N.check(N.lib().optigpu_tune_select(_OPS[op], dtype_code(dtype), int(config)), "optigpu_tune_select")


def tune_selected(op: str, dtype: torch.dtype) -> int:
    """Index of the configuration ``op`` uses for ``dtype`` (see tune_select)."""
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


# ------------------------------------------------------------------ batches

class BatchPlan:
    """Many transposes and sums in one persistent launch (optigpu_batch_*).

    ``items`` is a list of ``("transpose", src, dst)`` or
    ``("reduce", src, out)`` with CUDA tensors (``dst`` is cols x rows,
    ``out`` a 0-d int64 / float64 tensor).  The plan keeps references to the
    tensors so their memory stays valid while the plan lives.
    """

    def __init__(self, items, compensated: bool = False, graph: bool = True):
        import ctypes
        self._keep = []
        descs = (N.Desc * max(len(items), 1))()
        for k, (op, src, dst) in enumerate(items):
            d = descs[k]
            d.dtype = dtype_code(src.dtype)
            d.src = src.data_ptr() if src.numel() else None
            d.dst = dst.data_ptr() if dst.numel() else None
            if op == "transpose":
                d.op = N.OP_TRANSPOSE
                d.rows, d.cols = int(src.shape[0]), int(src.shape[1])
                if not (src.is_contiguous() and dst.is_contiguous()) or tuple(dst.shape) != (d.cols, d.rows):
                    raise ValueError(f"batch item {k}: contiguous src (r, c) and dst (c, r) required")
            elif op == "reduce":
                d.op = N.OP_REDUCE
                d.rows, d.cols = int(src.numel()), 1
                want = torch.int64 if src.dtype == torch.int32 else torch.float64
                if dst.dtype != want or dst.numel() != 1:
                    raise ValueError(f"batch item {k}: out must hold one {want}")
            else:
                raise ValueError(f"batch item {k}: unknown op {op!r}")
            self._keep.append((src, dst))
        flags = (N.REDUCE_COMPENSATED if compensated else 0) | (0 if graph else N.BATCH_NO_GRAPH)
        plan = ctypes.c_void_p()
        N.check(N.lib().optigpu_batch_plan_create(descs, len(items), flags, ctypes.byref(plan)),
                "optigpu_batch_plan_create")
        self._plan = plan

    def run(self, stream=None) -> None:
        N.check(N.lib().optigpu_batch_run(self._plan, _stream_ptr(stream)), "optigpu_batch_run")

    def info(self) -> dict:
        import ctypes
        items, nbytes, grid = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int32()
        N.check(N.lib().optigpu_batch_plan_info(self._plan, ctypes.byref(items), ctypes.byref(nbytes),
                                                ctypes.byref(grid)), "optigpu_batch_plan_info")
        return {"items": items.value, "bytes": nbytes.value, "grid": grid.value}

    def autotune(self, reps: int = 5, stream=None):
        import ctypes
        best, ms = ctypes.c_int(-1), ctypes.c_float()
        N.check(N.lib().optigpu_batch_autotune(self._plan, int(reps), _stream_ptr(stream), ctypes.byref(best),
                                               ctypes.byref(ms)), "optigpu_batch_autotune")
        return best.value, tune_configs("batch")[best.value], float(ms.value)

    def close(self) -> None:
        if getattr(self, "_plan", None) is not None and self._plan.value:
            torch.cuda.synchronize()
            N.lib().optigpu_batch_plan_destroy(self._plan)
            self._plan = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------------ serving

def _host_request(op: str, src: torch.Tensor, dst: torch.Tensor) -> "N.Request":
    r = N.Request()
    r.dtype = dtype_code(src.dtype)
    if src.is_cuda or dst.is_cuda:
        raise ValueError("served requests carry host (CPU) tensors")
    if op == "transpose":
        r.op = N.OP_TRANSPOSE
        r.rows, r.cols = int(src.shape[0]), int(src.shape[1])
        if tuple(dst.shape) != (r.cols, r.rows) or not dst.is_contiguous():
            raise ValueError("dst must be a contiguous (cols, rows) tensor")
    elif op == "reduce":
        r.op = N.OP_REDUCE
        r.rows, r.cols = int(src.numel()), 1
        want = torch.int64 if src.dtype == torch.int32 else torch.float64
        if dst.dtype != want or dst.numel() != 1:
            raise ValueError(f"out must hold one {want}")
    else:
        raise ValueError(f"unknown op {op!r}")
    if not src.is_contiguous():
        raise ValueError("src must be contiguous")
    r.host_src = src.data_ptr() if src.numel() else None
    r.host_dst = dst.data_ptr()
    return r


class Server:
    """Continuous-batching server (optigpu_server_*) over host tensors.

    Pinned host tensors (``tensor.pin_memory()``) make the copies
    asynchronous.  ``per_call=True`` is the baseline that launches one plain
    kernel per request.  ``copy`` picks the copy path of pinned buffers:
    None (batched: SM copy kernels; per-call: copy engines), ``"engines"``
    (copy-engine calls in both modes) or ``"kernels"`` (SM copy kernels in
    both modes).
    """

    def __init__(self, budget_bytes: int = 1 << 30, max_slots: int = 256, n_streams: int = 4,
                 per_call: bool = False, compensated: bool = False, copy: str | None = None):
        import ctypes
        flags = (N.SERVER_PER_CALL if per_call else 0) | (N.REDUCE_COMPENSATED if compensated else 0)
        if copy == "engines" and not per_call:
            flags |= N.SERVER_COPY_ENGINES
        elif copy == "kernels" and per_call:
            flags |= N.SERVER_COPY_KERNELS
        elif copy not in (None, "engines", "kernels"):
            raise ValueError("copy must be None, 'engines' or 'kernels'")
        h = ctypes.c_void_p()
        N.check(N.lib().optigpu_server_create(int(budget_bytes), int(max_slots), int(n_streams), flags,
                                              ctypes.byref(h)), "optigpu_server_create")
        self._h = h
        self._keep = {}

    def submit(self, op: str, src: torch.Tensor, dst: torch.Tensor) -> int:
        import ctypes
        r = _host_request(op, src, dst)
        tk = ctypes.c_uint64()
        N.check(N.lib().optigpu_server_submit(self._h, ctypes.byref(r), ctypes.byref(tk)), "optigpu_server_submit")
        self._keep[tk.value] = (src, dst)
        return tk.value

    def step(self) -> int:
        import ctypes
        n = ctypes.c_int32()
        N.check(N.lib().optigpu_server_step(self._h, ctypes.byref(n)), "optigpu_server_step")
        return n.value

    def poll(self, ticket: int) -> bool:
        import ctypes
        d = ctypes.c_int32()
        N.check(N.lib().optigpu_server_poll(self._h, int(ticket), ctypes.byref(d)), "optigpu_server_poll")
        if d.value:
            self._keep.pop(ticket, None)
        return bool(d.value)

    def drain(self) -> None:
        N.check(N.lib().optigpu_server_drain(self._h), "optigpu_server_drain")

    def inject_step_failure(self, nth: int = 1) -> None:
        """Testing hook: the nth step launch from now on fails on the host."""
        N.check(N.lib().optigpu_server_inject_step_failure(self._h, int(nth)),
                "optigpu_server_inject_step_failure")

    def stats(self) -> dict:
        import ctypes
        st = N.ServerStats()
        N.check(N.lib().optigpu_server_get_stats(self._h, ctypes.byref(st)), "optigpu_server_get_stats")
        return {name: getattr(st, name) for name, _ in N.ServerStats._fields_}

    def replay(self, requests, arrivals_s):
        """Open-loop replay of ``requests`` (list of (op, src, dst) host
        tensors) at ``arrivals_s`` seconds; returns per-request latencies (s)."""
        import ctypes
        import numpy as np
        n = len(requests)
        arr = (N.Request * max(n, 1))()
        for i, (op, src, dst) in enumerate(requests):
            arr[i] = _host_request(op, src, dst)
        t = np.ascontiguousarray(arrivals_s, dtype=np.float64)
        lat = np.zeros(n, dtype=np.float64)
        N.check(N.lib().optigpu_server_replay(self._h, ctypes.cast(arr, ctypes.c_void_p), t.ctypes.data, n,
                                              lat.ctypes.data), "optigpu_server_replay")
        return lat

    def close(self) -> None:
        if getattr(self, "_h", None) is not None and self._h.value:
            N.lib().optigpu_server_destroy(self._h)
            self._h = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
