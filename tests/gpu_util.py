"""Helpers for the GPU parity tests: numpy <-> torch device tensors.

16-bit floats travel as uint16 bit patterns on the host (numpy has no
bfloat16) and are reinterpreted, never converted, on the way to the device.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

TORCH_DT = {"int32": torch.int32, "float32": torch.float32,
            "bfloat16": torch.bfloat16, "float16": torch.float16}


def require_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def to_device(a: np.ndarray, dtype: str, offset_elems: int = 0) -> torch.Tensor:
    """Copy a host array to the device, optionally at an element offset inside
    a larger buffer (to exercise unaligned pointers)."""
    a = np.ascontiguousarray(a)
    if dtype in ("bfloat16", "float16"):
        host = torch.from_numpy(a.view(np.int16)).view(TORCH_DT[dtype])
    else:
        host = torch.from_numpy(a)
    if offset_elems == 0:
        return host.to("cuda")
    buf = torch.zeros(host.numel() + offset_elems + 8, dtype=host.dtype, device="cuda")
    view = buf[offset_elems:offset_elems + host.numel()].view(host.shape)
    view.copy_(host)
    return view


def to_host_bits(t: torch.Tensor) -> np.ndarray:
    """Device tensor -> host array of the raw element bits."""
    t = t.contiguous().cpu()
    if t.dtype in (torch.bfloat16, torch.float16):
        return t.view(torch.int16).numpy().view(np.uint16)
    if t.dtype == torch.float32:
        return t.numpy().view(np.uint32)
    return t.numpy()
