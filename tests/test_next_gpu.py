"""GPU parity of the neighbouring problems against the CPU oracle: stacks of
transposes (3-D TMA or padded tiles), and the other variants as they land.
Bit-exact for transposes."""
import numpy as np
import pytest

import oracle
from gpu_util import require_gpu, to_device, to_host_bits, torch
from paper_2605_13864_gb300 import _native as N
from paper_2605_13864_gb300 import api, workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def bits(a):
    return a.view(np.uint32) if a.dtype == np.float32 else a


@pytest.mark.parametrize("dtype", ["float32", "bfloat16", "int32"])
@pytest.mark.parametrize("batch,rows,cols", [(1, 64, 64), (3, 128, 64), (5, 136, 264), (4, 33, 17),
                                             (7, 1, 300), (2, 1000, 8)])
def test_transpose_batched_dense(dtype, batch, rows, cols):
    a = workloads.matrix(batch * rows, cols, dtype, seed=batch + rows).reshape(batch, rows, cols)
    d = to_device(a.reshape(batch * rows, cols), dtype).view(batch, rows, cols)
    out = api.transpose_batched(d)
    torch.cuda.synchronize()
    api.stream_status()
    got = to_host_bits(out.reshape(batch * cols, rows)).reshape(batch, cols, rows)
    assert np.array_equal(got, bits(oracle.transpose_batched(a)))


@pytest.mark.parametrize("dtype", ["float32", "bfloat16"])
@pytest.mark.parametrize("batch,rows,cols,gap_s,gap_d", [(3, 64, 128, 64, 32), (4, 40, 24, 8, 16),
                                                         (5, 33, 17, 3, 5)])
def test_transpose_batched_with_gaps(dtype, batch, rows, cols, gap_s, gap_d):
    """Matrices stride_src / stride_dst elements apart; the gaps between
    output matrices keep their canary."""
    n = rows * cols
    ss, sd = n + gap_s, n + gap_d
    flat = workloads.vector(batch * ss, dtype, seed=9)
    src = to_device(flat, dtype)
    tdt = src.dtype
    wide = torch.int16 if tdt == torch.bfloat16 else torch.int32
    dst_raw = torch.full((batch * sd,), 0x2B2B, dtype=wide, device="cuda")
    dst = dst_raw.view(tdt)
    st = N.lib().optigpu_transpose_batched(src.data_ptr(), ss, dst.data_ptr(), sd, batch, rows, cols,
                                           api.dtype_code(tdt), torch.cuda.current_stream().cuda_stream)
    assert st == N.OK, N.lib().optigpu_last_error()
    torch.cuda.synchronize()
    got = to_host_bits(dst)
    for b in range(batch):
        m = flat[b * ss:b * ss + n].reshape(rows, cols)
        assert np.array_equal(got[b * sd:b * sd + n].reshape(cols, rows), bits(oracle.transpose(m)))
        tail = got[b * sd + n:(b + 1) * sd]
        assert (tail.view(np.uint16 if tail.dtype == np.uint16 else np.uint32) == 0x2B2B).all()
