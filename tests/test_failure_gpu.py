"""Failure detection on the GPU without a fault: a bounded device-side wait
that nothing completes gives up after its limit, the host reads
OPTIGPU_ERR_TIMEOUT from optigpu_stream_status, and the context keeps
working.  Asynchronous argument errors never reach the device."""
import numpy as np
import pytest

import oracle
from gpu_util import require_gpu, torch
from paper_2605_13864_gb300 import _native as N
from paper_2605_13864_gb300 import api, workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def test_bounded_wait_times_out_and_context_survives():
    L = N.lib()
    s = torch.cuda.current_stream()
    api.stream_status()  # start from a clean status word
    assert L.optigpu_selftest_wait_timeout(2_000_000, s.cuda_stream) == N.OK  # 2 ms
    assert L.optigpu_stream_status(s.cuda_stream) == N.ERR_TIMEOUT
    assert b"limit" in L.optigpu_last_error()
    # The word was cleared by the read, and the device still computes.
    assert L.optigpu_stream_status(s.cuda_stream) == N.OK
    a = workloads.matrix(200, 136, "float32", seed=1)
    out = api.transpose(torch.from_numpy(a).cuda(), kernel="tma")
    assert np.array_equal(out.cpu().numpy(), oracle.transpose(a))
    api.stream_status()


def test_selftest_rejects_bad_limits():
    L = N.lib()
    assert L.optigpu_selftest_wait_timeout(0, None) == N.ERR_INVALID_ARG
    assert L.optigpu_selftest_wait_timeout(20_000_000_000, None) == N.ERR_INVALID_ARG
