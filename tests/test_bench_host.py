"""Host-side logic of bench.py on CPU: the max-over-ranks timing reduction
with two gloo ranks, the whole-job value, and the reference arm's rank
behaviour under a multi-rank launch (rank 0 alone prints one JSON line)."""
import json
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_q):
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    got = bench.max_over_ranks([1.0 + rank, 5.0 - rank], dist, device="cpu")
    out_q.put((rank, got))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res[0] == res[1] == [2.0, 5.0]


def test_max_over_ranks_single_rank_is_identity():
    assert bench.max_over_ranks([3, 4.5]) == [3.0, 4.5]


def test_job_value_counts_every_replica():
    one = bench.job_value(1, bench.STEP_BYTES, 0.5)
    assert bench.job_value(4, bench.STEP_BYTES, 0.5) == pytest.approx(4 * one)
    assert one == pytest.approx(bench.STEP_BYTES / 0.5e-3 / 1e9)


def _run_reference(env_extra):
    env = dict(os.environ, **env_extra)
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                           "--steps", "1", "--warmup", "1"], capture_output=True, text=True, env=env,
                          timeout=600, cwd=ROOT)


def test_reference_arm_other_ranks_exit_quietly():
    r = _run_reference({"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"})
    assert r.returncode == 0 and r.stdout.strip() == ""


def test_reference_arm_rank0_prints_one_json_line():
    r = _run_reference({"RANK": "0", "WORLD_SIZE": "2", "LOCAL_RANK": "0"})
    assert r.returncode == 0, r.stderr
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "GB/s" and d["metric"] == bench.METRIC
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["cpu_baseline"]["kind"] == "oracle"


def test_host_reference_agrees_with_the_oracle():
    # The bench's own result checks (served sample, precision errors) use
    # numpy references; here they are held to the oracle on small inputs.
    import numpy as np

    import oracle
    from paper_2605_13864_gb300 import workloads

    vb, vh = workloads.precision_vectors(1 << 16)
    rb = bench._host_reference(vb.view(np.uint16), "bfloat16")
    rh = bench._host_reference(vh.view(np.float16), "float16")
    assert rb["f64"] == oracle.reduce_reference(vb, "bfloat16")["f64"]   # exact sums
    assert rh["f64"] == oracle.reduce_reference(vh, "float16")["f64"]
    x = workloads.vector(100003, "float32", seed=9)
    r, o = bench._host_reference(x, "float32"), oracle.reduce_reference(x)
    assert abs(r["f64"] - o["f64"]) <= 1e-12 * o["abs"] and abs(r["abs"] - o["abs"]) <= 1e-12 * o["abs"]
    xi = workloads.vector(100003, "int32", seed=9)
    assert bench._host_reference(xi, "int32")["int"] == oracle.sum_i64(xi)
    m = workloads.matrix(37, 53, "float32", seed=9)
    assert np.array_equal(np.ascontiguousarray(m.T), oracle.transpose(m))
