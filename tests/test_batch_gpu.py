"""GPU parity of the batched persistent kernel (many transposes and sums in
one launch) against the CPU oracle and against the single calls.

Every transpose instance is bit-exact against the oracle; every int32 sum is
exact; every float sum is within 1e-6 * sum|x| of the FP64 oracle AND
bit-identical to the single-call optigpu_reduce_sum_ex result (same chunks,
same combine order), so each result is the same alone and in the mix.  The
full 4096-instance batched workload (seed 3) is checked instance by instance.
"""
import numpy as np
import pytest

import oracle
from gpu_util import TORCH_DT, require_gpu, to_device, to_host_bits, torch
from paper_2605_13864_gb300 import api, workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def make_items(instances, data):
    items, refs = [], []
    for inst, a in zip(instances, data):
        d = to_device(a, inst.dtype)
        if inst.op == 0:
            out = torch.empty((inst.cols, inst.rows), dtype=TORCH_DT[inst.dtype], device="cuda")
            items.append(("transpose", d, out))
        else:
            odt = torch.int64 if inst.dtype == "int32" else torch.float64
            out = torch.full((), -7, dtype=odt, device="cuda")
            items.append(("reduce", d, out))
        refs.append((inst, a))
    return items, refs


def check_items(items, refs, compensated=False, alone=True):
    for (op, d, out), (inst, a) in zip(items, refs):
        if op == "transpose":
            want = oracle.transpose(a)
            want = want.view(np.uint32) if want.dtype == np.float32 else want
            got = to_host_bits(out)
            assert np.array_equal(got, want), (inst, "transpose differs")
        else:
            got = out.item()
            if inst.dtype == "int32":
                assert got == oracle.sum_i64(a), inst
            else:
                ref = oracle.reduce_reference(a, inst.dtype)
                assert abs(got - ref["f64"]) <= 1e-6 * ref["abs"] + 1e-300, (inst, got, ref)
                if alone:
                    single = api.reduce_sum(d, compensated=compensated).item()
                    assert single == got or (np.isnan(single) and np.isnan(got)), (inst, single, got)


def mixed_instances():
    I = workloads.Instance
    out = []
    for dt in ("float32", "int32", "bfloat16", "float16"):
        for r, c in ((1, 1), (1, 67), (67, 1), (33, 65), (64, 64), (129, 257), (500, 3)):
            out.append(I(0, dt, r, c))
        for n in (0, 1, 7, 16384, 16385, 50000, 3 * 16384 + 9):
            out.append(I(1, dt, n, 1))
    return out


@pytest.mark.parametrize("compensated", [False, True])
def test_mixed_batch_every_dtype(compensated):
    inst = mixed_instances()
    data = workloads.batched_data(inst, seed=11)
    items, refs = make_items(inst, data)
    plan = api.BatchPlan(items, compensated=compensated)
    plan.run()
    torch.cuda.synchronize()
    api.stream_status()
    check_items(items, refs, compensated)
    plan.close()


def test_graph_replays_give_identical_results():
    inst = mixed_instances()
    data = workloads.batched_data(inst, seed=12)
    items, refs = make_items(inst, data)
    plan = api.BatchPlan(items)
    plan.run()
    torch.cuda.synchronize()
    first = [o.clone() for _, _, o in items]
    for _ in range(3):
        for _, _, o in items:
            o.fill_(0)
        plan.run()
    torch.cuda.synchronize()
    for f, (_, _, o) in zip(first, items):
        assert torch.equal(f.view(-1).view(torch.uint8), o.view(-1).view(torch.uint8))
    check_items(items, refs, alone=False)
    plan.close()


@pytest.mark.parametrize("config", range(4))
def test_every_batch_configuration(config):
    prev = api.tune_selected("batch", torch.float32)
    api.tune_select("batch", torch.float32, config)
    try:
        inst = mixed_instances()
        data = workloads.batched_data(inst, seed=13 + config)
        items, refs = make_items(inst, data)
        plan = api.BatchPlan(items, graph=(config % 2 == 0))
        plan.run()
        torch.cuda.synchronize()
        check_items(items, refs, alone=False)
        plan.close()
    finally:
        api.tune_select("batch", torch.float32, prev)


def test_batched_workload_4096_instances():
    """The full batched workload: 2048 transposes + 2048 sums, seed 3, in one
    persistent graph launch; every instance against the oracle, every sum
    also against its single call."""
    inst = workloads.batched_instances()
    data = workloads.batched_data(inst)
    items, refs = make_items(inst, data)
    plan = api.BatchPlan(items)
    info = plan.info()
    assert info["bytes"] == sum(i.algorithmic_bytes for i in inst)
    plan.run()
    torch.cuda.synchronize()
    api.stream_status()
    check_items(items, refs, alone=True)
    best = plan.autotune(reps=2)
    for _, _, o in items:
        o.fill_(0)
    plan.run()
    torch.cuda.synchronize()
    check_items(items, refs, alone=False)
    print("batched workload:", info, "autotuned:", best)
    plan.close()
