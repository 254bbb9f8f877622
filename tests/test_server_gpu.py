"""GPU tests of the continuous-batching server.

Every served result is checked against the CPU oracle (transposes bit-exact,
int32 sums exact, float sums within 1e-6 * sum|x|) and against the single
call on the same data (the same alone and in the mix: transposes bit for
bit, sums bit-identical).  Admission respects the slot count and the
device-memory budget; requests submitted while earlier steps run are launched
into further steps that overlap on the device; an open-loop Poisson trace is
replayed end to end.
"""
import numpy as np
import pytest

import oracle
from gpu_util import TORCH_DT, require_gpu, torch
from paper_2605_13864_gb300 import api, workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def host_tensor(a, dtype, pin=True):
    if dtype in ("bfloat16", "float16"):
        t = torch.from_numpy(np.ascontiguousarray(a).view(np.int16)).view(TORCH_DT[dtype])
    else:
        t = torch.from_numpy(np.ascontiguousarray(a))
    return t.pin_memory() if pin else t.clone()


def make_request(inst, a, pin=True):
    src = host_tensor(a, inst.dtype, pin)
    if inst.op == 0:
        dst = torch.empty((inst.cols, inst.rows), dtype=TORCH_DT[inst.dtype])
        op = "transpose"
    else:
        dst = torch.full((), -5, dtype=torch.int64 if inst.dtype == "int32" else torch.float64)
        op = "reduce"
    if pin:
        dst = dst.pin_memory()
    return op, src, dst


def bits(t):
    if t.dtype in (torch.bfloat16, torch.float16):
        return t.view(torch.int16).numpy()
    if t.dtype == torch.float32:
        return t.numpy().view(np.uint32)
    return t.numpy()


def check(inst, a, op, src, dst, compensated=False):
    if op == "transpose":
        want = oracle.transpose(a)
        want = want.view(np.uint32) if want.dtype == np.float32 else want
        got = bits(dst)
        if want.dtype == np.uint16:
            got = got.view(np.uint16)
        assert np.array_equal(got, want), inst
        single = api.transpose(src.cuda()).cpu()
        assert torch.equal(single.view(-1).view(torch.uint8), dst.view(-1).view(torch.uint8))
    else:
        got = dst.item()
        if inst.dtype == "int32":
            assert got == oracle.sum_i64(a), inst
        else:
            ref = oracle.reduce_reference(a, inst.dtype)
            assert abs(got - ref["f64"]) <= 1e-6 * ref["abs"] + 1e-300, (inst, got, ref)
        single = api.reduce_sum(src.cuda(), compensated=compensated).item()
        assert single == got, (inst, single, got)


def mixed(seed, count=60, max_side=300, max_len=1 << 18):
    rng = np.random.default_rng(seed)
    I = workloads.Instance
    out = []
    for k in range(count):
        dt = ("int32", "float32", "bfloat16")[k % 3]
        if k % 2 == 0:
            out.append(I(0, dt, int(rng.integers(1, max_side)), int(rng.integers(1, max_side))))
        else:
            out.append(I(1, dt, int(rng.integers(0, max_len)), 1))
    data = workloads.batched_data(out, seed=seed)
    return out, data


@pytest.mark.parametrize("per_call,compensated,copy", [(False, False, None), (False, True, None),
                                                        (True, False, None), (False, False, "engines"),
                                                        (True, False, "kernels")])
def test_served_results_equal_oracle_and_single_calls(per_call, compensated, copy):
    inst, data = mixed(21)
    sv = api.Server(budget_bytes=256 << 20, max_slots=64, n_streams=3, per_call=per_call,
                    compensated=compensated, copy=copy)
    reqs = [make_request(i, a) for i, a in zip(inst, data)]
    tickets = [sv.submit(op, s, d) for op, s, d in reqs]
    sv.drain()
    assert all(sv.poll(t) for t in tickets)
    st = sv.stats()
    assert st["completed"] == len(inst) and st["in_flight"] == 0 and st["bytes_in_use"] == 0
    for i, a, (op, s, d) in zip(inst, data, reqs):
        check(i, a, op, s, d, compensated)
    if not per_call:
        assert st["launches"] < len(inst)  # batched: fewer kernels than requests
    sv.close()


def test_growing_steps_reuse_the_step_workspace():
    """One stream serves a small step of multi-chunk sums, then larger ones:
    the step workspace is reused with a different table layout each time, so
    the completion counters must start at zero in every step."""
    I = workloads.Instance
    sv = api.Server(budget_bytes=512 << 20, max_slots=256, n_streams=1)
    for step, count in enumerate((3, 40, 120)):
        inst = [I(1, "int32", 16384 * 2 + 7 * k + step, 1) for k in range(count)]
        data = workloads.batched_data(inst, seed=60 + step)
        reqs = [make_request(i, a) for i, a in zip(inst, data)]
        for op, src, dst in reqs:
            sv.submit(op, src, dst)
        sv.drain()
        for i, a, (op, src, dst) in zip(inst, data, reqs):
            assert dst.item() == oracle.sum_i64(a), (step, i)
    sv.close()


def test_pageable_and_pinned_requests_mixed():
    """Pinned requests go through the step's copy kernels, pageable ones
    through copy-engine calls; both give the oracle's results."""
    inst, data = mixed(24, count=40)
    sv = api.Server(budget_bytes=256 << 20, max_slots=64, n_streams=2)
    reqs = [make_request(i, a, pin=(k % 2 == 0)) for k, (i, a) in enumerate(zip(inst, data))]
    for op, s, d in reqs:
        sv.submit(op, s, d)
    sv.drain()
    for i, a, (op, s, d) in zip(inst, data, reqs):
        check(i, a, op, s, d)
    sv.close()


def test_budget_and_slots_bound_admission():
    I = workloads.Instance
    inst = [I(0, "float32", 256, 256) for _ in range(12)]  # 256 KiB in + 256 KiB out each
    data = workloads.batched_data(inst, seed=5)
    sv = api.Server(budget_bytes=1 << 20, max_slots=8, n_streams=4)  # room for 2 requests
    reqs = [make_request(i, a) for i, a in zip(inst, data)]
    for op, s, d in reqs:
        sv.submit(op, s, d)
    sv.drain()
    st = sv.stats()
    assert st["peak_bytes"] <= 1 << 20
    assert st["max_in_flight"] <= 2
    assert st["completed"] == 12
    for i, a, (op, s, d) in zip(inst, data, reqs):
        check(i, a, op, s, d)
    sv.close()


def test_slot_limit_one():
    inst, data = mixed(22, count=10)
    sv = api.Server(budget_bytes=64 << 20, max_slots=1, n_streams=2)
    reqs = [make_request(i, a) for i, a in zip(inst, data)]
    for op, s, d in reqs:
        sv.submit(op, s, d)
    sv.drain()
    assert sv.stats()["max_in_flight"] == 1
    for i, a, (op, s, d) in zip(inst, data, reqs):
        check(i, a, op, s, d)
    sv.close()


def test_requests_arriving_during_a_step_overlap_with_it():
    """Continuous batching: a second wave submitted while the first step runs
    is launched on another stream before the first step completes."""
    I = workloads.Instance
    wave1 = [I(0, "float32", 2048, 2048) for _ in range(8)]   # ~128 MiB in + out
    wave2 = [I(1, "float32", 100_000, 1) for _ in range(4)]
    d1 = workloads.batched_data(wave1, seed=31)
    d2 = workloads.batched_data(wave2, seed=32)
    sv = api.Server(budget_bytes=1 << 30, max_slots=64, n_streams=4)
    r1 = [make_request(i, a) for i, a in zip(wave1, d1)]
    r2 = [make_request(i, a) for i, a in zip(wave2, d2)]
    for op, s, d in r1:
        sv.submit(op, s, d)
    assert sv.step() == 1
    for op, s, d in r2:
        sv.submit(op, s, d)
    launched = sv.step()
    st = sv.stats()
    assert launched == 1
    assert st["in_flight"] == len(wave1) + len(wave2)  # both steps on the device at once
    assert st["steps"] == 2
    sv.drain()
    for i, a, (op, s, d) in list(zip(wave1, d1, r1)) + list(zip(wave2, d2, r2)):
        check(i, a, op, s, d)
    sv.close()


def test_poll_and_unknown_tickets():
    inst, data = mixed(23, count=4)
    sv = api.Server(budget_bytes=64 << 20)
    reqs = [make_request(i, a) for i, a in zip(inst, data)]
    tickets = [sv.submit(op, s, d) for op, s, d in reqs]
    while not all(sv.poll(t) for t in tickets if t in sv._keep):
        sv.step()
    from paper_2605_13864_gb300 import OptigpuError
    with pytest.raises(OptigpuError):
        sv.poll(tickets[0])  # already reported
    sv.close()


@pytest.mark.parametrize("per_call", [False, True])
def test_replay_poisson_trace(per_call):
    reqs = workloads.serving_requests(count=1500, rate=20_000.0, seed=4, max_side=512, max_len=1 << 18)
    inst = [r.inst for r in reqs]
    data = workloads.batched_data(inst, seed=44)
    host = [make_request(i, a) for i, a in zip(inst, data)]
    sv = api.Server(budget_bytes=512 << 20, max_slots=256, n_streams=16 if per_call else 4,
                    per_call=per_call)
    lat = sv.replay(host, [r.arrival_s for r in reqs])
    assert (lat > 0).all() and np.isfinite(lat).all()
    st = sv.stats()
    assert st["completed"] == len(reqs) and st["in_flight"] == 0
    print(f"per_call={per_call}: p50 {np.percentile(lat, 50) * 1e3:.3f} ms, p99 "
          f"{np.percentile(lat, 99) * 1e3:.3f} ms, steps {st['steps']}, launches {st['launches']}")
    for i, a, (op, s, d) in zip(inst, data, host):
        check(i, a, op, s, d)
    sv.close()


@pytest.mark.parametrize("per_call,copy", [(False, None), (False, "engines"), (True, None)])
def test_failed_step_launch_rolls_back_and_retries(per_call, copy):
    """A step whose launch fails on the host (testing hook, no device fault)
    leaves nothing behind: its requests return to the queue with their arena
    space and slots freed, the error reaches the caller, and the next steps
    serve every request with results equal to the oracle's."""
    inst, data = mixed(23, count=24)
    sv = api.Server(budget_bytes=256 << 20, max_slots=16, n_streams=2, per_call=per_call, copy=copy)
    reqs = [make_request(i, a) for i, a in zip(inst, data)]
    tickets = [sv.submit(op, s, d) for op, s, d in reqs]
    sv.inject_step_failure(1)
    with pytest.raises(api.N.OptigpuError) as e:
        sv.step()
    assert "injected" in str(e.value)
    st = sv.stats()
    assert st["in_flight"] == 0 and st["bytes_in_use"] == 0 and st["pending"] == len(inst)
    sv.inject_step_failure(2)  # fails the second launch of a later step() round
    with pytest.raises(api.N.OptigpuError):
        sv.drain()
    sv.drain()
    assert all(sv.poll(t) for t in tickets)
    st = sv.stats()
    assert st["completed"] == len(inst) and st["in_flight"] == 0 and st["bytes_in_use"] == 0
    for i, a, (op, s, d) in zip(inst, data, reqs):
        check(i, a, op, s, d)
    sv.close()
