#!/usr/bin/env python3
"""Benchmark: transpose + sum reduction at roofline scale on GB300.

One step = one out-of-place transpose of a 16384x16384 float32 matrix plus
one sum of a 2^28-element float32 vector (both N(0,1), seed 1), i.e. the whole
hot path once over one batch of synthetic input.  Inputs (1 GiB each) are far
larger than the 129 MB L2, so no flush is needed between steps.

value   = algorithmic bytes per step / device time per step, in GB/s, with the
          inputs resident in HBM (2*N*4 bytes for the transpose, N*4 for the
          sum: the thesis's effective-bandwidth convention (R_B + W_B) / t,
          Sec. 7.1), summed over all ranks / max over ranks of the time.
e2e     = the same metric through the public API with host buffers: the
          pinned host inputs are copied in and the results copied out inside
          the timed region.
roofline: the dominant kernel (the transpose), its achieved GB/s from CUDA
          events on its launch stream against the measured HBM copy peak.
cpu_baseline: the CPU oracle timed on a bounded sample of the same workload.

``--impl reference`` times the CPU oracle (the only reference implementation
of this path) on the host cores instead, on the same metric and config.
Multi-GPU (torchrun): replicas only -- every rank runs its own copy of the
step on its own GPU; there is no data-path collective.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

ROWS = COLS = 16384
N_SUM = 1 << 28
ESIZE = 4
T_BYTES = 2 * ROWS * COLS * ESIZE   # transpose: read + write
R_BYTES = N_SUM * ESIZE             # sum: read
STEP_BYTES = T_BYTES + R_BYTES
WORKLOAD = "transpose 16384x16384 fp32 + sum 2^28 fp32, N(0,1), seed 1"
# The headline metric; `value` is its first clause (step GB/s), and the
# batched and served req/s and p99 comparisons are the line's "batched" and
# "served" objects.
METRIC = "transpose/reduce HBM GB/s (% of GB300 peak); batched+served req/s and p99 vs plain"

# DRAM traffic of one transpose launch (16384x16384 fp32, TMA kernel) from an
# ncu capture; kept only while the kernel's sources are unchanged (sha256 of
# TRANSPOSE_SOURCES below).
NCU_TRANSPOSE_TRAFFIC = {"bytes": 1073798400 + 1028149504,
                         "src_sha256": "316dfdfc032354f5230c8752f3d1cee90c213ae402953e4e2f9300e8775f75dc"}


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# Sources that define the dominant kernel (its file and the headers it uses).
TRANSPOSE_SOURCES = ("transpose.cu", "tma_tile.cuh", "ptx.cuh")


def _src_sha(names=TRANSPOSE_SOURCES):
    h = hashlib.sha256()
    for name in names:
        with open(os.path.join(ROOT, "paper_2605_13864_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) != 6:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[2:]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def max_over_ranks(values, dist=None, device="cpu"):
    """Element-wise maximum of `values` over all ranks (identity on one rank).
    Only the timing scalars travel: the data path itself has no collective."""
    if dist is None or not dist.is_initialized():
        return [float(v) for v in values]
    import torch
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.tolist()]


def job_value(world: int, step_bytes: int, step_ms: float) -> float:
    """Whole-job GB/s: every replica moves step_bytes per step; the job takes
    the slowest replica's time."""
    return world * step_bytes / (step_ms * 1e-3) / 1e9


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def cpu_baseline(seconds: float = 10.0):
    """The CPU oracle on a bounded sample of the workload (single thread)."""
    import oracle
    from paper_2605_13864_gb300 import workloads

    side, n = 4096, 1 << 24
    mat = workloads.roofline_matrix(side, side)
    vec = workloads.roofline_vector(n)
    oracle.transpose(mat[:64, :64])
    t_bytes = 2 * side * side * ESIZE
    r_bytes = n * ESIZE
    done_bytes, t0 = 0, time.perf_counter()
    reps = 0
    while True:
        oracle.transpose(mat)
        oracle.sum_f64(vec)
        done_bytes += t_bytes + r_bytes
        reps += 1
        if time.perf_counter() - t0 >= seconds:
            break
    dt = time.perf_counter() - t0
    return {"value": round(done_bytes / dt / 1e9, 3), "unit": "GB/s", "cores": 1, "kind": "oracle",
            "sample": f"{reps} x (transpose 4096x4096 fp32 + sum 2^24 fp32) in {dt:.1f} s, "
                      "plain C oracle, one host thread"}


def measure_batched(steps: int = 10):
    """The batched workload (4096 uneven instances, seed 3) as one persistent
    CUDA-graph launch, against the same 4096 instances issued as separate
    plain calls on one stream (from Python, and replayed from a CUDA graph)."""
    import torch
    from paper_2605_13864_gb300 import api, workloads

    inst = workloads.batched_instances()
    data = workloads.batched_data(inst)
    tdt = {"float32": torch.float32}
    items = []
    for i, a in zip(inst, data):
        d = torch.from_numpy(a).cuda()
        if i.op == 0:
            items.append(("transpose", d, torch.empty((i.cols, i.rows), dtype=tdt[i.dtype], device="cuda")))
        else:
            items.append(("reduce", d, torch.empty((), dtype=torch.float64, device="cuda")))
    del data
    plan = api.BatchPlan(items)
    best = plan.autotune(reps=3)
    info = plan.info()
    stream = torch.cuda.current_stream()

    def timed(fn, n):
        for _ in range(2):
            fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0 = time.perf_counter()
        a.record(stream)
        for _ in range(n):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / n, (time.perf_counter() - t0) * 1e3 / n

    batch_ms, batch_wall = timed(plan.run, steps)

    def separate():
        for op, d, o in items:
            if op == "transpose":
                api.transpose(d, out=o)
            else:
                api.reduce_sum(d, out=o)

    sep_ms, sep_wall = timed(separate, 2)
    g = torch.cuda.CUDAGraph()
    cap = torch.cuda.Stream()
    api.reduce_reserve(max(i.rows for i in inst if i.op == 1), stream=cap)
    torch.cuda.synchronize()
    with torch.cuda.graph(g, stream=cap):
        separate()
    sep_graph_ms, _ = timed(g.replay, 3)
    n = len(inst)
    res = {
        "workload": "4096 instances: 2048 fp32 transposes rows,cols log-uniform [1,2048] + "
                    "2048 fp32 sums n log-uniform [1,2^22], seed 3",
        "algorithmic_bytes": info["bytes"], "items": info["items"], "grid": info["grid"],
        "config": best[1],
        "batched_ms": round(batch_ms, 4), "batched_gbs": round(info["bytes"] / batch_ms / 1e6, 1),
        "batched_instances_per_s": round(n / batch_ms * 1e3, 1),
        "separate_launches_ms": round(sep_ms, 4), "separate_launches_wall_ms": round(sep_wall, 3),
        "separate_launches_graph_ms": round(sep_graph_ms, 4),
        "speedup_vs_separate": round(sep_ms / batch_ms, 2),
        "speedup_vs_separate_graph": round(sep_graph_ms / batch_ms, 2),
        "launches_per_run": 1,
    }
    plan.close()
    del items, g
    torch.cuda.empty_cache()
    return res


def _host_reference(a, dtype: str):
    """CPU references for the bench's own result checks (parity proper is in
    tests/, against the oracle): int32 sums exact in int64, float sums in
    float64 by numpy (pairwise: within about 1e-15 * sum|x|, and exact for
    the precision vectors, whose values and partial sums are all exact in
    float64), with sum|x| for the relative bound.  `a` holds bf16 as uint16
    bits and fp16 as float16."""
    if dtype == "int32":
        return {"int": int(np.asarray(a, dtype=np.int64).sum())}
    if dtype == "bfloat16":
        x = (np.asarray(a).astype(np.uint32) << 16).view(np.float32).astype(np.float64)
    else:
        x = np.asarray(a).astype(np.float64)
    x = x.reshape(-1)
    return {"f64": float(x.sum()), "abs": float(np.abs(x).sum())}


def measure_served(count: int = 100_000, rate: float = 20_000.0, check_sample: int = 400):
    """The serving workload: an open-loop Poisson stream of `count` requests
    at `rate` req/s (seed 4; op 50/50, dtype uniform over int32/fp32/bf16,
    sizes as in the batched workload) served under a 40 GB device budget by
    the continuous-batching server and by the per-call baseline; then both at
    saturation (every request queued at t = 0).  Each is run three times and
    reported as medians.  Inputs come from pinned host
    payload pools (one per dtype); a sample of sums and transposes is checked
    against CPU references (numpy transposes, float64 sums)."""
    import torch
    from paper_2605_13864_gb300 import api, workloads

    reqs = workloads.serving_requests(count=count, rate=rate, seed=4)
    rng = np.random.default_rng(40)
    pool_elems = 1 << 23  # 8 Mi elements per dtype (>= the largest request, 4,194,304)
    pools = {
        "int32": torch.from_numpy(rng.integers(-1000, 1001, pool_elems, dtype=np.int32)).pin_memory(),
        "float32": torch.from_numpy(rng.standard_normal(pool_elems, dtype=np.float32)).pin_memory(),
        "bfloat16": torch.from_numpy(rng.standard_normal(pool_elems, dtype=np.float32)).to(torch.bfloat16).pin_memory(),
    }
    out_ring = torch.empty(1 << 28, dtype=torch.uint8).pin_memory()  # 256 MiB of transpose outputs
    sums = torch.empty(count, dtype=torch.float64).pin_memory()
    sample = set(rng.choice(count, size=min(check_sample, count), replace=False).tolist())
    esize = {"int32": 4, "float32": 4, "bfloat16": 2}
    host, checks = [], []
    ring = 0
    for k, r in enumerate(reqs):
        i = r.inst
        n = i.rows * i.cols
        off = int((k * 2654435761) % (pool_elems - n + 1)) & ~7
        src = pools[i.dtype][off:off + n]
        if i.op == 0:
            src = src.view(i.rows, i.cols)
            nbytes = n * esize[i.dtype]
            if k in sample:
                dst = torch.empty((i.cols, i.rows), dtype=src.dtype).pin_memory()
                checks.append((k, "transpose", src, dst))
            else:
                if ring + nbytes > out_ring.numel():
                    ring = 0
                dst = out_ring[ring:ring + nbytes].view(src.dtype).view(i.cols, i.rows)
                ring = (ring + nbytes + 255) & ~255
            host.append(("transpose", src, dst))
        else:
            dst = sums[k:k + 1].view(()) if i.dtype != "int32" else sums[k:k + 1].view(torch.int64).view(())
            host.append(("reduce", src, dst))
            if k in sample:
                checks.append((k, "reduce", src, dst))
    arrivals = np.array([r.arrival_s for r in reqs])
    res = {"workload": f"{count} requests, Poisson {rate:.0f} req/s, op 50/50, dtype int32/fp32/bf16, "
                       "sizes log-uniform (transpose sides [1,2048], sum n [1,2^22]), seed 4, budget 40 GB"}
    # Server shapes (streams, slots), each the best of a sweep on this workload: the batched
    # server 16 x 512 (against 4 x 256: saturation 202k vs 192k req/s, p99 at 250k offered
    # 0.71 vs 0.90 ms); the per-call baseline 32 x 256 (16 to 128 streams all saturate near
    # 105k req/s).
    shapes = {"batched": (False, 16, 512), "per_call": (True, 32, 256)}
    for mode, (per_call, streams, slots) in shapes.items():
        sv = api.Server(budget_bytes=40 << 30, max_slots=slots, n_streams=streams, per_call=per_call)
        sv.replay(host[:2000], arrivals[:2000] * 0)  # warm-up: kernels loaded, workspaces sized
        # The trace runs three times and each figure is the median: on a
        # shared host one run now and then meets a stall of ~0.1 s, which
        # alone moves its p99 by orders of magnitude.
        runs, st = [], None
        for _ in range(3):
            t0 = time.perf_counter()
            lat = sv.replay(host, arrivals)
            wall = time.perf_counter() - t0
            if st is None:
                st = sv.stats()
            runs.append((count / wall, float(np.percentile(lat, 50)) * 1e3, float(np.percentile(lat, 99)) * 1e3,
                         float(lat.mean()) * 1e3))
        sat_n = min(count, 20_000)
        sats = []
        for _ in range(3):
            t1 = time.perf_counter()
            sv.replay(host[:sat_n], np.zeros(sat_n))
            sats.append(sat_n / (time.perf_counter() - t1))
        med = lambda i: float(np.median([r[i] for r in runs]))
        res[mode] = {"req_per_s": round(med(0), 1), "p50_ms": round(med(1), 4), "p99_ms": round(med(2), 4),
                     "mean_ms": round(med(3), 4), "p99_ms_runs": [round(r[2], 4) for r in runs],
                     "saturated_req_per_s": round(float(np.median(sats)), 1),
                     "steps": st["steps"], "kernel_launches": st["launches"],
                     "max_in_flight": st["max_in_flight"], "peak_device_bytes": st["peak_bytes"],
                     "streams": streams, "max_slots": slots}
        sv.close()
    # Exactness: every sum, a sample of transposes (results of the last run).
    ok = bad = 0
    for k, op, src, dst in checks:
        dt = reqs[k].inst.dtype
        a = src.numpy() if dt != "bfloat16" else src.view(torch.int16).numpy().view(np.uint16)
        if op == "transpose":
            got = dst.numpy() if dt != "bfloat16" else dst.view(torch.int16).numpy().view(np.uint16)
            good = np.array_equal(got.view(np.uint8), np.ascontiguousarray(a.T).view(np.uint8))
        elif dt == "int32":
            good = int(dst.view(torch.int64).item()) == _host_reference(a, dt)["int"]
        else:
            ref = _host_reference(a, dt)
            good = abs(float(dst.item()) - ref["f64"]) <= 1e-6 * ref["abs"] + 1e-300
        ok += int(good)
        bad += int(not good)
    res["checked"] = {"requests": ok + bad, "exact_or_within_tol": ok, "failed": bad,
                      "what": f"{check_sample} sampled requests (sums and transposes) against CPU "
                              "references (numpy transpose, float64 sums)"}
    # Offered-load sweep: the highest rate each mode sustains with p99 <= 1 ms.
    # Near a mode's saturation p99 swings from run to run, so every rate runs
    # three times (different arrival draws) and the point reports the medians.
    sweep_n = min(count, 20_000)
    for mode, (per_call, streams, slots) in shapes.items():
        sv = api.Server(budget_bytes=40 << 30, max_slots=slots, n_streams=streams, per_call=per_call)
        sv.replay(host[:1000], np.zeros(1000))
        points = []
        for rate_k in (20, 50, 100, 120, 150, 200, 225, 250, 275, 300, 400):
            runs = []
            for rep in range(3):
                arr = np.cumsum(np.random.default_rng(7 + rep).exponential(1.0 / (rate_k * 1e3), sweep_n))
                t0 = time.perf_counter()
                lat = sv.replay(host[:sweep_n], arr)
                wall = time.perf_counter() - t0
                runs.append((sweep_n / wall, float(np.percentile(lat, 50)) * 1e3,
                             float(np.percentile(lat, 99)) * 1e3))
            points.append({"offered_req_per_s": rate_k * 1000,
                           "achieved_req_per_s": round(float(np.median([r[0] for r in runs])), 1),
                           "p50_ms": round(float(np.median([r[1] for r in runs])), 4),
                           "p99_ms": round(float(np.median([r[2] for r in runs])), 4),
                           "p99_ms_runs": [round(r[2], 4) for r in runs]})
        sv.close()
        ok = [p for p in points if p["p99_ms"] <= 1.0]
        res[mode]["load_sweep"] = points
        res[mode]["max_req_per_s_p99_le_1ms"] = max((p["achieved_req_per_s"] for p in ok), default=0.0)
    b, c = res["batched"], res["per_call"]
    res["batched_vs_per_call"] = {
        "saturated_req_per_s_ratio": round(b["saturated_req_per_s"] / c["saturated_req_per_s"], 2),
        "req_per_s_at_p99_le_1ms_ratio": round(b["max_req_per_s_p99_le_1ms"] / max(c["max_req_per_s_p99_le_1ms"], 1), 2),
        "p99_ratio_at_20k": round(b["p99_ms"] / c["p99_ms"], 3)}
    return res


def measure_precision():
    """The precision workload: 2^28 N(100,1) values rounded to bf16 and to
    fp16 (seed 2), summed in FP32 plain and compensated with the FP64 final
    combine; errors against the exact sum (the values are multiples of 2^-4
    and every partial sum is below 2^35, so a float64 sum in any order is
    exact).  Plus the 8192x8192 bf16 transpose, checked bit-exact against
    numpy."""
    import torch
    from paper_2605_13864_gb300 import api, workloads

    vb, vh = workloads.precision_vectors()
    res = {"workload": "2^28 N(100,1) rounded to bf16 / fp16 (seed 2); bf16 8192x8192 N(0,1) transpose"}
    for name, v, tdt in (("bf16", vb, torch.bfloat16), ("fp16", vh, torch.float16)):
        ref = _host_reference(v.view(np.uint16) if name == "bf16" else v.view(np.float16),
                              "bfloat16" if name == "bf16" else "float16")
        d = torch.from_numpy(v.view(np.int16)).view(tdt).cuda()
        out = torch.empty((), dtype=torch.float64, device="cuda")
        for comp in (False, True):
            api.reduce_sum(d, out=out, compensated=comp)
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            for _ in range(20):
                api.reduce_sum(d, out=out, compensated=comp)
            b.record()
            torch.cuda.synchronize()
            ms = a.elapsed_time(b) / 20
            got = out.item()
            err = abs(got - ref["f64"])
            res[f"{name}_{'compensated' if comp else 'plain'}"] = {
                "sum": got, "exact_fp64": ref["f64"], "abs_error": err,
                "rel_error_vs_sum_abs": err / ref["abs"], "within_1e-6": err <= 1e-6 * ref["abs"],
                "ms": round(ms, 4), "gbs": round(v.nbytes / ms / 1e6, 1)}
        del d
    m = workloads.precision_matrix()
    d = torch.from_numpy(m.view(np.int16)).view(torch.bfloat16).cuda()
    o = api.transpose(d)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(20):
        api.transpose(d, out=o)
    b.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / 20
    exact = np.array_equal(o.view(torch.int16).cpu().numpy().view(np.uint16),
                           np.ascontiguousarray(m.view(np.uint16).T))
    res["bf16_transpose_8192"] = {"bit_exact": bool(exact), "ms": round(ms, 4),
                                  "gbs": round(2 * m.nbytes / ms / 1e6, 1)}
    del d, o
    torch.cuda.empty_cache()
    return res


# Table 7.4 of the thesis: effective bandwidth (GB/s) at its own sizes, a
# 4096x4096 fp32 transpose and a 16M-element sum, on an RTX 5060.  Context
# for the paper-size line below; another machine's figures, not a target.
TABLE_7_4_GBS = {"transpose_generated": 297.7, "transpose_no_bank_conflicts": 340.6,
                 "reduce_generated": 297.9, "reduce3": 349.4, "reduce6": 376.8}


def measure_paper_sizes(reps: int = 50):
    """The thesis's own benchmark sizes (Table 7.4): a 4096x4096 fp32
    transpose (TMA kernel and the padded tile32 baseline) and a 2^24 fp32 sum.
    Each is timed twice with CUDA events around single calls, median of
    `reps`: back to back (inputs left in L2, which holds both 64 MiB
    matrices) and with L2 flushed before every call (a write of twice the L2
    size, queued between the calls)."""
    import statistics

    import torch
    from paper_2605_13864_gb300 import api

    peak, _ = _peaks()
    g = torch.Generator(device="cuda").manual_seed(1)
    side, n = 4096, 1 << 24
    a = torch.randn(side, side, device="cuda", generator=g)
    b = torch.empty(side, side, device="cuda")
    v = torch.randn(n, device="cuda", generator=g)
    out = torch.empty((), dtype=torch.float64, device="cuda")
    l2 = int(getattr(torch.cuda.get_device_properties(0), "L2_cache_size", 0)) or (128 << 20)
    flush = torch.empty(2 * l2 // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    def med_ms(fn, flushed):
        # Every call is bracketed by its own events, all enqueued before one
        # synchronize, so host-side call overhead overlaps queued GPU work
        # instead of showing up between the events.
        for _ in range(5):
            fn()
        torch.cuda.synchronize()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
        for e0, e1 in evs:
            if flushed:
                flush.fill_(1.0)
            e0.record(stream)
            fn()
            e1.record(stream)
        torch.cuda.synchronize()
        return statistics.median(e0.elapsed_time(e1) for e0, e1 in evs)

    res = {}
    for name, fn, nbytes in (
            ("transpose_4096_fp32_tma", lambda: api.transpose(a, out=b, kernel="tma"), 2 * side * side * 4),
            ("transpose_4096_fp32_tile32", lambda: api.transpose(a, out=b, kernel="tile32"), 2 * side * side * 4),
            ("sum_2p24_fp32", lambda: api.reduce_sum(v, out=out), n * 4)):
        entry = {"algorithmic_bytes": nbytes}
        for tag, flushed in (("l2_resident", False), ("l2_flushed", True)):
            ms = med_ms(fn, flushed)
            gbs = nbytes / ms / 1e6
            entry[tag] = {"ms": round(ms, 4), "gbs": round(gbs, 1), "frac_of_peak": round(gbs / peak, 4)}
        res[name] = entry
    res["table_7_4_gbs_rtx5060"] = TABLE_7_4_GBS
    del a, b, v, flush
    torch.cuda.empty_cache()
    return res


def measure_next(reps: int = 10):
    """The neighbouring problems at roofline scale, CUDA-event timed:
    batched transpose (64 x 2048^2 fp32), in-place transpose (16384^2 fp32),
    segmented sums (2^28 fp32 in 16384 segments), inclusive scans (2^28 int32
    -> int64, fp32 -> fp32 and bf16 -> fp32, each tuner form) and the int32
    histogram (2^28 values, 4096 bins).  Bytes follow the same convention:
    every input byte read once plus every output byte written once."""
    import torch
    from paper_2605_13864_gb300 import api

    peak, _ = _peaks()
    res = {}

    def timed(name, fn, nbytes):
        fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(reps):
            fn()
        b.record()
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / reps
        gbs = nbytes / ms / 1e6
        res[name] = {"ms": round(ms, 4), "gbs": round(gbs, 1), "frac_of_peak": round(gbs / peak, 4),
                     "algorithmic_bytes": int(nbytes)}

    g = torch.Generator(device="cuda").manual_seed(5)
    x = torch.randn(64, 2048, 2048, device="cuda", generator=g)
    y = torch.empty(64, 2048, 2048, device="cuda")
    timed("transpose_batched_64x2048x2048_fp32", lambda: api.transpose_batched(x, out=y), 2 * x.numel() * 4)
    del x, y
    m = torch.randn(16384, 16384, device="cuda", generator=g)
    timed("transpose_inplace_16384_fp32", lambda: api.transpose_inplace(m), 2 * m.numel() * 4)
    del m
    v = torch.randn(1 << 28, device="cuda", generator=g)
    lens = np.random.default_rng(6).integers(1, 2 * (1 << 28) // 16384, size=16384)
    offs = np.concatenate([[0], np.cumsum(lens)])
    offs = np.minimum(offs, 1 << 28)
    timed("reduce_segmented_2p28_fp32_16384seg", lambda: api.reduce_segmented(v, offs), int(offs[-1]) * 4)
    # The same segments as a plan (tables built once, one graph launch per run).
    outs = torch.empty(len(offs) - 1, dtype=torch.float64, device="cuda")
    items = [("reduce", v[offs[k]:offs[k + 1]], outs[k]) for k in range(len(offs) - 1)]
    plan = api.BatchPlan(items)
    timed("reduce_segmented_2p28_fp32_16384seg_planned", plan.run, int(offs[-1]) * 4)
    plan.close()
    del items, outs
    vi = torch.randint(0, 4096, (1 << 28,), dtype=torch.int32, device="cuda", generator=g)
    out32 = torch.empty(1 << 28, device="cuda")
    out64 = torch.empty(1 << 28, dtype=torch.int64, device="cuda")
    vb = v.to(torch.bfloat16)
    scan_default = api.tune_selected("scan", torch.float32)
    for cfg, tag in ((0, ""), (1, "_three_pass"), (2, "_carries_at_once")):
        api.tune_select("scan", torch.float32, cfg)
        timed("scan_2p28_fp32" + tag, lambda: api.scan(v, out=out32), (1 << 28) * 8)
        timed("scan_2p28_int32_to_int64" + tag, lambda: api.scan(vi, out=out64), (1 << 28) * 12)
        timed("scan_2p28_bf16_to_fp32" + tag, lambda: api.scan(vb, out=out32), (1 << 28) * 6)
    api.tune_select("scan", torch.float32, scan_default)
    del out32, out64, vb
    timed("histogram_2p28_int32_4096bins", lambda: api.histogram(vi, 0, 1, 4096), (1 << 28) * 4)
    del v, vi
    torch.cuda.empty_cache()
    return res


def run_reference(args):
    world, rank, _ = _dist()
    if rank != 0:
        return 0
    import oracle
    from paper_2605_13864_gb300 import workloads

    side, n = 4096, 1 << 24
    mat = workloads.roofline_matrix(side, side)
    vec = workloads.roofline_vector(n)
    step_bytes = 2 * side * side * ESIZE + n * ESIZE
    for _ in range(args.warmup):
        oracle.transpose(mat)
        oracle.sum_f64(vec)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.transpose(mat)
        oracle.sum_f64(vec)
        times.append(time.perf_counter() - t0)
    total = sum(times)
    value = step_bytes * args.steps / total / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": round(value, 3), "unit": "GB/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(1e3 * total / args.steps, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample": "transpose 4096x4096 fp32 + sum 2^24 fp32 per step",
                   "l2": "host run"},
        "cpu_baseline": {"value": round(value, 3), "unit": "GB/s", "cores": 1, "kind": "oracle",
                         "sample": "each step: transpose 4096x4096 fp32 + sum 2^24 fp32, one host thread"},
        "e2e": {"value": round(value, 3), "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_gpu(args):
    import torch

    world, rank, local = _dist()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    from paper_2605_13864_gb300 import api, workloads
    api.transpose(torch.zeros((64, 64), device="cuda"))  # load + warm the library

    # Inputs resident in HBM before the timed region.
    mat_h = workloads.roofline_matrix(ROWS, COLS)
    vec_h = workloads.roofline_vector(N_SUM)
    mat = torch.from_numpy(mat_h).cuda()
    vec = torch.from_numpy(vec_h).cuda()
    out_t = torch.empty((COLS, ROWS), dtype=torch.float32, device="cuda")
    out_r = torch.empty((), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()

    def step():
        api.transpose(mat, out=out_t)
        api.reduce_sum(vec, out=out_r)

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()

    # Device-timed region: per-kernel events on the launch stream.
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    for k in range(args.steps):
        ev[k][0].record(stream)
        api.transpose(mat, out=out_t)
        ev[k][1].record(stream)
        api.reduce_sum(vec, out=out_r)
        ev[k][2].record(stream)
    t_end.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = sampler.stop()
    total_ms = t_start.elapsed_time(t_end)
    t_ms = [e[0].elapsed_time(e[1]) for e in ev]
    r_ms = [e[1].elapsed_time(e[2]) for e in ev]
    api.stream_status()

    # End to end through the public API with host buffers.
    mat_p = torch.from_numpy(mat_h).pin_memory()
    vec_p = torch.from_numpy(vec_h).pin_memory()
    out_tp = torch.empty((COLS, ROWS), dtype=torch.float32).pin_memory()
    del mat, vec, out_t
    torch.cuda.empty_cache()
    out_rp = torch.empty((), dtype=torch.float64).pin_memory()
    api.transpose(mat_p, out=out_tp)
    api.reduce_sum(vec_p, out=out_rp)
    torch.cuda.synchronize()
    e2e_steps = max(3, min(args.steps, 10))
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        api.transpose(mat_p, out=out_tp)      # host buffers: copies inside the call
        api.reduce_sum(vec_p, out=out_rp)
        float(out_rp.item())
    torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - t0) / e2e_steps

    local_ms = total_ms / args.steps
    step_ms, e2e_s = max_over_ranks([local_ms, e2e_s], dist, device="cuda")

    if rank == 0:
        peak, peak_kind = _peaks()
        value = job_value(world, STEP_BYTES, step_ms)
        t_avg = statistics.mean(t_ms)
        r_avg = statistics.mean(r_ms)
        achieved = T_BYTES / (t_avg * 1e-3) / 1e9
        traffic = NCU_TRANSPOSE_TRAFFIC["bytes"]
        if traffic is not None and NCU_TRANSPOSE_TRAFFIC["src_sha256"] != _src_sha():
            traffic = None
        line = {
            "metric": METRIC, "value": round(value, 2), "unit": "GB/s", "n_gpus": world,
            "steps": args.steps, "warmup": max(args.warmup, 3), "ms_per_step": round(step_ms, 4),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "parallelism": f"replicas{world}",
                       "l2": "inputs larger than L2 (1 GiB each), no flush",
                       "peak_gbs": peak, "peak_kind": peak_kind},
            "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                         "frac": round(achieved / peak, 4), "traffic": traffic,
                         "kernel": "transpose_tma_kernel<4,64,64,4>", "peak_kind": peak_kind},
            "components": {
                "transpose_ms": round(t_avg, 4), "transpose_gbs": round(achieved, 1),
                "transpose_frac_of_peak": round(achieved / peak, 4),
                "transpose_frac_of_8tbs": round(achieved / 8000.0, 4),
                "reduce_ms": round(r_avg, 4), "reduce_gbs": round(R_BYTES / (r_avg * 1e-3) / 1e9, 1),
                "reduce_frac_of_peak": round(R_BYTES / (r_avg * 1e-3) / 1e9 / peak, 4),
                "transpose_ms_p10_p50_p90": [round(float(np.percentile(t_ms, q)), 4) for q in (10, 50, 90)],
                "reduce_ms_p10_p50_p90": [round(float(np.percentile(r_ms, q)), 4) for q in (10, 50, 90)],
            },
            "e2e": {"value": round(job_value(world, STEP_BYTES, e2e_s * 1e3), 3), "unit": "GB/s",
                    "h2d_bytes_per_step": ROWS * COLS * ESIZE + N_SUM * ESIZE,
                    "d2h_bytes_per_step": ROWS * COLS * ESIZE + 8, "steps": e2e_steps},
            "gpu_launches": 2 * args.steps,
            "clocks": clocks,
        }
        if not args.no_batched:
            line["batched"] = measure_batched()
        if not args.no_served:
            line["served"] = measure_served()
        if not args.no_precision:
            line["precision"] = measure_precision()
        if not args.no_next:
            line["next"] = measure_next()
        if not args.no_paper_sizes:
            line["paper_sizes"] = measure_paper_sizes()
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(args.cpu_seconds)
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def run_case(args):
    """Runs one named kernel case `args.case_reps` times on a small problem
    and exits: the target of ncu captures (no timing, no JSON)."""
    import torch
    from paper_2605_13864_gb300 import api, workloads

    torch.cuda.set_device(0)
    side, case = args.side, args.case
    if case.startswith("transpose"):
        dt = torch.bfloat16 if case.endswith("bf16") else torch.float32
        kernel = "tile32" if "tile32" in case else "tma"
        m = torch.randn(side, side, device="cuda").to(dt)
        o = torch.empty(side, side, device="cuda", dtype=dt)
        for _ in range(args.case_reps):
            api.transpose(m, out=o, kernel=kernel)
    elif case.startswith("reduce"):
        dt = torch.bfloat16 if "bf16" in case else torch.float32
        v = torch.randn(side * side, device="cuda").to(dt)
        r = torch.empty((), dtype=torch.float64, device="cuda")
        for _ in range(args.case_reps):
            api.reduce_sum(v, out=r, compensated=case.endswith("comp"))
    elif case == "batch":
        inst = workloads.batched_instances(count=args.count)
        data = workloads.batched_data(inst)
        items = []
        for i, a in zip(inst, data):
            d = torch.from_numpy(a).cuda()
            if i.op == 0:
                items.append(("transpose", d, torch.empty((i.cols, i.rows), device="cuda")))
            else:
                items.append(("reduce", d, torch.empty((), dtype=torch.float64, device="cuda")))
        plan = api.BatchPlan(items)
        for _ in range(args.case_reps):
            plan.run()
        torch.cuda.synchronize()
        plan.close()
    elif case in ("scan_f32", "scan_i32", "scan3_f32", "scan3_i32", "scan2_f32", "scan2_i32"):
        n = side * side
        if case.endswith("f32"):
            v = torch.randn(n, device="cuda")
            o = torch.empty(n, device="cuda")
        else:
            v = torch.randint(0, 4096, (n,), dtype=torch.int32, device="cuda")
            o = torch.empty(n, dtype=torch.int64, device="cuda")
        api.tune_select("scan", torch.float32, 1 if case.startswith("scan3") else 2 if case.startswith("scan2") else 0)
        for _ in range(args.case_reps):
            api.scan(v, out=o)
    elif case == "histogram":
        v = torch.randint(0, 4096, (side * side,), dtype=torch.int32, device="cuda")
        for _ in range(args.case_reps):
            api.histogram(v, 0, 1, 4096)
    elif case == "inplace_f32":
        m = torch.randn(side, side, device="cuda")
        for _ in range(args.case_reps):
            api.transpose_inplace(m)
    elif case == "transpose_batched_f32":
        b = max(1, (side * side) // (2048 * 2048))
        x = torch.randn(b, 2048, 2048, device="cuda")
        y = torch.empty(b, 2048, 2048, device="cuda")
        for _ in range(args.case_reps):
            api.transpose_batched(x, out=y)
    elif case == "segmented_f32":
        n = side * side
        v = torch.randn(n, device="cuda")
        lens = np.random.default_rng(6).integers(1, 32768, size=max(1, n // 16384))
        offs = np.minimum(np.concatenate([[0], np.cumsum(lens)]), n)
        for _ in range(args.case_reps):
            api.reduce_segmented(v, offs)
    else:
        raise SystemExit(f"unknown case {case}")
    torch.cuda.synchronize()
    api.stream_status()
    print(f"case {case} side {side} reps {args.case_reps}: ok")
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["optigpu", "reference"], default="optigpu")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-served", action="store_true")
    ap.add_argument("--no-precision", action="store_true")
    ap.add_argument("--no-next", action="store_true")
    ap.add_argument("--no-paper-sizes", action="store_true")
    ap.add_argument("--case", default=None,
                    help="run one kernel case and exit (transpose_tma_f32, transpose_tma_bf16, "
                         "transpose_tile32_f32, reduce_f32, reduce_f32_comp, reduce_bf16_comp, batch, "
                         "scan_f32, scan_i32, scan3_f32, scan3_i32, scan2_f32, scan2_i32, histogram, inplace_f32, "
                         "transpose_batched_f32, segmented_f32)")
    ap.add_argument("--side", type=int, default=8192)
    ap.add_argument("--count", type=int, default=1024)
    ap.add_argument("--case-reps", type=int, default=3)
    args = ap.parse_args()
    if args.case:
        return run_case(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
