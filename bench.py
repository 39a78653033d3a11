#!/usr/bin/env python3
"""QMC-CPW Greeks throughput on GB300.

One step = one pass of the whole hot path (Sobol' + scramble, inverse normal,
path construction, conditional pathwise Greeks, per-replicate reduction and
statistics) over one batch: the d = 64 grid of 36 contracts
({arith, binary, lookback} x {bridge, PCA} x K in {90,100,110} x sigma in
{0.1, 0.3}, N = 2^20 points, R = 32 replicates), in MIXED precision.  The
FP64 form of the same batch is timed beside it.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun the batch is split over the ranks (strong scaling: the same
job on more GPUs): every contract's replicates in ranges, one per rank, each
rank computing its ranges with the job's seed; each step ends with one sum
over ranks (NCCL) of the replicate estimates and the statistics on the GPU,
so the result equals one GPU's.  Rank 0 prints one JSON line.
`--impl reference` times the CPU oracle (the test oracle, on the host cores)
on bounded samples of the same workload.
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads as W  # noqa: E402
from paper_2209_11337_gb300 import shard  # noqa: E402

METRIC = "QMC-CPW Greeks throughput (N·d points/s) mixed vs FP64; serving p50/p99 latency"
UNIT = "point-dates/s"
WORKLOAD = ("d=64 grid: {arith,binary,lookback} x {bridge,pca} x K{90,100,110} x sigma{0.1,0.3}, "
            "S0=100 r=0.05 T=1, N=2^20 points x R=32 replicates per contract (36 contracts)")
# The roofline of the float path (one element = one point-date): about 24
# FP32 operations (an FMA is one) and 2 SFU operations per element for the
# algorithmic minimum -- the uniform, an inverse normal of ~12 FMAs and a
# division, 3 FMAs of the bridge, an exponential, ~4 for the running sums --
# so the ceiling is min(FP32 op rate / 24, SFU rate / 2) point-dates/s; the
# tensor-core PCA adds 2n flops per split product per element on the tensor
# pipe (bf16: Ahat in three parts, five products; tf32: three).  Rates are the
# library's micro-benchmarks on this GPU (paper_2209_11337_gb300/pipe_peaks_gb300.json).
OPS_PER_ELEMENT, SFU_PER_ELEMENT = 24, 2
TC_PRODUCTS = {"tc-bf16": 5, "tc-tf32": 3}


def dist_info():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


class Ranks:
    """The job's ranks: one process per GPU, independent contracts per rank
    (no data-path collective); the only collectives are the timing barrier
    and the max over ranks of a step time.  `backend` "nccl" on the GPUs,
    "gloo" for host-side checks."""

    def __init__(self, world: int, backend: str = "nccl", local: int = 0):
        import torch
        self.world = world
        self.dist = None
        self.device = torch.device("cuda", local) if backend == "nccl" else torch.device("cpu")
        if world > 1:
            import torch.distributed as dist
            if backend == "nccl":
                dist.init_process_group("nccl", device_id=self.device)
            else:
                dist.init_process_group("gloo")
            self.dist = dist

    def barrier(self):
        if self.dist is not None:
            self.dist.barrier()

    def max_over_ranks(self, x: float) -> float:
        if self.dist is None:
            return x
        import torch
        t = torch.tensor([x], dtype=torch.float64, device=self.device)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX)
        return float(t.item())

    def close(self):
        if self.dist is not None:
            self.dist.destroy_process_group()


def job_value(job_point_dates: int, max_ms: float) -> float:
    """Whole-job throughput: the job's distinct point-dates (each replicate
    counted once, whichever rank ran it) over the slowest rank's step time."""
    return job_point_dates / (max_ms / 1e3)


def elements(contracts) -> int:
    return sum(c.N * c.R * c.d for c in contracts)


def pipe_peaks() -> dict:
    from paper_2209_11337_gb300 import peaks
    return peaks.load()


def measured_peaks() -> dict:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


# the kernel each launch segment of a batch runs, by grid precision
SEGMENT_KERNELS = {
    "mixed": ("fused_kernel<float, bridge>", "fused_kernel<float, standard>", "pca_tcs_kernel",
              "fused_kernel<float, pca>"),
    "tc-bf16": ("fused_kernel<float, bridge>", "fused_kernel<float, standard>", "pca_tcs_kernel<bf16>",
                "pca_tc_kernel<bf16>"),
    "tc-tf32": ("fused_kernel<float, bridge>", "fused_kernel<float, standard>", "pca_tcs_kernel<tf32>",
                "pca_tc_kernel<tf32>"),
}
# DRAM read + write bytes of one full-size launch of the grid's kernels from
# one ncu capture (profiles/dram_bytes_grid_d64_tcbf16.md); None for a kernel
# changed since
GRID_TRAFFIC = {"pca_tc_kernel<bf16>": 1408768 + 0, "fused_kernel<float, bridge>": 690944 + 0}
# launch segments of a batch: bridge, standard, streamed and resident PCA (the
# leading-coordinate segments that follow are not in the grid)
ROOFLINE_SEGMENTS = 4


def segment_contracts(contracts, seg: int):
    if seg == 0:
        return [c for c in contracts if c.construction == W.BB]
    if seg == 1:
        return [c for c in contracts if c.construction == W.STD]
    if seg < ROOFLINE_SEGMENTS:
        return [c for c in contracts if c.construction == W.PCA and ((c.d - 1 > 64) == (seg == 2))]
    return []


def ceilings(grid_precision: str, contracts, peaks: dict) -> dict:
    """Point-dates/s ceilings of a launch segment's contracts: FP32 op rate /
    24, SFU rate / 2, and for tensor-core PCA the bf16/tf32 rate over the
    split products' flops per element (averaged over the contracts' work)."""
    out = {}
    if peaks.get("fp32_fma_tflops"):
        out["fp32"] = peaks["fp32_fma_tflops"] * 1e12 / 2 / OPS_PER_ELEMENT
    sfu = peaks.get("sfu_ex2_gops")
    if sfu:
        out["sfu"] = sfu * 1e9 / SFU_PER_ELEMENT
    if grid_precision in TC_PRODUCTS and contracts and all(c.construction == W.PCA for c in contracts):
        rate = peaks.get("tc_bf16_tflops" if grid_precision == "tc-bf16" else "tc_tf32_tflops")
        work = sum(c.N * c.R * c.d for c in contracts)
        flops = sum(c.N * c.R * c.d * 2.0 * (c.d - 1) * TC_PRODUCTS[grid_precision] for c in contracts)
        if rate and flops > 0:
            out["tensor"] = rate * 1e12 / (flops / work)
    return out


def roofline(grid_precision: str, contracts, segment_ms, peaks: dict) -> dict:
    """Roofline of the launch segment that takes the most time (its kernel is
    the dominant one of the step): its point-dates over its event-timed
    duration against the lowest ceiling, reported as FP32 operations (24 per
    point-date) against the measured FP32 operation rate when that ceiling is
    the FP32 one.  `segments` gives the same for every segment with work."""
    segment_ms = list(segment_ms)[:ROOFLINE_SEGMENTS]
    segs = []
    for k, ms_k in enumerate(segment_ms):
        mine = segment_contracts(contracts, k)
        if not mine or ms_k <= 0:
            continue
        pd = sum(c.N * c.R * c.d for c in mine) / (ms_k / 1e3)
        ceil = ceilings(grid_precision if k >= 2 else "mixed", mine, peaks)
        bound = min(ceil, key=ceil.get) if ceil else None
        segs.append({"kernel": SEGMENT_KERNELS[grid_precision][k], "ms_per_launch": ms_k, "point_dates_per_s": pd,
                     "ceilings_point_dates_per_s": ceil, "limit": bound,
                     "frac": pd / ceil[bound] if bound else None})
    top = max(segs, key=lambda x: x["ms_per_launch"])
    op_peak = peaks.get("fp32_fma_tflops", 0.0) / 2  # tera-operations/s (an FMA is one)
    achieved_ops = top["point_dates_per_s"] * OPS_PER_ELEMENT / 1e12
    return {"bound": "alu", "achieved": achieved_ops, "peak": op_peak, "unit": "Top/s (FP32 operations)",
            "frac": achieved_ops / op_peak if op_peak else None,
            "traffic": GRID_TRAFFIC.get(top["kernel"]), "kernel": top["kernel"], "ms_per_launch": top["ms_per_launch"],
            "point_dates_per_s": top["point_dates_per_s"], "ceilings_point_dates_per_s": top["ceilings_point_dates_per_s"],
            "limit": top["limit"], "frac_of_lowest_ceiling": top["frac"],
            "peak_note": "of measured: FP32 operation rate = FFMA lane rate of the library's micro-benchmark "
                         "(pipe_peaks_gb300.json, burst); ceilings per point-date: FP32 ops/24, SFU(ex2)/2, "
                         "tensor/(2n x split products)",
            "segments": segs}


# ---------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
                power.append(float(f[3]))
            except ValueError:
                continue
            for name, val in zip(names, f[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "power_w_max": max(power) if power else None, "samples": len(sm), "reasons": sorted(reasons)}


# ---------------------------------------------------------------------------
def cpu_baseline(contracts, budget_s: float = 12.0) -> dict:
    """The oracle as it stands, on every host core, over a bounded sample of the workload:
    each contract with N = 2^11 points (all 32 replicates), contracts in order until the
    time budget is spent."""
    import oracle
    cores = os.cpu_count() or 1
    oracle.build()
    done, elems, t0 = 0, 0, time.perf_counter()
    for c in contracts:
        n = 2 ** 11
        oracle.greeks(W.SCRAMBLE_SEED, c.type, c.d, c.K, c.T, c.S0, c.r, c.sigma, c.construction, n, c.R,
                      threads=cores)
        done += 1
        elems += n * c.R * c.d
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    # one core, comparable to the paper's sequential CPU: the first contracts at N = 2^9
    t1, e1, done1 = time.perf_counter(), 0, 0
    for c in contracts:
        n = 2 ** 9
        oracle.greeks(W.SCRAMBLE_SEED, c.type, c.d, c.K, c.T, c.S0, c.r, c.sigma, c.construction, n, c.R, threads=1)
        done1 += 1
        e1 += n * c.R * c.d
        if time.perf_counter() - t1 > budget_s / 3:
            break
    dt1 = time.perf_counter() - t1
    return {"value": elems / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{done} of {len(contracts)} contracts at N=2^11, R=32, d=64 ({elems} point-dates, "
                      f"{dt:.1f} s wall)",
            "single_core": {"value": e1 / dt1, "unit": UNIT, "cores": 1,
                            "sample": f"{done1} contracts at N=2^9, R=32, d=64 ({e1} point-dates, {dt1:.1f} s)"}}


PILOT_N = 2 ** 12


def request_size(pilot_se: float, target_se: float, n_pilot: int = PILOT_N, n_max: int = 2 ** 22) -> int:
    """Points of a request: the smallest power of two in [n_pilot, n_max] whose
    standard error, the pilot's scaled as 1/N, meets the target."""
    ratio = max(pilot_se, 1e-300) / target_se
    N = n_pilot
    while N < n_max and ratio * n_pilot / N > 1.0:
        N *= 2
    return N


def combine_runs(per1, n1: int, per2, n2: int):
    """Per-replicate estimates of points 0 .. n1+n2-1 from a run over the
    first n1 points and a run over the next n2 (the point-weighted mean)."""
    return (n1 * per1 + n2 * per2) / (n1 + n2)


def serve(q, plan, precision, rate_hz, duration_s, warmup_s=1.0, seed=5):
    """Poisson arrivals through the device-resident serving loop.

    Each request is a book-like contract with a target delta standard error in
    {1e-3, 1e-4, 1e-5}: a pilot run (N1 = 2^12, R = 16) gives the delta SE at
    2^12, and N is the smallest power of two in [2^12, 2^22] whose SE, scaled
    as 1/N, meets the target.  The pilot's points are the first 2^12 of the N
    (the Sobol' sequence extends), so the main run covers points N1 .. N-1
    only (first_point = N1) and each replicate's estimate is the
    point-weighted mean of its two runs; a request whose pilot meets the
    target is answered by the pilot.  Latency = completion of the request's
    last run - arrival; `delta_se_target_met` is the share of requests whose
    answer's delta standard error meets the target (the 1/N scaling of the
    sizing rule is a prediction).  Offered load = the point-dates of the requests that
    arrive in the window (sum of N R d), per second of the window; requests
    arriving in the first `warmup_s` seconds are run but not counted."""
    import queue

    N1 = PILOT_N
    reqs = W.arrivals(rate_hz=rate_hz, duration_s=warmup_s + duration_s, seed=seed, R=16)
    # the requests are bridge contracts: the MIXED kernel without the PCA product fits three CTAs per SM
    q.qmccpw_server_start(plan, precision=precision, max_inflight=1024, max_inflight_bytes=256 << 20,
                          constructions=[q.QMCCPW_BB])
    pilots = queue.Queue()
    mains = queue.Queue()
    lat, offered_elems, Ns, met = [], [0], [], []
    t0 = time.perf_counter()

    def submitter():
        for i, rq in enumerate(reqs):
            delay = rq.arrival_s - (time.perf_counter() - t0)
            if delay > 0:
                time.sleep(delay)
            pilots.put((i, rq, q.qmccpw_submit(plan, rq.contract)))
        pilots.put(None)

    def sizer():
        while True:
            item = pilots.get()
            if item is None:
                mains.put(None)
                return
            i, rq, t = item
            _, se, per1 = q.qmccpw_wait(plan, t, rq.contract.R, 600000)
            N = request_size(se[1], rq.target_se)
            if N == N1:
                mains.put((i, rq, N, per1, None, time.perf_counter() - t0))
            else:
                rest = dataclasses.replace(rq.contract, N=N - N1, first_point=N1)
                mains.put((i, rq, N, per1, q.qmccpw_submit(plan, rest), None))

    def finisher():
        while True:
            item = mains.get()
            if item is None:
                return
            i, rq, N, per1, t, done = item
            if t is not None:
                _, _, per2 = q.qmccpw_wait(plan, t, rq.contract.R, 600000)
                done = time.perf_counter() - t0
                per1 = combine_runs(per1, N1, per2, N - N1)   # the request's per-replicate estimates
            if rq.arrival_s >= warmup_s:
                lat.append(done - rq.arrival_s)
                offered_elems[0] += N * rq.contract.R * rq.contract.d
                Ns.append(N)
                # the request's answer: its delta's standard error over the replicates, against the target
                met.append(per1[:, 1].std(ddof=1) / math.sqrt(per1.shape[0]) <= rq.target_se)

    threads = [threading.Thread(target=f) for f in (submitter, sizer, finisher)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    wall = time.perf_counter() - t0
    stats = q.qmccpw_server_get_stats(plan)
    q.qmccpw_server_stop(plan)
    lat_ms = sorted(1e3 * x for x in lat)
    pct = lambda p: lat_ms[min(len(lat_ms) - 1, int(p * len(lat_ms)))] if lat_ms else None
    return {"rate_hz": rate_hz, "window_s": duration_s, "requests": len(lat_ms), "p50_ms": pct(0.50),
            "p99_ms": pct(0.99), "max_ms": lat_ms[-1] if lat_ms else None,
            "throughput_point_dates_per_s": stats["point_dates"] / wall, "wall_s": wall,
            "offered_point_dates_per_s": offered_elems[0] / duration_s, "kernel_launches": stats["launches"],
            "idle_exits": stats["idle_exits"],
            "mean_N": statistics.mean(Ns) if Ns else None,
            "answered_by_pilot": (sum(1 for n in Ns if n == N1) / len(Ns)) if Ns else None,
            "delta_se_target_met": (sum(met) / len(met)) if met else None,
            "precision": {0: "fp64", 1: "mixed", 2: "tc-bf16", 3: "tc-tf32"}[precision]}


def latency_small(q, plan, stream, calls: int) -> dict:
    """The small case (arith, d=16, bridge, N=2^14, R=8, FP64): wall time of
    one synchronous public call, of a prepared batch launch + wait, of its
    CUDA-graph replay + wait, and the device time of one replay."""
    import torch
    c = W.small_arith()

    def quantiles(ts):
        ts = sorted(ts)
        return {"p50_us": 1e6 * ts[len(ts) // 2], "p99_us": 1e6 * ts[min(len(ts) - 1, int(0.99 * len(ts)))]}

    warm = 10
    ts = []
    for i in range(calls + warm):
        t0 = time.perf_counter()
        q.qmccpw_greeks(plan, c.type, c.d, c.K, c.T, c.S0, c.r, c.sigma, c.N, c.R, c.construction, q.QMCCPW_FP64)
        ts.append(time.perf_counter() - t0)
    out = {"workload": "arith Asian call, d=16, bridge, N=2^14, R=8, FP64 (one contract)",
           "sync_call": quantiles(ts[warm:])}
    def prepared(mode, dst):
        b = q.Batch(plan, [c], q.QMCCPW_FP64)
        if mode == "graph":
            b.use_graph(True)
        ts = []
        for i in range(calls + warm):
            t0 = time.perf_counter()
            b.launch(stream.cuda_stream)
            stream.synchronize()
            ts.append(time.perf_counter() - t0)
        dst[mode + "_and_wait"] = quantiles(ts[warm:])
        b.set_timing(calls)
        for _ in range(calls):
            b.launch(stream.cuda_stream)
        ms, n = b.timing()
        dst[mode + "_device_us"] = 1e3 * ms / max(1, n)
        dst[mode + "_kernels"] = b.launch_count()
        b.free()

    for mode in ("launch", "graph"):
        prepared(mode, out)
    # the same after the plan's tuner has chosen the tile for this contract
    # (a 2^14 x 8-point job is about one wave of 256-point tiles), then the
    # default restored for the rest of the run
    out["default_points_per_tile"] = q.qmccpw_tuning_get(plan, q.QMCCPW_FP64, c.construction, c.d)
    q.qmccpw_autotune(plan, [c], q.QMCCPW_FP64)
    tuned = {"points_per_tile": q.qmccpw_tuning_get(plan, q.QMCCPW_FP64, c.construction, c.d)}
    for mode in ("launch", "graph"):
        prepared(mode, tuned)
    out["tuned"] = tuned
    q.qmccpw_tuning_set(plan, q.QMCCPW_FP64, c.construction, c.d, 0)
    return out


def pca_stress(q, local, rank, stream, steps: int) -> dict:
    """d = 256 PCA (three products, N = 2^22, R = 16): CUDA-core MIXED and the
    tensor-core precisions, device time per step; error against FP64 at
    N = 2^16 (the same estimator on fewer points) in units of its SE."""
    import torch
    plan = q.qmccpw_plan(device=local, d_max=257, r_max=16, seed=W.SCRAMBLE_SEED, stream=stream.cuda_stream)
    full = W.pca_stress()
    small = W.pca_stress(N=2 ** 16)
    el = elements(full)
    out = {"workload": "PCA d=256 (n=255), {arith,binary,lookback}, S0=K=100 sigma=0.2 r=0.05 T=1, N=2^22, R=16",
           "point_dates": el}
    ref = q.qmccpw_greeks_batch(plan, small, q.QMCCPW_FP64)
    for name, prec in (("mixed", q.QMCCPW_MIXED), ("tc-bf16", q.QMCCPW_MIXED_TC_BF16X3),
                       ("tc-tf32", q.QMCCPW_MIXED_TC_TF32X3)):
        try:
            b = q.Batch(plan, full, prec)
        except q.QmcCpwError as e:
            out[name] = {"unsupported": str(e)}
            continue
        b.launch(stream.cuda_stream)
        torch.cuda.synchronize()
        b.set_timing(steps)
        for _ in range(steps):
            b.launch(stream.cuda_stream)
        ms, n = b.timing()
        b.free()
        res = q.qmccpw_greeks_batch(plan, small, prec)
        worst = max(abs(m[g] - m64[g]) / s64[g] for (m, _, _), (m64, s64, _) in zip(res, ref) for g in range(4))
        out[name] = {"value": el / (ms / n / 1e3), "unit": UNIT, "fused_ms": ms / n,
                     "max_err_in_se_vs_fp64_at_N_2^16": worst}
    q.qmccpw_free(plan)
    return out


def basket_section(q, local, stream, steps: int, N: int = 2 ** 18, R: int = 16) -> dict:
    """Basket of 4 correlated assets (d = 64, arithmetic call and binary on
    the basket average): MIXED and FP64 throughput in asset-point-dates
    (N R d m) per second, host wall time around the synchronous call (the
    kernel dominates at this size), and MIXED's worst error against FP64 in
    units of the FP64 standard error."""
    import time as _t
    plan = q.qmccpw_plan(device=local, d_max=257, r_max=R, seed=W.SCRAMBLE_SEED, stream=stream.cuda_stream)
    out = {"workload": f"basket of 4 assets (rho 0.5), d=64, N=2^{N.bit_length() - 1}, R={R}, "
                       "arithmetic call and binary on the basket average",
           "unit": "asset-point-dates/s"}
    for typ, tname in ((W.ARITH, "arith"), (W.BINARY, "binary")):
        b = W.basket_d64(typ)
        el = N * R * b.d * b.m
        res = {}
        for name, prec, k in (("mixed", q.QMCCPW_MIXED, steps), ("fp64", q.QMCCPW_FP64, 1)):
            q.qmccpw_basket_greeks(plan, b, N, R, prec)  # warm-up
            t0 = _t.perf_counter()
            for _ in range(k):
                mean, se, _ = q.qmccpw_basket_greeks(plan, b, N, R, prec)
            dt = (_t.perf_counter() - t0) / k
            res[name] = {"value": el / dt, "ms": dt * 1e3, "mean": mean.tolist(), "se": se.tolist()}
        err = [abs(res["mixed"]["mean"][g] - res["fp64"]["mean"][g]) / res["fp64"]["se"][g] for g in range(4)]
        res["mixed_vs_fp64_err_in_se"] = dict(zip(("price", "delta", "vega", "gamma"), err))
        out[tname] = res
    q.qmccpw_free(plan)
    return out


def run_reference(args):
    rank, world, _ = dist_info()
    if rank != 0:
        return
    import oracle
    oracle.build()
    cores = os.cpu_count() or 1
    contracts = W.grid_d64()
    n = 2 ** 10

    def step():
        for c in contracts:
            oracle.greeks(W.SCRAMBLE_SEED, c.type, c.d, c.K, c.T, c.S0, c.r, c.sigma, c.construction, n, c.R,
                          threads=cores)

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = (time.perf_counter() - t0) / max(1, args.steps)
    elems = sum(n * c.R * c.d for c in contracts)
    value = elems / dt
    sample = f"each step: the 36 contracts at N=2^10 (R=32, d=64), {elems} point-dates"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
        "scaling": "strong", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample": sample},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


# ---------------------------------------------------------------------------
def run_ours(args):
    import torch

    rank, world, local = dist_info()
    torch.cuda.set_device(local)
    ranks = Ranks(world, "nccl", local)
    barrier, max_over_ranks = ranks.barrier, ranks.max_over_ranks

    from paper_2209_11337_gb300 import build as lib_build
    from paper_2209_11337_gb300 import qmccpw as q
    lib_build.build()

    stream = torch.cuda.Stream()  # one non-default stream for the library, the events and the L2 flush
    torch.cuda.set_stream(stream)
    # every rank: the job's seed (a replicate is the same point set whichever rank runs it)
    plan = q.qmccpw_plan(device=local, d_max=max(65, args.case_d + 1), r_max=32, seed=W.SCRAMBLE_SEED,
                         stream=stream.cuda_stream)
    contracts = W.grid_d64()
    elems = elements(contracts)  # the job's distinct point-dates
    pieces = shard.replicate_shards(contracts, world)[rank]
    mine = shard.piece_contracts(contracts, pieces)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")  # > 129 MB L2
    peaks = pipe_peaks()

    def timed(precision, steps, warmup, with_clocks=False):
        """Per step: L2 flush, this rank's batch; with several ranks also the
        sum over ranks of the replicate estimates and the statistics."""
        batch = q.Batch(plan, mine, precision)
        rows = None
        if world > 1:
            rows = torch.zeros((shard.total_rows(contracts), 4), dtype=torch.float64, device="cuda")
            batch.scatter_replicates(rows.data_ptr(), shard.piece_rows(contracts, pieces))
        stats = [None]

        def step():
            if rows is not None:
                rows.zero_()
            batch.launch(stream.cuda_stream)
            if rows is not None:
                stats[0] = shard.gather_stats(rows, contracts, stream=stream.cuda_stream)

        for _ in range(warmup):
            flush.zero_()
            step()
        torch.cuda.synchronize()
        batch.set_timing(max(1, steps))
        sampler = ClockSampler(local) if with_clocks else None
        if sampler:
            sampler.start()
            time.sleep(0.3)
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        events = []
        for _ in range(steps):
            flush.zero_()  # L2 flush between timed steps
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step()
            e1.record(stream)
            events.append((e0, e1))
        torch.cuda.synchronize()
        barrier()
        wall = time.perf_counter() - t0
        clocks = sampler.stop() if sampler else None
        step_ms = [a.elapsed_time(b) for a, b in events]
        seg_ms, _ = batch.segment_timing()
        fused_ms, nl = batch.timing()
        launches = batch.launch_count() * steps
        if rows is None:
            res = [(m, s_, None) for m, s_, _ in batch.results()]
        else:
            st = stats[0].cpu().numpy()
            res = [(st[i, :4], st[i, 4:], None) for i in range(len(contracts))]
            launches += steps  # the statistics kernel
        batch.free()
        return {"ms_per_step": sum(step_ms) / steps, "wall_s": wall, "fused_ms": fused_ms / max(1, nl),
                "segment_ms": [x / max(1, nl) for x in seg_ms], "clocks": clocks, "launches": launches,
                "results": res}

    if args.case:
        # single-contract run for profiling: no JSON line
        typ, cons = args.case.split("-")
        tmap = {"arith": W.ARITH, "binary": W.BINARY, "lookback": W.LOOKBACK, "geometric": W.GEOMETRIC}
        one = [W.Contract(tmap[typ], args.case_d, 100.0, 1.0, 100.0, 0.05, 0.2, args.case_N, args.case_R,
                          {"bb": W.BB, "pca": W.PCA, "std": W.STD, "bblead": W.BB_LEAD,
                           "pcalead": W.PCA_LEAD}[cons])]
        prec = {"fp64": q.QMCCPW_FP64, "mixed": q.QMCCPW_MIXED, "tc-bf16": q.QMCCPW_MIXED_TC_BF16X3,
                "tc-tf32": q.QMCCPW_MIXED_TC_TF32X3}[args.case_precision]
        batch = q.Batch(plan, one, prec)
        batch.set_timing(args.steps)
        for _ in range(args.warmup):
            batch.launch(stream.cuda_stream)
        torch.cuda.synchronize()
        batch.timing()
        for _ in range(args.steps):
            batch.launch(stream.cuda_stream)
        ms, n = batch.timing()
        el = elements(one)
        print(f"case {args.case} d={args.case_d} N={args.case_N} R={args.case_R} {args.case_precision}: "
              f"fused {ms / n:.3f} ms/launch, {el / (ms / n / 1e3):.4g} point-dates/s")
        batch.free()
        q.qmccpw_free(plan)
        return

    grid_prec = {"mixed": q.QMCCPW_MIXED, "tc-bf16": q.QMCCPW_MIXED_TC_BF16X3,
                 "tc-tf32": q.QMCCPW_MIXED_TC_TF32X3}[args.grid_precision]
    mixed = timed(grid_prec, args.steps, args.warmup, with_clocks=True)
    # the same grid with PCA on the CUDA cores (MIXED), beside the headline
    cuda_core = timed(q.QMCCPW_MIXED, args.steps, 1) if args.grid_precision != "mixed" else None
    fp64 = timed(q.QMCCPW_FP64, args.fp64_steps, 1) if args.fp64_steps > 0 else None

    # end to end through the public API with host buffers: contracts in, results out
    def e2e_once():
        if world == 1:
            return q.qmccpw_greeks_batch(plan, contracts, grid_prec)
        return shard.sharded_greeks(plan, contracts, grid_prec, rank, world)

    e2e_once()
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        e2e_once()
    torch.cuda.synchronize()
    barrier()
    e2e_s = max_over_ranks((time.perf_counter() - t0) / args.steps)

    ms = max_over_ranks(mixed["ms_per_step"])
    value = job_value(elems, ms)
    seg_ms = [max_over_ranks(x) for x in mixed["segment_ms"]]

    # the float path against FP64 on the same points, in units of the FP64 standard error
    err_se = err_frac = per_greek = None
    if fp64 is not None:
        worst = np.zeros(4)
        table = []
        met = 0
        for c, (m32, _, _), (m64, se64, _) in zip(contracts, mixed["results"], fp64["results"]):
            e = np.abs(np.asarray(m32) - np.asarray(m64)) / np.asarray(se64)
            table.append({"contract": c.label(), "fp64": list(m64), "se": list(se64), "mixed": list(m32),
                          "err_in_se": e.tolist()})
            worst = np.maximum(worst, e)
            met += int(np.sum(e <= 0.1))
        err_se = float(worst.max())
        err_frac = met / (4.0 * len(contracts))
        per_greek = dict(zip(("price", "delta", "vega", "gamma"), worst.tolist()))
        if args.errors_out and rank == 0:
            with open(args.errors_out, "w") as f:
                json.dump(table, f, indent=1)

    sizeof_contract = 72  # bytes of one qmccpw_contract descriptor uploaded
    h2d = len(mine) * (sizeof_contract + 8) + sum(c.R for c in mine) * 8
    d2h = len(mine) * 8 * 8 + sum(c.R for c in mine) * 4 * 8
    if world > 1:
        h2d += shard.total_rows(contracts) * 4 * 8  # the assembled estimates, up for the sum over ranks
        d2h += shard.total_rows(contracts) * 4 * 8 + len(contracts) * 8 * 8
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "strong",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "contracts": len(contracts), "d": 64, "N": 2 ** 20, "R": 32,
                   "precision": {"mixed": "MIXED", "tc-bf16": "MIXED_TC_BF16X3",
                                 "tc-tf32": "MIXED_TC_TF32X3"}[args.grid_precision] +
                                ": inverse normal, path and exponentials in f32 from the library's own "
                                "polynomials with float-pair constants; switch point and per-point values in "
                                "float-float; tile and replicate sums in f64",
                   "point_dates_per_step": elems, "l2": "flushed between timed steps (512 MiB write)",
                   "parallelism": (f"{world} GPUs: each contract's 32 replicates in {world} ranges, one per GPU; "
                                   "one sum over GPUs of the replicate estimates per step" if world > 1 else
                                   "1 GPU")},
        "fp64": None if fp64 is None else {
            "value": job_value(elems, max_over_ranks(fp64["ms_per_step"])), "unit": UNIT,
            "ms_per_step": max_over_ranks(fp64["ms_per_step"]), "steps": args.fp64_steps},
        "mixed_vs_fp64_max_err_in_se": err_se,
        "mixed_vs_fp64_worst_in_se_per_greek": per_greek,
        "mixed_vs_fp64_share_within_0p1_se": err_frac,
        "roofline": roofline(args.grid_precision, mine, seg_ms, peaks),
        "segment_ms": {"bridge": seg_ms[0], "standard": seg_ms[1], "pca_streamed": seg_ms[2], "pca": seg_ms[3]},
        "mixed_cuda_core": None if cuda_core is None else {
            "value": job_value(elems, max_over_ranks(cuda_core["ms_per_step"])), "unit": UNIT,
            "ms_per_step": max_over_ranks(cuda_core["ms_per_step"]),
            "note": "the same grid in MIXED precision with the PCA product on the CUDA cores"},
        "e2e": {"value": elems / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": mixed["launches"],
        "clocks": mixed["clocks"],
    }
    if args.book_steps > 0:
        # the 4096-contract book: whole contracts spread over the ranks by point-dates, MIXED, plus an FP64 sample
        bplan = q.qmccpw_plan(device=local, d_max=366, r_max=16, seed=W.SCRAMBLE_SEED,
                              stream=stream.cuda_stream, workspace_bytes=8 << 30)
        bk = W.book(4096, seed=4, R=16)
        bel = elements(bk)
        bmine = shard.piece_contracts(bk, shard.contract_shards(bk, world)[rank])
        bb = q.Batch(bplan, bmine, q.QMCCPW_MIXED)
        bb.launch(stream.cuda_stream)
        torch.cuda.synchronize()
        bb.set_timing(args.book_steps)
        barrier()
        ev = []
        for _ in range(args.book_steps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            bb.launch(stream.cuda_stream)
            e1.record(stream)
            ev.append((e0, e1))
        torch.cuda.synchronize()
        bms = sum(a.elapsed_time(b) for a, b in ev) / args.book_steps
        bb.free()
        sample = bk[:64]
        sb = q.Batch(bplan, sample, q.QMCCPW_FP64)
        sb.launch(stream.cuda_stream)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sb.launch(stream.cuda_stream)
        e1.record(stream)
        torch.cuda.synchronize()
        f64ms = e0.elapsed_time(e1)
        sb.free()
        q.qmccpw_free(bplan)
        line["book"] = {"workload": "4096 contracts (seed 4): type U{3}, d U{12..365}, K U(80,120), sigma U(0.1,0.5), "
                                    "T U(0.25,2), r U(0,0.08), N=2^U{12..18}, R=16, bridge",
                        "point_dates": bel, "mixed": {"value": job_value(bel, max_over_ranks(bms)), "unit": UNIT,
                                                      "ms_per_step": max_over_ranks(bms), "steps": args.book_steps},
                        "fp64_sample": {"contracts": 64, "value": elements(sample) / (f64ms / 1e3), "unit": UNIT,
                                        "ms": f64ms}}
    # the latency, stress and serving sections run on rank 0's GPU only
    if rank == 0 and args.latency_calls > 0:
        line["latency_small"] = latency_small(q, plan, stream, args.latency_calls)
    if rank == 0 and args.stress_steps > 0:
        line["pca_stress"] = pca_stress(q, local, rank, stream, args.stress_steps)
    if rank == 0 and args.basket_steps > 0:
        line["basket"] = basket_section(q, local, stream, args.basket_steps)
    if rank == 0 and args.serving_s > 0:
        # at the configured rate (2000/s), at a rate well within what the GPU serves, and FP64 at a rate
        # its path sustains
        splan = q.qmccpw_plan(device=local, d_max=366, r_max=16, seed=W.SCRAMBLE_SEED)
        line["serving"] = {
            "mixed": serve(q, splan, q.QMCCPW_MIXED, args.serving_rate, args.serving_s),
            "mixed_sustained": serve(q, splan, q.QMCCPW_MIXED, args.serving_rate_sustained, args.serving_s),
            "fp64": serve(q, splan, q.QMCCPW_FP64, args.serving_rate_fp64, args.serving_s),
        }
        q.qmccpw_free(splan)
    barrier()
    if rank == 0 and not args.no_cpu_baseline and world == 1:
        line["cpu_baseline"] = cpu_baseline(contracts)
    elif rank == 0 and world == 1:
        line["cpu_baseline"] = None
    if rank == 0:
        print(json.dumps(line))
    q.qmccpw_free(plan)
    ranks.close()


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--fp64-steps", type=int, default=2)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--grid-precision", choices=["mixed", "tc-bf16", "tc-tf32"], default="tc-bf16",
                    help="precision of the timed grid (tc-*: float path with the PCA product on tensor cores)")
    ap.add_argument("--book-steps", type=int, default=1, help="timed steps of the 4096-contract book (0: skip)")
    ap.add_argument("--serving-s", type=float, default=3.0, help="seconds of Poisson arrivals (0: skip)")
    ap.add_argument("--latency-calls", type=int, default=200, help="calls timed in the small-case latency section")
    ap.add_argument("--stress-steps", type=int, default=1, help="timed steps of the d=256 PCA case (0: skip)")
    ap.add_argument("--basket-steps", type=int, default=3, help="timed MIXED calls of the 4-asset basket (0: skip)")
    ap.add_argument("--serving-rate", type=float, default=2000.0)
    ap.add_argument("--serving-rate-sustained", type=float, default=1000.0,
                    help="a second MIXED arrival rate, within what the GPU serves")
    ap.add_argument("--serving-rate-fp64", type=float, default=20.0)
    ap.add_argument("--errors-out", default=None, help="write the per-contract MIXED vs FP64 table (JSON)")
    ap.add_argument("--case", default=None, help="time one contract only, e.g. arith-bb or lookback-pca")
    ap.add_argument("--case-d", type=int, default=64)
    ap.add_argument("--case-N", type=int, default=2 ** 16)
    ap.add_argument("--case-R", type=int, default=4)
    ap.add_argument("--case-precision", choices=["mixed", "fp64", "tc-bf16", "tc-tf32"], default="mixed")
    args = ap.parse_args(argv)
    args.warmup = max(3, args.warmup)  # at least three untimed warm-up steps
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
