"""Measure the pipe peaks of this GPU and write them for the roofline.

    python -m paper_2209_11337_gb300.peaks [--device 0] [--write]

Runs qmccpw_measure_pipe_peaks (the library's own micro-benchmarks: FFMA,
packed FFMA2, DFMA, the SFU's ex2 / lg2 / rcp, tcgen05 kind::f16 and
kind::tf32) five times with nvidia-smi sampling the SM clock meanwhile (read
only: no clock or power setting is touched), keeps the best rate of each, and
prints one JSON object; with --write it also stores it as pipe_peaks_gb300.json
beside this file, where bench.py reads its roofline denominators.  The rates
are burst figures (each kernel runs a few milliseconds at the clock the GPU
holds then); the median SM clock of the run is recorded beside them.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

HERE = os.path.dirname(os.path.abspath(__file__))
PEAKS_PATH = os.path.join(HERE, "pipe_peaks_gb300.json")


def load() -> dict:
    """The committed measurement (empty if absent)."""
    try:
        with open(PEAKS_PATH) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def measure(device: int = 0, repeats: int = 5) -> dict:
    from . import build, qmccpw
    build.build()
    lines: list = []
    proc = None
    try:
        proc = subprocess.Popen(["nvidia-smi", f"--id={device}", "--query-gpu=clocks.sm,clocks.max.sm,power.draw",
                                 "--format=csv,noheader,nounits", "-lms", "50"],
                                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        reader = threading.Thread(target=lambda: lines.extend(x.strip() for x in proc.stdout), daemon=True)
        reader.start()
        time.sleep(0.2)
    except OSError:
        proc = None
    best: dict = {}
    for _ in range(repeats):
        r = qmccpw.qmccpw_measure_pipe_peaks(device)
        for k, v in r.items():
            best[k] = max(best.get(k, 0.0), v)
    clocks = {}
    if proc is not None:
        proc.terminate()
        proc.wait(timeout=5)
        sm = [float(x.split(",")[0]) for x in lines if x and x.split(",")[0].strip().replace(".", "").isdigit()]
        mx = [float(x.split(",")[1]) for x in lines if x and len(x.split(",")) > 1 and x.split(",")[1].strip().replace(".", "").isdigit()]
        clocks = {"sm_mhz_median": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                  "samples": len(sm)}
    import torch
    name = torch.cuda.get_device_name(device)
    sms = torch.cuda.get_device_properties(device).multi_processor_count
    out = dict(best)
    out.update({"gpu": name, "sms": sms, "clocks": clocks, "repeats": repeats,
                "how": "qmccpw_measure_pipe_peaks: best of 5 x (best of 5 CUDA-event-timed launches after a warm-up); "
                       "FFMA/FFMA2/DFMA: 8 chains x 16 steps per thread, 8 x 256-thread CTAs per SM; SFU: the same "
                       "with ex2/lg2/rcp.approx; tcgen05: one thread per CTA issues 4096 M=128 N=256 products, "
                       "two CTAs per SM",
                "when": time.strftime("%Y-%m-%dT%H:%M:%SZ", time.gmtime())})
    # per-SM per-clock rates at the median clock (the unit counts they imply)
    mhz = clocks.get("sm_mhz_median") or clocks.get("sm_max_mhz")
    if mhz:
        per = lambda v, scale: v * scale / (sms * mhz * 1e6)
        out["per_sm_per_clock"] = {"fp32_lanes": per(best["fp32_fma_tflops"], 1e12 / 2),
                                   "fp64_lanes": per(best["fp64_fma_tflops"], 1e12 / 2),
                                   "sfu_ex2": per(best["sfu_ex2_gops"], 1e9), "sfu_lg2": per(best["sfu_lg2_gops"], 1e9),
                                   "sfu_rcp": per(best["sfu_rcp_gops"], 1e9),
                                   "tc_bf16_flops": per(best["tc_bf16_tflops"], 1e12)}
    return out


def main(argv=None) -> None:
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--device", type=int, default=0)
    ap.add_argument("--write", action="store_true")
    args = ap.parse_args(argv)
    out = measure(args.device)
    print(json.dumps(out))
    if args.write:
        with open(PEAKS_PATH, "w") as f:
            json.dump(out, f, indent=1)
            f.write("\n")


if __name__ == "__main__":
    sys.exit(main())
