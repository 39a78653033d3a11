"""The bench's roofline object on CPU: six launch segments per batch (bridge,
standard, streamed and resident PCA, the two leading-coordinate forms), the
dominant one among those with a flop model, every working segment listed."""
import importlib.util
import os
import sys

import pytest

import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    sys.modules["bench_under_test"] = mod
    spec.loader.exec_module(mod)
    return mod


@pytest.mark.parametrize("prec", ["tc-bf16", "tc-tf32", "mixed"])
def test_roofline_of_the_grid_with_six_segments(bench, prec):
    cs = W.grid_d64()
    seg_ms = [91.7, 0.002, 0.002, 117.1, 0.002, 0.002]
    r = bench.roofline(prec, cs, seg_ms)
    assert r["kernel"] == bench.SEGMENT_KERNELS[prec][3]
    assert r["ms_per_launch"] == 117.1
    # 18 PCA contracts, N = 2^20, R = 32, d = 64
    per = bench.FLOPS_TC_FP32 if prec != "mixed" else bench.FLOPS_BRIDGE - 5 + 2 * 63
    flops = 18 * 2 ** 20 * 32 * 64 * per
    assert r["achieved"] == pytest.approx(flops / 0.1171 / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    kernels = [s["kernel"] for s in r["segments"]]
    assert kernels == [bench.SEGMENT_KERNELS[prec][0], bench.SEGMENT_KERNELS[prec][3]]
    assert ("tensor" in r) == (prec != "mixed")


def test_roofline_when_the_bridge_segment_dominates(bench):
    r = bench.roofline("tc-bf16", W.grid_d64(), [200.0, 0.0, 0.0, 100.0, 0.0, 0.0])
    assert r["kernel"] == "fused_kernel<float, bridge>"
    assert "tensor" not in r
