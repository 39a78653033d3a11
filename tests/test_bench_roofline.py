"""The bench's roofline object on CPU: six launch segments per batch (bridge,
standard, streamed and resident PCA, the two leading-coordinate forms), the
dominant one among the grid's four, every working segment listed with its
ceilings (FP32 operations / 24, SFU / 2, tensor / split-product flops)."""
import importlib.util
import os
import sys

import pytest

import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PEAKS = {"fp32_fma_tflops": 78.5, "sfu_ex2_gops": 10050.0, "tc_bf16_tflops": 2411.0, "tc_tf32_tflops": 1207.0}


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
    r = bench.roofline(prec, cs, seg_ms, PEAKS)
    assert r["kernel"] == bench.SEGMENT_KERNELS[prec][3]
    assert r["ms_per_launch"] == 117.1
    # 18 PCA contracts, N = 2^20, R = 32, d = 64
    pd = 18 * 2 ** 20 * 32 * 64 / 0.1171
    assert r["point_dates_per_s"] == pytest.approx(pd)
    assert r["achieved"] == pytest.approx(pd * 24 / 1e12)
    assert r["peak"] == pytest.approx(78.5 / 2)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    ceil = r["ceilings_point_dates_per_s"]
    assert ceil["fp32"] == pytest.approx(78.5e12 / 2 / 24) and ceil["sfu"] == pytest.approx(10050e9 / 2)
    if prec != "mixed":
        per = 2 * 63 * (5 if prec == "tc-bf16" else 3)
        rate = 2411e12 if prec == "tc-bf16" else 1207e12
        assert ceil["tensor"] == pytest.approx(rate / per)
    else:
        assert "tensor" not in ceil
    assert r["limit"] == min(ceil, key=ceil.get)
    assert r["frac_of_lowest_ceiling"] == pytest.approx(pd / ceil[r["limit"]])
    kernels = [s["kernel"] for s in r["segments"]]
    assert kernels == [bench.SEGMENT_KERNELS[prec][0], bench.SEGMENT_KERNELS[prec][3]]


def test_roofline_when_the_bridge_segment_dominates(bench):
    r = bench.roofline("tc-bf16", W.grid_d64(), [200.0, 0.0, 0.0, 100.0, 0.0, 0.0], PEAKS)
    assert r["kernel"] == "fused_kernel<float, bridge>"
    assert "tensor" not in r["ceilings_point_dates_per_s"]
