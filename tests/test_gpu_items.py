"""Work items of several tiles (one 32-byte slot per item).

A replicate's tiles are grouped into work items of up to 16 consecutive
tiles; the CTA that takes an item adds its tiles' sums in tile order and
writes one slot.  Here the tile counts leave a short last item (a single
tile in the first case) and a ragged last tile, and each replicate's
estimate must equal the exactly
rounded mean of the same kernel's own per-point values (qmccpw_point_values,
summed on the host with math.fsum): a grouping that dropped, repeated or
misplaced a tile, or summed an item into the wrong slot, would move it by
whole tiles' worth of points.
"""
import math

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def q():
    from paper_2209_11337_gb300 import build, qmccpw
    build.build()
    return qmccpw


@pytest.fixture(scope="module")
def plan(q):
    h = q.qmccpw_plan(device=0, d_max=201, r_max=4, seed=W.SCRAMBLE_SEED)
    yield h
    q.qmccpw_free(h)


CASES = [
    # FP64, 256-point tiles: 515 tiles, items of two, the last item one ragged tile
    (W.Contract(W.ARITH, 16, 100.0, 1.0, 100.0, 0.05, 0.2, 256 * 514 + 1, 2, W.BB), 0, 1e-12),
    # MIXED, shared-memory bridge with 64-point tiles: 1031 tiles, items of four, the last of three
    (W.Contract(W.LOOKBACK, 200, 95.0, 1.0, 100.0, 0.05, 0.25, 64 * 1030 + 3, 2, W.BB), 1, 1e-11),
    # tensor-core PCA (bf16), 128-point tiles: 1031 tiles, items of four, the last of three
    (W.Contract(W.BINARY, 64, 105.0, 1.0, 100.0, 0.05, 0.3, 128 * 1030 + 7, 2, W.PCA), 2, 1e-11),
    # standard construction, MIXED: 4100 tiles of 128 points (items of 16, the last of four) or 2050 of 256
    (W.Contract(W.ARITH, 64, 100.0, 1.0, 100.0, 0.05, 0.2, 128 * 4099 + 50, 2, W.STD), 1, 1e-11),
]


@pytest.mark.parametrize("c,prec,rtol", CASES, ids=lambda x: x.label() if hasattr(x, "label") else str(x))
def test_replicate_estimate_is_the_mean_of_its_points(q, plan, c, prec, rtol):
    (_, _, per), = q.qmccpw_greeks_batch(plan, [c], prec)
    for r in range(c.R):
        pts = q.qmccpw_point_values(plan, c.type, c.d, c.K, c.T, c.S0, c.r, c.sigma, c.construction, prec, r, 0,
                                    c.N)
        ref = np.array([math.fsum(pts[:, g]) for g in range(4)]) / c.N
        scale = np.mean(np.abs(pts), axis=0)
        assert np.all(np.abs(per[r] - ref) <= rtol * np.maximum(np.abs(ref), scale)), (c.label(), r, per[r], ref)
