"""CUDA-graph replay of a prepared batch: the same work, the same results."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu
SEED = W.SCRAMBLE_SEED


@pytest.fixture(scope="module")
def q():
    from paper_2209_11337_gb300 import build, qmccpw
    build.build()
    return qmccpw


@pytest.fixture(scope="module")
def plan(q):
    h = q.qmccpw_plan(device=0, d_max=65, r_max=16, seed=SEED)
    yield h
    q.qmccpw_free(h)


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_graph_replay_equals_plain_launch(q, plan, prec):
    cs = [W.small_arith(),
          W.Contract(W.LOOKBACK, 64, 95.0, 1.0, 100.0, 0.05, 0.3, 3000, 4, W.PCA),
          W.Contract(W.BINARY, 33, 105.0, 0.5, 100.0, 0.02, 0.2, 2 ** 12, 3, W.BB)]
    plain = q.Batch(plan, cs, prec)
    graph = q.Batch(plan, cs, prec)
    try:
        plain.launch()
        ref = plain.results()
        graph.use_graph(True)
        graph.set_timing(4)
        for _ in range(3):
            graph.launch()
            got = graph.results()
            for (m0, s0, p0), (m1, s1, p1) in zip(ref, got):
                assert np.array_equal(p0, p1) and np.array_equal(m0, m1) and np.array_equal(s0, s1)
        ms, n = graph.timing()
        assert n == 3 and ms > 0.0
        graph.use_graph(False)  # back to plain launches
        graph.launch()
        for (_, _, p0), (_, _, p1) in zip(ref, graph.results()):
            assert np.array_equal(p0, p1)
    finally:
        plain.free()
        graph.free()
