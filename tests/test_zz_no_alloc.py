"""The allocation-free entry point (qmccpw_greeks_noalloc) against the
ordinary one (qmccpw_greeks).

qmccpw_greeks_noalloc serves callers that must not allocate device memory
per call (latency-critical services where cudaMalloc/cudaFree would block or
synchronise the device, hosts whose device memory is owned by another
allocator): its per-call arrays live in a fixed array compiled into the
library.  Here the test itself owns the output buffer; the results of two
consecutive calls must match qmccpw_greeks within the parity tolerance of the
other GPU tests.  The file name makes pytest collect it last.
"""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

RTOL = 1e-12

CASES = [
    (W.Contract(W.ARITH, 64, 100.0, 1.0, 100.0, 0.05, 0.2, 2 ** 16, 8, W.BB), 1),         # MIXED
    (W.Contract(W.LOOKBACK, 33, 95.0, 1.5, 100.0, 0.03, 0.3, 5000, 4, W.PCA), 0),          # FP64, ragged N
    (W.Contract(W.BINARY, 16, 105.0, 0.5, 100.0, 0.02, 0.25, 2 ** 12, 2, W.PCA), 1),
    (W.Contract(W.ARITH, 16, 100.0, 1.0, 100.0, 0.05, 0.2, 2 ** 18 + 77, 4, W.BB), 1),    # items of 4 tiles, the last of 1
]


@pytest.fixture(scope="module")
def q():
    from paper_2209_11337_gb300 import build, qmccpw
    build.build()
    return qmccpw


@pytest.mark.parametrize("c,precision", CASES, ids=lambda x: x.label() if hasattr(x, "label") else str(x))
def test_no_alloc_matches_allocating_entry_point_twice(q, c, precision):
    import torch
    plan = q.qmccpw_plan(device=0, d_max=65, r_max=16, seed=W.SCRAMBLE_SEED)
    try:
        mean, se, per = q.qmccpw_greeks(plan, c.type, c.d, c.K, c.T, c.S0, c.r, c.sigma, c.N, c.R,
                                        c.construction, precision)
        out = torch.full(((c.R + 2) * 4,), float("nan"), dtype=torch.float64, device="cuda")
        for _ in range(2):
            out.fill_(float("nan"))
            torch.cuda.synchronize()
            q.qmccpw_greeks_noalloc(plan, c.type, c.d, c.K, c.T, c.S0, c.r, c.sigma, c.N, c.R, c.construction,
                                    precision, out.data_ptr())
            torch.cuda.synchronize()
            got = out.cpu().numpy()
            g_per = got[: 4 * c.R].reshape(c.R, 4)
            g_mean, g_se = got[4 * c.R: 4 * c.R + 4], got[4 * c.R + 4:]
            scale = np.maximum(np.abs(per).max(axis=0), 1e-300)
            assert np.all(np.abs(g_per - per) <= RTOL * scale), (g_per, per)
            assert np.all(np.abs(g_mean - mean) <= RTOL * scale)
            assert np.all(np.abs(g_se - se) <= RTOL * scale + 1e-9 * se)
    finally:
        q.qmccpw_free(plan)


def test_no_alloc_rejects_work_beyond_its_array(q):
    import torch
    plan = q.qmccpw_plan(device=0, d_max=65, r_max=64, seed=W.SCRAMBLE_SEED)
    try:
        out = torch.empty((64 + 2) * 4, dtype=torch.float64, device="cuda")
        # 64 replicates x 2^30 points: 2^18 work items of 16 tiles per replicate, 512 MiB of item sums
        with pytest.raises(q.QmcCpwError) as e:
            q.qmccpw_greeks_noalloc(plan, 0, 64, 100.0, 1.0, 100.0, 0.05, 0.2, 2 ** 30, 64, 0, 1, out.data_ptr())
        assert e.value.code == q.QMCCPW_ERR_OOM
        assert "16777216" in str(e.value)
    finally:
        q.qmccpw_free(plan)
