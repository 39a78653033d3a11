"""The single-GPU side of the multi-GPU split (paper Sec. 5: the estimate is
the mean of independently randomised replicates, so a job splits into
(contract, replicate range) pieces).  A contract run as replicate ranges
(first_replicate) gives the same replicate estimates, bit for bit, as one
call over all replicates; the pieces' estimates scattered into one device
array and reduced by the library's statistics kernel give the single call's
mean and standard error bit for bit; and the host-side split of a job run
rank by rank on one GPU, assembled by summing the ranks' arrays (what the
all-reduce does across GPUs), equals the unsplit job."""
import numpy as np
import pytest
import torch

import workloads as W
from paper_2209_11337_gb300 import shard

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def q():
    from paper_2209_11337_gb300 import build, qmccpw
    build.build()
    return qmccpw


@pytest.fixture(scope="module")
def plan(q):
    h = q.qmccpw_plan(device=0, d_max=130, r_max=32, seed=W.SCRAMBLE_SEED)
    yield h
    q.qmccpw_free(h)


def contracts():
    return [W.Contract(W.ARITH, 64, 100.0, 1.0, 100.0, 0.05, 0.2, 3000, 8, W.BB),
            W.Contract(W.BINARY, 17, 105.0, 0.5, 100.0, 0.02, 0.3, 2 ** 12, 5, W.PCA),
            W.Contract(W.LOOKBACK, 100, 95.0, 1.0, 100.0, 0.05, 0.25, 1000, 7, W.STD),
            W.Contract(W.ARITH, 33, 100.0, 1.0, 100.0, 0.05, 0.2, 2 ** 11, 6, W.PCA_LEAD)]


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_replicate_ranges_reproduce_the_whole_call(q, plan, prec):
    from dataclasses import replace
    cs = contracts()
    whole = q.qmccpw_greeks_batch(plan, cs, prec)
    for c, (_, _, per) in zip(cs, whole):
        for first, n in shard.replicate_ranges(c.R, 3):
            piece = replace(c, first_replicate=first, R=n)
            (_, _, p), = q.qmccpw_greeks_batch(plan, [piece], prec)
            assert np.array_equal(p, per[first:first + n]), (c.label(), first, n)


@pytest.mark.parametrize("prec", [0, 1])
def test_scattered_pieces_and_device_statistics_equal_one_call(q, plan, prec):
    cs = contracts()
    whole = q.qmccpw_greeks_batch(plan, cs, prec)
    pieces = shard.replicate_shards(cs, 3)
    rows = torch.zeros((shard.total_rows(cs), 4), dtype=torch.float64, device="cuda")
    for rank_pieces in pieces:  # every "rank" in turn on this GPU, one batch each
        b = q.Batch(plan, shard.piece_contracts(cs, rank_pieces), prec)
        try:
            b.scatter_replicates(rows.data_ptr(), shard.piece_rows(cs, rank_pieces))
            b.launch()
            b.results()
        finally:
            b.free()
    torch.cuda.synchronize()
    stats = shard.gather_stats(rows, cs).cpu().numpy()
    per_all = rows.cpu().numpy()
    for i, (c, (m, s, per), b0) in enumerate(zip(cs, whole, shard.rows(cs))):
        assert np.array_equal(per_all[b0:b0 + c.R], per), c.label()
        assert np.array_equal(stats[i, :4], m) and np.array_equal(stats[i, 4:], s), c.label()


def test_rank_by_rank_split_summed_equals_the_unsplit_job(q, plan):
    """Contract shards (whole contracts per rank) and replicate shards, each
    rank's rows zero elsewhere: the element-wise sum over ranks is exact."""
    cs = contracts()
    whole = q.qmccpw_greeks_batch(plan, cs, q.QMCCPW_MIXED)
    for split in (shard.replicate_shards, shard.contract_shards):
        total = np.zeros((shard.total_rows(cs), 4))
        for rank_pieces in split(cs, 2):
            part = np.zeros_like(total)
            res = q.qmccpw_greeks_batch(plan, shard.piece_contracts(cs, rank_pieces), q.QMCCPW_MIXED)
            for row, (_, _, per) in zip(shard.piece_rows(cs, rank_pieces), res):
                part[row:row + per.shape[0]] = per
            total += part
        for c, (_, _, per), b0 in zip(cs, whole, shard.rows(cs)):
            assert np.array_equal(total[b0:b0 + c.R], per), (split.__name__, c.label())
