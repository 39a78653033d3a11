"""The multi-GPU split of a job, on CPU: the partition rules and, with two
gloo ranks on 127.0.0.1, the assembly of replicate estimates by one
all-reduce.  Each rank computes its pieces with the oracle's per-replicate
sums as a stand-in worker (a replicate is the same point set whichever rank
runs it); the assembled array must equal the single-rank array bit for bit."""
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402
from paper_2209_11337_gb300 import shard  # noqa: E402


def free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("R", [2, 3, 5, 16, 31, 32])
@pytest.mark.parametrize("world", [1, 2, 3, 4, 8, 16])
def test_replicate_ranges_cover_every_replicate_once_in_ranges_of_two_or_more(R, world):
    ranges = shard.replicate_ranges(R, world)
    assert len(ranges) == min(world, R // 2)
    covered = [r for first, n in ranges for r in range(first, first + n)]
    assert covered == list(range(R))
    sizes = [n for _, n in ranges]
    assert min(sizes) >= 2 and max(sizes) - min(sizes) <= 1


@pytest.mark.parametrize("world", [1, 2, 3, 8])
def test_replicate_shards_give_every_rank_the_same_mix_on_the_grid(world):
    grid = W.grid_d64()
    shards = shard.replicate_shards(grid, world)
    work = [shard.point_dates(grid, s) for s in shards]
    assert sum(work) == shard.point_dates(grid)  # distinct work only: nothing counted twice
    if 32 % world == 0:
        assert len(set(work)) == 1
        for s in shards:  # every contract, R / world replicates
            assert sorted(i for i, _, _ in s) == list(range(len(grid)))
    seen = set()
    for s in shards:
        for i, f, n in s:
            for r in range(f, f + n):
                assert (i, r) not in seen
                seen.add((i, r))
    assert len(seen) == sum(c.R for c in grid)


def test_contract_shards_balance_a_book_by_point_dates():
    bk = W.book(512, seed=4, R=16)
    for world in (2, 4, 8):
        shards = shard.contract_shards(bk, world)
        assert sorted(i for s in shards for i, _, _ in s) == list(range(len(bk)))
        work = [shard.point_dates(bk, s) for s in shards]
        biggest = max(c.N * c.R * c.d for c in bk)
        assert max(work) - min(work) <= biggest  # greedy longest-first bound


def test_piece_contracts_and_rows():
    cs = [W.small_arith(), W.Contract(W.BINARY, 9, 90.0, 1.0, 100.0, 0.05, 0.1, 1000, 6, W.PCA)]
    pieces = shard.replicate_shards(cs, 2)
    assert pieces[0] == [(0, 0, 4), (1, 3, 3)] and pieces[1] == [(0, 4, 4), (1, 0, 3)]
    mine = shard.piece_contracts(cs, pieces[1])
    assert (mine[0].first_replicate, mine[0].R) == (4, 4) and (mine[1].first_replicate, mine[1].R) == (0, 3)
    assert shard.piece_rows(cs, pieces[1]) == [4, 8]
    assert shard.total_rows(cs) == 14


JOB = [W.Contract(W.ARITH, 8, 100.0, 1.0, 100.0, 0.05, 0.2, 256, 6, W.BB),
       W.Contract(W.LOOKBACK, 5, 95.0, 0.5, 100.0, 0.02, 0.3, 100, 4, W.PCA),
       W.Contract(W.BINARY, 4, 105.0, 1.0, 100.0, 0.05, 0.25, 77, 5, W.STD)]


def stand_in_worker(c, first, n):
    """Per-replicate estimates of replicates first..first+n-1 (the oracle)."""
    import oracle
    sums = oracle.partial_sums(W.SCRAMBLE_SEED, c.type, c.d, c.K, c.T, c.S0, c.r, c.sigma, c.construction,
                               first, n, 0, c.N, threads=1)
    return sums / c.N


def assemble(world, rank, dist=None):
    import torch
    buf = torch.zeros(shard.total_rows(JOB) * 4, dtype=torch.float64)
    pieces = shard.replicate_shards(JOB, world)[rank]
    for (i, f, n), row in zip(pieces, shard.piece_rows(JOB, pieces)):
        est = stand_in_worker(JOB[i], f, n)
        buf[row * 4:(row + n) * 4] = torch.from_numpy(est.reshape(-1))
    if dist is not None:
        dist.all_reduce(buf)  # the pieces' rows are disjoint: the sum is the assembly
    return buf.numpy().copy()


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    dist.init_process_group("gloo")
    got = assemble(world, rank, dist)
    out.put((rank, got.tobytes()))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_assemble_the_single_rank_replicate_estimates_bit_for_bit():
    world, port = 2, free_port()
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    got = dict(out.get(timeout=300) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    single = assemble(1, 0)
    for r in range(world):
        mine = np.frombuffer(got[r], dtype=np.float64)
        assert mine.tobytes() == single.tobytes()  # bit for bit, on every rank
    # and the single-rank rows are each contract's own replicates in order
    rows = shard.rows(JOB)
    for c, row in zip(JOB, rows):
        ref = stand_in_worker(c, 0, c.R).reshape(-1)
        assert single[row * 4:(row + c.R) * 4].tobytes() == ref.tobytes()
