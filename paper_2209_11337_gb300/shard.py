"""Splitting one QMC-CPW job over several GPUs (host-side scheduling only).

The estimate of a contract is the mean of R independently randomised
replicate estimates and its standard error their spread (Sec. 5), so the
work splits into (contract, replicate range) pieces that share nothing: a
replicate is the same point set whichever GPU computes it (plans with the same
seed; ``first_replicate`` of the contract descriptor), and the only exchange
is the R x 4 replicate estimates of each contract, assembled into one array
of the job (contract i's rows from ``rows(contracts)[i]``) and reduced once.
The pieces write disjoint rows of an array that is zero elsewhere, so a sum
over ranks (one all-reduce) assembles it exactly (x + 0 = x), and the mean
and standard error computed from it are those of one GPU running everything.

Two partitions:
  * ``replicate_shards``: each contract's replicates in contiguous ranges of
    at least two, one range per rank where R allows, so every rank runs the
    same mix of contracts (the d = 64 grid: 36 contracts x R/world replicates
    per rank);
  * ``contract_shards``: whole contracts, longest first on N * R * d to the
    least loaded rank (a book of many small contracts).

A piece is ``(contract index, first replicate within the contract, count)``.
"""
from __future__ import annotations

from dataclasses import replace
from typing import List, Sequence, Tuple

Piece = Tuple[int, int, int]


def replicate_ranges(R: int, parts: int) -> List[Tuple[int, int]]:
    """R replicates in min(parts, R // 2) contiguous ranges of at least two,
    sizes differing by at most one: [(first, count), ...]."""
    if R < 2:
        raise ValueError("a contract needs at least two replicates")
    k = max(1, min(parts, R // 2))
    base, extra = divmod(R, k)
    out, first = [], 0
    for j in range(k):
        n = base + (1 if j < extra else 0)
        out.append((first, n))
        first += n
    return out


def replicate_shards(contracts: Sequence, world: int) -> List[List[Piece]]:
    """Pieces of every rank: contract i's j-th replicate range goes to rank
    (i + j) mod world (the rotation spreads contracts whose R allows fewer
    ranges than ranks)."""
    if world < 1:
        raise ValueError("world must be >= 1")
    shards: List[List[Piece]] = [[] for _ in range(world)]
    for i, c in enumerate(contracts):
        for j, (first, n) in enumerate(replicate_ranges(c.R, world)):
            shards[(i + j) % world].append((i, first, n))
    return shards


def contract_shards(contracts: Sequence, world: int) -> List[List[Piece]]:
    """Whole contracts, largest N * R * d first, each to the rank with the
    least work so far (ties: the lowest rank); pieces in contract order."""
    if world < 1:
        raise ValueError("world must be >= 1")
    load = [0] * world
    shards: List[List[Piece]] = [[] for _ in range(world)]
    order = sorted(range(len(contracts)), key=lambda i: (-contracts[i].N * contracts[i].R * contracts[i].d, i))
    for i in order:
        r = min(range(world), key=lambda k: (load[k], k))
        load[r] += contracts[i].N * contracts[i].R * contracts[i].d
        shards[r].append((i, 0, contracts[i].R))
    for s in shards:
        s.sort()
    return shards


def rows(contracts: Sequence) -> List[int]:
    """First row of each contract's replicate block in the job's array."""
    out, at = [], 0
    for c in contracts:
        out.append(at)
        at += c.R
    return out


def total_rows(contracts: Sequence) -> int:
    return sum(c.R for c in contracts)


def piece_contracts(contracts: Sequence, pieces: Sequence[Piece]) -> list:
    """The contract descriptors a rank runs: each piece as its contract with
    ``first_replicate`` and ``R`` of the range."""
    return [replace(contracts[i], first_replicate=getattr(contracts[i], "first_replicate", 0) + f, R=n)
            for i, f, n in pieces]


def piece_rows(contracts: Sequence, pieces: Sequence[Piece]) -> List[int]:
    """Row of the job's array where each piece's first replicate lands."""
    base = rows(contracts)
    return [base[i] + f for i, f, _ in pieces]


def point_dates(contracts: Sequence, pieces: Sequence[Piece] = None) -> int:
    """Distinct work, N * R * d summed over the pieces (all contracts if None)."""
    if pieces is None:
        return sum(c.N * c.R * c.d for c in contracts)
    return sum(contracts[i].N * n * contracts[i].d for i, _, n in pieces)


def gather_stats(per_rep_rows, contracts, group=None, stream=None):
    """The job's statistics from a device array of replicate estimates.

    ``per_rep_rows``: float64 CUDA tensor of total_rows(contracts) x 4, this
    rank's rows filled and zeros elsewhere.  One sum over the ranks of
    ``group`` (torch.distributed, NCCL on the GPUs) assembles every rank's
    rows; the library's statistics kernel then forms mean and SE per contract
    on this GPU.  Returns a CUDA tensor of len(contracts) x 8 (mean[4], se[4])."""
    import torch
    import torch.distributed as dist
    from . import qmccpw as q
    if group is not None or (dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1):
        dist.all_reduce(per_rep_rows, group=group)
    dev = per_rep_rows.device
    first = torch.tensor(rows(contracts), dtype=torch.int64, device=dev)
    R = torch.tensor([c.R for c in contracts], dtype=torch.int32, device=dev)
    stats = torch.empty((len(contracts), 8), dtype=torch.float64, device=dev)
    cur = torch.cuda.current_stream(dev).cuda_stream if stream is None else stream
    q.qmccpw_replicate_stats(per_rep_rows.data_ptr(), first.data_ptr(), R.data_ptr(), len(contracts),
                             stats.data_ptr(), cur)
    return stats


def sharded_greeks(plan, contracts, precision, rank: int, world: int, mode: str = "replicates"):
    """One job over `world` GPUs, called on every rank (torch.distributed
    initialised, one GPU per rank, `plan` on this rank's GPU with the job's
    seed): this rank computes its pieces through qmccpw_greeks_batch (host
    buffers), the replicate estimates are assembled on the GPUs by one sum over
    ranks, and every rank gets (mean[C,4], se[C,4], per_replicate list of [R,4])
    for all contracts, identical to one GPU running the whole job."""
    import numpy as np
    import torch
    from . import qmccpw as q
    shards = replicate_shards(contracts, world) if mode == "replicates" else contract_shards(contracts, world)
    pieces = shards[rank]
    buf = torch.zeros((total_rows(contracts), 4), dtype=torch.float64)
    if pieces:
        res = q.qmccpw_greeks_batch(plan, piece_contracts(contracts, pieces), precision)
        for row, (_, _, per) in zip(piece_rows(contracts, pieces), res):
            buf[row:row + per.shape[0]] = torch.from_numpy(per)
    dev_buf = buf.cuda()
    stats = gather_stats(dev_buf, contracts).cpu().numpy()
    per_all = dev_buf.cpu().numpy()
    base = rows(contracts)
    per = [per_all[b:b + c.R] for b, c in zip(base, contracts)]
    return stats[:, :4].copy(), stats[:, 4:].copy(), per
