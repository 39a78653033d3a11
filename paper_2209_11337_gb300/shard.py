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
