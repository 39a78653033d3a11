"""Host side of the multi-GPU path, on CPU: two gloo ranks (127.0.0.1).

The job is split over the ranks (each contract's replicates in ranges, one
per rank, with the job's seed); the job's value counts each replicate once,
over the slowest rank's time; the reference arm runs on rank 0 only."""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import bench
    import workloads as W
    from paper_2209_11337_gb300 import shard
    r = bench.Ranks(world, "gloo")
    r.barrier()
    step_ms = 100.0 + 50.0 * rank  # rank 1 is the slower one
    worst = r.max_over_ranks(step_ms)
    r.barrier()
    grid = W.grid_d64()
    mine = shard.replicate_shards(grid, world)[rank]
    out.put((rank, worst, mine, bench.job_value(bench.elements(grid), worst)))
    r.close()


def test_two_gloo_ranks_take_the_max_time_and_split_the_replicates():
    import workloads as W
    from paper_2209_11337_gb300 import shard
    world, port = 2, free_port()
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    got = sorted(out.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [g[1] for g in got] == [150.0, 150.0]           # both ranks see the slowest step
    grid = W.grid_d64()
    reps = sorted((i, f + k) for g in got for i, f, n in g[2] for k in range(n))
    assert reps == sorted((i, r) for i, c in enumerate(grid) for r in range(c.R))  # each replicate once
    assert shard.point_dates(grid, got[0][2]) == shard.point_dates(grid, got[1][2])  # the same work per rank
    total = sum(c.N * c.R * c.d for c in grid)
    assert got[0][3] == pytest.approx(total / 0.150)         # the job's distinct point-dates / slowest time


def test_reference_arm_under_torchrun_prints_on_rank_zero_only():
    port = free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "3"]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=900, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["e2e"]["h2d_bytes_per_step"] == 0
