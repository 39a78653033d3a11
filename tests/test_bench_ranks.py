"""Host side of the multi-GPU path, on CPU: two gloo ranks (127.0.0.1).

Each rank runs the whole batch on its own randomisation (weak scaling, no
data-path collective); the job's value is all ranks' point-dates over the
slowest rank's time; the reference arm runs on rank 0 only."""
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
    r = bench.Ranks(world, "gloo")
    r.barrier()
    step_ms = 100.0 + 50.0 * rank  # rank 1 is the slower one
    worst = r.max_over_ranks(step_ms)
    r.barrier()
    out.put((rank, worst, bench.rank_seed(rank), bench.job_value(1000, world, worst)))
    r.close()


def test_two_gloo_ranks_take_the_max_time_and_distinct_seeds():
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
    assert got[0][2] != got[1][2]                           # independent randomisations
    assert got[0][3] == pytest.approx(2 * 1000 / 0.150)     # whole-job point-dates / slowest time


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
