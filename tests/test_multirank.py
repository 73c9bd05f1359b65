"""The N > 1 path of the benchmark on the CPU: one process per rank over gloo.

Replicas are independent, so ranks share no data: each runs its own seed, and
the only collectives are the barriers around the timed region and the maximum
of the ranks' times, from which the whole-job rate is formed.  The reference
arm under torchrun runs on rank 0 alone; the other ranks exit 0 at once.
"""
import json
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, r, local = bench._dist_env()
        # rank-dependent "times": the job's time is the slowest rank's
        t = 10.0 * (rank + 1)
        dist.barrier()
        t_max = bench.max_over_ranks(t, world, "cpu")
        value = bench.whole_job_rate(world, 1000.0, t_max)
        seeds = [None] * world
        dist.all_gather_object(seeds, bench.rank_seed(rank))
        out.put((rank, w, r, local, t_max, value, seeds))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_whole_job_rate_gloo():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, w, r, local, t_max, value, seeds in got:
        assert (w, r, local) == (world, rank, rank)
        assert t_max == 20.0                      # the slowest rank
        assert value == pytest.approx(2 * 1000.0 / 20.0)
        assert len(set(seeds)) == world           # independent replicas per rank


def test_single_rank_helpers():
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.whole_job_rate(1, 100.0, 2.0) == 50.0
    assert bench.rank_seed(0) != bench.rank_seed(1)


def test_reference_arm_under_torchrun_prints_one_line_from_rank_0():
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py",
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["n_gpus"] == 2
    assert line["value"] > 0 and line["cpu_baseline"]["kind"] == "oracle"
    assert line["e2e"]["h2d_bytes_per_step"] == 0
