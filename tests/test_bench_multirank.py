"""Host logic of the multi-rank benchmark on CPU: two gloo ranks take the
slowest rank's time as the job's time and report the whole-job value; the
reference arm runs on rank 0 only."""
import argparse
import json
import multiprocessing as mp
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank: int, world: int, port: int, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    elapsed = bench.reduce_max(0.5 + rank, dist, "cpu")  # rank r took 0.5 + r s
    value = bench.job_value(world, nodes=1000, steps=10, elapsed=elapsed)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, elapsed, value))


def test_two_gloo_ranks_take_the_slowest_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, elapsed, value in out:
        assert elapsed == 1.5
        assert value == pytest.approx(2 * 1000 * 10 / 1.5 / 1e9)


def test_reference_arm_runs_on_rank_zero_only(capsys):
    sys.path.insert(0, ROOT)
    import bench

    args = argparse.Namespace(ref_side=16, steps=3, warmup=1, n=4096)
    assert bench.run_reference(args, rank=1, world=2) is None
    assert capsys.readouterr().out == ""
    line = bench.run_reference(args, rank=0, world=2)
    printed = json.loads(capsys.readouterr().out.strip())
    assert printed == line
    assert printed["impl"] == "reference" and printed["n_gpus"] == 2
    assert printed["cpu_baseline"]["kind"] == "oracle" and printed["value"] > 0
    assert printed["e2e"]["h2d_bytes_per_step"] == 0
