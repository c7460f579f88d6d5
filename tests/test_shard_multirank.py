"""Sharding of batched and served work over ranks (no GPU): two gloo ranks
split a request trace and a list of grids deterministically, each serves its
share against a host stand-in of the batch backend, and the union of their
results on rank 0 equals the one-rank run, request by request."""
import multiprocessing as mp
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_1109_6672_gb300 import inputs, serve, shard  # noqa: E402


class _OOM(Exception):
    status = -2


class _Clock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t

    def sleep(self, dt):
        self.t += dt


class DetBatch:
    """Host stand-in of lbm.Batch whose 'moments' are a deterministic function
    of the request's parameters and steps (the same alone or in any mix)."""

    def __init__(self, clock, slots=6, budget=6 * 64 * 64):
        self.clock, self.slots, self.budget = clock, slots, budget
        self.active, self.next = {}, 0

    def add(self, p, f, steps):
        n = p["nx"] * p["ny"]
        if len(self.active) >= self.slots or sum(v[0] for v in self.active.values()) + n > \
                self.budget:
            raise _OOM()
        s = self.next
        self.next += 1
        self.active[s] = [n, steps, steps, p]
        return s

    def remaining(self, s):
        return self.active[s][1]

    def run(self, k):
        work = 0
        for v in self.active.values():
            d = min(k, v[1])
            v[1] -= d
            work += d * v[0]
        self.clock.t += work * 1e-9

    def moments(self, s):
        n, _, steps, p = self.active[s]
        return (float(n), float(steps), float(p["tau_f"]), float(p.get("T_wall", [1.0])[0]))

    def remove(self, s):
        del self.active[s]


def _trace():
    return serve.make_trace(40, seed=11, rate=500.0, cavity_sides=(16, 64), couette_ny=(17, 41),
                            steps_range=(20, 200))


def _serve(requests):
    clock = _Clock()
    srv = serve.Server(DetBatch(clock), precision=3, seg_max=32, seg_min=8, keep_moments=True,
                       clock=clock, sleep=clock.sleep)
    return [(r.rid, r.moments, r.error) for r in srv.run(requests)]


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    from paper_1109_6672_gb300 import shard as sh

    dist.init_process_group("gloo", rank=rank, world_size=world)
    mine = sh.shard_trace(_trace(), rank, world)
    got = sh.gather_results(_serve(mine), dist)
    grids = inputs.batch_cavities(count=24, seed=4, sides=tuple(range(16, 129, 16)))
    owned = [i for i, _ in sh.shard_grids(grids, rank, world)]
    all_owned = [None] * world
    dist.all_gather_object(all_owned, owned)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, got, all_owned, len(mine)))


def test_two_ranks_union_equals_one_rank_run():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = {}
    for _ in procs:
        rank, got, owned, n = q.get(timeout=180)
        out[rank] = (got, owned, n)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    one = sorted(_serve(_trace()))
    union = sorted(out[0][0])
    assert out[1][0] is None  # results gather on rank 0 only
    assert union == one
    assert out[0][2] > 0 and out[1][2] > 0  # both ranks served some requests
    # the grid split is a partition, the same on both ranks
    owned = out[0][1]
    assert owned == out[1][1]
    assert sorted(owned[0] + owned[1]) == list(range(24))
    assert not set(owned[0]) & set(owned[1])


def test_grid_split_balances_work():
    grids = inputs.batch_cavities(count=256, seed=4)
    for world in (2, 4, 8):
        owner = shard.assign_grids(grids, world)
        loads = [0] * world
        for (p, _), r in zip(grids, owner):
            loads[r] += p["nx"] * p["ny"]
        assert max(loads) <= 1.02 * sum(loads) / world
        assert owner == shard.assign_grids(grids, world)  # deterministic


def test_request_split_keeps_every_request_once():
    trace = serve.make_trace(200, seed=5)
    parts = [shard.shard_trace(trace, r, 4) for r in range(4)]
    rids = sorted(r.rid for p in parts for r in p)
    assert rids == sorted(r.rid for r in trace)
    work = [sum(r.nodes * r.steps for r in p) for p in parts]
    assert max(work) <= 1.3 * sum(work) / 4
    with pytest.raises(ValueError):
        shard.assign_requests(trace, 0)
