"""Host-side logic of the serving loop against a stand-in batch backend (no
GPU): admission by slots and footprint, continuous batching, completion of
every request, latency accounting."""
import pytest

from paper_1109_6672_gb300 import serve


class OOM(Exception):
    status = -2


class FakeBatch:
    """Slots and a node budget as the footprint; run(k) costs k * nodes * t."""

    def __init__(self, slots, node_budget, clock, t_per_update=1e-9):
        self.slots, self.budget, self.clock, self.t = slots, node_budget, clock, t_per_update
        self.active = {}
        self.max_active = 0
        self.max_nodes = 0
        self.next = 0

    def add(self, p, f, steps):
        n = p["nx"] * p["ny"]
        used = sum(v[0] for v in self.active.values())
        if len(self.active) >= self.slots or used + n > self.budget:
            raise OOM()
        s = self.next
        self.next += 1
        self.active[s] = [n, steps]
        self.max_active = max(self.max_active, len(self.active))
        self.max_nodes = max(self.max_nodes, used + n)
        return s

    def remaining(self, s):
        return self.active[s][1]

    def run(self, k):
        work = 0
        for v in self.active.values():
            d = min(k, v[1])
            v[1] -= d
            work += d * v[0]
        self.clock.advance(work * self.t)

    def moments(self, s):
        return None

    def remove(self, s):
        del self.active[s]


class Clock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t

    def advance(self, dt):
        self.t += dt

    def sleep(self, dt):
        self.t += dt


def small_trace(n=30, seed=3):
    return serve.make_trace(n, seed=seed, rate=200.0, cavity_sides=(32, 96), couette_ny=(17, 41),
                            steps_range=(50, 400))


def test_every_request_completes_within_capacity():
    clock = Clock()
    budget = 3 * 96 * 96
    fb = FakeBatch(slots=4, node_budget=budget, clock=clock)
    srv = serve.Server(fb, precision=3, seg_max=64, seg_min=8, clock=clock, sleep=clock.sleep)
    trace = small_trace()
    res = srv.run(trace)
    assert sorted(r.rid for r in res) == [r.rid for r in trace]
    assert fb.max_active <= 4 and fb.max_nodes <= budget
    for r in res:
        assert r.finished >= r.admitted >= r.arrival - 1e-12
    s = serve.summarize(res, srv.wall, srv.node_updates)
    assert s["requests"] == len(trace) and s["p99_s"] >= s["p50_s"] > 0
    assert srv.node_updates == sum(r.nodes * r.steps for r in trace)


def test_continuous_batching_overlaps_requests():
    """Requests that arrive while others run are admitted at the next segment
    boundary and share segments with them."""
    clock = Clock()
    fb = FakeBatch(slots=16, node_budget=10 ** 9, clock=clock, t_per_update=2e-8)
    srv = serve.Server(fb, precision=3, seg_max=32, seg_min=8, clock=clock, sleep=clock.sleep)
    trace = small_trace(20, seed=4)
    res = srv.run(trace)
    assert fb.max_active >= 3
    by_id = {r.rid: r for r in res}
    overlaps = sum(1 for a in res for b in res if a.rid < b.rid and
                   b.admitted < a.finished and a.admitted < b.finished)
    assert overlaps > 0
    assert len(by_id) == len(trace)


def test_request_too_big_waits_then_runs():
    clock = Clock()
    fb = FakeBatch(slots=2, node_budget=100 * 100, clock=clock)
    srv = serve.Server(fb, precision=3, seg_max=16, seg_min=4, clock=clock, sleep=clock.sleep)
    trace = [serve.Request(0, "cavity", 0.0, 40, dict(n=100, Ra=1e4, dT_over_T0=0.1)),
             serve.Request(1, "cavity", 0.0, 40, dict(n=50, Ra=1e4, dT_over_T0=0.1))]
    res = srv.run(trace)
    assert len(res) == 2
    second = [r for r in res if r.rid == 1][0]
    first = [r for r in res if r.rid == 0][0]
    assert second.admitted >= first.finished - 1e-12  # had to wait for room


def test_trace_is_seeded_and_has_the_mix():
    a = serve.make_trace(200, seed=5)
    b = serve.make_trace(200, seed=5)
    assert [(r.kind, r.arrival, r.steps) for r in a] == [(r.kind, r.arrival, r.steps) for r in b]
    frac = sum(r.kind == "cavity" for r in a) / len(a)
    assert 0.55 < frac < 0.85
    assert all(1000 <= r.steps <= 100000 for r in a)
    assert abs(a[-1].arrival / 200 - 1 / 50) < 0.01


def test_request_larger_than_the_pool_fails_alone():
    clock = Clock()
    fb = FakeBatch(slots=4, node_budget=60 * 60, clock=clock)
    srv = serve.Server(fb, precision=3, seg_max=16, seg_min=4, clock=clock, sleep=clock.sleep)
    trace = [serve.Request(0, "cavity", 0.0, 40, dict(n=50, Ra=1e4, dT_over_T0=0.1)),
             serve.Request(1, "cavity", 0.0, 40, dict(n=100, Ra=1e4, dT_over_T0=0.1)),
             serve.Request(2, "cavity", 1e-3, 40, dict(n=100, Ra=1e4, dT_over_T0=0.1))]
    res = {r.rid: r for r in srv.run(trace)}  # must end: nothing can ever admit 1 or 2
    assert set(res) == {0, 1, 2}
    assert res[0].error == ""
    assert res[1].error and res[2].error
    assert res[1].finished >= res[0].admitted  # tried again after 0 left, then failed
    s = serve.summarize(list(res.values()), srv.wall, srv.node_updates)
    assert s["failed"] == 2



@pytest.mark.parametrize("max_bypass", [0, 3, 10 ** 9])
def test_large_request_is_not_passed_without_limit(max_bypass):
    """A request refused for room waits a bounded number of segments: later,
    smaller requests pass it at most max_bypass segments running, then
    admission stops at it until it fits.  Without the bound (10**9) a steady
    stream of small requests keeps it out until the stream ends."""
    clock = Clock()
    small = 33 * 4
    # room for the 60^2 request beside at most two small channels
    fb = FakeBatch(slots=8, node_budget=60 * 60 + 2 * small, clock=clock, t_per_update=1e-9)
    srv = serve.Server(fb, precision=3, seg_max=16, seg_min=16, clock=clock, sleep=clock.sleep,
                       max_bypass=max_bypass)
    trace, t = [], 0.0
    for i in range(300):  # a steady stream of small channels, 3 segments each,
        # about one arrival per segment, so some are always running
        trace.append(serve.Request(1 + i, "couette", t, 48, dict(ny=33, nx=4, U=0.05)))
        t += 5e-6
    trace.append(serve.Request(0, "cavity", 1e-4 + 1e-9, 32, dict(n=60, Ra=1e4, dT_over_T0=0.1)))
    res = {r.rid: r for r in srv.run(trace)}
    assert len(res) == len(trace) and not any(r.error for r in res.values())
    big = res[0]
    passed = sum(1 for r in res.values() if r.rid >= 1 and big.arrival < r.arrival
                 and r.admitted < big.admitted)
    if max_bypass == 0:
        assert passed == 0
    elif max_bypass == 3:
        assert 0 < passed <= (max_bypass + 1) * 8
    else:  # unbounded bypass: the big request waits for (nearly) the whole stream
        assert passed > 250
