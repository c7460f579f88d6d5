"""Serving loop: continuous batching of cavity and Couette simulations.

Requests arrive over time (a seeded Poisson stream).  Each request is one
simulation: a grid, its parameters and initial fields, and a number of time
steps.  The server keeps the populations of every admitted request resident in
one device pool (``lbm.Batch``); a request is admitted as soon as a slot and its
footprint (``lbm_state_bytes``) are free, in arrival order: a later request
may pass a waiting one only while that one has waited fewer than
``max_bypass`` segments, after which nothing is admitted until it fits (so a
large request waits a bounded number of segments behind smaller ones; 0 gives
strict first-in-first-out).  The GPU advances
all admitted grids together in segments of k steps (one graph launch per
segment, one kernel launch per step covering every grid); between segments
finished requests are read back (moments) and released and queued requests are
admitted, so work that arrives while others run overlaps with them on the
device.  Latency = completion - arrival (queueing included).  A request that
does not fit even the empty pool fails alone (it could never be admitted).

The batch backend is injected, so the scheduling logic also runs against a
host-only stand-in in the CPU tests.
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass, field

import numpy as np

from . import inputs
from .lbm import LBM_ERR_NONFINITE, LBM_ERR_OOM


@dataclass
class Request:
    rid: int
    kind: str  # "cavity" or "couette"
    arrival: float  # seconds after the start of the trace
    steps: int
    spec: dict  # arguments of the inputs recipe
    params: dict = field(default=None, repr=False)
    fields: tuple = field(default=None, repr=False)
    passed: int = field(default=0, repr=False)  # segments waited after a refusal

    def materialize(self, precision: int):
        if self.params is None:
            if self.kind == "cavity":
                p, f = inputs.cavity(precision=precision, **self.spec)
            else:
                p, f = inputs.couette(precision=precision, **self.spec)
            self.params, self.fields = p, f
        return self.params, self.fields

    @property
    def nodes(self) -> int:
        if self.kind == "cavity":
            return self.spec["n"] ** 2
        return self.spec["ny"] * self.spec.get("nx", 4)


def make_trace(count: int, seed: int = 5, rate: float = 50.0, cavity_frac: float = 0.7,
               cavity_sides=(32, 2048), couette_ny=(17, 257), steps_range=(1000, 100000),
               dT_range=(0.01, 0.6), U_range=(0.01, 0.1), nu_min: float = 0.02):
    """Seeded request stream: exponential inter-arrival times at `rate` per
    second; cavity requests (side uniform in cavity_sides, dT/T0 uniform in
    dT_range, Ra log-uniform in [1e4, 1e6]) with probability cavity_frac, else
    Couette requests (ny uniform in couette_ny, nx = 4, U uniform in U_range);
    steps uniform in steps_range."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for i in range(count):
        t += float(rng.exponential(1.0 / rate))
        steps = int(rng.integers(steps_range[0], steps_range[1] + 1))
        if rng.uniform() < cavity_frac:
            n = int(rng.integers(cavity_sides[0], cavity_sides[1] + 1))
            spec = dict(n=n, dT_over_T0=float(rng.uniform(*dT_range)),
                        Ra=float(10.0 ** rng.uniform(4.0, 6.0)), seed=int(rng.integers(1 << 30)),
                        nu_min=nu_min)
            out.append(Request(i, "cavity", t, steps, spec))
        else:
            ny = int(rng.integers(couette_ny[0], couette_ny[1] + 1))
            spec = dict(ny=ny, nx=4, U=float(rng.uniform(*U_range)))
            out.append(Request(i, "couette", t, steps, spec))
    return out


def scale_arrivals(trace, factor: float):
    """Same requests with all arrival times multiplied by factor."""
    for r in trace:
        r.arrival *= factor
    return trace


def load_factor_scale(trace, glups: float, load: float = 0.7) -> float:
    """Arrival-time factor that makes the offered work (node updates per
    second) `load` times a sustained throughput of `glups`."""
    work = sum(r.nodes * r.steps for r in trace)
    span = trace[-1].arrival if trace else 1.0
    offered = work / max(span, 1e-9) / 1e9  # G node updates per second at the given times
    return offered / (load * glups)


@dataclass
class Result:
    rid: int
    kind: str
    nodes: int
    steps: int
    arrival: float
    admitted: float
    finished: float
    moments: tuple = field(default=None, repr=False)
    error: str = ""

    @property
    def latency(self) -> float:
        return self.finished - self.arrival


class Server:
    """Continuous-batching server over a batch backend with the ``lbm.Batch``
    interface (add / run / remaining / moments / remove / info)."""

    def __init__(self, batch, precision: int, seg_max: int = 256, seg_min: int = 16,
                 keep_moments: bool = False, clock=time.perf_counter, sleep=time.sleep,
                 max_bypass: int = 8):
        self.batch = batch
        self.max_bypass = max_bypass
        self.precision = precision
        self.seg_max = seg_max
        self.seg_min = seg_min
        self.keep_moments = keep_moments
        self.clock = clock
        self.sleep = sleep
        self.segments = 0
        self.node_updates = 0

    def run(self, trace):
        pending = sorted(trace, key=lambda r: r.arrival)
        for r in pending:
            r.passed = 0
        queue = []
        active = {}  # slot -> (request, admitted time)
        results = []
        t0 = self.clock()
        i = 0
        while i < len(pending) or queue or active:
            now = self.clock() - t0
            while i < len(pending) and pending[i].arrival <= now:
                queue.append(pending[i])
                i += 1
            # admit in arrival order while slots and pool space last; a
            # refused request may be passed by later ones only while it has
            # waited fewer than max_bypass segments (then admission stops at
            # it until it fits)
            still = []
            blocked = False
            for r in queue:
                if blocked:
                    still.append(r)
                    continue
                p, f = r.materialize(self.precision)
                try:
                    slot = self.batch.add(p, f, r.steps)
                except Exception as e:  # no slot / no room: keep waiting
                    if getattr(e, "status", None) != LBM_ERR_OOM:
                        raise
                    if not active:  # refused by the empty pool: never fits
                        t = self.clock() - t0
                        results.append(Result(r.rid, r.kind, r.nodes, r.steps, r.arrival, t, t,
                                              None, "does not fit the device pool"))
                    else:
                        blocked = r.passed >= self.max_bypass
                        still.append(r)
                    continue
                active[slot] = (r, self.clock() - t0)
            queue = still
            if not active:
                if i < len(pending):
                    wait = pending[i].arrival - (self.clock() - t0)
                    if wait > 0:
                        self.sleep(wait)
                continue
            rem = {s: self.batch.remaining(s) for s in active}
            k = max(self.seg_min, min(self.seg_max, min(rem.values())))
            self.batch.run(k)
            self.segments += 1
            for r in queue:  # segments the refused requests have waited through
                r.passed += 1
            for s, r0 in rem.items():
                r, _ = active[s]
                self.node_updates += r.nodes * min(k, r0)
            for s in [s for s in active if self.batch.remaining(s) == 0]:
                r, adm = active.pop(s)
                err = ""
                try:
                    mom = self.batch.moments(s)
                except Exception as e:  # a diverged simulation fails alone
                    if getattr(e, "status", None) != LBM_ERR_NONFINITE:
                        raise
                    mom, err = None, "non-finite result"
                self.batch.remove(s)
                results.append(Result(r.rid, r.kind, r.nodes, r.steps, r.arrival, adm,
                                      self.clock() - t0, mom if self.keep_moments else None, err))
        self.wall = self.clock() - t0
        return results


def summarize(results, wall: float, node_updates: int) -> dict:
    lat = np.array([r.latency for r in results]) if results else np.zeros(1)
    return {
        "requests": len(results),
        "failed": sum(1 for r in results if r.error),
        "p50_s": float(np.percentile(lat, 50)),
        "p99_s": float(np.percentile(lat, 99)),
        "mean_s": float(lat.mean()),
        "makespan_s": float(wall),
        "glups": float(node_updates / max(wall, 1e-12) / 1e9),
        "sims_per_s": float(len(results) / max(wall, 1e-12)),
    }
