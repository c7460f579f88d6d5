"""Benchmark of the fused coupled f+h D2Q9 step on GB300.

Workload (one "step" = one time step of the whole hot path over one grid):
periodic box 4096 x 4096, rho = 1, u ~ U(-1e-3, 1e-3), T = T0 (1 + U(-1e-2,
1e-2)) (seed 2), tau_f = 0.3, Pr = 0.71, b = 3, total-energy model,
correction on, FP32 storage and arithmetic.  The state (2.4 GB) is far larger
than L2 (129 MB), so no L2 flush is needed between steps.

Prints one JSON line.  ``--impl reference`` times the FP64 CPU oracle on the
host cores on a bounded sample of the same workload instead.
Multi-GPU (torchrun): every rank runs an independent replica (the single grid
is not sharded; weak scaling), max time over ranks.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "coupled f+h D2Q9 GLUPS and % HBM roofline; served p50/p99 latency"
UNIT = "GLUPS"

# DRAM bytes (read + write) of one step launch at 4096^2, from one ncu capture
# at 2048^2 scaled by the node count (profiles/step_pr_*_2048_full.md), keyed
# by the hash of the kernel sources they were measured on; a changed kernel
# reports null until it is captured again.
KERNEL_SOURCES = ("lbm_device.cuh", "lbm_step_tma.cuh", "lbm_step_pr.cuh")
MEASURED_TRAFFIC = {
    ("f35a03e90c75e143", "f32"): 2300.923904e6,
    ("f35a03e90c75e143", "bf16"): 1091.465216e6,
    ("f35a03e90c75e143", "f16"): 1096.441856e6,
}


def kernel_hash():
    """sha256/16 of the kernel sources' code: comments and blank lines are
    dropped, so that a comment edit does not void the measured traffic."""
    import hashlib
    import re

    csrc = os.path.join(ROOT, "paper_1109_6672_gb300", "csrc")
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(csrc, f), encoding="utf-8") as fh:
            code = re.sub(r"/\*.*?\*/", "", fh.read(), flags=re.S)
        code = re.sub(r"//[^\n]*", "", code)
        lines = [line.rstrip() for line in code.split("\n") if line.strip()]
        h.update("\n".join(lines).encode())
    return h.hexdigest()[:16]


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons: one sample just before the
    timed region, samples every 200 ms during it, and one just after (so a
    region shorter than the polling period still has a record)."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join("/tmp", f"lbm_clocks_{os.getpid()}.csv")

    def one_shot(self):
        try:
            r = subprocess.run(["nvidia-smi", f"--query-gpu={self.FIELDS}",
                                "--format=csv,noheader,nounits"], capture_output=True, text=True,
                               timeout=20)
            return r.stdout
        except Exception:
            return ""

    def __enter__(self):
        self.edges = [self.one_shot()]
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()
        self.edges.append(self.one_shot())

    def summary(self):
        lines = []
        if self.proc is not None:
            with open(self.path) as f:
                lines = f.read().splitlines()
        lines += [ln for chunk in self.edges for ln in chunk.splitlines()]
        if self.proc is None and not lines:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        for line in lines:
            parts = [s.strip() for s in line.split(",")]
            if len(parts) >= 9 and parts[1].replace(".", "").isdigit():
                rows.append(parts)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        mine = [r for r in rows if r[0] == str(self.gpu)]
        if mine and len({r[0] for r in rows}) > 1:
            rows = mine
        sm = [float(r[1]) for r in rows]
        mx = max(float(r[2]) for r in rows)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": reasons,
                "samples": len(rows), "power_w_max": max(float(r[3]) for r in rows)}


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def oracle_glups(n_side: int, steps: int, threads: int):
    """Time the FP64 oracle on an n_side^2 sample of the box workload."""
    from oracle import oracle
    from paper_1109_6672_gb300 import inputs

    p, fields = inputs.periodic_box(n=n_side, precision=inputs.P_FP64)
    o = oracle.Oracle(p).init(*fields)
    o.step(1, threads)
    t0 = time.perf_counter()
    o.step(steps, threads)
    dt = time.perf_counter() - t0
    return n_side * n_side * steps / dt / 1e9, dt


def reduce_max(value: float, dist, device) -> float:
    """Largest value over the ranks (the job's time is the slowest rank's);
    the value itself without a process group."""
    if dist is None:
        return float(value)
    import torch

    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(world: int, nodes: int, steps: int, elapsed: float) -> float:
    """Whole-job GLUPS: every rank advanced its own replica of `nodes` nodes
    by `steps` steps within `elapsed` seconds (max over ranks)."""
    return world * nodes * steps / elapsed / 1e9


def run_reference(args, rank, world):
    """The oracle as it stands on the host cores, on a side x side sample of
    the benchmark workload (same recipe), W untimed and K timed steps; rank 0
    only (other ranks of a multi-rank launch exit without work)."""
    if rank != 0:
        return None
    from oracle import oracle
    from paper_1109_6672_gb300 import inputs

    cores = cpu_cores()
    side = args.ref_side
    p, fields = inputs.periodic_box(n=side, precision=inputs.P_FP64)
    o = oracle.Oracle(p).init(*fields)
    o.step(args.warmup, cores)
    t0 = time.perf_counter()
    o.step(args.steps, cores)
    total_t = time.perf_counter() - t0
    value = side * side * args.steps / total_t / 1e9
    sample = (f"{side}x{side} periodic box of the same recipe (seed 2), {args.steps} timed "
              f"steps after {args.warmup} untimed, FP64, OpenMP over rows")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total_t / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": f"periodic box {args.n}x{args.n}, coupled f+h D2Q9 BGK, total "
                               "energy, correction on (FP64 CPU oracle on a bounded sample)",
                   "nx": args.n, "ny": args.n, "sample_side": side},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return line


def batch_and_serving(torch, args):
    """Config 4: the 256-cavity batch (sides 64..512) run to completion,
    10 000 steps per grid, in each 16/32-bit storage, against the same grids
    stepped one grid per launch in FP64; the error of each storage against
    FP64 after 10 000 steps; and a served trace (quick leg by default, the
    configured 500-request trace with --config5)."""
    from paper_1109_6672_gb300 import inputs, lbm, serve

    out = {}
    names = {lbm.LBM_P_FP32_BF16: "bf16", lbm.LBM_P_FP32_FP16: "f16", lbm.LBM_P_FP32: "f32"}
    sim_steps = args.batch_sim_steps

    def batched(precision):
        """Completed simulations: every grid admitted with a budget of
        sim_steps, then segments of up to 4096 steps until none is left; the
        wall time runs from the first segment to the last completion (graph
        captures included; the autotuner before it is timed apart)."""
        grids = inputs.batch_cavities(count=args.batch_grids, seed=4, precision=precision)
        nodes = sum(p["nx"] * p["ny"] for p, _ in grids)
        pool = sum(lbm.lbm_state_bytes(p) for p, _ in grids) + (64 << 20)
        b = lbm.Batch(precision, len(grids), pool)
        slots = [b.add(p, f, sim_steps) for p, f in grids]
        t0 = time.perf_counter()
        tuned = b.autotune(3)
        t_tune = time.perf_counter() - t0
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        left = sim_steps
        while left > 0:
            k = min(4096, left)
            b.run(k)
            left -= k
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        assert all(b.remaining(s) == 0 for s in slots)
        b.close()
        return grids, nodes, dt, tuned, t_tune

    res = {}
    for prec in (lbm.LBM_P_FP32_BF16, lbm.LBM_P_FP32_FP16, lbm.LBM_P_FP32):
        grids, nodes, dt, tuned, t_tune = batched(prec)
        res[prec] = {"glups": nodes * sim_steps / dt / 1e9, "seconds": dt,
                     "sims_per_s": len(grids) / dt, "autotune": tuned,
                     "autotune_seconds": t_tune}
    # the plain one-grid-per-launch FP64 path, each grid for fp64_steps
    # steps (its own graph replays), sequentially
    f64 = [lbm.Lbm(dict(p, precision=lbm.LBM_P_FP64)).init(*f) for p, f in grids]
    for g in f64:
        g.step(32)
    torch.cuda.synchronize()
    k64 = args.batch_fp64_steps
    t0 = time.perf_counter()
    for g in f64:
        g.step(k64)
    torch.cuda.synchronize()
    dt64 = time.perf_counter() - t0
    for g in f64:
        g.close()
    glups64 = nodes * k64 / dt64 / 1e9
    sims64 = len(grids) * k64 / sim_steps / dt64  # 10 000-step simulations per second
    # error of each storage precision (batched) against the FP64 path after
    # 10 000 steps, on grids of side <= 256 spanning the dT range of the batch
    small = sorted((g for g in grids if g[0]["nx"] <= 256),
                   key=lambda g: abs(g[0]["T_wall"][0] - g[0]["T_wall"][1]))
    pick = [small[round(i * (len(small) - 1) / max(args.batch_err_grids - 1, 1))]
            for i in range(args.batch_err_grids)] if small else []
    errs = {names[q]: [] for q in names}
    for p, f in pick:
        ref = lbm.Lbm(dict(p, precision=lbm.LBM_P_FP64)).init(*f).step(10000)
        rho64, ux64, uy64, T64 = ref.moments()
        ref.close()
        dTw = abs(p["T_wall"][0] - p["T_wall"][1])
        umax = max(np.abs(ux64).max(), np.abs(uy64).max())
        for q in names:
            pq = dict(p, precision=q)
            bb = lbm.Batch(q, 1, lbm.lbm_state_bytes(pq) + (1 << 20))
            sl = bb.add(pq, f, 10000)
            while bb.remaining(sl):
                bb.run(min(1000, bb.remaining(sl)))
            rho, ux, uy, T = bb.moments(sl)
            bb.close()
            du = np.sqrt((ux - ux64) ** 2 + (uy - uy64) ** 2)
            errs[names[q]].append({
                "n": p["nx"], "dT_over_T0": dTw,
                "T_max_rel": float(np.abs(T - T64).max() / np.abs(T64).max()),
                "T_l2_rel": float(np.sqrt(np.mean((T - T64) ** 2) / np.mean(T64 ** 2))),
                "T_max_over_dT": float(np.abs(T - T64).max() / dTw),
                "u_max_over_umax": float(du.max() / umax),
                "u_l2_over_umax": float(np.sqrt(np.mean(du ** 2)) / umax)})
    meets = {k: all(e["T_max_rel"] <= 1e-3 for e in v) for k, v in errs.items()}
    # headline: FP32 storage, the storage that meets the 1e-3 relative T
    # target on every sampled grid (and the fastest: the 16-bit kernels are
    # instruction-bound); the configured BF16 storage beside it
    out["batch"] = {
        "grids": len(grids), "nodes": nodes, "steps_per_sim": sim_steps,
        "completed": "every grid ran all its steps inside the timed wall time",
        "precision": "f32 arithmetic, f32 storage (the storage meeting the 1e-3 T target)",
        "glups": res[lbm.LBM_P_FP32]["glups"],
        "seconds": res[lbm.LBM_P_FP32]["seconds"],
        "sims_per_s": res[lbm.LBM_P_FP32]["sims_per_s"],
        "autotune": res[lbm.LBM_P_FP32]["autotune"],
        "bf16_storage_configured": res[lbm.LBM_P_FP32_BF16],
        "f16_storage": res[lbm.LBM_P_FP32_FP16], "f32_storage": res[lbm.LBM_P_FP32],
        "fp64_one_grid_per_launch": {"glups": glups64, "sims_per_s_10k_steps": sims64,
                                     "steps_timed_per_grid": k64, "seconds": dt64,
                                     "note": "every grid stepped k steps, one grid per "
                                             "launch sequence; sims/s = grids x k / 10 000 "
                                             "/ seconds"},
        "speedup_sims_per_s": res[lbm.LBM_P_FP32]["sims_per_s"] / sims64,
        "speedup_sims_per_s_bf16": res[lbm.LBM_P_FP32_BF16]["sims_per_s"] / sims64,
        "meets_1e-3_T": meets,
        "error_vs_fp64_after_10k_steps": errs,
    }
    if args.serve_requests <= 0:
        return out
    glups_bf16 = res[lbm.LBM_P_FP32_BF16]["glups"]

    def served(key, prec, trace, desc, factor):
        for r in trace:  # inputs are materialised per precision
            r.params = r.fields = None
        sb = lbm.Batch(prec, 64, args.serve_pool_gb << 30)
        srv = serve.Server(sb, prec, seg_max=256, seg_min=16)
        t0 = time.perf_counter()
        res_ = srv.run(trace)
        wall = time.perf_counter() - t0
        sb.close()
        st = serve.summarize(res_, srv.wall, srv.node_updates)
        st.update({"precision": names[prec] + " storage", "load_factor": 0.7,
                   "arrival_time_scale": factor, "trace": desc, "wall_seconds": wall})
        out[key] = st

    # quick leg: 40 requests, sides 32-512, 1e3-1e4 steps, load 0.7
    trace = serve.make_trace(args.serve_requests, seed=5, rate=50.0, cavity_sides=(32, 512),
                             couette_ny=(17, 257), steps_range=(1000, 10000))
    factor = serve.load_factor_scale(trace, glups_bf16, load=0.7)
    serve.scale_arrivals(trace, factor)
    desc = (f"{args.serve_requests} requests, 70 % cavity (side 32-512) / 30 % Couette (ny "
            "17-257), 1e3-1e4 steps, Poisson arrivals (seed 5) time-scaled to 0.7 of the BF16 "
            "batched throughput")
    for key, prec in (("serving", lbm.LBM_P_FP32_BF16), ("serving_f16", lbm.LBM_P_FP32_FP16),
                      ("serving_f32", lbm.LBM_P_FP32)):
        served(key, prec, trace, desc, factor)
    if args.config5_sample > 0:
        # a sample of the configured ranges (sides 32-2048, 1e3-1e5 steps), the
        # first requests of the configured seeded stream, load 0.7, BF16
        trace = serve.make_trace(args.config5_sample, seed=5, rate=50.0)
        factor = serve.load_factor_scale(trace, glups_bf16, load=0.7)
        serve.scale_arrivals(trace, factor)
        desc = (f"the first {args.config5_sample} requests of the configured stream: 70 % "
                "cavity (side 32-2048, dT/T0 0.01-0.6, Ra 1e4-1e6) / 30 % Couette (ny 17-257), "
                "1e3-1e5 steps, Poisson arrivals (seed 5) time-scaled to 0.7 of the BF16 batched "
                "throughput")
        served("serving_config5_sample", lbm.LBM_P_FP32_BF16, trace, desc, factor)
    if args.config5:
        # the configured trace: 500 requests, cavity sides 32-2048, 1e3-1e5
        # steps, Couette ny 17-257, time-scaled to load 0.7
        trace = serve.make_trace(500, seed=5, rate=50.0)
        factor = serve.load_factor_scale(trace, glups_bf16, load=0.7)
        serve.scale_arrivals(trace, factor)
        desc = ("500 requests, 70 % cavity (side 32-2048, dT/T0 0.01-0.6, Ra 1e4-1e6) / 30 % "
                "Couette (ny 17-257, U 0.01-0.1), 1e3-1e5 steps, Poisson arrivals (seed 5, "
                "50/s) time-scaled to 0.7 of the BF16 batched throughput")
        for which in args.config5.split(","):
            prec = {"bf16": lbm.LBM_P_FP32_BF16, "f32": lbm.LBM_P_FP32}[which]
            served("serving_config5" + ("" if which == "bf16" else "_" + which), prec, trace,
                   desc, factor)
    return out


def sharded_batch(torch, args, rank, world, dist):
    """Config 4 over the ranks of a multi-GPU job: each rank takes its share
    of the 256 cavities (paper_1109_6672_gb300.shard, no data-path exchange)
    and runs it to completion in BF16 storage; the job's time is the slowest
    rank's, sims/s counts every rank's completed grids."""
    from paper_1109_6672_gb300 import inputs, lbm, shard

    grids = inputs.batch_cavities(count=args.batch_grids, seed=4)
    mine = [g for _, g in shard.shard_grids(grids, rank, world)]
    nodes = sum(p["nx"] * p["ny"] for p, _ in mine)
    b = lbm.Batch(lbm.LBM_P_FP32_BF16, max(1, len(mine)),
                  sum(lbm.lbm_state_bytes(p) for p, _ in mine) + (64 << 20))
    for p, f in mine:
        b.add(p, f, args.batch_sim_steps)
    b.autotune(3)
    dist.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    left = args.batch_sim_steps
    while left > 0:
        k = min(4096, left)
        b.run(k)
        left -= k
    torch.cuda.synchronize()
    dt = reduce_max(time.perf_counter() - t0, dist, "cuda")
    b.close()
    total_nodes = reduce_sum(nodes, dist, "cuda")
    return {"batch_sharded": {
        "grids": len(grids), "ranks": world, "seconds": dt,
        "sims_per_s": len(grids) / dt,
        "glups": total_nodes * args.batch_sim_steps / dt / 1e9,
        "split": "longest-first greedy by nodes, whole grids per rank, no exchange"}}


def reduce_sum(value: float, dist, device) -> float:
    import torch

    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def large_dT_study(torch, args):
    """Large-dT cavity (1024^2, dT/T0 = 0.6, Ra = 1e6, Pr = 0.71, noise 1e-4,
    seed 3): FP32 storage and FP16 / BF16 deviation storage against FP64 after
    `args.config3_steps` steps: max and L2 error of u and T, and the mean
    wall heat flux (Nusselt number at both walls).  The FP64 run is the CUDA
    FP64 path (the tests hold it to 1e-12 of the oracle, which is too slow for
    this size)."""
    from paper_1109_6672_gb300 import inputs, lbm

    n, steps = 1024, args.config3_steps

    def wall_nu(p, T):
        Th, Tl = p["T_wall"][0], p["T_wall"][1]
        cold = ((9 * T[:, -1] - T[:, -2] - 8 * Tl) / 3).mean() * n / (Th - Tl)
        hot = (-(9 * T[:, 0] - T[:, 1] - 8 * Th) / 3).mean() * n / (Th - Tl)
        return float(hot), float(cold)

    out = {"grid": f"{n}x{n}", "dT_over_T0": 0.6, "Ra": 1e6, "steps": steps,
           "note": "bf16 / f16: the TMA step kernel, whose 16-bit T recovery ends in one FP32 "
                   "subtraction of deviation terms; bf16_fp64_recovery: the register-pull "
                   "kernel (launch variant 128), which forms rho E in FP64 from the FP32 "
                   "deviation sums (its other arithmetic also rounds in another order)"}
    ref = None
    mom_bf16 = None
    dTw = 0.6
    for name, q, variant in (("f64", lbm.LBM_P_FP64, 0), ("f32", lbm.LBM_P_FP32, 0),
                             ("f16", lbm.LBM_P_FP32_FP16, 0), ("bf16", lbm.LBM_P_FP32_BF16, 0),
                             ("bf16_fp64_recovery", lbm.LBM_P_FP32_BF16, 128)):
        p, f = inputs.cavity(n=n, Ra=1e6, dT_over_T0=0.6, seed=3, precision=q)
        g = lbm.Lbm(p)
        if variant:
            g.set_launch(variant)
        g.init(*f)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        g.step(steps)
        mom = g.moments()
        dt = time.perf_counter() - t0
        g.close()
        hot, cold = wall_nu(p, mom[3])
        rec = {"seconds": dt, "glups": n * n * steps / dt / 1e9, "Nu_hot": hot, "Nu_cold": cold}
        if ref is None:
            ref = mom
        else:
            rho0, ux0, uy0, T0_ = ref
            rho, ux, uy, T = mom
            du = np.sqrt((ux - ux0) ** 2 + (uy - uy0) ** 2)
            umax = float(np.sqrt(ux0 ** 2 + uy0 ** 2).max())
            rec.update({
                "T_max_rel": float(np.abs(T - T0_).max() / np.abs(T0_).max()),
                "T_l2_rel": float(np.sqrt(np.mean((T - T0_) ** 2) / np.mean(T0_ ** 2))),
                "T_max_over_dT": float(np.abs(T - T0_).max() / dTw),
                "u_max_over_umax": float(du.max() / umax),
                "u_l2_over_umax": float(np.sqrt(np.mean(du ** 2)) / umax),
                "Nu_cold_rel": abs(cold - out["f64"]["Nu_cold"]) / abs(out["f64"]["Nu_cold"]),
            })
            if name == "bf16":
                mom_bf16 = mom
            elif name == "bf16_fp64_recovery" and mom_bf16 is not None:
                # the two BF16 forms against each other
                T16 = mom_bf16[3]
                du16 = np.sqrt((ux - mom_bf16[1]) ** 2 + (uy - mom_bf16[2]) ** 2)
                rec["vs_bf16_fp32_recovery"] = {
                    "T_max_over_dT": float(np.abs(T - T16).max() / dTw),
                    "u_max_over_umax": float(du16.max() / umax)}
        out[name] = rec
    return out


def time_steps(torch, lbm_mod, g, stream, steps):
    """CUDA-event time of `steps` back-to-back step launches on `stream`."""
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    g.step(steps)
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1) / 1e3


def run_ours(args, rank, world, local_rank):
    import torch

    from paper_1109_6672_gb300 import build as cuda_build
    from paper_1109_6672_gb300 import inputs, lbm

    cuda_build.build()
    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist_mod

        dist = dist_mod
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))

    prec = {"f64": lbm.LBM_P_FP64, "f32": lbm.LBM_P_FP32, "f16": lbm.LBM_P_FP32_FP16,
            "bf16": lbm.LBM_P_FP32_BF16}[args.precision]
    n = args.n
    coll = dict(collision=lbm.LBM_COLL_MRT, s_e=1.3, s_eps=1.1, s_q=1.6) \
        if args.collision == "mrt" else {}
    p, fields = inputs.periodic_box(n=n, precision=prec, **coll)
    stream = torch.cuda.Stream()
    g = lbm.Lbm(p, stream=stream.cuda_stream)
    if args.threads:
        g.set_launch(args.threads, args.rows)
    # inputs resident in HBM before the timed region
    dev_fields = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in fields]
    with torch.cuda.stream(stream):
        lbm.lbm_init_device(g.h, *[t.data_ptr() for t in dev_fields])
    stream.synchronize()
    g.step(args.warmup)
    g.sync()

    gpu_index = int(os.environ.get("CUDA_VISIBLE_DEVICES", str(local_rank)).split(",")[local_rank]) \
        if os.environ.get("CUDA_VISIBLE_DEVICES", "").replace(",", "").isdigit() else local_rank
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(gpu_index) as clk:
        elapsed = time_steps(torch, lbm, g, stream, args.steps)
    torch.cuda.synchronize()
    elapsed = reduce_max(elapsed, dist, "cuda")
    if dist:
        dist.barrier()
    nodes = n * n
    value = job_value(world, nodes, args.steps, elapsed)
    per_launch = elapsed / args.steps
    bpn = lbm.BYTES_PER_NODE_UPDATE[prec]
    hbm, peak_kind = peaks()
    achieved = nodes * bpn / per_launch / 1e9

    # e2e through the C ABI with host buffers: H2D of the fields from pinned
    # memory, `steps` steps, D2H of the moments, all inside the timed region;
    # median of args.e2e_reps repetitions (the handle's staging is allocated
    # at create, so no repetition allocates)
    pinned = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in fields]
    out = [torch.empty((n, n), dtype=torch.float64).pin_memory() for _ in range(4)]
    e2e_steps = args.steps
    e2e_times = []
    for _ in range(max(1, args.e2e_reps)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        lbm.lbm_init(g.h, *[t.numpy() for t in pinned])
        g.step(e2e_steps)
        rc = lbm.load().lbm_moments(g.h, *[lbm._dp(t.numpy()) for t in out])
        if rc != 0:
            raise lbm.LbmError(rc, lbm.lbm_last_error(g.h))
        e2e_times.append(time.perf_counter() - t0)
    e2e_t = reduce_max(statistics.median(e2e_times), dist, "cuda")
    e2e_value = job_value(world, nodes, e2e_steps, e2e_t)
    io_bytes = 2 * 4 * nodes * 8  # four FP64 fields in, four out
    e2e_io_s = max(e2e_t - e2e_steps * per_launch, 1e-12)
    # the host link's own copy rate for the same bytes (pinned, one copy per
    # field each way, torch's copies): what the transfers of the e2e leg
    # could reach at best
    dev_tmp = [torch.empty((n, n), dtype=torch.float64, device="cuda") for _ in range(4)]
    link = []
    for _ in range(3):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for a, d in zip(pinned, dev_tmp):
            d.copy_(a, non_blocking=True)
        for d, o in zip(dev_tmp, out):
            o.copy_(d, non_blocking=True)
        torch.cuda.synchronize()
        link.append(time.perf_counter() - t0)
    link_gbs = io_bytes / statistics.median(link) / 1e9
    del dev_tmp

    variants = {}
    cavity = inputs.cavity(n=n, Ra=1e5, dT_over_T0=0.3, seed=3)[0]
    if args.variants and world == 1:
        for name, pv, opts in (("f64", lbm.LBM_P_FP64, {}), ("f16dev", lbm.LBM_P_FP32_FP16, {}),
                                ("bf16dev", lbm.LBM_P_FP32_BF16, {}),
                                ("mrt_f32", lbm.LBM_P_FP32,
                                 dict(collision=lbm.LBM_COLL_MRT, s_e=1.3, s_eps=1.1, s_q=1.6)),
                                # the same size as a walled cavity: halfway walls, and the
                                # walls of non-equilibrium extrapolation (second pass)
                                ("cavity_f32", lbm.LBM_P_FP32, dict(base=cavity)),
                                ("cavity_nee_f32", lbm.LBM_P_FP32, dict(base=cavity, wall_nee=15))):
            if pv == prec and not opts:
                continue
            g.close()
            opts = dict(opts)
            pp = dict(opts.pop("base", p), precision=pv, **opts)
            gv = lbm.Lbm(pp, stream=stream.cuda_stream)
            with torch.cuda.stream(stream):
                lbm.lbm_init_device(gv.h, *[t.data_ptr() for t in dev_fields])
            ksteps = max(3, args.steps // (16 if pv == lbm.LBM_P_FP64 else 2))
            gv.step(args.warmup)
            gv.sync()
            tv = time_steps(torch, lbm, gv, stream, ksteps)
            gl = nodes * ksteps / tv / 1e9
            variants[name] = {"glups": gl, "bytes_per_node_update": lbm.BYTES_PER_NODE_UPDATE[pv],
                              "achieved_gbs": gl * lbm.BYTES_PER_NODE_UPDATE[pv],
                              "hbm_frac": gl * lbm.BYTES_PER_NODE_UPDATE[pv] / hbm,
                              "steps": ksteps}
            gv.close()
    else:
        g.close()
    if args.variants and world == 1 and args.n3d > 0:
        # the 3-D (D3Q19) extension: periodic n3d^3 box of the same recipe,
        # 38 populations per node (304 B per node update in FP32, 608 in FP64)
        from paper_1109_6672_gb300 import lbm3d

        p3, f3 = inputs.periodic_box3d(n=args.n3d)
        d3 = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in f3]
        for name, pv in (("d3q19_f32", lbm.LBM_P_FP32), ("d3q19_f64", lbm.LBM_P_FP64)):
            g3 = lbm3d.Lbm3d(dict(p3, precision=pv), stream=stream.cuda_stream)
            with torch.cuda.stream(stream):
                g3.init_device(*[t.data_ptr() for t in d3])
            g3.step(args.warmup)
            g3.sync()
            k3 = max(3, args.steps // (16 if pv == lbm.LBM_P_FP64 else 4))
            t3 = time_steps(torch, lbm, g3, stream, k3)
            g3.close()
            gl = args.n3d ** 3 * k3 / t3 / 1e9
            bpn3 = lbm3d.BYTES_PER_NODE_UPDATE_3D[pv]
            variants[name] = {"glups": gl, "bytes_per_node_update": bpn3,
                              "achieved_gbs": gl * bpn3, "hbm_frac": gl * bpn3 / hbm, "steps": k3,
                              "workload": f"periodic box {args.n3d}^3, D3Q19, total energy, "
                                          "correction on"}
        del d3

    extra = {}
    if rank == 0 and world == 1 and args.batch:
        extra = batch_and_serving(torch, args)
    elif world > 1 and args.batch:
        extra = sharded_batch(torch, args, rank, world, dist)
    if rank == 0 and world == 1 and args.config3_steps > 0:
        extra["large_dT_cavity"] = large_dT_study(torch, args)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cores = cpu_cores()
        side = args.ref_side
        gl, dt = oracle_glups(side, args.ref_steps, cores)
        gl1, dt1 = oracle_glups(256, 60, 1)
        cpu = {"value": gl, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"{side}x{side} periodic box of the same workload, {args.ref_steps} steps "
                         f"({dt:.1f} s), FP64, OpenMP over rows",
               "single_thread": {"value": gl1, "unit": UNIT, "cores": 1,
                                 "sample": f"256x256 periodic box, 60 steps ({dt1:.1f} s), FP64"}}

    traffic = None
    if n == 4096 and args.threads in (0, 1) and args.rows == 0 and args.collision == "bgk":
        traffic = MEASURED_TRAFFIC.get((kernel_hash(), args.precision))
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * elapsed / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {"f64": "f64", "f32": "f32", "f16": "f32 (f16 storage)",
                      "bf16": "f32 (bf16 storage)"}[args.precision],
            "data": "synthetic",
            "config": {"workload": f"periodic box {n}x{n}, coupled f+h D2Q9 "
                                   f"{args.collision.upper()}, total energy, "
                                   f"correction on, {lbm.PRECISION_NAMES[prec]} storage",
                       "nx": n, "ny": n, "precision": args.precision,
                       "bytes_per_node_update": bpn,
                       "l2": "state 2x18 populations per node >> 129 MB L2; no flush",
                       "replicas": world},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                         "frac": achieved / hbm, "traffic": traffic, "peak_kind": peak_kind,
                         "kernel": "step_pr_kernel", "algorithmic_bytes_per_launch": nodes * bpn,
                         "traffic_note": "DRAM read+write bytes per launch from ncu at 2048^2, "
                                         "scaled x4 (node count); null if the kernel changed"},
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": UNIT,
                    "h2d_bytes_per_step": int(4 * nodes * 8 / e2e_steps),
                    "d2h_bytes_per_step": int(4 * nodes * 8 / e2e_steps),
                    "reps": len(e2e_times), "seconds_median": e2e_t,
                    "seconds_all": e2e_times,
                    "transfer_gbs": io_bytes / e2e_io_s / 1e9,
                    "link_copy_gbs": link_gbs,
                    "transfer_note": "host<->device bytes (fields in, moments out) / (e2e time "
                                     "- steps x device step time); includes the init and "
                                     "export kernels"},
            "gpu_launches": args.steps,
            "clocks": clk.summary(),
            "variants": variants,
        }
        line.update(extra)
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="f32", choices=["f64", "f32", "f16", "bf16"])
    ap.add_argument("--collision", default="bgk", choices=["bgk", "mrt"],
                    help="collision of the timed box (MRT: Eqs. 40-47, rates 1.3 / 1.1 / 1.6)")
    ap.add_argument("--n", type=int, default=4096)
    ap.add_argument("--threads", type=int, default=0)
    ap.add_argument("--rows", type=int, default=0)
    ap.add_argument("--ref-side", type=int, default=1024)
    ap.add_argument("--ref-steps", type=int, default=800)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-variants", dest="variants", action="store_false")
    ap.add_argument("--no-batch", dest="batch", action="store_false")
    ap.add_argument("--batch-grids", type=int, default=256)
    ap.add_argument("--batch-sim-steps", type=int, default=10000,
                    help="steps every grid of the 256-cavity batch runs to completion")
    ap.add_argument("--batch-fp64-steps", type=int, default=500,
                    help="steps per grid of the FP64 one-grid-per-launch comparison")
    ap.add_argument("--config5", default="",
                    help="also serve the configured 500-request trace (sides to 2048, steps "
                         "to 1e5, load 0.7: about 20 minutes per storage) in these storages, "
                         "comma-separated: bf16, f32")
    ap.add_argument("--serve-pool-gb", type=int, default=24)
    ap.add_argument("--config5-sample", type=int, default=40,
                    help="requests of the configured serving stream served by default (about "
                         "90 s at 40; 0 skips it)")
    ap.add_argument("--batch-err-grids", type=int, default=4)
    ap.add_argument("--serve-requests", type=int, default=40)
    ap.add_argument("--e2e-reps", type=int, default=3)
    ap.add_argument("--n3d", type=int, default=256,
                    help="side of the D3Q19 box variant (0: skip it)")
    ap.add_argument("--config3-steps", type=int, default=200000,
                    help="steps of the large-dT cavity precision study (1024^2, about three "
                         "minutes at 200 000; 0 skips it)")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
