"""Parity at the benchmark's full sizes and launch configurations, on sampled
outputs the oracle computes window by window.

The state of a node after k steps depends only on the initial values within
2k nodes of it (per step: the pull reaches 1 node, the correction's
neighbour moments 1 more).  So the oracle, run for k steps on a window of
the initial fields whose cut edges are at least 2k + 1 nodes away (periodic
wrap or walls at the cuts), reproduces the window's centre exactly; real walls
and corners of the grid stay in the window where it touches them."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1109_6672_gb300 import inputs
from paper_1109_6672_gb300 import lbm

pytestmark = pytest.mark.gpu

K = 4           # steps
W = 32          # window side
M = 2 * K + 1   # margin to a cut edge
P, ADI = inputs.PERIODIC, inputs.WALL_ADIABATIC


def window_fields(fields, x0, y0, nx, ny):
    """fields[.][y0 : y0 + W, x0 : x0 + W] with periodic wrap."""
    ys = np.arange(y0, y0 + W) % ny
    xs = np.arange(x0, x0 + W) % nx
    return [np.ascontiguousarray(a[np.ix_(ys, xs)]) for a in fields]


def field_errors(gpu, ref):
    """max |gpu - ref| per moment, normalised by the oracle's scale of that
    moment (rho - 1, |u|, T - T0 spread)."""
    rho_g, ux_g, uy_g, T_g = gpu
    rho_o, ux_o, uy_o, T_o = ref
    umax = max(np.abs(ux_o).max(), np.abs(uy_o).max(), 1e-300)
    return {
        "rho": np.abs(rho_g - rho_o).max() / np.abs(rho_o).max(),
        "u": max(np.abs(ux_g - ux_o).max(), np.abs(uy_g - uy_o).max()) / umax,
        "T": np.abs(T_g - T_o).max() / np.abs(T_o).max(),
    }


BOX_TOL = {lbm.LBM_P_FP64: dict(rho=1e-12, u=1e-12, T=1e-12),
           lbm.LBM_P_FP32: dict(rho=2e-6, u=2e-4, T=2e-6),
           lbm.LBM_P_FP32_BF16: dict(rho=2e-3, u=5e-1, T=2e-3)}


@pytest.mark.parametrize("precision", sorted(BOX_TOL))
def test_box_4096_default_launch_windows(precision):
    """The bench workload (4096^2 periodic box) in its default launch shape;
    16 windows, four of them across the periodic wrap."""
    n = 4096
    p, fields = inputs.periodic_box(n=n, precision=precision)
    g = lbm.Lbm(p).init(*fields).step(K)
    gpu = g.moments()
    g.close()
    rng = np.random.default_rng(11)
    corners = [(n - W // 2, n - W // 2), (n - 5, 100), (100, n - 7), (0, 0)]
    corners += [tuple(int(v) for v in rng.integers(0, n, 2)) for _ in range(12)]
    pw = dict(p, nx=W, ny=W, precision=lbm.LBM_P_FP64)
    for x0, y0 in corners:
        o = orc.Oracle(pw).init(*window_fields(fields, x0, y0, n, n)).step(K)
        ref = [a[M:W - M, M:W - M] for a in o.moments()]
        ys = np.arange(y0 + M, y0 + W - M) % n
        xs = np.arange(x0 + M, x0 + W - M) % n
        got = [a[np.ix_(ys, xs)] for a in gpu]
        err = field_errors(got, ref)
        for k, tol in BOX_TOL[precision].items():
            assert err[k] <= tol, (x0, y0, k, err[k])


def test_batch_of_256_cavities_autotuned_windows():
    """The batched workload (256 cavities, sides 64..512, BF16 storage) in the
    schedule the autotuner picks, as the bench runs it; windows at a hot-wall
    corner, a cold-wall corner and the interior of four grids."""
    prec = lbm.LBM_P_FP32_BF16
    grids = inputs.batch_cavities(count=256, seed=4, precision=prec)
    pool = sum(lbm.lbm_state_bytes(p) for p, _ in grids) + (64 << 20)
    b = lbm.Batch(prec, len(grids), pool)
    slots = [b.add(p, f, K) for p, f in grids]
    b.autotune(3)
    b.run(K)
    order = np.argsort([abs(p["T_wall"][0] - p["T_wall"][1]) for p, _ in grids])
    picks = [int(order[0]), int(order[85]), int(order[170]), int(order[-1])]
    for i in picks:
        p, fields = grids[i]
        s = p["nx"]
        gpu = b.moments(slots[i])
        for x0, y0 in ((0, 0), (s - W, s - W), (s // 2 - W // 2, s // 3)):
            # the grid's own walls where the window touches them, walls at the cuts
            bc = [p["bc"][0] if x0 == 0 else ADI, p["bc"][1] if x0 + W == s else ADI,
                  p["bc"][2] if y0 == 0 else ADI, p["bc"][3] if y0 + W == s else ADI]
            pw = dict(p, nx=W, ny=W, bc=bc, precision=lbm.LBM_P_FP64)
            win = [np.ascontiguousarray(a[y0:y0 + W, x0:x0 + W]) for a in fields]
            o = orc.Oracle(pw).init(*win).step(K)
            lo_x = 0 if x0 == 0 else M
            hi_x = W if x0 + W == s else W - M
            lo_y = 0 if y0 == 0 else M
            hi_y = W if y0 + W == s else W - M
            ref = [a[lo_y:hi_y, lo_x:hi_x] for a in o.moments()]
            got = [a[y0 + lo_y:y0 + hi_y, x0 + lo_x:x0 + hi_x] for a in gpu]
            err = field_errors(got, ref)
            # BF16 deviations: a few storage quanta of the deviation scale
            dT = abs(p["T_wall"][0] - p["T_wall"][1])
            assert err["rho"] <= 2e-3, (i, x0, y0, err)
            assert err["T"] <= 8 * 2.0 ** -8 * dT, (i, x0, y0, err)
    b.close()
