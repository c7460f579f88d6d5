"""The CUDA path on the paper's cavity benchmark (Table II, fixture
tests/golden/table2_cavity.txt) at Ra = 1e4 and 1e5, where the CPU oracle is
too slow to reach steady state.  Pr = 0.71, internal-energy model, gravity
force, stratification g H / R T0 = 0.05 dT/T0 (near the Boussinesq regime the
table compares).  dT/T0 = 0.2 rather than the paper's 0.1: at a fixed Ra and
grid the viscosity grows with dT, and at dT/T0 = 0.1 these grids need
tau_f < 0.05, where the BGK scheme diverged (the paper used MRT).  BGK with
bounce-back walls on coarser grids than the paper's, so the agreement is to
a few percent (measured: within 1 %)."""
import os

import numpy as np
import pytest

from paper_1109_6672_gb300 import inputs
from paper_1109_6672_gb300 import lbm

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table2_cavity.txt")


def table2():
    rows = {}
    for line in open(GOLDEN):
        if line.strip() and not line.startswith("#"):
            ra, *vals = line.split()
            rows[float(ra)] = dict(zip(["Nu", "u_max", "y_max", "v_max", "x_max"], map(float, vals)))
    return rows


def steady_cavity(n, Ra, precision, chunk, max_steps, dT=0.2):
    p, f = inputs.cavity(n=n, Ra=Ra, dT_over_T0=dT, strat=0.05 * dT, nu_min=0.0, seed=1,
                         precision=precision)
    g = lbm.Lbm(p).init(*f)
    Th, Tl = p["T_wall"][0], p["T_wall"][1]
    chi = p["tau_h"] * inputs.RT0
    prev, steps = None, 0
    while steps < max_steps:
        g.step(chunk)
        steps += chunk
        rho, ux, uy, T = g.moments()
        Nu = float(((9 * T[:, n - 1] - T[:, n - 2] - 8 * Tl) / 3).mean() * n / (Th - Tl))
        if prev is not None and abs(Nu - prev) < 1e-5 * Nu:
            break
        prev = Nu
    g.close()
    mid = n // 2
    u_line, v_line = ux[:, mid], uy[mid, :]
    return dict(Nu=Nu, u_max=u_line.max() * n / chi, y_max=(u_line.argmax() + 0.5) / n,
                v_max=v_line.max() * n / chi, x_max=(v_line.argmax() + 0.5) / n, steps=steps)


@pytest.mark.parametrize("Ra,n,precision,chunk,max_steps,tol",
                         [(1e4, 97, lbm.LBM_P_FP32, 50000, 1500000, 0.02),
                          (1e5, 257, lbm.LBM_P_FP32, 100000, 3000000, 0.02)])
def test_cavity_matches_table2(Ra, n, precision, chunk, max_steps, tol):
    ref = table2()[Ra]
    got = steady_cavity(n, Ra, precision, chunk, max_steps)
    assert got["steps"] < max_steps, "not converged"
    for k in ("Nu", "u_max", "v_max"):
        assert got[k] == pytest.approx(ref[k], rel=tol), (k, got)
    assert abs(got["y_max"] - ref["y_max"]) <= 2 / n, got
    assert abs(got["x_max"] - ref["x_max"]) <= 2 / n, got
