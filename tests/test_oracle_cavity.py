"""The oracle against the paper's printed cavity results (Table II, fixture
tests/golden/table2_cavity.txt): natural convection at Ra = 1e3, Pr = 0.71,
dT/T0 = 0.1 (the paper's 315 K / 285 K), internal-energy model with the
gravity force a = (0, -rho g), run to steady state.  The paper used the MRT
scheme with non-equilibrium-extrapolation walls on 100^2 nodes; the oracle
runs BGK with the bounce-back / ghost-equilibrium walls on 49^2, so the
agreement is to about a percent.  The hydrostatic stratification g H / R T0
is held at 0.05 dT/T0 so that the flow is in the near-Boussinesq regime the
paper compares against."""
import os

import numpy as np
import pytest

from oracle import oracle as orc
from paper_1109_6672_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table2_cavity.txt")


def table2():
    rows = {}
    for line in open(GOLDEN):
        if line.strip() and not line.startswith("#"):
            ra, *vals = line.split()
            rows[float(ra)] = dict(zip(["Nu", "u_max", "y_max", "v_max", "x_max"], map(float, vals)))
    return rows


def cavity_results(n, Ra, dT=0.1, chunk=20000, max_steps=240000):
    p, f = inputs.cavity(n=n, Ra=Ra, dT_over_T0=dT, strat=0.05 * dT, nu_min=0.0, seed=1)
    o = orc.Oracle(p).init(*f)
    Th, Tl = p["T_wall"][0], p["T_wall"][1]
    chi = p["tau_h"] * inputs.RT0  # thermal diffusivity tau_h R T0
    nu_prev, steps = None, 0
    while steps < max_steps:
        o.step(chunk, threads=os.cpu_count() or 1)
        steps += chunk
        rho, ux, uy, T = o.moments()
        # cold wall halfway beyond x = n - 1: second-order one-sided gradient
        # through the wall value and the nodes at distances 1/2 and 3/2
        dTds = (9 * T[:, n - 1] - T[:, n - 2] - 8 * Tl) / 3
        Nu = float(dTds.mean() * n / (Th - Tl))
        if nu_prev is not None and abs(Nu - nu_prev) < 1e-5:
            break
        nu_prev = Nu
    mid = n // 2  # node n // 2 sits on the midplane for odd n
    u_line, v_line = ux[:, mid], uy[mid, :]
    return dict(Nu=Nu, u_max=u_line.max() * n / chi, y_max=(u_line.argmax() + 0.5) / n,
                v_max=v_line.max() * n / chi, x_max=(v_line.argmax() + 0.5) / n, steps=steps)


def test_cavity_ra1e3_matches_table2():
    ref = table2()[1e3]
    got = cavity_results(49, 1e3)
    assert got["steps"] < 240000, "not converged"
    assert got["Nu"] == pytest.approx(ref["Nu"], rel=0.01)
    assert got["u_max"] == pytest.approx(ref["u_max"], rel=0.01)
    assert got["v_max"] == pytest.approx(ref["v_max"], rel=0.01)
    # locations within one node spacing of the 49^2 grid
    assert abs(got["y_max"] - ref["y_max"]) <= 1 / 49
    assert abs(got["x_max"] - ref["x_max"]) <= 1 / 49
