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


# ---- grid convergence ---------------------------------------------------------
#
# The same cavity on three grids, H = 24, 48, 96, in diffusive scaling: the
# lattice viscosity is held (tau_f = 0.1) and g follows from Ra, so the Mach
# number falls as 1/H and the hydrostatic stratification as 1/H^2 while Ra,
# Pr and dT/T0 stay fixed.  Every error of the scheme (lattice truncation, the
# halfway walls, compressibility, stratification) is then of second order in
# the spacing, and Nu, u_max and v_max must converge at Richardson order
# about 2.  Each grid starts from the previous grid's steady fields,
# interpolated, and runs until Nu changes by less than 1e-6 over 1000 steps.

def _convergence_params(n, Ra=1e3, Pr=0.71, dT=0.1, nu=0.1 / 3):
    chi = nu / Pr
    g = Ra * nu * chi / (dT * n ** 3)  # Eqs. 57-58 with beta = 1 / T0
    tau_f = nu / inputs.RT0
    p = inputs.base_params(n, n, tau_f=tau_f, tau_h=tau_f / Pr, b=5.0, g=g,
                           energy_model=inputs.E_INTERNAL,
                           bc=[inputs.WALL_ISOTHERMAL, inputs.WALL_ISOTHERMAL,
                               inputs.WALL_ADIABATIC, inputs.WALL_ADIABATIC],
                           T_wall=[1 + dT / 2, 1 - dT / 2, 1.0, 1.0])
    return p, chi


def _refine(a):
    """Cell-centred field of side n to side 2n by linear interpolation (edges
    held): only a starting guess."""
    n = a.shape[0]
    c = np.arange(2 * n) / 2 - 0.25
    x = np.arange(n)
    rows = np.array([np.interp(c, x, r) for r in a])
    return np.array([np.interp(c, x, col) for col in rows.T]).T


def _peak(a):
    """Maximum of a sampled profile through the parabola on its largest sample
    and the two neighbours."""
    k = int(np.argmax(a))
    y0, y1, y2 = a[k - 1], a[k], a[k + 1]
    d = 0.5 * (y0 - y2) / (y0 - 2 * y1 + y2)
    return y1 - 0.25 * (y0 - y2) * d


def _steady(n, start, tol=1e-6, chunk=1000, max_steps=400000):
    p, chi = _convergence_params(n)
    fields = inputs.uniform_fields(n, n, seed=1, u_amp=0.0) if start is None else \
        tuple(_refine(a) for a in start)
    o = orc.Oracle(p).init(*fields)
    Th, Tl = p["T_wall"][0], p["T_wall"][1]
    prev, steps = None, 0
    while steps < max_steps:
        o.step(chunk, threads=os.cpu_count() or 1)
        steps += chunk
        mom = o.moments()
        T = mom[3]
        Nu = float(((9 * T[:, n - 1] - T[:, n - 2] - 8 * Tl) / 3).mean() * n / (Th - Tl))
        if prev is not None and abs(Nu - prev) < tol:
            break
        prev = Nu
    assert steps < max_steps, f"{n}^2 cavity did not reach steady state"
    rho, ux, uy, T = mom
    m = n // 2  # the midplanes lie between nodes m - 1 and m
    u_mid = 0.5 * (ux[:, m - 1] + ux[:, m])
    v_mid = 0.5 * (uy[m - 1, :] + uy[m, :])
    return dict(Nu=Nu, u_max=_peak(u_mid) * n / chi, v_max=_peak(v_mid) * n / chi), mom


def test_cavity_grid_convergence_second_order():
    res, mom = [], None
    for n in (24, 48, 96):
        r, mom = _steady(n, mom)
        res.append(r)
    ref = table2()[1e3]
    for k in ("Nu", "u_max", "v_max"):
        a, b, c = (r[k] for r in res)
        order = np.log2(abs(a - b) / abs(b - c))
        assert 1.5 <= order <= 2.5, (k, order, res)
        # the Richardson extrapolation lands on the paper's Table II
        assert c + (c - b) / 3 == pytest.approx(ref[k], rel=0.01), (k, res)
