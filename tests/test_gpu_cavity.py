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


# ---- grid convergence on the CUDA path ----------------------------------------
#
# Ra = 1e4 on H = 64, 128, 256 in diffusive scaling (tau_f = 0.06 held, g
# from Ra, dT/T0 = 0.2): Mach number ~ 1/H, stratification ~ 1/H^2, so every
# error of the scheme is of second order in the spacing.  FP64 storage: the
# rounding drift of FP32 storage over the millions of steps these runs take
# (a Ra = 1e5, 128/256/512 FP32 attempt needed 5.9 million steps at 512^2)
# shows in Nu at the level of the differences between the finer grids.
# Each grid starts from the previous grid's steady fields, interpolated.

def _conv_params(n, Ra=1e4, Pr=0.71, dT=0.2, tau_f=0.06, precision=lbm.LBM_P_FP64):
    nu = tau_f * inputs.RT0
    chi = nu / Pr
    g = Ra * nu * chi / (dT * n ** 3)
    p = inputs.base_params(n, n, tau_f=tau_f, tau_h=tau_f / Pr, b=5.0, g=g,
                           energy_model=inputs.E_INTERNAL, precision=precision,
                           bc=[inputs.WALL_ISOTHERMAL, inputs.WALL_ISOTHERMAL,
                               inputs.WALL_ADIABATIC, inputs.WALL_ADIABATIC],
                           T_wall=[1 + dT / 2, 1 - dT / 2, 1.0, 1.0])
    return p, chi


def _refine(a):
    n = a.shape[0]
    c = np.arange(2 * n) / 2 - 0.25
    x = np.arange(n)
    rows = np.array([np.interp(c, x, r) for r in a])
    return np.array([np.interp(c, x, col) for col in rows.T]).T


def _peak(a):
    k = int(np.argmax(a))
    y0, y1, y2 = a[k - 1], a[k], a[k + 1]
    d = 0.5 * (y0 - y2) / (y0 - 2 * y1 + y2)
    return y1 - 0.25 * (y0 - y2) * d


def _steady_gpu(n, start, chunk, max_steps, tol=1e-7):
    p, chi = _conv_params(n)
    fields = inputs.uniform_fields(n, n, seed=1, u_amp=1e-4) if start is None else \
        tuple(_refine(a) for a in start)
    g = lbm.Lbm(p).init(*fields)
    Th, Tl = p["T_wall"][0], p["T_wall"][1]
    prev, steps = None, 0
    while steps < max_steps:
        g.step(chunk)
        steps += chunk
        mom = g.moments()
        T = mom[3]
        Nu = float(((9 * T[:, n - 1] - T[:, n - 2] - 8 * Tl) / 3).mean() * n / (Th - Tl))
        if prev is not None and abs(Nu - prev) < tol * Nu:
            break
        prev = Nu
    g.close()
    rho, ux, uy, T = mom
    m = n // 2
    u_mid = 0.5 * (ux[:, m - 1] + ux[:, m])
    v_mid = 0.5 * (uy[m - 1, :] + uy[m, :])
    return dict(Nu=Nu, u_max=_peak(u_mid) * n / chi, v_max=_peak(v_mid) * n / chi,
                steps=steps), mom


def test_cavity_grid_convergence_gpu():
    res, mom = [], None
    for n, chunk, cap in ((64, 10000, 1000000), (128, 20000, 2000000), (256, 50000, 4000000)):
        r, mom = _steady_gpu(n, mom, chunk, cap)
        assert r["steps"] < cap, f"{n}^2 not converged: {r}"
        res.append(r)
    print("grid convergence (64, 128, 256):", res)
    ref = table2()[1e4]
    for k in ("Nu", "u_max", "v_max"):
        a, b, c = (r[k] for r in res)
        order = np.log2(abs(a - b) / abs(b - c))
        print(k, "order", order, "extrapolated", c + (c - b) / 3, "Table II", ref[k])
        assert 1.5 <= order <= 2.5, (k, order, res)
        assert c + (c - b) / 3 == pytest.approx(ref[k], rel=0.02), (k, res)


def test_rayleigh_benard_onset_gpu():
    """The Rayleigh-Benard onset on the CUDA path (FP64) at a fourth of the
    oracle test's stratification (H = 64, g H / (R T0) = 0.014): growth
    rates at 0.95, 1.0 and 1.05 Ra_c interpolate to Ra_c = 1707.76 within
    1 % (the oracle pin at H = 32 brackets it)."""
    from test_oracle_convection import RA_C, growth_rate, rb_case

    H = 64
    rates = {}
    for ratio in (0.95, 1.0, 1.05):
        p, f, chi = rb_case(ratio, H=H)
        g = lbm.Lbm(p).init(*f)
        rates[ratio] = growth_rate(g, H, chi, int(2.5 * H * H / chi))
        g.close()
    r = sorted(rates)
    slope, icpt = np.polyfit(r, [rates[k] for k in r], 1)
    assert slope > 0, rates
    assert abs(-icpt / slope - 1.0) < 0.01, (rates, -icpt / slope * RA_C)
