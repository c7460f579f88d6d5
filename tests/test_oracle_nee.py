"""Oracle pins for walls of non-equilibrium extrapolation (the paper's wall
method, ref. [45], Secs. IV.A and IV.C), with the wall on the ghost node one
spacing outside the boundary node (so H = n + 1 between two such walls):

* the independent NumPy restatement (walls on every side, mixed with halfway
  walls in both orders, along a periodic axis, MRT) to 1e-13;
* pure conduction between isothermal walls: T exactly linear;
* thermal Couette flow: u linear, the viscous-heating rise on the closed form;
* the large-temperature-difference cavity without gravity stays at rest
  (the halfway walls drive a spurious flow from the corners there);
* the paper's mu ~ T Couette of Table I (10 x 60 nodes with the wall nodes,
  adiabatic lower wall) within the paper's own error of Eq. 52a.
"""
import math
import os

import numpy as np
import pytest

import brute_lbm as B
from oracle import oracle as O
from paper_1109_6672_gb300 import inputs

RT0 = 1.0 / 3.0
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table1_couette.txt")

CASES = {
    "cavity_all": dict(bc=[1, 1, 2, 2], wall_nee=15, energy_model=1, g=1e-3, b=5.0,
                       T_wall=[1.1, 0.9, 1, 1]),
    "couette_y": dict(bc=[0, 0, 2, 1], wall_nee=12, u_wall=[[0, 0], [0, 0], [0, 0], [0.05, 0]],
                      T_wall=[1, 1, 1, 1.05]),
    "x_nee_y_halfway": dict(bc=[1, 2, 1, 2], wall_nee=3,
                            u_wall=[[0, 0.02], [0, 0], [0.01, 0], [0, 0]], T_wall=[1.1, 1, 0.95, 1]),
    "x_halfway_y_nee": dict(bc=[1, 2, 1, 2], wall_nee=12,
                            u_wall=[[0, 0.02], [0, 0], [0.01, 0], [0, 0]], T_wall=[1.1, 1, 0.95, 1]),
    "x_nee_y_periodic": dict(bc=[1, 1, 0, 0], wall_nee=3, T_wall=[1.1, 0.9, 1, 1]),
    "mrt_all": dict(bc=[1, 2, 2, 1], wall_nee=15, collision=1, s_e=1.3, s_q=1.6,
                    T_wall=[1.1, 1, 1, 0.95]),
    "adiabatic_moving": dict(bc=[0, 0, 2, 2], wall_nee=12, u_wall=[[0, 0], [0, 0], [0.03, 0],
                                                                     [-0.04, 0]]),
}


def nee_case(name, nx=7, ny=6, seed=5):
    rng = np.random.default_rng(seed)
    p = dict(nx=nx, ny=ny, tau_f=0.4, tau_h=0.5, R=1 / 3, T0=1.0, b=3.0, energy_model=0,
             correction=1, z_full=1, collision=0, g=0.0, u_wall=[[0, 0]] * 4, T_wall=[1, 1, 1, 1])
    p.update(CASES[name])
    f = (1 + 0.01 * rng.standard_normal((ny, nx)), 0.01 * rng.standard_normal((ny, nx)),
         0.01 * rng.standard_normal((ny, nx)), 1 + 0.02 * rng.standard_normal((ny, nx)))
    return p, f


@pytest.mark.parametrize("name", sorted(CASES))
def test_nee_matches_brute_force(name):
    p, f = nee_case(name)
    o = O.Oracle(p).init(*f).step(40)
    b = B.Brute(p).init(*f).step(40)
    np.testing.assert_allclose(o.pops(), b.pops(), rtol=0, atol=1e-13)


@pytest.mark.parametrize("em", [O.E_TOTAL, O.E_INTERNAL])
def test_nee_conduction_is_exact(em):
    ny = 15
    p, f = inputs.couette(ny=ny)
    p.update(wall_nee=12, u_wall=[[0, 0]] * 4, T_wall=[1, 1, 1.05, 0.95], energy_model=em,
             b=3.0 if em == O.E_TOTAL else 5.0)
    o = O.Oracle(p).init(*f).step(60000, threads=4)
    rho, ux, uy, T = o.moments()
    y = np.arange(ny) + 1.0  # walls on the nodes y = -1 and y = ny
    np.testing.assert_allclose(T[:, 0], 1.05 - 0.1 * y / (ny + 1), rtol=0, atol=1e-12)
    assert np.abs(uy).max() < 1e-13


def test_nee_couette_viscous_heating():
    ny = 31
    p, f = inputs.couette(ny=ny, U=0.1)
    p["wall_nee"] = 12
    o = O.Oracle(p).init(*f).step(60000, threads=4)
    rho, ux, uy, T = o.moments()
    eta = (np.arange(ny) + 1.0) / (ny + 1)
    U = p["u_wall"][3][0]
    assert np.abs(ux[:, 0] - U * eta).max() < 1e-5 * U
    Pr = p["tau_f"] / p["tau_h"]
    rise = Pr * U ** 2 / ((p["b"] + 2) * RT0) * eta * (1 - eta)
    assert np.abs((T[:, 0] - 1) - rise).max() < 0.01 * rise.max()


@pytest.mark.parametrize("collision", [O.BGK, O.MRT], ids=["bgk", "mrt"])
def test_nee_couette_adiabatic_moving_wall(collision):
    """Bottom wall at rest and T0, top wall moving and adiabatic, both of
    non-equilibrium extrapolation (walls on the ghost nodes, eta = (y + 1) /
    (ny + 1)): no heat crosses the moving wall, its viscous work does, and the
    heating is theta - 1 = Pr U^2 / ((b + 2) R T0) (2 eta - eta^2), exact to
    the steady state's convergence (measured 6e-12 at ny = 8)."""
    H, U, nu, Pr, b = 8, 0.2, 0.2, 1.0, 5.0
    tau_f = nu / RT0
    p = inputs.base_params(2, H, tau_f=tau_f, tau_h=tau_f / Pr, b=b, collision=collision,
                           bc=[0, 0, inputs.WALL_ISOTHERMAL, inputs.WALL_ADIABATIC],
                           u_wall=[[0, 0], [0, 0], [0, 0], [U, 0]], wall_nee=12)
    rho, ux, uy, T = O.Oracle(p).init(*inputs.uniform_fields(2, H, seed=0)).step(
        3000, threads=4).moments()
    eta = (np.arange(H) + 1.0) / (H + 1)
    assert np.abs(ux[:, 0] - U * eta).max() < 1e-10 * U
    rise = Pr * U * U / ((b + 2) * RT0) * (2 * eta - eta * eta)
    assert np.abs((T[:, 0] - 1) - rise).max() < 1e-8 * rise.max()


def test_nee_large_dt_cavity_has_no_spurious_flow():
    n = 20
    flows = {}
    for nee in (0, 15):
        p, f = inputs.cavity_large_dT(Ra=1e3, n=n)
        p.update(g=0.0, wall_nee=nee)
        m = O.Oracle(p).init(*f).step(60000, threads=4).moments()
        flows[nee] = max(np.abs(m[1]).max(), np.abs(m[2]).max())
    assert flows[15] < 1e-12
    assert flows[0] > 1e-3  # the halfway walls' creep along the adiabatic walls


def test_nee_table1_couette_pr1():
    """The paper's set-up with its own wall method: 60 nodes across including
    the two wall nodes (58 fluid rows), adiabatic lower wall at rest, upper
    wall at T0 moving at U, mu = mu0 T/T0, mu0 = 0.25, b = 3, MRT rates 1.5,
    correction omitted; Pr = 1, Ma = 0.35.  The lower-wall temperature (the
    wall node's, zero slope there) within Table I's E_r."""
    rows = [dict(zip(["Pr", "Ma", "T", "Ta", "Er"], map(float, l.split())))
            for l in open(GOLDEN) if l.strip() and not l.startswith("#")]
    row = [r for r in rows if r["Pr"] == 1 and r["Ma"] == 0.35][0]
    U = 0.35 * math.sqrt(5.0 / 3.0 * RT0)
    tau_f = 0.25 / RT0
    p = inputs.base_params(10, 58, tau_f=tau_f, tau_h=tau_f, b=3.0, correction=0,
                           bc=[inputs.PERIODIC, inputs.PERIODIC, inputs.WALL_ADIABATIC,
                               inputs.WALL_ISOTHERMAL],
                           u_wall=[[0, 0], [0, 0], [0, 0], [U, 0]], mu_law=O.MU_POWER, mu_n=1.0,
                           collision=O.MRT, s_e=1.5, s_eps=1.5, s_q=1.5, wall_nee=12)
    o = O.Oracle(p).init(*inputs.uniform_fields(10, 58, seed=0))
    o.step(100000, threads=os.cpu_count() or 1)
    T = o.moments()[3][:, 0]
    Tw = (4 * T[0] - T[1]) / 3
    Er = abs((Tw - 1) - (row["Ta"] - 1)) / (row["Ta"] - 1)
    assert Er <= row["Er"] / 100
