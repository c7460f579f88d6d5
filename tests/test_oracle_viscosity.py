"""Temperature-dependent viscosity (the premise of Eq. 52, Sutherland's law
Eq. 59): the oracle's per-node relaxation times against the shear-wave decay
they imply, and the thermal Couette flow with mu proportional to T and an
adiabatic lower wall against the analytical solution Eq. 52 and the paper's
Table I (fixture tests/golden/table1_couette.txt)."""
import math
import os

import numpy as np
import pytest

from oracle import oracle as orc
from paper_1109_6672_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table1_couette.txt")
RT0 = 1.0 / 3.0


def table1():
    rows = []
    for line in open(GOLDEN):
        if line.strip() and not line.startswith("#"):
            rows.append(dict(zip(["Pr", "Ma", "T", "Ta", "Er"], map(float, line.split()))))
    return rows


def test_fixture_matches_eq52a():
    """The analytical column is Eq. 52a at the lower wall (u_x = 0)."""
    for r in table1():
        assert 1 + r["Pr"] * (2.0 / 3.0) / 2 * r["Ma"] ** 2 == pytest.approx(r["Ta"], abs=1e-4)


@pytest.mark.parametrize("law,theta0", [(orc.MU_POWER, 1.2), (orc.MU_SUTHERLAND, 0.8)])
def test_shear_decay_follows_the_viscosity_law(law, theta0):
    """mu(T) sets tau_f = mu / (rho R T): a shear wave at uniform theta0 decays
    at nu k^2 with nu = mu(theta0) / rho, not at tau_f R T."""
    L, A = 128, 1e-3
    p = inputs.base_params(4, L, tau_f=0.3, tau_h=0.3 / 0.71, b=5.0, mu_law=law, mu_n=0.0,
                           energy_model=inputs.E_INTERNAL,
                           mu_S=0.1)
    k = 2 * math.pi / L
    y = np.arange(L)[:, None] * np.ones((1, 4))
    o = orc.Oracle(p).init(np.ones((L, 4)), A * np.sin(k * y), np.zeros((L, 4)),
                           np.full((L, 4), theta0))
    s = np.sin(k * np.arange(L))
    o.step(200)
    a1 = float(o.moments()[1][:, 0] @ s)
    o.step(2000)
    a2 = float(o.moments()[1][:, 0] @ s)
    rate = math.log(a1 / a2) / 2000
    mu0 = 0.3 * RT0
    mu = mu0 if law == orc.MU_POWER else mu0 * theta0 ** 1.5 * 1.1 / (theta0 + 0.1)
    assert rate == pytest.approx(mu * k * k, rel=0.01)
    assert abs(rate / (0.3 * RT0 * theta0 * k * k) - 1) > 0.05  # not the constant-tau value


def couette_mu(Pr, Ma, collision=orc.MRT, chunk=25000, max_steps=400000):
    """The paper's set-up: 10 x 60, adiabatic lower wall at rest, upper wall at
    T0 moving at U, mu = mu0 T/T0 with mu0 = 0.25 (tau_f = mu0 / (R T0) at T0),
    b = 3, correction omitted, MRT with s_e = s_eps = s_q = 1.5."""
    b, gamma = 3.0, 5.0 / 3.0
    U = Ma * math.sqrt(gamma * RT0)
    tau_f = 0.25 / RT0
    p = inputs.base_params(10, 60, tau_f=tau_f, tau_h=tau_f / Pr, b=b, correction=0,
                           bc=[inputs.PERIODIC, inputs.PERIODIC, inputs.WALL_ADIABATIC,
                               inputs.WALL_ISOTHERMAL],
                           u_wall=[[0, 0], [0, 0], [0, 0], [U, 0]], mu_law=orc.MU_POWER, mu_n=1.0,
                           collision=collision, s_e=1.5, s_eps=1.5, s_q=1.5)
    o = orc.Oracle(p).init(*inputs.uniform_fields(10, 60, seed=0))
    prev, steps = None, 0
    while steps < max_steps:
        o.step(chunk, threads=os.cpu_count() or 1)
        steps += chunk
        rho, ux, uy, T = o.moments()
        Tw = T[0, 0] - (T[1, 0] - T[0, 0]) / 8  # zero-gradient extrapolation to y = -1/2
        if prev is not None and abs(Tw - prev) < 1e-9:
            break
        prev = Tw
    return Tw, ux[:, 0] / U, T[:, 0], steps


def test_couette_mu_proportional_to_T_matches_eq52_and_table1():
    """Pr = 1, Ma = 0.35: the lower-wall temperature within the paper's own
    error of Eq. 52a (E_r 0.74 % in Table I), and the whole u(y), T(y)
    profile on Eqs. 52a/52b."""
    row = [r for r in table1() if r["Pr"] == 1 and r["Ma"] == 0.35][0]
    Tw, u, T, steps = couette_mu(1.0, 0.35)
    assert steps < 400000, "not converged"
    Er = abs((Tw - 1) - (row["Ta"] - 1)) / (row["Ta"] - 1)
    assert Er <= row["Er"] / 100
    c = (2.0 / 3.0) / 2 * 0.35 ** 2  # Pr (gamma - 1)/2 Ma^2
    # Eq. 52a: T(u); Eq. 52b: y(u), with the walls halfway: y/H = (j + 1/2)/60
    np.testing.assert_allclose(T - 1, c * (1 - u ** 2), rtol=0.02, atol=0.01 * c)
    eta = (np.arange(60) + 0.5) / 60
    y_of_u = (u + c * (u - u ** 3 / 3)) / (1 + (2.0 / 3.0) * c)
    assert np.abs(y_of_u - eta).max() < 5e-3
