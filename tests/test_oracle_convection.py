"""Rayleigh-Benard onset: a layer of gas between a hot isothermal wall below
and a cold one above, periodic sideways, under gravity.  Linear stability
theory of the Boussinesq equations with rigid isothermal walls puts the onset
of convection at Ra_c = 1707.76 (wavelength 2.016 H; Chandrasekhar,
Hydrodynamic and Hydromagnetic Stability, 1961, ch. II).  The oracle's D2Q9
step with gravity (Guo force, the internal-energy model of Eq. 38) and
halfway walls has to damp a roll below the onset and amplify it above: this
pins gravity, buoyancy through p = rho R T, the thermal walls and the
momentum and heat transport together against a textbook number.  The gas is
near the Boussinesq limit (dT/T0 = 0.05, stratification g H / (R T0) =
0.056); measured, the onset lies at 1.011 Ra_c here.  The isothermal ghost
carries the node's pressure with the hydrostatic drop across the spacing;
with equal pressure instead, the floor and ceiling sat g / (2 R) off their
temperatures and the onset moved to 1.047 Ra_c."""
import math

import numpy as np
import pytest

from oracle import oracle as orc
from paper_1109_6672_gb300 import inputs

RT0 = 1.0 / 3.0
RA_C = 1707.76


def rb_case(ratio, H=32, dT=0.05, tau_f=0.06, Pr=0.71, b=5.0, precision=inputs.P_FP64):
    """Parameters and initial fields at Ra = ratio Ra_c: conduction profile,
    isothermal-hydrostatic density, and a roll of one wavelength 2 H seeded
    in T at 1e-3 dT.  Returns (params, fields, chi)."""
    nx = 2 * H
    nu = tau_f * RT0
    chi = nu / Pr
    g = ratio * RA_C * nu * chi / (dT * H ** 3)  # Ra = g (dT / T0) H^3 / (nu chi)
    p = inputs.base_params(nx, H, tau_f=tau_f, tau_h=tau_f / Pr, b=b, g=g,
                           energy_model=inputs.E_INTERNAL, precision=precision,
                           bc=[inputs.PERIODIC, inputs.PERIODIC, inputs.WALL_ISOTHERMAL,
                               inputs.WALL_ISOTHERMAL],
                           T_wall=[1.0, 1.0, 1 + dT / 2, 1 - dT / 2])
    y = (np.arange(H) + 0.5) / H
    x = np.arange(nx)
    T = (1 + dT / 2 - dT * y)[:, None] * np.ones((1, nx))
    T = T + 1e-3 * dT * np.sin(2 * math.pi * x / nx)[None, :] * np.sin(math.pi * y)[:, None]
    rho = np.exp(-3 * g * (np.arange(H) - H / 2))[:, None] * np.ones((1, nx))
    return p, (rho, 0.0, 0.0, T), chi


def growth_rate(sim, H, chi, steps, chunks=40):
    """sigma H^2 / chi of the roll's kinetic energy (sum of u_y^2), fitted
    over the second half of the run (after the acoustic settling)."""
    every = max(1, steps // chunks)
    E = []
    for _ in range(chunks):
        sim.step(every, **({"threads": 8} if isinstance(sim, orc.Oracle) else {}))
        E.append(float((sim.moments()[2] ** 2).sum()))
    t = (np.arange(chunks) + 1) * every
    h = chunks // 2
    return np.polyfit(t[h:], 0.5 * np.log(np.array(E[h:])), 1)[0] * H * H / chi


def test_rayleigh_benard_onset():
    """Growth rates at 0.95 and 1.05 Ra_c (a decay and a growth) put the
    onset, by linear interpolation, within 2.5 % of Ra_c (measured 1.01)."""
    s = {r: growth_rate(orc.Oracle(p).init(*f), 32, chi, 80000)
         for r, (p, f, chi) in ((r, rb_case(r)) for r in (0.95, 1.05))}
    assert s[0.95] < 0 < s[1.05], s
    onset = 0.95 + 0.1 * (-s[0.95]) / (s[1.05] - s[0.95])
    assert abs(onset - 1.0) < 0.025, (s, onset)
