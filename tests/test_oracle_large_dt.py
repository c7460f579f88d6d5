"""Oracle pins for natural convection with a large temperature difference
(arXiv:1109.6672, Sec. IV.C: T_h = 960 K, T_l = 240 K, Sutherland's law of
Eq. 59 with constant Pr).  The paper prints figures only, so the pins are:

* the conduction limit (no gravity, periodic in y): at steady state the heat
  flux -lambda(T) dT/dx is uniform and lambda is proportional to mu at
  constant Pr, so the Kirchhoff integral F(theta) = int_{0.4}^{theta} mu
  d(theta') is linear in x between the walls; with Sutherland's law theta
  itself is far from linear (0.12 off at its worst), with constant mu it is
  linear; F converges at second order in the grid spacing;
* the paper's description of Figs. 7-8: the centre of the primary vortex
  moves towards the right (cold) wall and downwards (with the paper's walls
  of non-equilibrium extrapolation), where the small temperature difference
  keeps it at the centre by symmetry.
"""
import math

import numpy as np
import pytest
from scipy.integrate import quad

from oracle import oracle as O
from paper_1109_6672_gb300 import inputs


def sutherland(p):
    S = p["mu_S"]
    return lambda th: th ** 1.5 * (1.0 + S) / (th + S)


def conduction_profile(n, law):
    p, _ = inputs.cavity_large_dT(Ra=1e3, n=n, nee=False)
    p.update(g=0.0, mu_law=law, ny=4, bc=[inputs.WALL_ISOTHERMAL, inputs.WALL_ISOTHERMAL,
                                          inputs.PERIODIC, inputs.PERIODIC])
    f = inputs.uniform_fields(n, 4, seed=1, u_amp=1e-4)
    o = O.Oracle(p).init(*f).step(int(60000 * (n / 32) ** 2), threads=4)
    th = o.moments()[3].mean(axis=0) / p["T0"]
    mu = sutherland(p) if law == O.MU_SUTHERLAND else (lambda t: 1.0)
    F = np.array([quad(mu, 0.4, t)[0] for t in th])
    Fw = quad(mu, 0.4, 1.6)[0]
    x = np.arange(n) + 0.5  # halfway walls at x = 0 (theta 1.6) and x = n (theta 0.4)
    return th, np.abs(F - Fw * (1.0 - x / n)).max() / Fw, np.abs(th - (1.6 - 1.2 * x / n)).max()


def test_conduction_limit_kirchhoff_profile():
    th16, e16, off16 = conduction_profile(16, O.MU_SUTHERLAND)
    th32, e32, off32 = conduction_profile(32, O.MU_SUTHERLAND)
    assert e32 < 1e-3 and e16 / e32 > 3.0  # second order
    assert off32 > 0.1  # the profile is not linear in theta
    _, e_const, off_const = conduction_profile(32, O.MU_TAU)
    assert e_const < 1e-5 and off_const < 1e-5


def vortex_centre(o, n, nee=False):
    """Centre of the largest |psi| (mass stream function, psi = 0 on the bottom
    wall) in units of the wall distance (halfway walls: node i at i + 1/2 of
    n; walls on the ghost nodes: node i at i + 1 of n + 1)."""
    rho, ux, uy, T = o.moments()
    psi = np.cumsum(rho * ux, axis=0)
    j, i = np.unravel_index(np.argmax(np.abs(psi)), psi.shape)
    if nee:
        return (i + 1.0) / (n + 1), (j + 1.0) / (n + 1)
    return (i + 0.5) / n, (j + 0.5) / n


def test_primary_vortex_moves_right_and_down():
    n = 40
    p, f = inputs.cavity_large_dT(Ra=1e3, n=n)
    xc, yc = vortex_centre(O.Oracle(p).init(*f).step(15000, threads=4), n, nee=True)
    assert xc > 0.6 and yc < 0.45
    # small temperature difference, same Ra and grid: centred by symmetry
    q, g = inputs.cavity(n=n, Ra=1e3, dT_over_T0=0.1, nu_min=0.05, strat=0.005, seed=1)
    xs, ys = vortex_centre(O.Oracle(q).init(*g).step(10000, threads=4), n)
    assert abs(xs - 0.5) <= 1.0 / n and abs(ys - 0.5) <= 1.0 / n
