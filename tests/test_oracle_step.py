"""Whole-step pins of the oracle: brute-force agreement with an independent
NumPy restatement on tiny grids, exact conservation in a periodic box
(collision invariants of Eqs. 34-38 with Eq. 26), and the momentum input of
the gravity force (text under Eq. 51)."""
import zlib

import numpy as np
import pytest

from oracle import oracle as orc
from paper_1109_6672_gb300 import inputs
from brute_lbm import Brute

P, ISO, ADI = inputs.PERIODIC, inputs.WALL_ISOTHERMAL, inputs.WALL_ADIABATIC


def _fields(nx, ny, seed, u_amp=0.05, T_amp=0.2, rho_amp=0.1):
    return inputs.uniform_fields(nx, ny, seed, u_amp=u_amp, T_amp=T_amp, rho_amp=rho_amp)


TINY = {
    "periodic_total": dict(nx=5, ny=4, bc=[P, P, P, P]),
    "periodic_total_zsimple": dict(nx=5, ny=4, bc=[P, P, P, P], z_full=0),
    "periodic_nocorr": dict(nx=5, ny=4, bc=[P, P, P, P], correction=0),
    "couette_walls": dict(nx=4, ny=6, bc=[P, P, ISO, ISO], T_wall=[1, 1, 1.1, 0.9],
                          u_wall=[[0, 0], [0, 0], [0.02, 0.0], [0.05, 0.01]]),
    "adiabatic_walls": dict(nx=4, ny=6, bc=[P, P, ADI, ADI],
                            u_wall=[[0, 0], [0, 0], [0.03, 0.0], [-0.04, 0.0]]),
    "cavity_internal_gravity": dict(nx=5, ny=5, bc=[ISO, ISO, ADI, ADI], T_wall=[1.2, 0.8, 1, 1],
                                    energy_model=inputs.E_INTERNAL, g=1e-3, b=5.0),
    "x_walls_y_periodic": dict(nx=6, ny=4, bc=[ISO, ADI, P, P], T_wall=[1.1, 1, 1, 1],
                               u_wall=[[0, 0.02], [0, -0.01], [0, 0], [0, 0]]),
    "all_iso_moving": dict(nx=5, ny=6, bc=[ISO, ISO, ISO, ISO], T_wall=[1.1, 0.9, 1.05, 0.95],
                           u_wall=[[0, 0.01], [0.0, -0.02], [0.03, 0], [-0.02, 0.01]]),
    "gravity_iso_floor_ceiling": dict(nx=5, ny=6, bc=[P, P, ISO, ISO], T_wall=[1, 1, 1.1, 0.9],
                                      energy_model=inputs.E_INTERNAL, g=2e-3, b=5.0),
}


@pytest.mark.parametrize("name", sorted(TINY))
def test_oracle_matches_bruteforce(name):
    kw = dict(TINY[name])
    p = inputs.base_params(kw.pop("nx"), kw.pop("ny"), tau_f=0.35, tau_h=0.6, **kw)
    fields = _fields(p["nx"], p["ny"], seed=zlib.crc32(name.encode()) % 1000)
    o = orc.Oracle(p).init(*fields)
    b = Brute(p).init(*fields)
    np.testing.assert_allclose(o.pops(), b.pops(), rtol=1e-14, atol=1e-15)
    for _ in range(5):
        o.step(10)
        b.step(10)
        np.testing.assert_allclose(o.pops(), b.pops(), rtol=1e-11, atol=1e-13)


@pytest.mark.parametrize("model", [inputs.E_TOTAL, inputs.E_INTERNAL])
@pytest.mark.parametrize("z_full", [1, 0])
def test_periodic_conservation(model, z_full):
    """Periodic box: sum rho, sum rho u and sum hbar are invariants of the
    collision (sum C = sum e C = 0; sum Z (fbar - f^eq + C/2) = 0) and of
    streaming."""
    p = inputs.base_params(24, 20, energy_model=model, z_full=z_full, b=3.0)
    fields = _fields(24, 20, seed=5, u_amp=0.05, T_amp=0.2, rho_amp=0.05)
    o = orc.Oracle(p).init(*fields)
    c0 = o.conserved()
    o.step(500)
    c1 = o.conserved()
    rel = np.abs(c1 - c0) / np.array([abs(c0[0]), abs(c0[0]), abs(c0[0]), abs(c0[3])])
    assert np.all(rel < 1e-13), (c0, c1, rel)
    rho, ux, uy, T = o.moments()
    assert np.all(np.isfinite(T))


def test_gravity_momentum_input():
    """a = (0, -rho g) enters the momentum at rate sum a per step in a periodic
    box (first moment of F_a is a, Eq. 26 for C)."""
    g = 1e-4
    p = inputs.base_params(12, 10, g=g, energy_model=inputs.E_INTERNAL, b=5.0)
    fields = _fields(12, 10, seed=6, u_amp=0.01, T_amp=0.05, rho_amp=0.02)
    o = orc.Oracle(p).init(*fields)
    c0 = o.conserved()
    steps = 50
    o.step(steps)
    c1 = o.conserved()
    assert np.isclose(c1[0], c0[0], rtol=1e-14)
    assert abs(c1[1] - c0[1]) < 1e-13
    assert np.isclose(c1[2] - c0[2], -g * c0[0] * steps, rtol=1e-9)


def test_init_moments_roundtrip():
    """Moments of the initial equilibrium state return the input fields."""
    p = inputs.base_params(7, 9, b=3.0)
    rho, ux, uy, T = _fields(7, 9, seed=8)
    o = orc.Oracle(p).init(rho, ux, uy, T)
    r2, ux2, uy2, T2 = o.moments()
    for a, b in ((rho, r2), (ux, ux2), (uy, uy2), (T, T2)):
        np.testing.assert_allclose(a, b, rtol=1e-13, atol=1e-15)


@pytest.mark.parametrize("g", [0.0, 1e-4])
def test_closed_adiabatic_box_conserves_mass_and_energy(g):
    """All four walls adiabatic and at rest: bounce-back keeps sum rho and
    sum hbar (internal energy) constant; gravity only adds momentum."""
    p = inputs.base_params(10, 12, bc=[ADI] * 4, energy_model=inputs.E_INTERNAL, b=5.0, g=g,
                           tau_f=0.4, tau_h=0.5)
    fields = _fields(10, 12, seed=9, u_amp=0.01, T_amp=0.1, rho_amp=0.02)
    o = orc.Oracle(p).init(*fields)
    c0 = o.conserved()
    o.step(400)
    c1 = o.conserved()
    assert abs(c1[0] / c0[0] - 1) < 1e-13
    assert abs(c1[3] / c0[3] - 1) < 1e-13


def test_isothermal_box_relaxes_to_wall_temperature():
    """All walls isothermal at theta_w = 1.05, fluid at rest at theta = 1:
    the interior approaches the wall temperature (Dirichlet data reached)."""
    p = inputs.base_params(8, 8, bc=[ISO] * 4, T_wall=[1.05] * 4, energy_model=inputs.E_INTERNAL,
                           b=5.0, tau_f=0.4, tau_h=1.0)
    o = orc.Oracle(p).init(*inputs.uniform_fields(8, 8, seed=0))
    o.step(3000)
    T = o.moments()[3]
    np.testing.assert_allclose(T, 1.05, rtol=1e-6)
