"""Pins of the oracle's MRT scheme (Sec. III.C.2: Eqs. 40-47, Appendix B)
against the velocity set, the BGK scheme it reduces to, an independent NumPy
restatement, conservation, and the shear-wave closed form."""
import math

import zlib

import numpy as np
import pytest

from oracle import oracle as orc
from paper_1109_6672_gb300 import inputs
from brute_lbm import MB, Brute
from test_oracle_step import TINY, _fields

P, ISO, ADI = inputs.PERIODIC, inputs.WALL_ISOTHERMAL, inputs.WALL_ADIABATIC
RT0 = 1.0 / 3.0


def test_oracle_matrices_are_the_velocity_set_moments():
    """B1 rows are the moments rho, e, eps, j, q, p of the velocity set and B2
    is its inverse."""
    M, Minv = orc.mrt_matrices()
    np.testing.assert_array_equal(M, MB)
    np.testing.assert_allclose(M @ Minv, np.eye(9), atol=1e-15)


def test_eq41_is_M_times_eq18a():
    rng = np.random.default_rng(41)
    for _ in range(50):
        rho, th = rng.uniform(0.5, 1.5, 2)
        ux, uy = rng.uniform(-0.2, 0.2, 2)
        np.testing.assert_allclose(orc.meq(rho, ux, uy, th), MB @ orc.feq(RT0, rho, ux, uy, th),
                                   rtol=1e-13, atol=1e-15)


MRT_RATES = dict(collision=orc.MRT, s_e=1.3, s_eps=1.1, s_q=1.6)


@pytest.mark.parametrize("name", sorted(TINY))
def test_uniform_rates_reduce_to_bgk(name):
    """With every rate of S equal to omega_f (the rates of the conserved
    moments drop out) Eq. 44 is Eq. 34 and the Eq. 47 coupling equals the
    BGK (w_h - w_f)."""
    kw = dict(TINY[name])
    p = inputs.base_params(kw.pop("nx"), kw.pop("ny"), tau_f=0.35, tau_h=0.6, **kw)
    fields = _fields(p["nx"], p["ny"], seed=zlib.crc32(name.encode()) % 1000)
    bgk = orc.Oracle(p).init(*fields).step(40)
    mrt = orc.Oracle(dict(p, collision=orc.MRT)).init(*fields).step(40)
    np.testing.assert_allclose(mrt.pops(), bgk.pops(), rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("name", sorted(TINY))
def test_mrt_matches_bruteforce(name):
    kw = dict(TINY[name])
    p = inputs.base_params(kw.pop("nx"), kw.pop("ny"), tau_f=0.35, tau_h=0.6, **kw, **MRT_RATES)
    fields = _fields(p["nx"], p["ny"], seed=zlib.crc32(name.encode()) % 1000 + 7)
    o = orc.Oracle(p).init(*fields)
    b = Brute(p).init(*fields)
    for _ in range(4):
        o.step(10)
        b.step(10)
        np.testing.assert_allclose(o.pops(), b.pops(), rtol=1e-11, atol=1e-13)


@pytest.mark.parametrize("model", [inputs.E_TOTAL, inputs.E_INTERNAL])
def test_mrt_periodic_conservation(model):
    p = inputs.base_params(24, 20, energy_model=model, b=3.0, **MRT_RATES)
    fields = _fields(24, 20, seed=6, u_amp=0.05, T_amp=0.1, rho_amp=0.05)
    o = orc.Oracle(p).init(*fields)
    c0 = o.conserved()
    o.step(500)
    c1 = o.conserved()
    rel = np.abs(c1 - c0) / np.array([abs(c0[0]), abs(c0[0]), abs(c0[0]), abs(c0[3])])
    assert np.all(rel < 1e-13), (c0, c1, rel)


@pytest.mark.parametrize("theta0", [0.9, 1.0, 1.1])
def test_mrt_shear_wave_viscosity(theta0):
    """mu = (tau - 1/2) p with the discrete MRT shear time tau = tau_f + 1/2:
    the decay rate is nu k^2, nu = tau_f R T, whatever the rates of the
    non-hydrodynamic moments."""
    L, A = 128, 1e-3
    p = inputs.base_params(4, L, tau_f=0.3, tau_h=0.3 / 0.71, b=3.0, **MRT_RATES)
    k = 2 * math.pi / L
    y = np.arange(L)[:, None] * np.ones((1, 4))
    fields = (np.ones((L, 4)), A * np.sin(k * y), np.zeros((L, 4)), np.full((L, 4), theta0))
    o = orc.Oracle(p).init(*fields)
    s = np.sin(k * np.arange(L))

    def amp():
        return float(o.moments()[1][:, 0] @ s) * 2 / L

    o.step(200)
    a1 = amp()
    o.step(2000)
    a2 = amp()
    rate = math.log(a1 / a2) / 2000
    assert rate == pytest.approx(p["tau_f"] * RT0 * theta0 * k * k, rel=0.01)
