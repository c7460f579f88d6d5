"""Physical pins of the oracle's whole step against closed forms of the
Navier-Stokes-Fourier equations the scheme recovers (Eqs. 29-30, Appendix A):

* shear-wave decay at rate nu k^2 with nu = tau_f R T (mu = tau_f p): the
  theta coupling shows as nu proportional to T, not to T0;
* entropy-wave decay at rate chi k^2 with chi = tau_h R T (lambda = tau_h
  (b+2)/2 p R, c_p = (b+2) R / 2);
* standing sound wave: frequency c_s k with c_s = sqrt(gamma R T) (p = rho R T)
  and damping k^2 / (2 rho) [(2 - 2/b) mu + (gamma - 1) lambda / c_p]
  (Eq. 56 times c_s, with mu_B = 2 (1/3 - 1/b) mu), which only holds with the
  correction term C_a of Eqs. 48-50 entering with a plus sign;
* thermal Couette flow: linear velocity and the viscous-heating parabola
  theta - 1 = Pr U^2 / ((b+2) R T0) eta (1 - eta), with second-order
  convergence in H; under a moving adiabatic wall
  theta - 1 = Pr U^2 / ((b+2) R T0) (2 eta - eta^2).
"""
import math

import numpy as np
import pytest
from scipy.optimize import curve_fit

from oracle import oracle as orc
from paper_1109_6672_gb300 import inputs

RT0 = 1.0 / 3.0


def _proj(field, k, axis):
    n = field.shape[axis]
    s = np.sin(k * np.arange(n))
    return 2.0 / n * np.tensordot(field.mean(axis=1 - axis), s, axes=(0, 0))


# The total-energy h^eq rest population is proportional to 2b - (b+2) theta,
# so with b = 3 the BGK scheme needs theta < 1.2 (in practice ~1.1, the
# bound at which it stays stable here); the cases stay below that.
@pytest.mark.parametrize("theta0", [0.8, 1.0, 1.1])
def test_shear_wave_viscosity(theta0):
    L, A = 128, 1e-3
    p = inputs.base_params(4, L, tau_f=0.3, tau_h=0.3 / 0.71, b=3.0)
    k = 2 * math.pi / L
    y = np.arange(L)[:, None] * np.ones((1, 4))
    fields = (np.ones((L, 4)), A * np.sin(k * y), np.zeros((L, 4)), np.full((L, 4), theta0))
    o = orc.Oracle(p).init(*fields)
    o.step(200)
    a1 = _proj(o.moments()[1], k, 0)
    o.step(2000)
    a2 = _proj(o.moments()[1], k, 0)
    rate = math.log(a1 / a2) / 2000
    nu = p["tau_f"] * RT0 * theta0
    assert rate == pytest.approx(nu * k * k, rel=0.01)
    if theta0 != 1.0:  # the decoupled model would give tau_f R T0
        assert abs(rate / (p["tau_f"] * RT0 * k * k) - 1) > 0.08


@pytest.mark.parametrize("model,theta0", [(inputs.E_TOTAL, 1.0), (inputs.E_TOTAL, 1.1),
                                          (inputs.E_INTERNAL, 1.0), (inputs.E_INTERNAL, 0.8)])
def test_entropy_wave_diffusivity(model, theta0):
    L, eps = 128, 1e-3
    p = inputs.base_params(L, 4, tau_f=0.3, tau_h=0.5, b=3.0, energy_model=model)
    k = 2 * math.pi / L
    x = np.ones((4, 1)) * np.arange(L)[None, :]
    pert = 1 + eps * np.sin(k * x)
    fields = (1.0 / pert, np.zeros((4, L)), np.zeros((4, L)), theta0 * pert)
    o = orc.Oracle(p).init(*fields)
    o.step(200)
    a1 = _proj(o.moments()[3] / theta0, k, 1)
    o.step(2000)
    a2 = _proj(o.moments()[3] / theta0, k, 1)
    rate = math.log(a1 / a2) / 2000
    chi = p["tau_h"] * RT0 * theta0
    assert rate == pytest.approx(chi * k * k, rel=0.02)


def _sound_run(theta0, correction, b=3.0, L=64, steps=1500):
    eps = 1e-3
    gamma = (b + 2) / b
    p = inputs.base_params(L, 4, tau_f=0.3, tau_h=0.3 / 0.71, b=b, correction=correction)
    k = 2 * math.pi / L
    x = np.ones((4, 1)) * np.arange(L)[None, :]
    s = np.sin(k * x)
    fields = (1 + eps * s, np.zeros((4, L)), np.zeros((4, L)), theta0 * (1 + (gamma - 1) * eps * s))
    o = orc.Oracle(p).init(*fields)
    amp = [_proj(fields[0], k, 1)]
    for _ in range(steps):
        o.step(1)
        amp.append(_proj(o.moments()[0], k, 1))
    t = np.arange(steps + 1, dtype=float)
    amp = np.array(amp) / eps

    def model(t, a, G, w, ph, c, d):
        return a * np.exp(-G * t) * np.cos(w * t + ph) + c * np.exp(-d * t)

    cs = math.sqrt(gamma * RT0 * theta0)
    p0 = [1.0, 1e-3, cs * k, 0.0, 0.0, 1e-3]
    popt, _ = curve_fit(model, t, amp, p0=p0, maxfev=20000)
    pr = theta0 * RT0  # p at rho = 1
    mu = p["tau_f"] * pr
    lam_cp = p["tau_h"] * pr
    Gamma = k * k / 2 * ((2 - 2 / b) * mu + (gamma - 1) * lam_cp)
    return popt[1], abs(popt[2]), Gamma, cs * k


@pytest.mark.parametrize("theta0", [0.8, 1.0, 1.1])
def test_sound_wave_speed_and_damping(theta0):
    G, w, G_th, w_th = _sound_run(theta0, correction=1)
    assert w == pytest.approx(w_th, rel=0.005)
    assert G == pytest.approx(G_th, rel=0.03)


def test_sound_wave_needs_correction_with_plus_sign():
    """Away from theta0 = 1 dropping C_a changes the longitudinal viscosity
    by tau_f rho c^2 (1 - theta0) (the Eq. 20 defect), far outside the
    tolerance above."""
    for theta0 in (0.8, 1.1):
        G, _, G_th, _ = _sound_run(theta0, correction=0)
        assert abs(G / G_th - 1) > 0.1, theta0


def _couette_error(p, fields, steps):
    o = orc.Oracle(p).init(*fields)
    o.step(steps)
    rho, ux, uy, T = o.moments()
    H = p["ny"]
    U = p["u_wall"][3][0]
    eta = (np.arange(H) + 0.5) / H
    Pr = p["tau_f"] / p["tau_h"]
    th_a = 1 + Pr * U * U / ((p["b"] + 2) * RT0) * eta * (1 - eta)
    th = T[:, 0] / p["T0"]
    Er = np.abs((th - 1) - (th_a - 1)).max() / (th_a - 1).max()
    return np.abs(ux[:, 0] / U - eta).max(), Er, (th - 1).max()


def test_couette_config():
    """4 x 33, U = 0.05, nu = 0.1, Pr = 0.71, 20 000 steps."""
    p, fields = inputs.couette()
    uerr, Er, rise = _couette_error(p, fields, 20000)
    assert uerr < 1e-6
    assert Er < 0.005  # Table I reports E_r below 1 %
    assert rise == pytest.approx(2.6625e-4, rel=0.01)


def test_couette_b_five_percent_rise_and_convergence():
    errs = []
    for H in (17, 33):
        p, fields = inputs.couette_b(ny=H)
        chi = p["tau_h"] * RT0
        uerr, Er, rise = _couette_error(p, fields, int(5 * H * H / chi))
        assert uerr < 1e-10  # halfway bounce-back: the linear profile is exact
        errs.append(Er)
    assert errs[1] < 0.001
    assert rise == pytest.approx(0.05, rel=0.01)
    assert errs[0] / errs[1] > 3.0  # second order in H


@pytest.mark.parametrize("collision", [orc.BGK, orc.MRT], ids=["bgk", "mrt"])
def test_couette_adiabatic_moving_wall(collision):
    """Bottom wall at rest and T0, top wall moving and adiabatic (halfway):
    the wall's work enters the gas, no heat crosses the wall, and the heating
    is theta - 1 = Pr U^2 / ((b + 2) R T0) (2 eta - eta^2), largest at the
    moving wall; second order in H (measured 3.9e-3, 9.8e-4)."""
    errs = []
    for H, steps in ((8, 3000), (16, 8000)):
        U, nu, Pr, b = 0.2, 0.2, 1.0, 5.0
        tau_f = nu / RT0
        p = inputs.base_params(2, H, tau_f=tau_f, tau_h=tau_f / Pr, b=b, collision=collision,
                               bc=[0, 0, inputs.WALL_ISOTHERMAL, inputs.WALL_ADIABATIC],
                               u_wall=[[0, 0], [0, 0], [0, 0], [U, 0]])
        rho, ux, uy, T = orc.Oracle(p).init(*inputs.uniform_fields(2, H, seed=0)).step(
            steps, threads=4).moments()
        eta = (np.arange(H) + 0.5) / H
        assert np.abs(ux[:, 0] - U * eta).max() < 1e-10 * U
        rise = Pr * U * U / ((b + 2) * RT0) * (2 * eta - eta * eta)
        errs.append(np.abs((T[:, 0] - 1) - rise).max() / rise.max())
    assert errs[1] < 2e-3 and 3.0 < errs[0] / errs[1] < 5.0, errs


@pytest.mark.parametrize("model,b,stable_tau,unstable_tau", [(inputs.E_INTERNAL, 5.0, 0.06, 0.03),
                                                             (inputs.E_TOTAL, 5.0, 0.15, 0.1),
                                                             (inputs.E_TOTAL, 3.0, 0.25, 0.2)])
def test_small_tau_stability_range(model, b, stable_tau, unstable_tau):
    """Where the coupled BGK scheme stays bounded (Pr = 0.71, periodic box
    seeded with grid-scale velocity noise 1e-4): internal energy down to
    tau_f = 0.06 (omega_f = 1.79), total energy down to 0.15 at b = 5 and 0.25
    at b = 3, whose h^eq rest weight is small; below these the thermal
    coupling (theta in f^eq, tau_h != tau_f) grows.  Every configured workload
    lies inside these ranges."""
    n = 32
    for tau_f, stable in ((stable_tau, True), (unstable_tau, False)):
        p = inputs.base_params(n, n, tau_f=tau_f, tau_h=tau_f / 0.71, energy_model=model, b=b)
        o = orc.Oracle(p).init(*inputs.uniform_fields(n, n, seed=1, u_amp=1e-4))
        o.step(3000)
        T = o.moments()[3]
        bounded = bool(np.isfinite(T).all() and np.abs(T - 1).max() < 1e-6)
        assert bounded == stable, (tau_f, np.abs(T - 1).max())
