"""Seeded synthetic inputs and workload recipes.

This module holds no step arithmetic of the method: it draws the initial
macroscopic fields (rho, u, T) from a seeded generator and fills the parameter
dictionaries of the named workloads.  Both the CUDA path and the CPU oracle
receive exactly these arrays and parameters.

Sides are ordered x-, x+, y-, y+ everywhere.  Lattice units: dx = dt = 1,
c = sqrt(3 R T0) = 1, so R T0 = 1/3 (Eq. 6 and Eq. 28 of arXiv:1109.6672).

Parameter mapping used by the recipes (BGK scheme, Eq. 30 and text around it):
the shear viscosity is mu = tau_f p, so nu = tau_f R T; the thermal
diffusivity is chi = tau_h R T; Pr = tau_f / tau_h.
"""
from __future__ import annotations

import math

import numpy as np

PERIODIC, WALL_ISOTHERMAL, WALL_ADIABATIC, INLET, OUTLET = 0, 1, 2, 3, 4
E_TOTAL, E_INTERNAL = 0, 1
P_FP64, P_FP32, P_FP32_FP16, P_FP32_BF16 = 0, 1, 2, 3
RT0 = 1.0 / 3.0


def base_params(nx: int, ny: int, **kw) -> dict:
    p = dict(
        nx=int(nx), ny=int(ny), bc=[PERIODIC] * 4, tau_f=0.3, tau_h=0.3 / 0.71, Pr=0.0,
        R=1.0 / 3.0, T0=1.0, b=3.0, u_wall=[[0.0, 0.0] for _ in range(4)],
        T_wall=[1.0] * 4, g=0.0, energy_model=E_TOTAL, correction=1, z_full=1,
        precision=P_FP64,
    )
    p.update(kw)
    return p


def uniform_fields(nx: int, ny: int, seed: int, rho0: float = 1.0, u_amp: float = 0.0,
                   T0: float = 1.0, T_amp: float = 0.0, rho_amp: float = 0.0):
    """rho, ux, uy, T as [ny, nx] float64: constant means plus independent
    uniform noise U(-amp, amp) from numpy's PCG64 seeded with ``seed``.
    T_amp is relative to T0."""
    rng = np.random.default_rng(seed)
    shape = (ny, nx)
    rho = rho0 + rho_amp * rng.uniform(-1.0, 1.0, shape) if rho_amp else np.full(shape, rho0)
    ux = u_amp * rng.uniform(-1.0, 1.0, shape) if u_amp else np.zeros(shape)
    uy = u_amp * rng.uniform(-1.0, 1.0, shape) if u_amp else np.zeros(shape)
    T = T0 * (1.0 + T_amp * rng.uniform(-1.0, 1.0, shape)) if T_amp else np.full(shape, T0)
    return rho, ux, uy, T


# ---- named workloads -------------------------------------------------------

def couette(ny: int = 33, nx: int = 4, U: float = 0.05, nu: float = 0.1, Pr: float = 0.71,
            b: float = 3.0, **kw):
    """Thermal Couette flow: periodic in x, halfway walls at y = -1/2 and
    y = ny - 1/2 (H = ny); bottom at rest, top moving at (U, 0); both walls at
    T = T0 = 1.  Starts from uniform rest."""
    tau_f = nu / RT0
    p = base_params(nx, ny, tau_f=tau_f, tau_h=tau_f / Pr, b=b,
                    bc=[PERIODIC, PERIODIC, WALL_ISOTHERMAL, WALL_ISOTHERMAL],
                    u_wall=[[0.0, 0.0], [0.0, 0.0], [0.0, 0.0], [U, 0.0]], **kw)
    return p, uniform_fields(nx, ny, seed=0)


def couette_b(ny: int = 33, nx: int = 4, **kw):
    """Couette variant with a 5 % viscous-heating rise: Pr = 3, b = 3
    (gamma = 5/3), U = 1/3 (Ma = U / sqrt(gamma R T0) = 0.447), nu = 0.2.
    The peak rise of the constant-property solution is
    Pr U^2 / (4 (b + 2) R T0) = 0.05.  (Pr = 5 with tau_h = tau_f / 5 is
    outside the stable range of the BGK scheme, so Pr = 3 is used.)"""
    return couette(ny=ny, nx=nx, U=1.0 / 3.0, nu=0.2, Pr=3.0, b=3.0, **kw)


def periodic_box(n: int = 4096, seed: int = 2, precision: int = P_FP32, nx: int | None = None,
                 ny: int | None = None, **kw):
    """Fully periodic box: rho = 1, u ~ U(-1e-3, 1e-3), T = T0 (1 + U(-1e-2, 1e-2)),
    tau_f = 0.3 (nu = 0.1), Pr = 0.71, b = 3, total-energy model, correction on."""
    nx = n if nx is None else nx
    ny = n if ny is None else ny
    p = base_params(nx, ny, precision=precision, **kw)
    return p, uniform_fields(nx, ny, seed=seed, u_amp=1e-3, T_amp=1e-2)


def cavity_gravity(H: int, dT_over_T0: float, Ma: float = 0.1, strat: float = 0.05) -> float:
    """Gravity for a cavity of height H: the smaller of the value that keeps the
    hydrostatic stratification g H / (R T0) at ``strat`` and the value whose
    free-fall velocity sqrt(g beta dT H) equals Ma * sqrt(gamma R T0) with
    gamma = 1.4 (beta = 1/T_r, T_r = T0)."""
    g_strat = strat * RT0 / H
    U = Ma * math.sqrt(1.4 * RT0)
    g_ma = U * U / (dT_over_T0 * H)
    return min(g_strat, g_ma)


def cavity(n: int = 256, Ra: float = 1e5, Pr: float = 0.71, dT_over_T0: float = 0.01,
           seed: int = 1, noise: float = 1e-4, b: float = 5.0, precision: int = P_FP64,
           nu_min: float = 0.02, strat: float = 0.05, **kw):
    """Differentially heated square cavity (natural convection): hot wall at
    x-, cold wall at x+ (isothermal, T0 (1 +- dT/2)), adiabatic top and bottom,
    internal-energy model (Eq. 38), gravity a = (0, -rho g), b = 5
    (gamma = 1.4).  Ra = g beta dT H^3 Pr / nu^2 with beta = 1/T0 (Eq. 57-58),
    hence nu = sqrt(g (dT/T0) H^3 Pr / Ra).  ``strat`` caps the hydrostatic
    stratification g H / (R T0); near the Boussinesq limit it has to be small
    against dT/T0 (0.05 dT/T0 keeps its effect on Nu below 1 %).  A nu below
    ``nu_min`` (0.02: tau_f = 0.06, where the scheme with the internal-energy
    model is still stable) is raised by raising g (keeping Ra), up to the
    Ma = 0.1 free-fall limit; beyond it nu is floored and the effective Ra
    drops (recorded as Ra_effective)."""
    H = n
    g = cavity_gravity(H, dT_over_T0, strat=strat)
    nu = math.sqrt(g * dT_over_T0 * H ** 3 * Pr / Ra)
    if nu < nu_min:
        g_ma = cavity_gravity(H, dT_over_T0, strat=math.inf)
        g = min(nu_min * nu_min * Ra / (dT_over_T0 * H ** 3 * Pr), g_ma)
        nu = max(math.sqrt(g * dT_over_T0 * H ** 3 * Pr / Ra), nu_min)
    tau_f = nu / RT0
    Th, Tl = 1.0 + 0.5 * dT_over_T0, 1.0 - 0.5 * dT_over_T0
    p = base_params(n, n, tau_f=tau_f, tau_h=tau_f / Pr, b=b, g=g, energy_model=E_INTERNAL,
                    bc=[WALL_ISOTHERMAL, WALL_ISOTHERMAL, WALL_ADIABATIC, WALL_ADIABATIC],
                    T_wall=[Th, Tl, 1.0, 1.0], precision=precision, **kw)
    p["Ra_effective"] = g * dT_over_T0 * H ** 3 * Pr / (nu * nu)
    return p, uniform_fields(n, n, seed=seed, u_amp=noise)


def batch_cavities(count: int = 256, seed: int = 4, sides=tuple(range(64, 513, 32)),
                   precision: int = P_FP32_BF16, nu_min: float = 0.02):
    """Batch of independent cavities: side uniform over ``sides``, dT/T0 ~
    U[0.01, 0.6], Ra log-uniform in [1e4, 1e6], Pr = 0.71, nu >= nu_min
    (see ``cavity``)."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(count):
        n = int(rng.choice(sides))
        dT = float(rng.uniform(0.01, 0.6))
        Ra = float(10.0 ** rng.uniform(4.0, 6.0))
        p, fields = cavity(n=n, Ra=Ra, dT_over_T0=dT, seed=seed * 100003 + k, precision=precision,
                           nu_min=nu_min)
        out.append((p, fields))
    return out


def acoustic_channel(Pr: float = 2.0, gamma: float = 5.0 / 3.0, nx: int = 600, ny: int = 4,
                     mu: float = 0.1, wavelength: float = 50.0, drho: float = 0.01,
                     precision: int = P_FP64, **kw):
    """Attenuation-driven acoustic streaming (Sec. IV.B): a plane sound wave
    enters a channel periodic in y through an inlet at x- and leaves through a
    zero-gradient outlet at x+ (600 x 4 nodes).  rho0 = T0 = 1, mu = 0.1
    (tau_f = mu / p0), wavelength 50, b = 2 / (gamma - 1), total-energy model;
    the correction term is off, as the paper runs it.  The inlet state is
    Eq. 53, rho0 + drho sin(w t) and T0 (1 + (gamma - 1) drho/rho0 sin(w t)),
    with w = 2 pi c_s / wavelength, c_s = sqrt(gamma R T0), and the velocity of
    the travelling wave, c_s drho/rho0 sin(w t) (the amplitude U of Eq. 54).
    Starts from uniform rest.  The returned parameters also carry c_s, w and U
    (keys cs, omega, U) for the analysis."""
    cs = math.sqrt(gamma * RT0)
    omega = 2.0 * math.pi * cs / wavelength
    tau_f = mu / RT0
    kw.setdefault("correction", 0)
    p = base_params(nx, ny, tau_f=tau_f, tau_h=tau_f / Pr, b=2.0 / (gamma - 1.0),
                    bc=[INLET, OUTLET, PERIODIC, PERIODIC], energy_model=E_TOTAL,
                    precision=precision, in_rho=1.0, in_drho=drho, in_du=cs * drho,
                    in_dT=(gamma - 1.0) * drho, in_omega=omega, cs=cs, omega=omega,
                    U=cs * drho, **kw)
    return p, uniform_fields(nx, ny, seed=0)


# Sec. IV.C, large temperature difference: Ra -> (grid side, mu_r)
LARGE_DT_CASES = {1e3: (100, 0.1), 1e4: (150, 0.1), 1e5: (200, 0.06)}


def cavity_large_dT(Ra: float = 1e5, n: int | None = None, mu_r: float | None = None,
                    Pr: float = 0.71, seed: int = 1, noise: float = 1e-4,
                    precision: int = P_FP64, nee: bool = True, **kw):
    """Natural convection with a large temperature difference (Sec. IV.C):
    T_h = 960 K, T_l = 240 K, T0 = T_r = 600 K (theta 1.6 at x-, 0.4 at x+),
    adiabatic top and bottom.  Sutherland's law (Eq. 59, S = 110.5 K) referred
    to T_r (mu* taken from mu(T_r) = mu_r); Pr = 0.71 constant; mu_r and the
    grid per Ra as the paper takes them (100, 150, 200 nodes; mu_r = 0.1, 0.1,
    0.06 for Ra = 1e3, 1e4, 1e5).  MRT with tau_e = tau_eps = tau_f and
    1/tau_q = 1.5, internal-energy model (Eq. 38), correction on.  ``nee``:
    the paper's walls of non-equilibrium extrapolation on the wall nodes (the
    paper's grid counts them: n = grid - 2 fluid nodes, H = n + 1); else
    halfway walls (n = grid, H = n).  ``n`` overrides the fluid nodes per side.
    Gravity from Eq. 57 with beta = 1/T_r (Eq. 58): g = Ra nu_r^2 /
    (Pr beta dT H^3), nu_r = mu_r / rho0, rho0 = 1."""
    n0, mu0 = LARGE_DT_CASES.get(Ra, (200, 0.06))
    if n is None:
        n = n0 - 2 if nee else n0
    mu_r = mu0 if mu_r is None else mu_r
    H = n + 1 if nee else n
    dT = (960.0 - 240.0) / 600.0
    g = Ra * mu_r * mu_r / (Pr * dT * H ** 3)
    tau_f = mu_r / RT0
    p = base_params(n, n, tau_f=tau_f, tau_h=tau_f / Pr, b=5.0, g=g, energy_model=E_INTERNAL,
                    bc=[WALL_ISOTHERMAL, WALL_ISOTHERMAL, WALL_ADIABATIC, WALL_ADIABATIC],
                    T_wall=[1.6, 0.4, 1.0, 1.0], precision=precision, mu_law=2,
                    mu_S=110.5 / 600.0, collision=1, s_q=1.5, wall_nee=15 if nee else 0, **kw)
    return p, uniform_fields(n, n, seed=seed, u_amp=noise)


# ---- three-dimensional (D3Q19) workloads ------------------------------------

def base_params3d(nx: int, ny: int, nz: int, **kw) -> dict:
    """Parameters of a 3-D grid (periodic unless bc_z is given): the same physical
    parameters as base_params, without walls or gravity."""
    p = dict(nx=int(nx), ny=int(ny), nz=int(nz), tau_f=0.3, tau_h=0.3 / 0.71, R=1.0 / 3.0,
             T0=1.0, b=3.0, energy_model=E_TOTAL, correction=1, z_full=1, precision=P_FP64)
    p.update(kw)
    return p


def uniform_fields3d(nx: int, ny: int, nz: int, seed: int, rho0: float = 1.0,
                     u_amp: float = 0.0, T0: float = 1.0, T_amp: float = 0.0,
                     rho_amp: float = 0.0):
    """rho, ux, uy, uz, T as [nz, ny, nx] float64: constant means plus
    independent uniform noise U(-amp, amp) from numpy's PCG64 seeded with
    ``seed``.  T_amp is relative to T0."""
    rng = np.random.default_rng(seed)
    shape = (nz, ny, nx)
    rho = rho0 + rho_amp * rng.uniform(-1.0, 1.0, shape) if rho_amp else np.full(shape, rho0)
    u = [u_amp * rng.uniform(-1.0, 1.0, shape) if u_amp else np.zeros(shape) for _ in range(3)]
    T = T0 * (1.0 + T_amp * rng.uniform(-1.0, 1.0, shape)) if T_amp else np.full(shape, T0)
    return (rho, *u, T)


def periodic_box3d(n: int = 256, seed: int = 2, precision: int = P_FP32, **kw):
    """Fully periodic n^3 box, the 3-D counterpart of periodic_box: rho = 1,
    u ~ U(-1e-3, 1e-3), T = T0 (1 + U(-1e-2, 1e-2)), tau_f = 0.3, Pr = 0.71,
    b = 3, total-energy model, correction on."""
    p = base_params3d(n, n, n, precision=precision, **kw)
    return p, uniform_fields3d(n, n, n, seed=seed, u_amp=1e-3, T_amp=1e-2)
