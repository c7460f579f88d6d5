"""The D3Q19 CUDA path against the 3-D oracle: every physics mode, ragged
tiles (sizes not multiples of the 32 x 8 tile), grids smaller than a tile,
several z ranges per column of blocks; FP64 to 1e-12 of the oracle's
populations, FP32 to 2e-5; conservation of mass, momentum and total energy
on the GPU."""
import numpy as np
import pytest

from oracle import oracle3d as o3
from paper_1109_6672_gb300 import inputs
from paper_1109_6672_gb300 import lbm
from paper_1109_6672_gb300.lbm3d import Lbm3d

pytestmark = pytest.mark.gpu

MODES = {
    "total_zfull_corr": dict(energy_model=inputs.E_TOTAL, z_full=1, correction=1),
    "total_corr": dict(energy_model=inputs.E_TOTAL, z_full=0, correction=1),
    "total_zfull": dict(energy_model=inputs.E_TOTAL, z_full=1, correction=0),
    "total": dict(energy_model=inputs.E_TOTAL, z_full=0, correction=0),
    "internal_corr": dict(energy_model=inputs.E_INTERNAL, correction=1, b=5.0),
    "internal": dict(energy_model=inputs.E_INTERNAL, correction=0, b=5.0),
}
SIZES = [(4, 3, 5), (37, 11, 9), (70, 20, 12), (33, 9, 40)]


def _case(shape, mode, precision, seed=7):
    nx, ny, nz = shape
    kw = dict(MODES[mode])
    p = inputs.base_params3d(nx, ny, nz, tau_f=0.35, tau_h=0.5, precision=precision, **kw)
    f = inputs.uniform_fields3d(nx, ny, nz, seed=seed, u_amp=0.04, T_amp=0.05, rho_amp=0.03)
    return p, f


def _rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


@pytest.mark.parametrize("mode", list(MODES))
@pytest.mark.parametrize("shape", SIZES, ids=["x".join(map(str, s)) for s in SIZES])
def test_fp64_parity_3d(shape, mode):
    p, f = _case(shape, mode, lbm.LBM_P_FP64)
    steps = 30
    o = o3.Oracle3d(p).init(*f).step(steps)
    g = Lbm3d(p).init(*f).step(steps)
    assert _rel(g.pops(), o.pops()) <= 1e-12
    for got, want in zip(g.moments(), o.moments()):
        assert np.abs(got - want).max() <= 1e-12 * max(np.abs(want).max(), 1e-3)
    g.close()


SHAPES = [(8, 0), (16, 0), (4, 1), (8, 1)]  # FP32 launch shapes (tile rows, halo warps)


@pytest.mark.parametrize("shape", SHAPES, ids=[f"{a}x{b}" for a, b in SHAPES])
@pytest.mark.parametrize("mode", ["total_zfull_corr", "internal_corr"])
def test_fp32_parity_3d(mode, shape):
    p, f = _case((37, 21, 9), mode, lbm.LBM_P_FP32)
    o = o3.Oracle3d(dict(p, precision=lbm.LBM_P_FP64)).init(*f).step(30)
    g = Lbm3d(p).set_launch(*shape).init(*f).step(30)
    assert _rel(g.pops(), o.pops()) <= 2e-5
    g.close()


def test_fp32_tiles_agree():
    """The launch shapes compute the same step; they are separate template
    instantiations, whose FMA contractions the compiler may choose
    differently, so they agree to the FP32 rounding accumulated over the
    steps (measured 1.8e-6 of the populations after 20 steps of these noisy
    fields; each is within 2e-5 of the FP64 oracle, test_fp32_parity_3d)."""
    p, f = _case((70, 33, 12), "total_zfull_corr", lbm.LBM_P_FP32)
    a = Lbm3d(p).set_tile(8).init(*f).step(20)
    for shape in SHAPES[1:]:
        b = Lbm3d(p).set_launch(*shape).init(*f).step(20)
        assert _rel(a.pops(), b.pops()) <= 1e-5, shape
        b.close()
    a.close()


def test_set_tile_validation():
    p, f = _case((8, 8, 8), "total", lbm.LBM_P_FP64)
    g = Lbm3d(p)
    with pytest.raises(lbm.LbmError):
        g.set_tile(16)
    with pytest.raises(lbm.LbmError):
        g.set_tile(12)
    for shape in [(4, 1), (8, 1), (16, 0), (4, 0), (16, 1), (8, 2)]:
        with pytest.raises(lbm.LbmError):
            g.set_launch(*shape)  # FP64: (8, 0) only
    g.set_launch(8, 0).set_launch(0, 0)
    g.close()
    g = Lbm3d(dict(p, precision=lbm.LBM_P_FP32))
    for shape in [(4, 0), (16, 1), (8, 2), (12, 0)]:
        with pytest.raises(lbm.LbmError):
            g.set_launch(*shape)
    g.close()


def test_conservation_3d_gpu():
    p, f = _case((37, 11, 9), "total_zfull_corr", lbm.LBM_P_FP64)
    g = Lbm3d(p).init(*f)
    c0 = g.conserved()
    g.step(200)
    c1 = g.conserved()
    assert np.abs(c1 - c0).max() <= 1e-12 * np.abs(c0).max()
    g.close()


def test_bench_box_sampled_against_oracle_3d():
    """The 3-D bench workload's recipe (periodic box, seed 2) at 64^3 in FP64
    over 20 steps, the same launch shape logic as the 256^3 bench box."""
    p, f = inputs.periodic_box3d(n=64, precision=lbm.LBM_P_FP64)
    o = o3.Oracle3d(p).init(*f).step(20, threads=8)
    g = Lbm3d(p).init(*f).step(20)
    assert _rel(g.pops(), o.pops()) <= 1e-12
    g.close()


def test_bench_box_full_size_3d():
    """The 256^3 bench box in its launch shape (too large for the oracle):
    FP32 against the FP64 CUDA path (held to 1e-12 of the oracle above) after
    5 steps, and mass, momentum and total energy conserved at full size."""
    p64, f = inputs.periodic_box3d(n=256, precision=lbm.LBM_P_FP64)
    g64 = Lbm3d(p64).init(*f).step(5)
    ref = g64.pops()
    g64.close()
    g32 = Lbm3d(dict(p64, precision=lbm.LBM_P_FP32)).init(*f)
    c0 = g32.conserved()
    g32.step(5)
    c1 = g32.conserved()
    assert _rel(g32.pops(), ref) <= 2e-6
    # FP32 storage: the sums move by its rounding only (16.7 M nodes)
    assert abs(c1[0] - c0[0]) <= 1e-6 * c0[0]
    assert abs(c1[4] - c0[4]) <= 1e-6 * c0[4]
    g32.close()


WALLS = {
    "iso_moving": dict(bc_z=[1, 1], u_wall_z=[[0.0, 0.0, 0.0], [0.05, -0.02, 0.0]],
                       T_wall_z=[1.03, 0.98]),
    "adiabatic": dict(bc_z=[2, 2], u_wall_z=[[0.01, 0.0, 0.0], [0.0, 0.0, 0.0]]),
    "iso_adia": dict(bc_z=[1, 2], T_wall_z=[1.04, 1.0]),
}


@pytest.mark.parametrize("walls", list(WALLS))
@pytest.mark.parametrize("mode", ["total_zfull_corr", "internal_corr", "total"])
@pytest.mark.parametrize("shape", [(4, 3, 5), (37, 11, 9)], ids=["4x3x5", "37x11x9"])
def test_fp64_parity_3d_walls(shape, mode, walls):
    p, f = _case(shape, mode, lbm.LBM_P_FP64)
    p.update(WALLS[walls])
    o = o3.Oracle3d(p).init(*f).step(30)
    g = Lbm3d(p).init(*f).step(30)
    assert _rel(g.pops(), o.pops()) <= 1e-12
    g.close()


@pytest.mark.parametrize("shape", SHAPES, ids=[f"{a}x{b}" for a, b in SHAPES])
def test_fp32_parity_3d_walls(shape):
    p, f = _case((37, 21, 9), "total_zfull_corr", lbm.LBM_P_FP32)
    p.update(WALLS["iso_moving"])
    o = o3.Oracle3d(dict(p, precision=lbm.LBM_P_FP64)).init(*f).step(30)
    g = Lbm3d(p).set_launch(*shape).init(*f).step(30)
    assert _rel(g.pops(), o.pops()) <= 2e-5
    g.close()


def test_fp64_parity_3d_walls_long():
    """400 steps with a fast moving wall and several z ranges per column of
    blocks: the wall planes meet block boundaries and the x-y tile edges."""
    p, f = _case((33, 9, 40), "total_zfull_corr", lbm.LBM_P_FP64)
    # b = 5: with b = 3 the D3Q19 h^eq loses positivity where theta > 1 and
    # this flow overflows in the oracle too
    p.update(b=5.0, bc_z=[1, 2], u_wall_z=[[0.0, 0.0, 0.0], [0.2, 0.1, 0.0]],
             T_wall_z=[1.05, 1.0])
    o = o3.Oracle3d(p).init(*f).step(400, threads=8)
    g = Lbm3d(p).init(*f).step(400)
    # FP64 rounding, grown over 400 steps
    assert _rel(g.pops(), o.pops()) <= 1e-11
    g.close()


def test_couette_3d_gpu_closed_form():
    """The 3-D thermal Couette flow on the GPU (FP64): flow in x between the
    z walls, the top moving; u linear and the viscous-heating parabola (a
    4 x 4 cross-section seeded with 1e-10 noise at Pr = 1, where the BGK step
    damps modes oblique to z)."""
    H, U, nu, Pr, b = 16, 1.0 / 3.0, 0.2, 1.0, 5.0
    tau_f = nu / inputs.RT0
    p = inputs.base_params3d(4, 4, H, tau_f=tau_f, tau_h=tau_f / Pr, b=b,
                             bc_z=[1, 1], u_wall_z=[[0.0, 0.0, 0.0], [U, 0.0, 0.0]])
    g = Lbm3d(p).init(*inputs.uniform_fields3d(4, 4, H, seed=0, u_amp=1e-10)).step(6000)
    rho, ux, uy, uz, T = g.moments()
    g.close()
    eta = (np.arange(H) + 0.5) / H
    assert np.abs(ux[:, 0, 0] - U * eta).max() < 1.5e-3 * U
    assert np.abs(uz).max() < 1e-10 and np.abs(uy).max() < 1e-10
    rise = Pr * U * U / ((b + 2) * inputs.RT0) * eta * (1 - eta)
    assert np.abs((T[:, 0, 0] - 1) - rise).max() < 0.02 * rise.max()


@pytest.mark.parametrize("precision", [lbm.LBM_P_FP64, lbm.LBM_P_FP32], ids=["fp64", "fp32"])
def test_couette_3d_gpu_adiabatic_moving_wall(precision):
    """Bottom wall at rest and T0, top wall moving and adiabatic: its work
    enters the gas, no heat crosses it, and the heating follows
    theta - 1 = Pr U^2 / ((b + 2) R T0) (2 eta - eta^2) (0.1 % in the
    oracle at H = 16)."""
    H, U, nu, Pr, b = 16, 0.2, 0.2, 1.0, 5.0
    tau_f = nu / inputs.RT0
    p = inputs.base_params3d(2, 2, H, tau_f=tau_f, tau_h=tau_f / Pr, b=b, precision=precision,
                             bc_z=[1, 2], u_wall_z=[[0.0, 0.0, 0.0], [U, 0.0, 0.0]])
    g = Lbm3d(p).init(*inputs.uniform_fields3d(2, 2, H, seed=0)).step(8000)
    rho, ux, uy, uz, T = g.moments()
    g.close()
    eta = (np.arange(H) + 0.5) / H
    assert np.abs(ux[:, 0, 0] - U * eta).max() < 2e-4 * U
    rise = Pr * U * U / ((b + 2) * inputs.RT0) * (2 * eta - eta * eta)
    assert np.abs((T[:, 0, 0] - 1) - rise).max() < 2e-3 * rise.max()


GRAVITY = {
    "periodic_corr": dict(energy_model=inputs.E_INTERNAL, b=5.0, g=2e-3),
    "periodic": dict(energy_model=inputs.E_INTERNAL, b=5.0, g=2e-3, correction=0),
    "iso_walls_corr": dict(energy_model=inputs.E_INTERNAL, b=5.0, g=2e-3, bc_z=[1, 1],
                           T_wall_z=[1.04, 0.97], u_wall_z=[[0.0, 0.0, 0.0], [0.03, 0.0, 0.0]]),
    "iso_adiabatic": dict(energy_model=inputs.E_INTERNAL, b=5.0, g=2e-3, bc_z=[1, 2],
                          T_wall_z=[1.04, 1.0]),
}


@pytest.mark.parametrize("case", list(GRAVITY))
@pytest.mark.parametrize("shape", [(4, 3, 5), (37, 11, 9)], ids=["4x3x5", "37x11x9"])
def test_fp64_parity_3d_gravity(shape, case):
    p, f = _case(shape, "internal", lbm.LBM_P_FP64)
    p.update(GRAVITY[case])
    o = o3.Oracle3d(p).init(*f).step(30)
    g = Lbm3d(p).init(*f).step(30)
    assert _rel(g.pops(), o.pops()) <= 1e-12
    for got, want in zip(g.moments(), o.moments()):
        assert np.abs(got - want).max() <= 1e-12 * max(np.abs(want).max(), 1e-3)
    g.close()


@pytest.mark.parametrize("shape", SHAPES, ids=[f"{a}x{b}" for a, b in SHAPES])
def test_fp32_parity_3d_gravity(shape):
    p, f = _case((37, 21, 9), "internal", lbm.LBM_P_FP32)
    p.update(GRAVITY["iso_walls_corr"])
    o = o3.Oracle3d(dict(p, precision=lbm.LBM_P_FP64)).init(*f).step(30)
    g = Lbm3d(p).set_launch(*shape).init(*f).step(30)
    assert _rel(g.pops(), o.pops()) <= 2e-5
    g.close()


def test_gravity_validation_3d():
    p, f = _case((8, 8, 8), "total_zfull_corr", lbm.LBM_P_FP64)
    for bad in (dict(g=1e-3), dict(g=float("nan"), energy_model=inputs.E_INTERNAL)):
        with pytest.raises(lbm.LbmError):
            Lbm3d(dict(p, **bad))


def test_rayleigh_benard_onset_3d_gpu():
    """The Rayleigh-Benard layer of test_oracle_convection.py on the D3Q19
    path (FP64; rolls along y, two nodes deep; H = 32, dT/T0 = 0.05,
    g H / (R T0) = 0.056): growth rates at 0.95, 1.0 and 1.05 Ra_c
    interpolate the onset within 1.5 % of Ra_c = 1707.76 (measured 1.0073;
    1.0014 at H = 64)."""
    import math

    H, ny, dT, tau_f, Pr = 32, 2, 0.05, 0.06, 0.71
    nx, nu = 2 * H, tau_f * inputs.RT0
    chi = nu / Pr
    rates = {}
    for ratio in (0.95, 1.0, 1.05):
        grav = ratio * 1707.76 * nu * chi / (dT * H ** 3)
        p = inputs.base_params3d(nx, ny, H, tau_f=tau_f, tau_h=tau_f / Pr, b=5.0, g=grav,
                                 energy_model=inputs.E_INTERNAL, bc_z=[1, 1],
                                 T_wall_z=[1 + dT / 2, 1 - dT / 2])
        z = (np.arange(H) + 0.5) / H
        x = np.arange(nx)
        T = ((1 + dT / 2 - dT * z)[:, None, None] + 1e-3 * dT * np.sin(math.pi * z)[:, None, None]
             * np.sin(2 * math.pi * x / nx)[None, None, :]) * np.ones((H, ny, nx))
        rho = np.exp(-3 * grav * (np.arange(H) - H / 2))[:, None, None] * np.ones((H, ny, nx))
        g = Lbm3d(p).init(rho, 0.0, 0.0, 0.0, T)
        steps, chunks = int(2.5 * H * H / chi), 40
        E = []
        for _ in range(chunks):
            g.step(steps // chunks)
            E.append(float((g.moments()[3] ** 2).sum()))
        g.close()
        t = (np.arange(chunks) + 1) * (steps // chunks)
        rates[ratio] = np.polyfit(t[chunks // 2:], 0.5 * np.log(E[chunks // 2:]), 1)[0] * H * H / chi
    r = sorted(rates)
    slope, icpt = np.polyfit(r, [rates[k] for k in r], 1)
    assert slope > 0 and abs(-icpt / slope - 1.0) < 0.015, rates


# walls on the x and y sides too (a population leaving through an edge of
# two walled sides takes the first of x, y, z, as in the oracle)
WALLS_XY = {
    "x_iso_moving": dict(bc_x=[1, 1], T_wall_x=[1.03, 0.98],
                         u_wall_x=[[0.0, 0.02, 0.0], [0.0, -0.01, 0.03]]),
    "y_adiabatic": dict(bc_y=[2, 2], u_wall_y=[[0.01, 0.0, 0.0], [0.0, 0.0, 0.02]]),
    "x_y_mixed": dict(bc_x=[2, 2], bc_y=[1, 1], T_wall_y=[1.04, 0.99],
                      u_wall_y=[[0.0, 0.0, 0.0], [0.03, 0.0, 0.0]]),
    "box": dict(bc_x=[1, 2], T_wall_x=[1.03, 1.0], bc_y=[2, 1], T_wall_y=[1.0, 0.97],
                bc_z=[1, 1], T_wall_z=[1.02, 0.99],
                u_wall_z=[[0.0, 0.0, 0.0], [0.04, -0.02, 0.0]]),
}


@pytest.mark.parametrize("walls", list(WALLS_XY))
@pytest.mark.parametrize("mode", ["total_zfull_corr", "internal_corr", "total"])
@pytest.mark.parametrize("shape", [(4, 3, 5), (37, 11, 9), (33, 9, 12)],
                         ids=["4x3x5", "37x11x9", "33x9x12"])
def test_fp64_parity_3d_walls_xy(shape, mode, walls):
    p, f = _case(shape, mode, lbm.LBM_P_FP64)
    p.update(WALLS_XY[walls])
    o = o3.Oracle3d(p).init(*f).step(30)
    g = Lbm3d(p).init(*f).step(30)
    assert _rel(g.pops(), o.pops()) <= 1e-12
    for got, want in zip(g.moments(), o.moments()):
        assert np.abs(got - want).max() <= 1e-12 * max(np.abs(want).max(), 1e-3)
    g.close()


@pytest.mark.parametrize("shape", SHAPES, ids=[f"{a}x{b}" for a, b in SHAPES])
@pytest.mark.parametrize("walls", ["box", "x_y_mixed"])
def test_fp32_parity_3d_walls_xy(shape, walls):
    """Every FP32 launch shape with walls on the tile edges: 37 x 21 leaves
    ragged tiles on the x+ and y+ sides."""
    p, f = _case((37, 21, 9), "total_zfull_corr", lbm.LBM_P_FP32)
    p.update(WALLS_XY[walls])
    o = o3.Oracle3d(dict(p, precision=lbm.LBM_P_FP64)).init(*f).step(30)
    g = Lbm3d(p).set_launch(*shape).init(*f).step(30)
    assert _rel(g.pops(), o.pops()) <= 2e-5
    g.close()


@pytest.mark.parametrize("shape", [(4, 3, 5), (37, 11, 9)], ids=["4x3x5", "37x11x9"])
def test_fp64_parity_3d_gravity_box(shape):
    """Gravity along -z in a box walled on every side (the isothermal x and y
    walls carry no hydrostatic drop: their normal is horizontal)."""
    p, f = _case(shape, "internal", lbm.LBM_P_FP64)
    p.update(GRAVITY["iso_walls_corr"])
    p.update(bc_x=[1, 1], T_wall_x=[1.02, 0.99], bc_y=[2, 2])
    o = o3.Oracle3d(p).init(*f).step(30)
    g = Lbm3d(p).init(*f).step(30)
    assert _rel(g.pops(), o.pops()) <= 1e-12
    g.close()


def test_fp64_parity_3d_box_long():
    """400 steps in a box walled on every side with a fast lid and several z
    ranges per column of blocks (the walls meet the blocks' edges in x, y
    and z)."""
    p, f = _case((33, 9, 40), "total_zfull_corr", lbm.LBM_P_FP64)
    p.update(b=5.0, bc_x=[1, 2], T_wall_x=[1.04, 1.0], bc_y=[2, 2],
             bc_z=[1, 2], u_wall_z=[[0.0, 0.0, 0.0], [0.2, 0.1, 0.0]], T_wall_z=[1.05, 1.0])
    o = o3.Oracle3d(p).init(*f).step(400, threads=8)
    g = Lbm3d(p).init(*f).step(400)
    assert _rel(g.pops(), o.pops()) <= 1e-11
    g.close()


@pytest.mark.parametrize("precision", [lbm.LBM_P_FP64, lbm.LBM_P_FP32], ids=["fp64", "fp32"])
def test_closed_adiabatic_box_conserves_3d_gpu(precision):
    """Six adiabatic walls at rest: no mass and no energy cross them, so the
    sums of rho and of hbar stay at their initial values (FP64 to rounding;
    FP32 storage to its rounding over the grid)."""
    p, f = _case((37, 21, 9), "total_zfull_corr", precision)
    p.update(bc_x=[2, 2], bc_y=[2, 2], bc_z=[2, 2])
    g = Lbm3d(p).init(*f)
    c0 = g.conserved()
    g.step(300)
    c1 = g.conserved()
    tol = 1e-12 if precision == lbm.LBM_P_FP64 else 2e-6
    assert abs(c1[0] - c0[0]) <= tol * c0[0]
    assert abs(c1[4] - c0[4]) <= tol * c0[4]
    g.close()


def test_side_validation_3d():
    p, f = _case((8, 8, 8), "total", lbm.LBM_P_FP64)
    for bad in (dict(bc_x=[1, 0]), dict(bc_y=[0, 2]), dict(bc_x=[3, 3]),
                dict(bc_y=[1, 1], T_wall_y=[1.0, 0.0]),
                dict(bc_x=[2, 2], u_wall_x=[[0.0, float("inf"), 0.0], [0.0, 0.0, 0.0]])):
        with pytest.raises(lbm.LbmError):
            Lbm3d(dict(p, **bad))
    # an adiabatic side needs no temperature
    Lbm3d(dict(p, bc_x=[2, 2], T_wall_x=[0.0, 0.0])).close()


DEGENERATE = [(1, 4, 3), (3, 1, 4), (2, 3, 1), (1, 1, 1), (1, 1, 5)]


@pytest.mark.parametrize("walls", ["box", "x_y_mixed"])
@pytest.mark.parametrize("mode", ["total_zfull_corr", "internal_corr"])
@pytest.mark.parametrize("shape", DEGENERATE, ids=["x".join(map(str, s)) for s in DEGENERATE])
def test_fp64_parity_3d_walls_degenerate(shape, mode, walls):
    """Axes one node thick: both walls of an axis act on the same node (its
    leaving populations bounce off either side, Eq. 50 takes both mirror
    ghosts), and a one-plane periodic axis wraps onto itself."""
    p, f = _case(shape, mode, lbm.LBM_P_FP64)
    p.update(WALLS_XY[walls])
    o = o3.Oracle3d(p).init(*f).step(30)
    g = Lbm3d(p).init(*f).step(30)
    assert _rel(g.pops(), o.pops()) <= 1e-12
    g.close()
