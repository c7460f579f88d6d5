"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Tolerances (max |gpu - oracle| / max |oracle| per compared array):
* FP64 path: 1e-12 (the spec bar).  Both sides compute the same
  formulas in FP64; they differ only in rounding order and FMA contraction,
  about 1e-16 per operation, a few hundred operations per node and step.
* FP32 path: 2e-5 on populations after 50 steps: FP32 rounding (6e-8 relative
  per operation) accumulated over the same operation count and steps.
* 16-bit deviation storage: bounded by the storage quantum of the deviations
  (2^-11 relative for FP16, 2^-8 for BF16) times the deviation scale.
"""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1109_6672_gb300 import inputs
from paper_1109_6672_gb300 import lbm

pytestmark = pytest.mark.gpu

P, ISO, ADI = inputs.PERIODIC, inputs.WALL_ISOTHERMAL, inputs.WALL_ADIABATIC


def rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


CASES = {
    # name: (params overrides, field amplitudes, steps)
    "periodic_total": (dict(nx=150, ny=41, bc=[P] * 4), (0.03, 0.08, 0.03)),
    "periodic_total_zsimple": (dict(nx=150, ny=41, bc=[P] * 4, z_full=0), (0.03, 0.08, 0.03)),
    "periodic_nocorr": (dict(nx=150, ny=41, bc=[P] * 4, correction=0), (0.03, 0.08, 0.03)),
    "periodic_internal_gravity": (dict(nx=130, ny=45, bc=[P] * 4, energy_model=inputs.E_INTERNAL,
                                       b=5.0, g=2e-4), (0.02, 0.1, 0.02)),
    "couette_walls": (dict(nx=70, ny=33, bc=[P, P, ISO, ISO], T_wall=[1, 1, 1.05, 0.97],
                           u_wall=[[0, 0], [0, 0], [0.02, 0], [0.05, 0.0]]), (0.02, 0.03, 0.02)),
    "adiabatic_walls_moving": (dict(nx=70, ny=33, bc=[P, P, ADI, ADI],
                                    u_wall=[[0, 0], [0, 0], [0.03, 0], [-0.04, 0]]),
                               (0.02, 0.03, 0.02)),
    "cavity": (dict(nx=140, ny=70, bc=[ISO, ISO, ADI, ADI], T_wall=[1.2, 0.8, 1, 1],
                    energy_model=inputs.E_INTERNAL, b=5.0, g=1e-4), (0.01, 0.05, 0.01)),
    "x_walls_y_periodic": (dict(nx=131, ny=29, bc=[ISO, ADI, P, P], T_wall=[1.04, 1, 1, 1],
                                u_wall=[[0, 0.02], [0, -0.01], [0, 0], [0, 0]]),
                           (0.02, 0.03, 0.02)),
    "all_iso_moving": (dict(nx=67, ny=45, bc=[ISO] * 4, T_wall=[1.03, 0.98, 1.02, 0.99],
                            energy_model=inputs.E_INTERNAL, b=5.0,
                            u_wall=[[0, 0.01], [0, -0.02], [0.03, 0], [-0.02, 0.01]]),
                       (0.02, 0.03, 0.02)),
    "gravity_iso_floor_ceiling": (dict(nx=70, ny=33, bc=[P, P, ISO, ISO], T_wall=[1, 1, 1.05, 0.95],
                                       energy_model=inputs.E_INTERNAL, b=5.0, g=1e-3),
                                  (0.02, 0.03, 0.02)),
    "narrow_periodic_4x33": (dict(nx=4, ny=33, bc=[P] * 4), (0.02, 0.05, 0.02)),
    "single_column_1x20": (dict(nx=1, ny=20, bc=[P] * 4), (0.02, 0.05, 0.02)),
    "min_walls_3x3": (dict(nx=3, ny=3, bc=[ISO, ISO, ADI, ADI], T_wall=[1.05, 0.95, 1, 1],
                           energy_model=inputs.E_INTERNAL, b=5.0), (0.01, 0.02, 0.01)),
}


def make_case(name, precision):
    kw, (ua, ta, ra) = CASES[name]
    kw = dict(kw)
    p = inputs.base_params(kw.pop("nx"), kw.pop("ny"), tau_f=0.35, tau_h=0.5,
                           precision=precision, **kw)
    fields = inputs.uniform_fields(p["nx"], p["ny"], seed=len(name) * 7 + 1, u_amp=ua, T_amp=ta,
                                   rho_amp=ra)
    return p, fields


def run_both(name, precision, steps, launch=None):
    p, fields = make_case(name, precision)
    o = orc.Oracle(p).init(*fields).step(steps)
    g = lbm.Lbm(p)
    if launch:
        g.set_launch(*launch)
    g.init(*fields).step(steps)
    return p, o, g


@pytest.mark.parametrize("launch", [None, (1, 3), (2, 0), (2, 5), (64, 7)])
@pytest.mark.parametrize("name", sorted(CASES))
def test_fp64_parity(name, launch):
    p, o, g = run_both(name, lbm.LBM_P_FP64, 60, launch)
    assert rel(g.pops(), o.pops()) <= 1e-12
    mo, mg = o.moments(), g.moments()
    for k in range(4):
        scale = np.abs(mo[k]).max() if k in (0, 3) else max(np.abs(mo[1]).max(), np.abs(mo[2]).max())
        assert np.abs(mg[k] - mo[k]).max() / scale <= 1e-12, k
    np.testing.assert_allclose(g.conserved(), o.conserved(), rtol=1e-12, atol=1e-12)
    g.close()


@pytest.mark.parametrize("launch", [None, (1, 1), (2, 3), (96, 5)])
@pytest.mark.parametrize("name", sorted(CASES))
def test_fp32_parity(name, launch):
    p, o, g = run_both(name, lbm.LBM_P_FP32, 50, launch)
    assert rel(g.pops(), o.pops()) <= 2e-5
    g.close()


@pytest.mark.parametrize("launch", [None, (1, 2), (2, 1), (128, 0)])
@pytest.mark.parametrize("precision,quantum", [(lbm.LBM_P_FP32_FP16, 2.0 ** -11),
                                               (lbm.LBM_P_FP32_BF16, 2.0 ** -8)])
@pytest.mark.parametrize("name", ["periodic_total", "cavity", "couette_walls"])
def test_16bit_deviation_storage(name, precision, quantum, launch):
    p, o, g = run_both(name, precision, 50, launch)
    po, pg = o.pops(), g.pops()
    # reference (rest) equilibria the deviations are taken from
    ref = orc.Oracle(dict(p, nx=1, ny=1, bc=[P] * 4)).init(1.0, 0.0, 0.0, p["T0"]).pops()
    dev_scale = np.abs(po - ref).max()
    # each stored value is rounded once per step; BGK relaxation keeps the
    # accumulated error within a few quanta of the deviation scale
    assert np.abs(pg - po).max() <= 8 * quantum * dev_scale
    g.close()


def test_fp64_long_couette_matches_oracle_and_closed_form():
    """Couette 4 x 33, U = 0.05, Pr = 0.71, 20 000 steps (full configured
    count): FP64 GPU within 1e-12 of the oracle, and of the closed form."""
    p, fields = inputs.couette()
    o = orc.Oracle(p).init(*fields).step(20000)
    g = lbm.Lbm(p).init(*fields).step(20000)
    assert rel(g.pops(), o.pops()) <= 1e-12
    rho, ux, uy, T = g.moments()
    H, U = p["ny"], p["u_wall"][3][0]
    eta = (np.arange(H) + 0.5) / H
    assert np.abs(ux[:, 0] / U - eta).max() < 1e-6
    th_a = 1 + 0.71 * U * U / (5 / 3) * eta * (1 - eta)
    assert np.abs((T[:, 0] - 1) - (th_a - 1)).max() / (th_a - 1).max() < 0.005
    g.close()


@pytest.mark.parametrize("precision", [lbm.LBM_P_FP64, lbm.LBM_P_FP32, lbm.LBM_P_FP32_BF16])
def test_launch_shape_does_not_change_result(precision):
    """Within one kernel the row blocking (and, for the register-pull kernel,
    the block width) does not change a single bit; different kernels compile
    the same formulas with different FMA contraction and order, so they agree
    to rounding."""
    p, fields = make_case("cavity", precision)
    families = {"pr1": [(0, 0), (1, 1), (1, 4), (0, 33), (1, 7)], "pr2": [(2, 0), (2, 9), (2, 1)],
                "ldg": [(64, 1), (128, 3), (256, 0), (192, 17)]}
    results = {}
    for fam, launches in families.items():
        ref = None
        for launch in launches:
            g = lbm.Lbm(p).set_launch(*launch).init(*fields).step(30)
            pops = g.pops()
            g.close()
            if ref is None:
                ref = pops
            else:
                np.testing.assert_array_equal(pops, ref, err_msg=f"{fam} {launch}")
        results[fam] = ref
    tol = {lbm.LBM_P_FP64: 1e-13, lbm.LBM_P_FP32: 1e-5, lbm.LBM_P_FP32_BF16: 1e-2}[precision]
    for fam in ("pr2", "ldg"):
        assert rel(results[fam], results["pr1"]) <= tol, fam


@pytest.mark.parametrize("precision", [lbm.LBM_P_FP64, lbm.LBM_P_FP32, lbm.LBM_P_FP32_FP16,
                                       lbm.LBM_P_FP32_BF16])
def test_checkpoint_resume_bitwise(precision):
    p, fields = make_case("couette_walls", precision)
    straight = lbm.Lbm(p).init(*fields).step(70).pops()
    a = lbm.Lbm(p).init(*fields).step(30)
    snap = a.pops()
    b = lbm.Lbm(p).set_pops(snap, steps_done=a.steps_done).step(40)
    np.testing.assert_array_equal(b.pops(), straight)


def test_errors_are_reported():
    p, fields = make_case("periodic_total", lbm.LBM_P_FP64)
    g = lbm.Lbm(p)
    with pytest.raises(lbm.LbmError) as e:
        g.step(1)
    assert e.value.status == lbm.LBM_ERR_STATE
    with pytest.raises(lbm.LbmError) as e:
        lbm.Lbm(dict(p, tau_f=-1.0))
    assert e.value.status == lbm.LBM_ERR_PARAM
    with pytest.raises(lbm.LbmError) as e:
        lbm.Lbm(dict(p, R=0.5))
    assert e.value.status == lbm.LBM_ERR_PARAM
    g.init(*fields)
    g.step(0)
    assert g.steps_done == 0


def test_nonfinite_is_reported():
    """An unstable parameter set (total-energy h^eq rest weight negative at
    theta = 1.5, b = 3) blows up; lbm_moments reports LBM_ERR_NONFINITE and
    keeps the state."""
    p = inputs.base_params(32, 32, tau_f=0.3, tau_h=0.42)
    fields = inputs.uniform_fields(32, 32, seed=1, u_amp=1e-3, T0=1.5, T_amp=1e-3)
    g = lbm.Lbm(p).init(*fields).step(2000)
    with pytest.raises(lbm.LbmError) as e:
        g.moments()
    assert e.value.status == lbm.LBM_ERR_NONFINITE


@pytest.mark.parametrize("precision", [lbm.LBM_P_FP64, lbm.LBM_P_FP32])
@pytest.mark.parametrize("name", ["cavity", "couette_walls"])
def test_graph_replay_equals_single_launches(name, precision):
    """Long lbm_step calls replay a captured graph of 32 steps; the result is
    the same bit for bit as one launch per call (also across a change of
    launch shape, which drops the graphs, and with walls of non-equilibrium
    extrapolation, whose second pass is captured too)."""
    for extra in ({}, {"wall_nee": 15} if name == "cavity" else {"wall_nee": 12}):
        p, fields = make_case(name, precision)
        p = dict(p, **extra)
        a = lbm.Lbm(p).init(*fields)
        for _ in range(70):
            a.step(1)
        b = lbm.Lbm(p).init(*fields).step(33).step(37)
        np.testing.assert_array_equal(a.pops(), b.pops())
        c = lbm.Lbm(p).init(*fields).step(40).set_launch(1, 3).step(30)
        d = lbm.Lbm(p).init(*fields).step(40).set_launch(1, 3)
        for _ in range(30):
            d.step(1)
        np.testing.assert_array_equal(c.pops(), d.pops())
        for g in (a, b, c, d):
            g.close()


@pytest.mark.parametrize("nee", [False, True], ids=["halfway", "nee"])
@pytest.mark.parametrize("precision", [lbm.LBM_P_FP64, lbm.LBM_P_FP32], ids=["fp64", "fp32"])
def test_couette_adiabatic_moving_wall_gpu(precision, nee):
    """Bottom wall at rest and T0, top wall moving and adiabatic: the wall's
    work enters the gas, no heat crosses it, and the heating follows
    theta - 1 = Pr U^2 / ((b + 2) R T0) (2 eta - eta^2) (halfway walls at
    eta = (y + 1/2) / H: 0.1 % at H = 16 in the oracle; walls of
    non-equilibrium extrapolation on the ghost nodes, eta = (y + 1) / (H + 1):
    exact in the oracle)."""
    H, U, nu, Pr, b = 16, 0.2, 0.2, 1.0, 5.0
    tau_f = nu / inputs.RT0
    p = inputs.base_params(4, H, tau_f=tau_f, tau_h=tau_f / Pr, b=b, precision=precision,
                           bc=[P, P, ISO, ADI], u_wall=[[0, 0], [0, 0], [0, 0], [U, 0]],
                           wall_nee=12 if nee else 0)
    g = lbm.Lbm(p).init(*inputs.uniform_fields(4, H, seed=0)).step(8000)
    rho, ux, uy, T = g.moments()
    g.close()
    eta = (np.arange(H) + 1.0) / (H + 1) if nee else (np.arange(H) + 0.5) / H
    assert np.abs(ux[:, 0] - U * eta).max() < 1e-5 * U
    rise = Pr * U * U / ((b + 2) * inputs.RT0) * (2 * eta - eta * eta)
    # FP32 storage adds about 1e-6 to theta (6e-5 of the rise)
    assert np.abs((T[:, 0] - 1) - rise).max() < (5e-4 if nee else 2e-3) * rise.max()
