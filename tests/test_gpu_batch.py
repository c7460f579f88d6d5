"""Batched grids (lbm_batch_*): parity with the oracle and with the
single-grid path, independence from the other grids in the batch and from the
schedule, admission by pool footprint, budgets, autotuner."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1109_6672_gb300 import inputs
from paper_1109_6672_gb300 import lbm

pytestmark = pytest.mark.gpu

P, ISO, ADI = inputs.PERIODIC, inputs.WALL_ISOTHERMAL, inputs.WALL_ADIABATIC


def rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def mixed_grids(precision):
    """Different sizes, physics modes and boundary conditions."""
    out = []
    p, f = inputs.cavity(n=70, Ra=1e4, dT_over_T0=0.2, precision=precision, seed=5)
    out.append((p, f))
    p, f = inputs.couette(ny=33, nx=4, precision=precision)
    out.append((p, f))
    p = inputs.base_params(300, 41, precision=precision, tau_f=0.35, tau_h=0.5)
    out.append((p, inputs.uniform_fields(300, 41, seed=7, u_amp=0.02, T_amp=0.05, rho_amp=0.02)))
    p = inputs.base_params(131, 29, precision=precision, bc=[ISO, ADI, P, P], T_wall=[1.04, 1, 1, 1],
                           u_wall=[[0, 0.02], [0, -0.01], [0, 0], [0, 0]], tau_f=0.35, tau_h=0.5)
    out.append((p, inputs.uniform_fields(131, 29, seed=8, u_amp=0.02, T_amp=0.03, rho_amp=0.02)))
    p = inputs.base_params(3, 3, precision=precision, bc=[ISO, ISO, ADI, ADI],
                           T_wall=[1.05, 0.95, 1, 1], energy_model=inputs.E_INTERNAL, b=5.0,
                           tau_f=0.35, tau_h=0.5)
    out.append((p, inputs.uniform_fields(3, 3, seed=9, u_amp=0.01, T_amp=0.02)))
    return out


def test_fp64_batch_matches_oracle_with_budgets():
    grids = mixed_grids(lbm.LBM_P_FP64)
    budgets = [45, 30, 60, 17, 52]
    b = lbm.Batch(lbm.LBM_P_FP64, 8, 1 << 30)
    slots = [b.add(p, f, n) for (p, f), n in zip(grids, budgets)]
    for _ in range(4):
        b.run(20)
    for (p, f), n, s in zip(grids, budgets, slots):
        assert b.remaining(s) == 0
        o = orc.Oracle(p).init(*f).step(n)
        assert rel(b.pops(s), o.pops()) <= 1e-12, p["nx"]
    b.close()


def test_batch_result_independent_of_mix_and_schedule():
    grids = mixed_grids(lbm.LBM_P_FP32_BF16)
    alone = lbm.Batch(lbm.LBM_P_FP32_BF16, 2, 1 << 28)
    s0 = alone.add(*grids[0], 40)
    alone.run(40)
    ref = alone.pops(s0)
    alone.close()
    for rows, dyn in ((0, 1), (4, 0), (16, 1), (7, 0)):
        mix = lbm.Batch(lbm.LBM_P_FP32_BF16, 8, 1 << 28)
        mix.set_schedule(rows, dyn)
        others = [mix.add(p, f, 100) for p, f in grids[1:]]
        s = mix.add(*grids[0], 40)
        mix.run(25).run(25)
        np.testing.assert_array_equal(mix.pops(s), ref, err_msg=f"rows {rows} dyn {dyn}")
        mix.close()


def test_fp32_batch_matches_single_grid():
    grids = mixed_grids(lbm.LBM_P_FP32)
    b = lbm.Batch(lbm.LBM_P_FP32, 8, 1 << 28)
    slots = [b.add(p, f, 50) for p, f in grids]
    b.run(50)
    for (p, f), s in zip(grids, slots):
        g = lbm.Lbm(p).init(*f).step(50)
        assert rel(b.pops(s), g.pops()) <= 1e-5
        g.close()
    b.close()


def test_admission_by_footprint_and_slots():
    p, f = inputs.cavity(n=64, precision=lbm.LBM_P_FP32_BF16)
    need = lbm.lbm_state_bytes(p)
    b = lbm.Batch(lbm.LBM_P_FP32_BF16, 3, 2 * need + 1024)
    a0 = b.add(p, f, 10)
    a1 = b.add(p, f, 10)
    with pytest.raises(lbm.LbmError) as e:  # pool full
        b.add(p, f, 10)
    assert e.value.status == lbm.LBM_ERR_OOM
    b.remove(a0)
    a2 = b.add(p, f, 10)  # the freed range is reused
    assert b.info()["grids"] == 2
    with pytest.raises(lbm.LbmError) as e:  # wrong precision
        b.add(dict(p, precision=lbm.LBM_P_FP32), f, 10)
    assert e.value.status == lbm.LBM_ERR_PARAM
    b.close()
    small = lbm.Batch(lbm.LBM_P_FP32_BF16, 1, 4 * need)
    small.add(p, f, 1)
    with pytest.raises(lbm.LbmError) as e:  # no slot
        small.add(p, f, 1)
    assert e.value.status == lbm.LBM_ERR_OOM
    small.close()


def test_autotune_does_not_advance_state():
    grids = mixed_grids(lbm.LBM_P_FP32_BF16)
    b = lbm.Batch(lbm.LBM_P_FP32_BF16, 8, 1 << 28)
    slots = [b.add(p, f, 30) for p, f in grids]
    b.run(10)
    before = [b.pops(s) for s in slots]
    best = b.autotune(3)
    assert best["rows"] in (4, 6, 8, 12, 16, 24) and best["dynamic"] in (0, 1)
    for s, ref in zip(slots, before):
        np.testing.assert_array_equal(b.pops(s), ref)
        assert b.remaining(s) == 20
    b.run(20)
    ref_b = lbm.Batch(lbm.LBM_P_FP32_BF16, 8, 1 << 28)
    ref_slots = [ref_b.add(p, f, 30) for p, f in grids]
    ref_b.run(30)
    for s, rs in zip(slots, ref_slots):
        np.testing.assert_array_equal(b.pops(s), ref_b.pops(rs))
    b.close()
    ref_b.close()
