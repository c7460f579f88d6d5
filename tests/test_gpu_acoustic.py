"""Open x sides (inlet of Eq. 53, zero-gradient outlet) on the CUDA path:
parity with the oracle in every kernel family, precision, and in a batch;
resume with the step count; and the attenuation-driven acoustic streaming of
Sec. IV.B against Eq. 56 in FP32 and 16-bit storage."""
import math

import numpy as np
import pytest

from oracle import oracle as orc
from paper_1109_6672_gb300 import inputs
from paper_1109_6672_gb300 import lbm
from test_gpu_parity import rel
from test_oracle_acoustic import analyse, envelope, eq56_beta

pytestmark = pytest.mark.gpu

# launch shapes: pulled-row TMA kernel (one and two nodes per thread, BGK
# constant tau only for two) and the register-pull kernel
LAUNCHES = [None, (1, 3), (2, 5), (96, 4)]


def noisy_channel(precision, em=inputs.E_TOTAL, coll=lbm.LBM_COLL_BGK, nx=157, ny=13, seed=7,
                  **kw):
    """A 2-D channel with both open sides, a moving inlet mean and noise in
    every field (the correction term off: open sides need it off)."""
    p = inputs.base_params(nx, ny, bc=[inputs.INLET, inputs.OUTLET, inputs.PERIODIC,
                                       inputs.PERIODIC],
                           tau_f=0.35, tau_h=0.5, b=3.0 if em == inputs.E_TOTAL else 5.0,
                           energy_model=em, precision=precision, collision=coll,
                           s_q=1.5 if coll == lbm.LBM_COLL_MRT else 0.0,
                           u_wall=[[0.01, 0.003], [0, 0], [0, 0], [0, 0]],
                           T_wall=[1.04, 1.0, 1.0, 1.0], in_rho=1.01, in_drho=0.02, in_du=0.015,
                           in_dT=0.03, in_omega=0.21, correction=0, **kw)
    if em == inputs.E_INTERNAL:
        p["g"] = 2e-5
    fields = inputs.uniform_fields(nx, ny, seed=seed, u_amp=0.02, T_amp=0.03, rho_amp=0.02)
    return p, fields


@pytest.mark.parametrize("launch", LAUNCHES)
@pytest.mark.parametrize("case", ["total_bgk", "internal_gravity", "total_mrt"])
def test_open_sides_fp64_parity(case, launch):
    em = inputs.E_INTERNAL if case == "internal_gravity" else inputs.E_TOTAL
    coll = lbm.LBM_COLL_MRT if case == "total_mrt" else lbm.LBM_COLL_BGK
    if coll == lbm.LBM_COLL_MRT and launch is not None and launch[0] == 2:
        pytest.skip("two nodes per thread: BGK with constant tau only")
    p, fields = noisy_channel(lbm.LBM_P_FP64, em, coll)
    o = orc.Oracle(p).init(*fields).step(80)
    g = lbm.Lbm(p)
    if launch:
        g.set_launch(*launch)
    g.init(*fields).step(80)
    assert rel(g.pops(), o.pops()) <= 1e-12
    assert g.steps_done == o.t == 80
    g.close()


@pytest.mark.parametrize("precision,tol", [(lbm.LBM_P_FP32, 2e-5), (lbm.LBM_P_FP32_FP16, 2e-3),
                                           (lbm.LBM_P_FP32_BF16, 1.5e-2)])
def test_open_sides_reduced_precision(precision, tol):
    p, fields = noisy_channel(precision)
    o = orc.Oracle(p).init(*fields).step(50)
    g = lbm.Lbm(p).init(*fields).step(50)
    assert rel(g.pops(), o.pops()) <= tol
    g.close()


def test_acoustic_channel_fp64_parity_full_size():
    """The paper's 600 x 4 channel (Pr = 0.5, gamma = 5/3) for 400 steps."""
    p, fields = inputs.acoustic_channel(Pr=0.5)
    o = orc.Oracle(p).init(*fields).step(400, threads=4)
    g = lbm.Lbm(p).init(*fields).step(400)
    assert rel(g.pops(), o.pops()) <= 1e-12
    g.close()


def test_open_sides_in_a_batch():
    grids = [noisy_channel(lbm.LBM_P_FP64, seed=s, nx=nx)
             for s, nx in ((1, 157), (2, 70), (3, 300))]
    p, fields = inputs.acoustic_channel(Pr=2.0, gamma=1.4, nx=200)
    grids.append((p, fields))
    b = lbm.Batch(lbm.LBM_P_FP64, len(grids), 1 << 28)
    slots = [b.add(p, f, 35) for p, f in grids]
    b.run(35)
    for (p, f), s in zip(grids, slots):
        assert rel(b.pops(s), orc.Oracle(p).init(*f).step(35).pops()) <= 1e-12
    b.close()


@pytest.mark.parametrize("precision", [lbm.LBM_P_FP64, lbm.LBM_P_FP32_BF16])
def test_open_sides_resume_bitwise(precision):
    """The inlet's phase follows the step count, which lbm_set_steps_done restores."""
    p, fields = noisy_channel(precision)
    straight = lbm.Lbm(p).init(*fields).step(47).pops()
    a = lbm.Lbm(p).init(*fields).step(20)
    b = lbm.Lbm(p).set_pops(a.pops(), steps_done=a.steps_done).step(27)
    np.testing.assert_array_equal(b.pops(), straight)


@pytest.mark.parametrize("Pr,gamma,precision,tol", [
    (0.2, 5 / 3, lbm.LBM_P_FP32, 0.03), (5.0, 5 / 3, lbm.LBM_P_FP32, 0.03),
    (2.0, 9 / 7, lbm.LBM_P_FP32, 0.03), (0.2, 5 / 3, lbm.LBM_P_FP32_BF16, 0.05),
    (2.0, 9 / 7, lbm.LBM_P_FP32_BF16, 0.05)])
def test_acoustic_attenuation_on_gpu(Pr, gamma, precision, tol):
    """Sec. IV.B on the GPU: the amplitude decays at Eq. 56's rate, starts at
    U = c_s drho / rho0 and has the coupled model's wavelength."""
    p, fields = inputs.acoustic_channel(Pr=Pr, gamma=gamma, precision=precision)
    g = lbm.Lbm(p).init(*fields)
    amp, ux = envelope(lambda n: g.step(n), g.moments, p)
    g.close()
    beta, u0, lam = analyse(amp, ux, p)
    assert beta == pytest.approx(eq56_beta(p), rel=tol)
    assert u0 == pytest.approx(1.0, abs=0.02)
    assert lam == pytest.approx(50.0, rel=0.02)
