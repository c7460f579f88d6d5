"""The large-temperature-difference cavity of Sec. IV.C on the CUDA path
(T_h = 960 K, T_l = 240 K, Sutherland's law, MRT, correction on, internal
energy, the paper's walls of non-equilibrium extrapolation): parity with the
oracle at theta from 0.4 to 1.6, and the paper's
grid for Ra = 1e4 run to steady state, where the primary vortex
centre lies right of and below the cavity centre (the paper's description of
Figs. 7-8)."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1109_6672_gb300 import inputs
from paper_1109_6672_gb300 import lbm
from test_gpu_parity import rel

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision,tol", [(lbm.LBM_P_FP64, 1e-12), (lbm.LBM_P_FP32, 5e-5)])
def test_large_dt_cavity_parity(precision, tol):
    p, f = inputs.cavity_large_dT(Ra=1e5, n=48, precision=precision)
    o = orc.Oracle(p).init(*f).step(300, threads=4)
    g = lbm.Lbm(p).init(*f).step(300)
    assert rel(g.pops(), o.pops()) <= tol
    g.close()


@pytest.mark.parametrize("Ra", [1e4])
def test_large_dt_cavity_vortex_shift(Ra):
    p, f = inputs.cavity_large_dT(Ra=Ra, precision=lbm.LBM_P_FP32)
    n = p["nx"]
    # the vortex structure settles within 60 000 steps; the walls of
    # non-equilibrium extrapolation keep leaking a little mass (a known
    # property of the method), so there is no strict steady state to wait for
    g = lbm.Lbm(p).init(*f).step(100000)
    rho, ux, uy, T = g.moments()
    g.close()
    assert np.isfinite(T).all() and 0.39 < T.min() and T.max() < 1.61
    psi = np.cumsum(rho * ux, axis=0)
    j, i = np.unravel_index(np.argmax(np.abs(psi)), psi.shape)
    # walls on the ghost nodes: node i at i + 1 of n + 1 spacings
    assert (i + 1.0) / (n + 1) > 0.55 and (j + 1.0) / (n + 1) < 0.45
