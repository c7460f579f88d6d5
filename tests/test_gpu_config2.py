"""The small-dT cavity at its configured size and step count: 256 x 256,
dT/T0 = 0.01, Ra = 1e5, Pr = 0.71, noise 1e-4 (seed 1), 50 000 steps, FP64
and FP32.  The FP64 CUDA path matches the oracle to 1e-12 after all 50 000
steps (populations, rho and T relative, u relative to the lattice speed;
u relative to its own maximum to 1e-11);
FP32 stays within the 1e-3 relative T target."""
import os

import numpy as np
import pytest

from oracle import oracle as orc
from paper_1109_6672_gb300 import inputs
from paper_1109_6672_gb300 import lbm

pytestmark = pytest.mark.gpu

STEPS = 50000


def rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


def test_small_dT_cavity_full_run():
    p, f = inputs.cavity(n=256, Ra=1e5, dT_over_T0=0.01, seed=1, precision=lbm.LBM_P_FP64)
    o = orc.Oracle(p).init(*f).step(STEPS, threads=os.cpu_count() or 1)
    g64 = lbm.Lbm(p).init(*f).step(STEPS)
    assert rel(g64.pops(), o.pops()) <= 1e-12
    rho_o, ux_o, uy_o, T_o = o.moments()
    rho, ux, uy, T = g64.moments()
    # velocities relative to the lattice speed c = 1, and relative to the
    # flow's own max |u|: u is 8.6e-3 of c here and comes from differences
    # of populations of order 1, so their rounding shows about 100x larger
    # in that norm (measured 5.0e-14 of c = 5.8e-12 of max |u| after the
    # full run); the gate in that norm is therefore 1e-11, not 1e-12
    du = max(np.abs(ux - ux_o).max(), np.abs(uy - uy_o).max())
    umax = max(np.abs(ux_o).max(), np.abs(uy_o).max())
    print(f"u error after {STEPS} steps: {du:.3e} of c, {du / umax:.3e} of max|u| ({umax:.3e})")
    assert du <= 1e-12
    assert du / umax <= 1e-11
    assert rel(rho, rho_o) <= 1e-12
    assert rel(T, T_o) <= 1e-12
    g64.close()
    g32 = lbm.Lbm(dict(p, precision=lbm.LBM_P_FP32)).init(*f).step(STEPS)
    T32 = g32.moments()[3]
    g32.close()
    # FP32 storage rounds to nearest at every step: in the nearly steady flow
    # those errors repeat and add up (measured 1.5e-4 after 50 000 steps);
    # the bar is the 1e-3 relative T target of the reduced-precision paths
    assert rel(T32, T_o) <= 1e-3
