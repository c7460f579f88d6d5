"""The D3Q19 oracle against the independent NumPy restatement
(tests/brute_lbm3d.py) on tiny noisy grids: every physics mode, periodic and
walled sides (z alone, x alone, all six, with edges and corners).  This is the only check of the -u^2/2 part of Z_a in the
Eq. 36 coupling in 3-D, which no closed form or decay rate can see (the
paper notes that Z_a reduces to e_a.u at the Navier-Stokes level)."""
import numpy as np
import pytest

from oracle import oracle3d as o3
from paper_1109_6672_gb300 import inputs
from brute_lbm3d import Brute3d

CASES = {
    "total_zfull_corr": dict(),
    "total_corr": dict(z_full=0),
    "total_zfull": dict(correction=0),
    "internal_corr": dict(energy_model=inputs.E_INTERNAL),
    "iso_moving_walls": dict(bc_z=[1, 1], u_wall_z=[[0.02, -0.01, 0.0], [0.05, 0.03, 0.0]],
                             T_wall_z=[1.04, 0.97]),
    "adiabatic_moving_walls": dict(bc_z=[2, 2], u_wall_z=[[0.03, 0.0, 0.0], [-0.02, 0.04, 0.0]]),
    "iso_adiabatic_internal": dict(bc_z=[1, 2], energy_model=inputs.E_INTERNAL,
                                   u_wall_z=[[0.0, 0.0, 0.0], [0.04, 0.0, 0.0]],
                                   T_wall_z=[1.05, 1.0]),
    "gravity_walls_internal": dict(bc_z=[1, 1], energy_model=inputs.E_INTERNAL, g=2e-3,
                                   T_wall_z=[1.05, 0.97]),
    "gravity_periodic_internal": dict(energy_model=inputs.E_INTERNAL, g=2e-3, correction=0),
    "x_walls": dict(bc_x=[1, 2], u_wall_x=[[0.0, 0.03, 0.0], [0.0, 0.0, -0.02]],
                    T_wall_x=[1.05, 1.0]),
    "box_all_walls": dict(bc_x=[1, 1], bc_y=[2, 2], bc_z=[1, 2], T_wall_x=[1.04, 0.97],
                          T_wall_z=[1.02, 1.0],
                          u_wall_y=[[0.02, 0.0, 0.0], [0.0, 0.0, 0.03]],
                          u_wall_z=[[0.0, 0.0, 0.0], [0.04, -0.01, 0.0]]),
    "box_internal_gravity": dict(bc_x=[1, 1], bc_y=[2, 2], bc_z=[2, 2], T_wall_x=[1.05, 0.95],
                                 energy_model=inputs.E_INTERNAL, g=2e-3),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_oracle3d_matches_restatement(name):
    p = inputs.base_params3d(5, 4, 6, tau_f=0.35, tau_h=0.5, b=5.0, **CASES[name])
    f = inputs.uniform_fields3d(5, 4, 6, seed=11, u_amp=0.04, T_amp=0.05, rho_amp=0.03)
    o = o3.Oracle3d(p).init(*f)
    b = Brute3d(p).init(*f)
    np.testing.assert_allclose(o.pops(), b.pops(), rtol=1e-14, atol=1e-15)
    for _ in range(3):
        o.step(10)
        b.step(10)
        np.testing.assert_allclose(o.pops(), b.pops(), rtol=1e-12, atol=1e-13)


def test_restatement_sees_the_full_z():
    """The two forms of Z differ by more than the comparison's tolerance
    over these steps, so the comparison above pins the -u^2/2 part."""
    p = inputs.base_params3d(5, 4, 6, tau_f=0.35, tau_h=0.5, b=5.0)
    f = inputs.uniform_fields3d(5, 4, 6, seed=11, u_amp=0.04, T_amp=0.05, rho_amp=0.03)
    a = Brute3d(p).init(*f).step(30).pops()
    c = Brute3d(dict(p, z_full=0)).init(*f).step(30).pops()
    assert np.abs(a - c).max() > 1e3 * 1e-13 * np.abs(a).max()
