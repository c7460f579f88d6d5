"""Pins of the correction term (Eqs. 26, 28, 48, 49) and the Guo forcing term
(text above Eq. 51) against the paper's constraints and its Appendix B
transformation matrices."""
import numpy as np
import pytest

from oracle import oracle as orc

EX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1], float)
EY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1], float)
RT0 = 1.0 / 3.0

# Eq. B1, typed from the paper (rows: rho, e, eps, jx, qx, jy, qy, pxx, pxy).
M = np.array([
    [1, 1, 1, 1, 1, 1, 1, 1, 1],
    [-4, -1, -1, -1, -1, 2, 2, 2, 2],
    [4, -2, -2, -2, -2, 1, 1, 1, 1],
    [0, 1, 0, -1, 0, 1, -1, -1, 1],
    [0, -2, 0, 2, 0, 1, -1, -1, 1],
    [0, 0, 1, 0, -1, 1, 1, -1, -1],
    [0, 0, -2, 0, 2, 1, 1, -1, -1],
    [0, 1, -1, 1, -1, 0, 0, 0, 0],
    [0, 0, 0, 0, 0, 1, -1, 1, -1],
], float)

# Eq. B2, typed from the paper.
_a, _b, _c, _d, _e, _f = 1 / 9, 1 / 36, 1 / 18, 1 / 6, 1 / 12, 1 / 4
MINV = np.array([
    [_a, -_a, _a, 0, 0, 0, 0, 0, 0],
    [_a, -_b, -_c, _d, -_d, 0, 0, _f, 0],
    [_a, -_b, -_c, 0, 0, _d, -_d, -_f, 0],
    [_a, -_b, -_c, -_d, _d, 0, 0, _f, 0],
    [_a, -_b, -_c, 0, 0, -_d, _d, -_f, 0],
    [_a, _c, _b, _d, _e, _d, _e, 0, _f],
    [_a, _c, _b, -_d, -_e, _d, _e, 0, -_f],
    [_a, _c, _b, -_d, -_e, -_d, -_e, 0, _f],
    [_a, _c, _b, _d, _e, -_d, -_e, 0, -_f],
])


def test_appendix_b_matrices_are_inverse():
    np.testing.assert_allclose(M @ MINV, np.eye(9), atol=1e-15)


def test_rows_of_M_match_velocity_set():
    """Row 0 is 1, rows 3 and 5 are e_x and e_y (Eq. 6 ordering)."""
    np.testing.assert_array_equal(M[3], EX)
    np.testing.assert_array_equal(M[5], EY)


def qcases(n=30, seed=21):
    rng = np.random.default_rng(seed)
    return [tuple(rng.normal(0, 0.05, 2)) for _ in range(n)]


@pytest.mark.parametrize("dqx,dqy", qcases())
def test_correction_constraints_eq26_eq28(dqx, dqy):
    C = orc.correction(dqx, dqy)
    assert abs(C.sum()) < 1e-16
    assert abs(EX @ C) < 1e-16 and abs(EY @ C) < 1e-16
    assert abs((EX * EY) @ C) < 1e-16
    assert np.isclose((EX * EX) @ C, dqx, rtol=1e-14, atol=1e-17)
    assert np.isclose((EY * EY) @ C, dqy, rtol=1e-14, atol=1e-17)


@pytest.mark.parametrize("dqx,dqy", qcases(seed=22))
def test_correction_is_minv_of_moment_space_eq48(dqx, dqy):
    """C = M^-1 C_hat with C_hat = (0, phi_x, 0, 0, 0, 0, 0, phi_y, 0) (Eq. 48)."""
    phx, phy = 3 * (dqx + dqy), dqx - dqy
    Chat = np.array([0, phx, 0, 0, 0, 0, 0, phy, 0])
    C = orc.correction(dqx, dqy)
    np.testing.assert_allclose(C, np.linalg.solve(M, Chat), atol=1e-17)
    np.testing.assert_allclose(M @ C, Chat, atol=1e-16)


def fcases(n=30, seed=23):
    rng = np.random.default_rng(seed)
    return [tuple(rng.uniform(-0.2, 0.2, 4)) for _ in range(n)]


@pytest.mark.parametrize("ux,uy,ax,ay", fcases())
def test_force_moments(ux, uy, ax, ay):
    """Guo forcing: zeroth moment 0, first moment a, second moment u a + a u."""
    F = orc.force(RT0, ux, uy, ax, ay)
    assert abs(F.sum()) < 1e-16
    np.testing.assert_allclose([EX @ F, EY @ F], [ax, ay], atol=1e-16)
    second = np.array([[(EX * EX) @ F, (EX * EY) @ F], [(EY * EX) @ F, (EY * EY) @ F]])
    u, a = np.array([ux, uy]), np.array([ax, ay])
    np.testing.assert_allclose(second, np.outer(u, a) + np.outer(a, u), atol=1e-16)


@pytest.mark.parametrize("ux,uy,ax,ay", fcases(seed=24))
def test_force_moment_space_eq51(ux, uy, ax, ay):
    """Eq. 51 with its seventh entry read as 2 (u_x a_x - u_y a_y) (the
    printed 2 (u_x a_x - u_x a_y) is not symmetric under x <-> y)."""
    F = orc.force(RT0, ux, uy, ax, ay)
    ua = ux * ax + uy * ay
    Fhat = np.array([0, 6 * ua, -6 * ua, ax, -ax, ay, -ay, 2 * (ux * ax - uy * ay),
                     ux * ay + uy * ax])
    np.testing.assert_allclose(M @ F, Fhat, atol=1e-15)
