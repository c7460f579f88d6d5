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


# ---- Eq. 50 at a wall: the ghost Q across the halfway wall -------------------
#
# Eq. 50 is a central difference; the paper does not say what stands for the
# neighbour across a wall.  The oracle reads it as the ghost of a linear
# extrapolation through the wall value, Q_g = 2 Q_w - Q(node), with
# Q_w = rho u_w (1 - theta_w) (Eq. 48's definition of Q at the wall).  What the
# mathematics fixes: for any smooth field whose Q takes the value Q_w at the
# halfway wall, the difference at the boundary node must tend to the true
# derivative as the grid is refined.  A linear ghost makes it exact for linear
# Q and leaves a first-order error (the second derivative over the uneven
# stencil); a zero-gradient ghost, or the mirror's sign flipped, leaves half
# the derivative however fine the grid.  Interior nodes: second order.

def _wall_field(H, axis, moving):
    """Fields on an H-node walled axis (4 periodic nodes across) whose Q along
    that axis is Q(eta) = u(eta) (1 - theta(eta)), rho = 1, eta = (i + 1/2)/H:
    u = u_n + A eta (1 - eta)(1 + 2 eta), theta = theta_w - B (eta - eta^2/2).
    Both walls carry the normal velocity u_n (0, or a transpiring pair), the
    first is isothermal at theta_w and the second adiabatic, where theta has
    no normal slope; so Q takes its wall value Q_w at both walls.  Returns the
    oracle parameters, the fields and Q as a function of eta."""
    from paper_1109_6672_gb300 import inputs

    A, B = 0.02, 0.05
    un = 0.01 if moving else 0.0
    thw = 1.04
    walls = [inputs.WALL_ISOTHERMAL, inputs.WALL_ADIABATIC]
    if axis == 0:
        bc = walls + [inputs.PERIODIC, inputs.PERIODIC]
        nx, ny = H, 4
    else:
        bc = [inputs.PERIODIC, inputs.PERIODIC] + walls
        nx, ny = 4, H
    p = inputs.base_params(nx, ny, bc=bc)
    side0 = 2 * axis  # the isothermal wall at eta = 0
    p["T_wall"] = [1.0] * 4
    p["T_wall"][side0] = thw * p["T0"]
    p["u_wall"] = [[0.0, 0.0] for _ in range(4)]
    p["u_wall"][side0][axis] = un  # a normal wall velocity (transpiring walls)
    p["u_wall"][side0 + 1][axis] = un

    def u(e):
        return un + A * e * (1 - e) * (1 + 2 * e)

    def th(e):
        return thw - B * (e - 0.5 * e * e)

    i = np.arange(H, dtype=float)
    eta = (i + 0.5) / H
    prof_u, prof_t = u(eta), th(eta)
    if axis == 0:
        U = np.broadcast_to(prof_u[None, :], (ny, nx))
        T = np.broadcast_to(prof_t[None, :], (ny, nx))
        fields = (1.0, U, 0.0, T * p["T0"])
    else:
        U = np.broadcast_to(prof_u[:, None], (ny, nx))
        T = np.broadcast_to(prof_t[:, None], (ny, nx))
        fields = (1.0, 0.0, U, T * p["T0"])
    return p, fields, (lambda e: u(e) * (1 - th(e)))


def _wall_gradient_errors(H, axis, moving):
    p, fields, Q = _wall_field(H, axis, moving)
    o = orc.Oracle(p).init(*fields)
    dqx, dqy = o.gradients()
    d = dqx[0, :] if axis == 0 else dqy[:, 0]  # along the walled axis
    i = np.arange(H, dtype=float)
    eta = (i + 0.5) / H
    eps = 1e-6
    exact = (Q(eta + eps) - Q(eta - eps)) / (2 * eps) / H  # dQ/di, one node = 1/H
    scale = np.abs(exact).max()
    first, last = abs(d[0] - exact[0]) / scale, abs(d[-1] - exact[-1]) / scale
    interior = np.abs(d[1:-1] - exact[1:-1]).max() / scale
    return first, last, interior


@pytest.mark.parametrize("axis", [0, 1], ids=["x_walls", "y_walls"])
@pytest.mark.parametrize("moving", [False, True], ids=["still", "transpiring"])
def test_eq50_wall_ghost_is_consistent(axis, moving):
    errs = [_wall_gradient_errors(H, axis, moving) for H in (16, 32, 64, 128)]
    for k in range(3):  # first node, last node, interior
        e = [x[k] for x in errs]
        assert e[-1] < e[0] / 5, f"no convergence at {('first', 'last', 'interior')[k]}: {e}"
    for (f0, l0, _), (f1, l1, _) in zip(errs, errs[1:]):
        # at least first order at the boundary nodes (ratio 2 when H doubles)
        assert f0 / f1 > 1.6 and l0 / l1 > 1.6, errs
    for (_, _, i0), (_, _, i1) in zip(errs, errs[1:]):
        assert 3.0 < i0 / i1 < 4.6, errs  # second order inside
    assert errs[-1][0] < 0.01 and errs[-1][1] < 0.01
