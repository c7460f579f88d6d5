"""Pins of the oracle's discrete equilibria against closed forms printed in
arXiv:1109.6672: the moment identities Eq. 19a/19b, the third-moment defect
Eq. 20/21, the theta = 1 reduction to the decoupled Eq. 8, and the
internal-energy form under Eq. 38."""
import numpy as np
import pytest

from oracle import oracle as orc

EX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1], float)
EY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1], float)
E = np.stack([EX, EY])
W = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
RT0 = 1.0 / 3.0


def cases(n=40, seed=11):
    rng = np.random.default_rng(seed)
    for _ in range(n):
        yield (rng.uniform(0.4, 1.6), rng.uniform(-0.3, 0.3), rng.uniform(-0.3, 0.3),
               rng.uniform(0.4, 1.6))


@pytest.mark.parametrize("rho,ux,uy,th", list(cases()))
def test_feq_moments_eq19a(rho, ux, uy, th):
    f = orc.feq(RT0, rho, ux, uy, th)
    u = np.array([ux, uy])
    RT = RT0 * th
    assert np.isclose(f.sum(), rho, rtol=1e-14, atol=1e-15)
    np.testing.assert_allclose(E @ f, rho * u, rtol=1e-13, atol=1e-15)
    second = np.einsum("ia,ja,a->ij", E, E, f)
    np.testing.assert_allclose(second, rho * np.outer(u, u) + rho * RT * np.eye(2), rtol=1e-13,
                               atol=1e-15)


@pytest.mark.parametrize("rho,ux,uy,th", list(cases(seed=12)))
def test_feq_third_moment_eq20(rho, ux, uy, th):
    """Eq. 20: sum f e_i e_j e_k = rho RT (u_k d_ij + u_j d_ik + u_i d_jk)
    + 3 rho RT0 u_l (1 - theta) d_ijkl (diagonal entries carry RT0, Eq. 21)."""
    f = orc.feq(RT0, rho, ux, uy, th)
    u = np.array([ux, uy])
    RT = RT0 * th
    d = np.eye(2)
    third = np.einsum("ia,ja,ka,a->ijk", E, E, E, f)
    want = np.zeros((2, 2, 2))
    for i in range(2):
        for j in range(2):
            for k in range(2):
                want[i, j, k] = rho * RT * (u[k] * d[i, j] + u[j] * d[i, k] + u[i] * d[j, k])
                if i == j == k:
                    want[i, j, k] += 3 * rho * RT0 * u[i] * (1 - th)
    np.testing.assert_allclose(third, want, rtol=1e-13, atol=1e-15)
    # Eq. 21, diagonal: rho RT0 * 3 u_i
    assert np.isclose(third[0, 0, 0], 3 * rho * RT0 * ux, rtol=1e-13, atol=1e-15)


@pytest.mark.parametrize("rho,ux,uy,th", list(cases(seed=13)))
@pytest.mark.parametrize("b", [2.0, 3.0, 5.0])
def test_heq_moments_eq19b(rho, ux, uy, th, b):
    RT = RT0 * th
    usq = ux * ux + uy * uy
    Etot = 0.5 * (b * RT + usq)
    p = rho * RT
    h = orc.heq(RT0, rho, ux, uy, th, Etot)
    u = np.array([ux, uy])
    assert np.isclose(h.sum(), rho * Etot, rtol=1e-13)
    np.testing.assert_allclose(E @ h, (rho * Etot + p) * u, rtol=1e-13, atol=1e-15)
    second = np.einsum("ia,ja,a->ij", E, E, h)
    want = (rho * Etot + 2 * p) * np.outer(u, u) + p * (Etot + RT) * np.eye(2)
    np.testing.assert_allclose(second, want, rtol=1e-13, atol=1e-15)


def decoupled_eq8(rho, ux, uy, Etot):
    """Eq. 8a/8b (Guo et al.'s decoupled model), retyped from the paper."""
    p0 = rho * RT0
    f = np.empty(9)
    h = np.empty(9)
    usq = ux * ux + uy * uy
    for a in range(9):
        eu = EX[a] * ux + EY[a] * uy
        e2 = EX[a] ** 2 + EY[a] ** 2
        f[a] = rho * W[a] * (1 + eu / RT0 + 0.5 * (eu / RT0) ** 2 - usq / (2 * RT0))
    for a in range(9):
        eu = EX[a] * ux + EY[a] * uy
        e2 = EX[a] ** 2 + EY[a] ** 2
        h[a] = Etot * f[a] + W[a] * p0 * (eu / RT0 + (eu / RT0) ** 2 - usq / RT0
                                          + 0.5 * (e2 / RT0 - 2))
    return f, h


@pytest.mark.parametrize("rho,ux,uy,_", list(cases(n=10, seed=14)))
def test_theta_one_reduces_to_eq8(rho, ux, uy, _):
    """Text under Eq. 18: theta = 1, p = p0 gives the decoupled Eq. 8."""
    Etot = 0.5 * (3 * RT0 + ux * ux + uy * uy)
    f = orc.feq(RT0, rho, ux, uy, 1.0)
    h = orc.heq(RT0, rho, ux, uy, 1.0, Etot)
    f8, h8 = decoupled_eq8(rho, ux, uy, Etot)
    np.testing.assert_allclose(f, f8, rtol=1e-14, atol=1e-16)
    np.testing.assert_allclose(h, h8, rtol=1e-14, atol=1e-16)


@pytest.mark.parametrize("rho,ux,uy,th", list(cases(n=10, seed=15)))
def test_internal_energy_equilibrium(rho, ux, uy, th):
    """Text under Eq. 38: h^eq = b R T f^eq / 2, so sum h^eq = rho b R T / 2."""
    b = 5.0
    h = orc.heq_internal(RT0, b, rho, ux, uy, th)
    assert np.isclose(h.sum(), rho * b * RT0 * th / 2, rtol=1e-13)
    f = orc.feq(RT0, rho, ux, uy, th)
    np.testing.assert_allclose(h, 0.5 * b * RT0 * th * f, rtol=1e-14)


def test_rest_state_weights():
    """rho = 1, u = 0, theta = 1: f^eq = w (weights under Eq. 8)."""
    np.testing.assert_allclose(orc.feq(RT0, 1.0, 0.0, 0.0, 1.0), W, rtol=1e-15)
