"""Independent NumPy restatement of one step of the D3Q19 extension of the
coupled DDF scheme (arXiv:1109.6672, Sec. III.C.1 with D = 3), used only to
cross-check the C oracle (oracle/lbm3d_oracle.c) on tiny grids.  It is written
separately from the oracle and takes different routes to the same quantities:

* Eq. 18a and Eq. 18b are expanded per speed shell (rest, axis, face
  diagonal) by hand, with R T0 = 1/3, instead of being evaluated from the
  generic Hermite forms;
* the deviation of the third-order moment is written out (D_iii = Q_i,
  D_iik = D_iki = D_kii = Q_k / 6 for i != k, zero with three distinct
  indices, Q = rho u (1 - theta)) instead of being summed over the lattice,
  and the correction's second-moment conditions are solved in closed form
  (A_kk = (G_kk + 4/7 tr G) / 6, A_ij = G_ij / 8, kappa = 10/19) instead of
  by elimination;
* moments are array contractions; streaming is pull-based (np.roll); the
  walls are applied on the pull, node by node from the receiving side;
* gravity along -z: Guo's force term with the half-force velocity shift.
"""
from __future__ import annotations

import numpy as np

# the population order of the C ABI and of the oracle
E = np.array([(0, 0, 0), (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1),
              (1, 1, 0), (-1, -1, 0), (1, -1, 0), (-1, 1, 0), (1, 0, 1), (-1, 0, -1), (1, 0, -1),
              (-1, 0, 1), (0, 1, 1), (0, -1, -1), (0, 1, -1), (0, -1, 1)])
E2 = (E * E).sum(1)
W = np.where(E2 == 0, 1 / 3, np.where(E2 == 1, 1 / 18, 1 / 36))
OPP = np.array([int(np.flatnonzero((E == -e).all(1))[0]) for e in E])
PERIODIC, ISO, ADIA = 0, 1, 2
KAPPA = 10.0 / 19.0


def feq_shells(rho, u, th):
    """Eq. 18a, D = 3, R T0 = 1/3, per shell (u: [3, ...]):
    rest  rho/3  [1 - 3/2 u^2 - 3/2 (th - 1)]
    axis  rho/18 [1 + (6 - 3 th) eu + 9/2 eu^2 - 3/2 u^2]
    diag  rho/36 [1 + (3/2 + 3/2 th) eu + 9/2 eu^2 - 3/2 u^2 + 3/2 (th - 1)]"""
    usq = (u * u).sum(0)
    out = []
    for a in range(19):
        eu = E[a, 0] * u[0] + E[a, 1] * u[1] + E[a, 2] * u[2]
        if E2[a] == 0:
            t = 1 - 1.5 * usq - 1.5 * (th - 1)
        elif E2[a] == 1:
            t = 1 + (6 - 3 * th) * eu + 4.5 * eu * eu - 1.5 * usq
        else:
            t = 1 + (1.5 + 1.5 * th) * eu + 4.5 * eu * eu - 1.5 * usq + 1.5 * (th - 1)
        out.append(rho * W[a] * t)
    return np.array(out)


def heq_total(rho, u, th, b, f):
    """Eq. 18b, D = 3, R T0 = 1/3, per shell: h = E f + w p B with p = rho th / 3,
    E = b th / 6 + u^2 / 2 and
    rest  B = -3 u^2 - 3/2 th
    axis  B = 3 eu + 9 eu^2 - 3 u^2
    diag  B = 3 eu + 9 eu^2 - 3 u^2 + 3/2 th"""
    usq = (u * u).sum(0)
    En = b * th / 6 + 0.5 * usq
    p = rho * th / 3
    out = []
    for a in range(19):
        eu = E[a, 0] * u[0] + E[a, 1] * u[1] + E[a, 2] * u[2]
        if E2[a] == 0:
            B = -3 * usq - 1.5 * th
        elif E2[a] == 1:
            B = 3 * eu + 9 * eu * eu - 3 * usq
        else:
            B = 3 * eu + 9 * eu * eu - 3 * usq + 1.5 * th
        out.append(En * f[a] + W[a] * p * B)
    return np.array(out)


def heq_internal(th, b, f):
    """The internal-energy form under Eq. 38: b R T f / 2 = b th f / 6."""
    return b * th / 6 * f


def correction(dQ):
    """C_a from dQ[k, j] = dQ_j/dx_k (arrays over the grid): G_ij =
    sum_k dD_ijk/dx_k with the D above, then the closed-form A."""
    G = np.zeros((3, 3) + dQ.shape[2:])
    for i in range(3):
        for j in range(3):
            for k in range(3):
                if i == j == k:
                    Dc = dQ[k, i]  # dD_iii/dx_i = dQ_i/dx_i
                elif i == j:
                    Dc = dQ[k, k] / 6 if k != i else 0  # D_iik = Q_k / 6
                elif i == k:
                    Dc = dQ[k, j] / 6  # D_iji = Q_j / 6
                elif j == k:
                    Dc = dQ[k, i] / 6  # D_ijj = Q_i / 6
                else:
                    Dc = 0
                G[i, j] = G[i, j] + Dc
    tr = G[0, 0] + G[1, 1] + G[2, 2]
    A = np.zeros_like(G)
    for i in range(3):
        A[i, i] = (G[i, i] + 4.0 / 7.0 * tr) / 6
        for j in range(3):
            if j != i:
                A[i, j] = 0.5 * (G[i, j] + G[j, i]) / 8
    trA = A[0, 0] + A[1, 1] + A[2, 2]
    C = []
    for a in range(19):
        c = -KAPPA * trA
        for i in range(3):
            for j in range(3):
                c = c + A[i, j] * E[a, i] * E[a, j]
        C.append(c)
    return np.array(C)


class Brute3d:
    """Arrays [nz, ny, nx]; parameters as the oracle's dictionary."""

    def __init__(self, p: dict):
        self.p = dict(p)
        self.shape = (int(p["nz"]), int(p["ny"]), int(p["nx"]))
        self.total = int(p.get("energy_model", 0)) == 0
        # sides 2 axis + (0 low, 1 high), axes x, y, z
        self.bc, self.uw, self.thw = [], [], []
        for ax in "xyz":
            self.bc += list(p.get("bc_" + ax, [PERIODIC, PERIODIC]))
            self.uw += [np.array(v, dtype=float) for v in p.get("u_wall_" + ax, [[0.0] * 3] * 2)]
            self.thw += [float(v) / p["T0"] for v in p.get("T_wall_" + ax, [1.0, 1.0])]

    def _eq(self, rho, u, th):
        f = feq_shells(rho, u, th)
        h = heq_total(rho, u, th, self.p["b"], f) if self.total else heq_internal(th, self.p["b"], f)
        return f, h

    def init(self, rho, ux, uy, uz, T):
        rho, ux, uy, uz, T = [np.broadcast_to(np.asarray(v, float), self.shape).copy()
                              for v in (rho, ux, uy, uz, T)]
        self.F, self.H = self._eq(rho, np.array([ux, uy, uz]), T / self.p["T0"])
        return self

    def moments(self):
        rho = self.F.sum(0)
        j = np.tensordot(E.T.astype(float), self.F, axes=(1, 0))
        j[2] = j[2] - 0.5 * rho * float(self.p.get("g", 0.0))  # half the force a = -rho g e_z
        u = j / rho
        es = self.H.sum(0) / rho
        if self.total:
            th = 6 / self.p["b"] * (es - 0.5 * (u * u).sum(0))
        else:
            th = 6 / self.p["b"] * es
        return rho, u, th

    def pops(self):
        return np.concatenate([self.F, self.H], 0)

    def _grad(self, Q, rho, th):
        """dQ[k, j] = dQ_j / dx_k by central differences; across a wall the
        mirror ghost 2 rho u_w (1 - theta_w) - Q (theta_w: the node's own on
        an adiabatic wall)."""
        dQ = np.zeros((3,) + Q.shape)
        for k in range(3):
            ax = 2 - k  # array axis of x, y, z in [nz, ny, nx]
            up = np.roll(Q, -1, axis=1 + ax)
            dn = np.roll(Q, 1, axis=1 + ax)
            for hi in (0, 1):
                side = 2 * k + hi
                if self.bc[side] == PERIODIC:
                    continue
                sl = [slice(None)] * 3
                sl[ax] = -1 if hi else 0
                sl = tuple(sl)
                thw = self.thw[side] if self.bc[side] == ISO else th[sl]
                uw = self.uw[side].reshape((3,) + (1,) * rho[sl].ndim)
                ghost = 2 * rho[sl] * uw * (1 - thw) - Q[(slice(None),) + sl]
                if hi:
                    up[(slice(None),) + sl] = ghost
                else:
                    dn[(slice(None),) + sl] = ghost
            dQ[k] = 0.5 * (up - dn)
        return dQ

    def step(self, n: int = 1):
        for _ in range(n):
            self._step()
        return self

    def _step(self):
        p = self.p
        wf = 2 / (2 * p["tau_f"] + 1)
        wh = 2 / (2 * p["tau_h"] + 1)
        rho, u, th = self.moments()
        if int(p.get("correction", 1)):
            C = correction(self._grad(rho * u * (1 - th), rho, th))
        else:
            C = np.zeros_like(self.F)
        g = float(p.get("g", 0.0))
        if g:
            # Guo's force term with cs^2 = 1/3, a = (0, 0, -rho g):
            # w [3 (e - u).a + 9 (e.u)(e.a)]
            az = -rho * g
            for a in range(19):
                eu = E[a, 0] * u[0] + E[a, 1] * u[1] + E[a, 2] * u[2]
                C[a] = C[a] + W[a] * (3 * (E[a, 2] - u[2]) * az + 9 * eu * E[a, 2] * az)
        feq, heq = self._eq(rho, u, th)
        # Eq. 37 / Eq. 38: h^eq from the node's own energy (sum h = rho E)
        es = self.H.sum(0) / rho
        if self.total:
            f = feq_shells(rho, u, th)
            usq = (u * u).sum(0)
            heq = heq_total(rho, u, th, p["b"], f) + (es - (p["b"] * th / 6 + 0.5 * usq)) * f
        fneq = self.F - feq
        fs = self.F - wf * fneq + (1 - 0.5 * wf) * C
        hs = self.H - wh * (self.H - heq)
        if self.total:
            usq = (u * u).sum(0)
            for a in range(19):
                eu = E[a, 0] * u[0] + E[a, 1] * u[1] + E[a, 2] * u[2]
                Z = eu - 0.5 * usq if int(p.get("z_full", 1)) else eu
                hs[a] = hs[a] + (wh - wf) * Z * (fneq[a] + 0.5 * C[a])
        # pull streaming (periodic), then, node by node on the faces, the
        # populations that came back from a wall replaced from the receiving
        # node's side (a left through the first walled side it crossed, of
        # x, y, z; b = its opposite arrives)
        Fn = np.empty_like(fs)
        Hn = np.empty_like(hs)
        for a in range(19):
            sh = (E[a, 2], E[a, 1], E[a, 0])
            Fn[a] = np.roll(fs[a], sh, axis=(0, 1, 2))
            Hn[a] = np.roll(hs[a], sh, axis=(0, 1, 2))
        nz, ny, nx = self.shape
        n = (nx, ny, nz)
        for z in range(nz):
            for y in range(ny):
                for x in range(nx):
                    c = (x, y, z)
                    if all(0 < c[k] < n[k] - 1 for k in range(3)):
                        continue
                    for a in range(1, 19):
                        side = -1
                        for k in range(3):
                            t = c[k] + E[a, k]
                            sk = 2 * k if t < 0 else (2 * k + 1 if t >= n[k] else -1)
                            if sk >= 0 and self.bc[sk] != PERIODIC:
                                side = sk
                                break
                        if side < 0:
                            continue
                        b = OPP[a]
                        r, tn = rho[z, y, x], th[z, y, x]
                        un = u[:, z, y, x]
                        uw = self.uw[side]
                        fw, hw = self._eq(r, uw, tn)  # node's rho, theta; wall velocity
                        Fn[b, z, y, x] = fs[a, z, y, x] + (fw[b] - fw[a])
                        if self.bc[side] == ISO:
                            tg = max(2 * self.thw[side] - tn, 0.5 * self.thw[side])
                            # the node's pressure less the hydrostatic drop
                            # to the ghost (gravity along -z)
                            nz_out = -1 if side == 4 else (1 if side == 5 else 0)
                            rg = r * (tn - 3 * float(p.get("g", 0.0)) * nz_out) / tg
                            fg, hg = self._eq(rg, 2 * uw - un, tg)
                            Hn[b, z, y, x] = hg[b] + (hs[b, z, y, x] - heq[b, z, y, x])
                        else:
                            hin = hs[a, z, y, x] + (hw[b] - hw[a])
                            if self.total:  # the moving wall's work on the pair
                                hin = hin - float(E[a] @ uw) * (Fn[b, z, y, x] + fs[a, z, y, x])
                            Hn[b, z, y, x] = hin
        self.F, self.H = Fn, Hn
