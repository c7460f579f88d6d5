"""Independent NumPy restatement of one step of the BGK coupled DDF scheme
(arXiv:1109.6672, Sec. III.C), used only to cross-check the C oracle on tiny
grids.  It is written from the paper separately from the oracle and takes
different routes to the same quantities:

* Eq. 18a is expanded per speed shell (rest, axis, diagonal) by hand instead of
  being evaluated from the generic Hermite form;
* moments use array contractions;
* streaming is pull-based (``np.roll``), and the wall rules are applied from the
  receiving node's side instead of the sending node's side;
* for the MRT scheme (Sec. III.C.2) the moment basis is built from its
  defining polynomials of the velocity set and inverted numerically, and
  m^eq is M f^eq rather than Eq. 41;
* the open sides of the acoustic set-up (Sec. IV.B) are applied on the pull:
  a first-column node takes its e_x = +1 populations from the inlet state of
  Eq. 53, a last-column node takes its e_x = -1 populations from the ghost
  column x = nx, whose state is the last column's (zero gradient) and whose
  non-equilibrium part is the last column's too;
* walls of non-equilibrium extrapolation are applied on the pull as well: the
  ghost node a population comes from, and the fluid node next to it (the
  x side's for a corner ghost), are found from the receiving node.
"""
from __future__ import annotations

import numpy as np

EX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
EY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])
OPP = np.array([0, 3, 4, 1, 2, 7, 8, 5, 6])
W = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
PERIODIC, ISO, ADIA, INLET, OUTLET = 0, 1, 2, 3, 4

# moments rho, e, eps, jx, qx, jy, qy, pxx, pxy as polynomials of e_a
_E2 = EX * EX + EY * EY
MB = np.array([np.ones(9), 3 * _E2 - 4, (9 * _E2 ** 2 - 21 * _E2 + 8) / 2, EX, (3 * _E2 - 5) * EX,
               EY, (3 * _E2 - 5) * EY, EX * EX - EY * EY, EX * EY], float)
MB_INV = np.linalg.inv(MB)


def feq_shells(rho, ux, uy, th):
    """Eq. 18a with R T0 = 1/3, D = 2, expanded per shell:
    rest:     rho 4/9  [1 - 3/2 u^2 - (th - 1)]
    axis:     rho 1/9  [1 + 3 eu (1 - (th-1)/2) + 9/2 eu^2 - 3/2 u^2 + (th-1)/2]
    diagonal: rho 1/36 [1 + 3 th eu + 9/2 eu^2 - 3/2 u^2 + 2 (th-1)]"""
    usq = ux * ux + uy * uy
    out = []
    for a in range(9):
        eu = EX[a] * ux + EY[a] * uy
        if a == 0:
            v = rho * (4 / 9) * (1 - 1.5 * usq - (th - 1))
        elif a <= 4:
            v = rho / 9 * (1 + 3 * eu * (1 - 0.5 * (th - 1)) + 4.5 * eu * eu - 1.5 * usq + 0.5 * (th - 1))
        else:
            v = rho / 36 * (1 + 3 * th * eu + 4.5 * eu * eu - 1.5 * usq + 2 * (th - 1))
        out.append(v)
    return np.array(out)


def heq_total(rho, ux, uy, th, b, feq):
    """Eq. 18b with E = (b R T + u^2)/2, p = rho R T, R T = th/3."""
    usq = ux * ux + uy * uy
    E = 0.5 * (b * th / 3 + usq)
    p = rho * th / 3
    out = []
    for a in range(9):
        eu = EX[a] * ux + EY[a] * uy
        e2 = EX[a] ** 2 + EY[a] ** 2
        out.append(E * feq[a] + W[a] * p * (3 * eu + 9 * eu * eu - 3 * usq + 0.5 * th * (3 * e2 - 2)))
    return np.array(out)


def heq_internal(th, b, feq):
    return 0.5 * b * (th / 3) * feq


class Brute:
    def __init__(self, p: dict):
        self.p = p
        self.nx, self.ny = p["nx"], p["ny"]
        self.t = 0
        assert abs(p["R"] * p["T0"] - 1 / 3) < 1e-14

    def inlet(self):
        """Eq. 53 at the current time: rho, u_x, u_y, theta of the inlet node."""
        p = self.p
        s = np.sin(p.get("in_omega", 0.0) * self.t)
        return (p.get("in_rho", 1.0) + p.get("in_drho", 0.0) * s,
                p["u_wall"][0][0] + p.get("in_du", 0.0) * s, p["u_wall"][0][1],
                (p["T_wall"][0] + p.get("in_dT", 0.0) * s) / p["T0"])

    def init(self, rho, ux, uy, T):
        p = self.p
        th = T / p["T0"]
        self.F = feq_shells(rho, ux, uy, th)
        self.H = (heq_total(rho, ux, uy, th, p["b"], self.F) if p["energy_model"] == 0
                  else heq_internal(th, p["b"], self.F))
        return self

    def moments(self):
        p = self.p
        rho = self.F.sum(0)
        jx = np.tensordot(EX, self.F, 1)
        jy = np.tensordot(EY, self.F, 1) - 0.5 * rho * p["g"]
        ux, uy = jx / rho, jy / rho
        sh = self.H.sum(0)
        if p["energy_model"] == 0:
            th = 6 / p["b"] * (sh / rho - 0.5 * (ux * ux + uy * uy))
        else:
            th = 6 * sh / (rho * p["b"])
        return rho, ux, uy, th

    def _wall_theta(self, side, th_node):
        if self.p["bc"][side] == ISO:
            return self.p["T_wall"][side] / self.p["T0"] + 0 * th_node
        return th_node

    def _grad(self, Q, axis, rho, th, comp):
        """Eq. 50 with periodic wrap or a mirror ghost across a wall."""
        lo_side, hi_side = (0, 1) if axis == 1 else (2, 3)
        n = Q.shape[axis]
        plus = np.roll(Q, -1, axis=axis)
        minus = np.roll(Q, 1, axis=axis)
        for side, arr, idx in ((hi_side, plus, n - 1), (lo_side, minus, 0)):
            if self.p["bc"][side] == PERIODIC:
                continue
            sl = [slice(None), slice(None)]
            sl[axis] = idx
            sl = tuple(sl)
            if self.p["bc"][side] == OUTLET:
                arr[sl] = Q[sl]
                continue
            if self.p["bc"][side] == INLET:
                ri, uxi, uyi, ti = self.inlet()
                arr[sl] = ri * (uxi, uyi)[comp] * (1 - ti)
                continue
            thw = self._wall_theta(side, th[sl])
            Qw = rho[sl] * self.p["u_wall"][side][comp] * (1 - thw)
            arr[sl] = 2 * Qw - Q[sl]
        return 0.5 * (plus - minus)

    def _collide(self, F, H, rho, ux, uy, th, C):
        """Equilibria and post-collision populations of nodes (arrays over
        the grid, or one node with scalar moments)."""
        p = self.p
        usq = ux * ux + uy * uy
        feq = feq_shells(rho, ux, uy, th)
        if p["energy_model"] == 0:
            heq = heq_total(rho, ux, uy, th, p["b"], feq)
        else:
            heq = heq_internal(th, p["b"], feq)
        wf = 1 / (p["tau_f"] + 0.5)
        wh = 1 / (p["tau_h"] + 0.5)
        if p.get("collision", 0) == 1:
            # rates: conserved moments 1, e / eps / q as given (0: omega_f), shear omega_f
            r = [p.get(k, 0.0) or wf for k in ("s_e", "s_eps", "s_q")]
            S = np.array([1, r[0], r[1], 1, r[2], 1, r[2], wf, wf]).reshape((9,) + (1,) * (F.ndim - 1))
            m = np.tensordot(MB, F, 1)
            meq = np.tensordot(MB, feq, 1)
            Ch = np.tensordot(MB, C, 1)
            fs = np.tensordot(MB_INV, m - S * (m - meq) + (1 - S / 2) * Ch, 1)
            # Eq. 47: (1 - w_h/2) Z / tau_hf, tau_hf = (tau_f + 1/2)/(Pr - 1)
            kz = (1 - wh / 2) * (p["tau_f"] / p["tau_h"] - 1) / (p["tau_f"] + 0.5)
        else:
            fs = F + wf * (feq - F) + (1 - wf / 2) * C
            kz = wh - wf
        hs = H + wh * (heq - H)
        if p["energy_model"] == 0:
            for a in range(9):
                eu = EX[a] * ux + EY[a] * uy
                Z = eu - 0.5 * usq if p["z_full"] else eu
                hs[a] = hs[a] + kz * Z * (F[a] - feq[a] + 0.5 * C[a])
        return np.asarray(feq), np.asarray(heq), fs, hs

    def step(self, n=1):
        for _ in range(n):
            self._step()
            self.t += 1
        return self

    def _step(self):
        p = self.p
        rho, ux, uy, th = self.moments()
        usq = ux * ux + uy * uy
        Qx, Qy = rho * ux * (1 - th), rho * uy * (1 - th)
        C = np.zeros_like(self.F)
        if p["correction"]:
            dqx = self._grad(Qx, 1, rho, th, 0)
            dqy = self._grad(Qy, 0, rho, th, 1)
            phx, phy = 3 * (dqx + dqy), dqx - dqy
            C[0] = -phx / 9
            C[1] = C[3] = -phx / 36 + phy / 4
            C[2] = C[4] = -phx / 36 - phy / 4
            C[5:] = phx / 18
        ay = -rho * p["g"]
        for a in range(9):  # Guo force, R T0 = 1/3
            ea = EY[a] * ay
            eu = EX[a] * ux + EY[a] * uy
            C[a] += W[a] * (3 * ea + 9 * (eu * ea - (uy * ay) / 3))
        feq, heq, fs, hs = self._collide(self.F, self.H, rho, ux, uy, th, C)
        # pull streaming with wrap, then overwrite wall-crossing pulls
        Fn = np.empty_like(fs)
        Hn = np.empty_like(hs)
        for a in range(9):
            Fn[a] = np.roll(fs[a], (EY[a], EX[a]), axis=(0, 1))
            Hn[a] = np.roll(hs[a], (EY[a], EX[a]), axis=(0, 1))
        nx, ny = self.nx, self.ny
        ri, uxi, uyi, ti = self.inlet()
        fin = feq_shells(ri, uxi, uyi, ti)
        hin = heq_total(ri, uxi, uyi, ti, p["b"], fin) if p["energy_model"] == 0 else heq_internal(
            ti, p["b"], fin)
        for y in range(ny):
            for x in range(nx):
                if 0 < x < nx - 1 and 0 < y < ny - 1:
                    continue
                for a in range(1, 9):
                    sx, sy = x - EX[a], y - EY[a]
                    out_x = 0 if sx < 0 else (1 if sx >= nx else -1)
                    out_y = 2 if sy < 0 else (3 if sy >= ny else -1)
                    side = -1
                    if out_x >= 0 and p["bc"][out_x] != PERIODIC:
                        side = out_x
                    elif out_y >= 0 and p["bc"][out_y] != PERIODIC:
                        side = out_y
                    if side < 0:
                        continue
                    if p["bc"][side] == INLET:
                        Fn[a, y, x], Hn[a, y, x] = fin[a], hin[a]
                        continue
                    if p["bc"][side] == OUTLET:
                        Fn[a, y, x] = fs[a, (y - EY[a]) % ny, nx - 1]
                        Hn[a, y, x] = hs[a, (y - EY[a]) % ny, nx - 1]
                        continue
                    if p.get("wall_nee", 0) >> side & 1:
                        # ghost G = (sx, sy); its fluid node F is the first
                        # node inward along the side's normal (wrapped along
                        # a periodic axis, clamped at a corner)
                        if side < 2:
                            fx = 0 if side == 0 else nx - 1
                            fy = sy % ny if p["bc"][2] == PERIODIC else min(max(sy, 0), ny - 1)
                        else:
                            fy = 0 if side == 2 else ny - 1
                            fx = sx % nx
                        r, t = rho[fy, fx], th[fy, fx]
                        uw = p["u_wall"][side]
                        if p["bc"][side] == ISO:
                            tG = p["T_wall"][side] / p["T0"]
                        else:  # zero slope at the wall node: quadratic through F, F2
                            nxo, nyo = [(-1, 0), (1, 0), (0, -1), (0, 1)][side]
                            tG = max((4 * t - th[fy - nyo, fx - nxo]) / 3, 0.5 * t)
                        nyo = [0, 0, -1, 1][side]
                        rG = r * (t - 3 * p["g"] * nyo) / tG  # hydrostatic pressure at G
                        fG = feq_shells(rG, uw[0], uw[1], tG)
                        hG = (heq_total(rG, uw[0], uw[1], tG, p["b"], fG) if p["energy_model"] == 0
                              else heq_internal(tG, p["b"], fG))
                        fbG = np.array(fG) + self.F[:, fy, fx] - feq[:, fy, fx]
                        hneq = self.H[:, fy, fx] - heq[:, fy, fx]
                        if p["bc"][side] == ADIA:  # no normal heat flux at the wall node
                            nxo, nyo = [(-1, 0), (1, 0), (0, -1), (0, 1)][side]
                            en = EX * nxo + EY * nyo
                            # the heat part of h^neq: less the viscous work
                            # Z f^neq at the wall velocity (total energy)
                            heat = hneq
                            if p["energy_model"] == 0:
                                Zw = EX * uw[0] + EY * uw[1]
                                if p["z_full"]:
                                    Zw = Zw - 0.5 * (uw[0] ** 2 + uw[1] ** 2)
                                heat = hneq - Zw * (self.F[:, fy, fx] - feq[:, fy, fx])
                            hneq = hneq - W * en * (en @ heat) / (W @ (en * en))
                        hbG = np.array(hG) + hneq
                        CG = np.array([W[k] * (3 * EY[k] * (-rG * p["g"]) + 9 * (
                            (EX[k] * uw[0] + EY[k] * uw[1]) * EY[k] * (-rG * p["g"]) -
                            (uw[1] * (-rG * p["g"])) / 3)) for k in range(9)])
                        _, _, fsG, hsG = self._collide(fbG, hbG, rG, uw[0], uw[1], tG, CG)
                        Fn[a, y, x], Hn[a, y, x] = fsG[a], hsG[a]
                        continue
                    r, t = rho[y, x], th[y, x]
                    uw = p["u_wall"][side]
                    iso = p["bc"][side] == ISO
                    thw = p["T_wall"][side] / p["T0"] if iso else t
                    fw = feq_shells(r, uw[0], uw[1], t)
                    o = OPP[a]
                    Fn[a, y, x] = fs[o, y, x] + (fw[a] - fw[o])
                    if iso:
                        # ghost node one spacing outside: linear in u and theta
                        # through the wall; its pressure the node's less the
                        # hydrostatic drop over the spacing (y sides)
                        tg = max(2 * thw - t, 0.5 * thw)
                        ny_out = [0, 0, -1, 1][side]
                        rg = r * (t - 3 * p["g"] * ny_out) / tg
                        ugx, ugy = 2 * uw[0] - ux[y, x], 2 * uw[1] - uy[y, x]
                        fg = feq_shells(rg, ugx, ugy, tg)
                        hg = (heq_total(rg, ugx, ugy, tg, p["b"], fg) if p["energy_model"] == 0
                              else heq_internal(tg, p["b"], fg))
                        Hn[a, y, x] = hg[a] + hs[a, y, x] - heq[a, y, x]
                    else:
                        fa = feq_shells(r, uw[0], uw[1], t)
                        ha = (heq_total(r, uw[0], uw[1], t, p["b"], fa) if p["energy_model"] == 0
                              else heq_internal(t, p["b"], fa))
                        Hn[a, y, x] = hs[o, y, x] + (ha[a] - ha[o])
                        if p["energy_model"] == 0:  # the moving wall's work on the pair
                            Hn[a, y, x] += (EX[a] * uw[0] + EY[a] * uw[1]) * (
                                Fn[a, y, x] + fs[o, y, x])
        self.F, self.H = Fn, Hn

    def pops(self):
        return np.concatenate([self.F, self.H], 0)
