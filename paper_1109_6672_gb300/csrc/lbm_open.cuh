// Ghost slots that the step kernels leave to a second pass: open x sides and
// walls of non-equilibrium extrapolation.
//
// Open x sides of the attenuation-driven acoustic streaming set-up
// (arXiv:1109.6672, Sec. IV.B): an inlet at x- reset every step to the
// equilibria of the Eq. 53 state, and a zero-gradient outlet at x+ with
// non-equilibrium extrapolation.  y is periodic.
//
// The step kernels handle an open side as if it were a wall and write wall
// values into its ghost slots; the kernels here, launched right after each
// step on the same stream, overwrite every one of those slots:
//  - inlet: node (0, y) pulls populations 1, 5, 8 from the inlet node one
//    spacing outside, whose post-collision populations are its equilibria
//    (Eq. 18a, Eq. 18b or the Eq. 38 form) at step t;
//  - outlet: the ghost column's (rho, u, T) are the last column's (zero
//    gradient), so its equilibria are the last column's and non-equilibrium
//    extrapolation makes its post-collision populations the last column's;
//    populations 3, 6, 7 are copied from the stored post-collision values
//    (bit for bit, deviation storage included) to where the nodes they reach
//    pull them, wrapping in y as a periodic copy does.
// What leaves through an open side is dropped.  Keeping this out of the step
// kernels leaves their inner loops untouched.
#pragma once

#include "lbm_device.cuh"

namespace lbm {

// State of the inlet node at step t, Eq. 53 (FP64).
__device__ __forceinline__ void inlet_state(const Grid& g, unsigned t, double& rho, double& ux,
                                            double& uy, double& th) {
  const double sn = sin(g.in_omega * (double)t);
  rho = g.in_rho + g.in_drho * sn;
  ux = g.pd.uw[0][0] + g.in_du * sn;
  uy = g.pd.uw[0][1];
  th = g.pd.thw[0] + g.in_dth * sn;
}

// Ghost slots of the open sides for rows y = first, first + stride, ... of
// one grid whose state at t + 1 is dst (g.t = t: the step just taken).
template <class S>
__device__ void open_rows(const Grid& g, S* __restrict__ dst, int first, int stride) {
  using C = typename Io<S>::C;
  const bool in = g.bc[0] == BC_INLET, out = g.bc[1] == BC_OUTLET;
  C fin[9], hin[9];
  if (in) {
    double r, vx, vy, th;
    inlet_state(g, g.t, r, vx, vy, th);
    double fd[9], hd[9];
    equilibria<double>(r, vx, vy, th, g.pd.b6, g.energy_model == E_TOTAL, fd, hd);
    for (int a = 0; a < 9; ++a) {
      fin[a] = C(fd[a]);
      hin[a] = C(hd[a]);
    }
  }
  const int x = g.nx - 1;
  for (int y = first; y < g.ny; y += stride) {
    if (in) {
      // random streams of wall values (18 + a, 27 + a) of node (0, y)
      const unsigned hs = Io<S>::sr ? sr_hash(g, 0, y) : 0u;
      put<S>(g, dst, 1, -1, y, fin[1], hs, 19);
      put<S>(g, dst, 5, -1, y - 1, fin[5], hs, 23);
      put<S>(g, dst, 8, -1, y + 1, fin[8], hs, 26);
      put<S>(g, dst, 10, -1, y, hin[1], hs, 28);
      put<S>(g, dst, 14, -1, y - 1, hin[5], hs, 32);
      put<S>(g, dst, 17, -1, y + 1, hin[8], hs, 35);
    }
    if (out) {
      const int y6 = (y + 1) % g.ny - 1, y7 = (y - 1 + g.ny) % g.ny + 1;  // wrap(y + e_y) - e_y
      dst[slot(g, 3, x + 1, y)] = dst[slot(g, 3, x, y)];
      dst[slot(g, 12, x + 1, y)] = dst[slot(g, 12, x, y)];
      dst[slot(g, 6, x + 1, y6)] = dst[slot(g, 6, x, y)];
      dst[slot(g, 15, x + 1, y6)] = dst[slot(g, 15, x, y)];
      dst[slot(g, 7, x + 1, y7)] = dst[slot(g, 7, x, y)];
      dst[slot(g, 16, x + 1, y7)] = dst[slot(g, 16, x, y)];
    }
  }
}

// Walls of non-equilibrium extrapolation (the paper's wall method, ref.
// [45]; side s flagged in Grid::nee).  The wall sits on the ghost node G one
// spacing outside the boundary node F.  G's state: the wall velocity, theta_G
// (the wall's on an isothermal side; on an adiabatic side zero slope at G to
// second order, (4 theta_F - theta_F2)/3 with F2 the next node inward,
// floored at theta_F / 2 so that the density below stays finite), and
// F's pressure carried to G by hydrostatic balance,
// rho_G = rho_F (theta_F - 3 g n_y) / theta_G.  Its pre-collision
// populations are its equilibria plus F's non-equilibrium part
// fbar(F) - f^eq(F) (likewise h; on an adiabatic side without the normal
// energy flux of that part); it collides like a fluid node (rates of
// its own rho and theta, the Guo force of its own density, no correction
// term), and the populations it sends into the domain are stored where the
// receiving nodes pull them.  Ghost k of a grid: 0 .. ny + 1 the x- column
// (G at y = k - 1, the corners included), then the x+ column, then nx per
// y side; the step kernels treat these sides as halfway walls and this
// rewrites every slot those wrote.
__host__ __device__ inline int nee_ghosts(const Grid& g) { return 2 * (g.ny + 2) + 2 * g.nx; }

template <class S>
__device__ void nee_ghost(const Grid& g, const S* __restrict__ src, S* __restrict__ dst, int k) {
  using C = typename Io<S>::C;
  int side, gx, gy;
  if (k < 2 * (g.ny + 2)) {
    side = k < g.ny + 2 ? 0 : 1;
    gx = side == 0 ? -1 : g.nx;
    gy = k - (side == 0 ? 0 : g.ny + 2) - 1;
  } else {
    k -= 2 * (g.ny + 2);
    side = k < g.nx ? 2 : 3;
    gx = k - (side == 2 ? 0 : g.nx);
    gy = side == 2 ? -1 : g.ny;
  }
  if (!(g.nee >> side & 1)) return;
  const bool xs = side < 2;
  const bool yper = g.bc[2] == BC_PERIODIC, xper = g.bc[0] == BC_PERIODIC;
  const int nxo = side == 0 ? -1 : (side == 1 ? 1 : 0), nyo = side == 2 ? -1 : (side == 3 ? 1 : 0);
  // F: the first node inward (an x side's corner ghost: the corner node)
  int fx, fy;
  bool corner = false;
  if (xs) {
    fx = gx - nxo;
    if (gy < 0 || gy >= g.ny) {
      if (yper) return;  // along a periodic y the column has no corner ghosts
      corner = true;
      fy = gy < 0 ? 0 : g.ny - 1;
    } else {
      fy = gy;
    }
  } else {
    fx = gx;
    fy = gy - nyo;
  }
  const bool total = g.energy_model == E_TOTAL;
  const Phys<C>& kp = phys<C>(g);
  C d[NPOP], rho, ux, uy, th, Es;
  pull<S>(g, src, fx, fy, d);
  moments<S>(g, d, rho, ux, uy, th, Es);
  C feq[9], heq[9];
  collision_equilibria<C>(rho, ux, uy, th, Es, kp.b6, total, feq, heq);
  C thG;
  if (g.bc[side] == BC_ISO) {
    thG = kp.thw[side];
  } else {
    C d2[NPOP], r2, u2, v2, t2, e2;
    pull<S>(g, src, fx - nxo, fy - nyo, d2);
    moments<S>(g, d2, r2, u2, v2, t2, e2);
    thG = fmax((C(4) * th - t2) * C(1.0 / 3.0), C(0.5) * th);  // floored: rho_G = rho th / thG
  }
  // F's pressure carried to G by hydrostatic balance, p_G = p_F - rho_F g n_y
  const C rG = rho * (th - C(3) * kp.g * C(nyo)) / thG;
  const C uwx = kp.uw[side][0], uwy = kp.uw[side][1];
  const C EsG = kp.b6 * thG + (total ? C(0.5) * (uwx * uwx + uwy * uwy) : C(0));
  C fqG[9], hqG[9], fb[9], hb[9];
  collision_equilibria<C>(rG, uwx, uwy, thG, EsG, kp.b6, total, fqG, hqG);
  C hn[9], qn = C(0);
  const C zw2 = (total && g.z_full) ? C(0.5) * (uwx * uwx + uwy * uwy) : C(0);
#pragma unroll
  for (int a = 0; a < 9; ++a) {
    const C fneq = (pref<S>(g, a) + d[a]) - feq[a];
    fb[a] = fqG[a] + fneq;
    hn[a] = (pref<S>(g, 9 + a) + d[9 + a]) - heq[a];
    // the heat part of h^neq: less the viscous work Z f^neq at the wall
    // velocity (h - Z f relaxes at the thermal rate, Eq. 36)
    const C zw = total ? C(ex(a)) * uwx + C(ey(a)) * uwy - zw2 : C(0);
    qn += C(ex(a) * nxo + ey(a) * nyo) * (hn[a] - zw * fneq);
  }
  // an adiabatic wall node carries no normal heat flux: that part's normal
  // moment is taken out (sum w e_n^2 = 1/3); a moving wall's work passes
  const bool adia = g.bc[side] != BC_ISO;
#pragma unroll
  for (int a = 0; a < 9; ++a) {
    const C en = C(ex(a) * nxo + ey(a) * nyo);
    hb[a] = hqG[a] + (adia ? hn[a] - wgt<C>(a) * en * qn * C(3) : hn[a]);
  }
  // collision of G
  C wf, wh, kz;
  node_rates<C>(g, kp, rG, thG, g.collision == COLL_MRT, wf, wh, kz);
  C cc[9];
  const C ay = -rG * kp.g;
#pragma unroll
  for (int a = 0; a < 9; ++a) {
    const C ea = C(ey(a)) * ay;
    const C eu = C(ex(a)) * uwx + C(ey(a)) * uwy;
    cc[a] = g.has_force ? wgt<C>(a) * (C(3) * ea + C(9) * eu * ea - C(3) * uwy * ay) : C(0);
  }
  C fs[9], fn[9];
#pragma unroll
  for (int a = 0; a < 9; ++a) fn[a] = fb[a] - fqG[a];
  if (g.collision == COLL_MRT) {
    C mc[9];
    mrt_source<C>(false, C(0), C(0), g.has_force != 0, uwx, uwy, ay, mc);
    mrt_collide<C, false>(kp, wf, fb, fn, mc, fs);
  } else {
#pragma unroll
    for (int a = 0; a < 9; ++a) fs[a] = fb[a] - wf * fn[a] + (C(1) - C(0.5) * wf) * cc[a];
  }
  const C usq = uwx * uwx + uwy * uwy;
  const unsigned hs = Io<S>::sr ? sr_hash(g, gx, gy) : 0u;
#pragma unroll
  for (int a = 1; a < 9; ++a) {
    if (ex(a) * nxo + ey(a) * nyo >= 0) continue;  // not into the domain
    int dx = gx + ex(a), dy = gy + ey(a);
    if (corner) {
      if (dx != fx || dy != fy) continue;  // a corner ghost feeds the corner node only
    } else {
      if (dx < 0 || dx >= g.nx) {
        if (!xper) continue;  // the x side's rule has it
        dx = (dx + g.nx) % g.nx;
      }
      if (dy < 0 || dy >= g.ny) {
        if (!yper) continue;
        dy = (dy + g.ny) % g.ny;
      }
    }
    C hsa = hb[a] - wh * (hb[a] - hqG[a]);
    if (total) {
      const C eu = C(ex(a)) * uwx + C(ey(a)) * uwy;
      const C Z = g.z_full ? eu - C(0.5) * usq : eu;
      hsa += kz * Z * (fn[a] + C(0.5) * cc[a]);
    }
    put<S>(g, dst, a, dx - ex(a), dy - ey(a), fs[a], hs, 18 + a);
    put<S>(g, dst, 9 + a, dx - ex(a), dy - ey(a), hsa, hs, 27 + a);
  }
}

// Every ghost slot of the open sides and of the walls of non-equilibrium
// extrapolation of one grid (state at t in src, at t + 1 in dst, g.t = t),
// work units first, first + stride, ...
template <class S>
__device__ void fixup_grid(const Grid& g, const S* __restrict__ src, S* __restrict__ dst,
                           int first, int stride) {
  if (g.bc[0] == BC_INLET || g.bc[1] == BC_OUTLET) open_rows<S>(g, dst, first, stride);
  if (g.nee) {
    const int n = nee_ghosts(g);
    for (int k = first; k < n; k += stride) nee_ghost<S>(g, src, dst, k);
  }
}

// One grid: work spread over the launch.
template <class S>
__global__ void __launch_bounds__(128)
    side_fixup_kernel(const Grid g, const S* __restrict__ src, S* __restrict__ dst) {
  fixup_grid<S>(g, src, dst, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x);
}

}  // namespace lbm
