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

// One grid: rows spread over the launch.
template <class S>
__global__ void __launch_bounds__(128) open_fixup_kernel(const Grid g, S* __restrict__ dst) {
  open_rows<S>(g, dst, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x);
}

}  // namespace lbm
