// Device side of the three-dimensional extension of the coupled DDF thermal
// lattice Boltzmann step (arXiv:1109.6672, BGK scheme of Sec. III.C.1
// carried to D3Q19; the paper states that its formulation extends to 3-D).
//
// Equilibria: Eq. 18a / 18b with D = 3 (R T0 = 1/3, c = 1).  Correction
// term: on D3Q19 the third-order moment of f^eq deviates from Eq. 10d by
//   D_iii = Q_i   and   D_iik = D_iki = D_kii = Q_k / 6   (i != k),
// Q = rho u (1 - theta) (the diagonal is Eq. 20; the cross entries come from
// the missing (1,1,1) velocities), so the argument that gives Eq. 28 from
// Eq. 27 asks for second moments
//   G_ii = dQ_i/dx_i + (1/6) sum_{k != i} dQ_k/dx_k,
//   G_ij = (dQ_j/dx_i + dQ_i/dx_j) / 6   (i != j),
// with the central differences of Eq. 50 along every axis.  C_a is the
// even quadratic polynomial of e_a orthogonal to the constants (the D3Q19
// counterpart of Eq. 49: only second-order moments):
//   C_a = sum_ij A_ij (e_ai e_aj - kappa d_ij), kappa = 10/19,
//   A_kk = (G_kk + (4/7) tr G) / 6,  A_ij = G_ij / 8,
// i.e. C_0 = -(5/21) tr G, C_(+-x) = A_xx - (5/21) tr G,
// C_(+-1,+-1,0) = A_xx + A_yy - (5/21) tr G +- G_xy / 4 (sign of e_x e_y).
//
// State layout (one buffer; two buffers ping-pong): element (a, x, y, z),
// a = 0..37 (f_0..f_18, h_0..h_18), x in [-1, nx], y in [-1, ny], z in
// [-1, nz] (a one-node ghost ring) at
//     ((z + 1) * (ny + 2) + (y + 1)) * 38 * pitch + a * pitch + x + 32,
// pitch a multiple of 32 and >= nx + 33.  As in 2-D, a buffer holds the
// post-collision value f*_a(s) at the slot s from which node s + e_a pulls
// it: the canonical pre-collision state of node x is buf_a(x - e_a), the
// nodes on the faces write the periodic copies into the ghost slots.
//
// Kernel: a block owns a 32 x TY tile of (x, y) and marches along z over
// its z range.  For each plane it first computes the moments (and Q) of the
// tile plus a one-node halo ring (wrapped periodically) into a 3-plane ring
// of Q in shared memory, then collides the plane below, whose own moments
// the thread kept in registers and whose pulled populations it parked in
// shared memory (a per-thread column, two planes deep, so no barrier guards
// it).  Each side of the box is periodic or a halfway wall.
#pragma once

#include "lbm_device.cuh"

namespace lbm3 {

using lbm::Io;

constexpr int Q19 = 19;
constexpr int NP3 = 38;
constexpr int XOFF3 = 32;

// D3Q19: rest, +-x, +-y, +-z, then the face diagonals (+-1,+-1,0),
// (+-1,0,+-1), (0,+-1,+-1), each velocity followed by its opposite.
__host__ __device__ constexpr int e3x(int a) {
  return (a == 1 || a == 7 || a == 9 || a == 11 || a == 13) ? 1
         : (a == 2 || a == 8 || a == 10 || a == 12 || a == 14) ? -1 : 0;
}
__host__ __device__ constexpr int e3y(int a) {
  return (a == 3 || a == 7 || a == 10 || a == 15 || a == 17) ? 1
         : (a == 4 || a == 8 || a == 9 || a == 16 || a == 18) ? -1 : 0;
}
__host__ __device__ constexpr int e3z(int a) {
  return (a == 5 || a == 11 || a == 14 || a == 15 || a == 18) ? 1
         : (a == 6 || a == 12 || a == 13 || a == 16 || a == 17) ? -1 : 0;
}
__host__ __device__ constexpr int e3sq(int a) {
  return e3x(a) * e3x(a) + e3y(a) * e3y(a) + e3z(a) * e3z(a);
}
template <class C>
__host__ __device__ constexpr C w3(int a) {
  return a == 0 ? C(1) / C(3) : (a <= 6 ? C(1) / C(18) : C(1) / C(36));
}

enum { M3_TOTAL = 1, M3_ZFULL = 2, M3_CORR = 4, M3_FORCE = 8 };

template <class C>
struct Phys3 {
  C omega_f, omega_h;  // 2 / (2 tau + 1)
  C kz;                // omega_h - omega_f (Eq. 36)
  C b6, six_b;         // b / 6, 6 / b
  C uw[6][3];          // wall velocities of the sides x-, x+, y-, y+, z-, z+
  C thw[6];            // wall theta = T_w / T0 (isothermal walls)
  C g;                 // gravity along -z: a = (0, 0, -rho g)
};

enum { BC3_PERIODIC = 0, BC3_ISO = 1, BC3_ADIA = 2 };

struct Grid3 {
  void* src;
  void* dst;
  int nx, ny, nz, pitch;
  long long lp, zs;  // line stride (38 pitch) and plane stride ((ny + 2) lp)
  int energy_model, correction, z_full;
  int bc[6];  // sides x-, x+, y-, y+, z-, z+ (2 axis + high end): BC3_PERIODIC
              // or a halfway wall
  Phys3<double> pd;
  Phys3<float> pf;
};

template <class C>
__host__ __device__ __forceinline__ const Phys3<C>& phys3(const Grid3& g) {
  if constexpr (sizeof(C) == 8)
    return g.pd;
  else
    return g.pf;
}

__host__ __device__ __forceinline__ long long slot3(const Grid3& g, int a, int x, int y, int z) {
  return (long long)(z + 1) * g.zs + (long long)(y + 1) * g.lp + (long long)a * g.pitch +
         (x + XOFF3);
}

__device__ __forceinline__ int wrap3(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

// Pull the 38 values of node (x, y, z): d[a] = buf_a(x - e_a).
template <class S>
__device__ __forceinline__ void pull3(const Grid3& g, const S* __restrict__ src, int x, int y,
                                      int z, typename Io<S>::C d[NP3]) {
  const S* p = src + slot3(g, 0, x, y, z);
#pragma unroll
  for (int a = 0; a < NP3; ++a) {
    const int q = a % Q19;
    d[a] = Io<S>::to(Io<S>::ld(p + (long long)a * g.pitch - (long long)e3z(q) * g.zs -
                               (long long)e3y(q) * g.lp - e3x(q)));
  }
}

// Eq. 35 and Eq. 37 (or the internal-energy form under Eq. 38): rho, u,
// theta and the specific energy Es = sum h / rho.
template <class C, int M>
__device__ __forceinline__ void moments3(const Grid3& g, const C d[NP3], C& rho, C& ux, C& uy,
                                         C& uz, C& th, C& es) {
  const Phys3<C>& k = phys3<C>(g);
  C sf = d[0], sh = d[Q19];
  C jx = 0, jy = 0, jz = 0;
#pragma unroll
  for (int a = 1; a < Q19; a += 2) {
    sf += d[a] + d[a + 1];
    sh += d[Q19 + a] + d[Q19 + a + 1];
    if (e3x(a)) jx += C(e3x(a)) * (d[a] - d[a + 1]);
    if (e3y(a)) jy += C(e3y(a)) * (d[a] - d[a + 1]);
    if (e3z(a)) jz += C(e3z(a)) * (d[a] - d[a + 1]);
  }
  rho = sf;
  if constexpr ((M & M3_FORCE) != 0) jz -= C(0.5) * rho * k.g;  // rho u = sum e f + a / 2
  const C inv = C(1) / rho;
  ux = jx * inv;
  uy = jy * inv;
  uz = jz * inv;
  es = sh * inv;
  if constexpr ((M & M3_TOTAL) != 0)
    th = k.six_b * (es - C(0.5) * (ux * ux + uy * uy + uz * uz));
  else
    th = k.six_b * es;
}

// f^eq (Eq. 18a, D = 3) and h^eq (Eq. 18b, D = 3, or Es f^eq) per pair of
// opposite velocities:
//   axis (e^2 = 1):     f = rho w [1 - 3/2 u^2 + 9/2 eu^2 +- (6 - 3 theta) eu]
//   diagonal (e^2 = 2): f = rho w [1 - 3/2 u^2 + 9/2 eu^2 + 3/2 (theta - 1)
//                                  +- (3/2 + 3/2 theta) eu]
//   h = Es f + w p [+-3 eu + 9 eu^2 - 3 u^2 + (0 axis | 3/2 theta diagonal)]
// The rest populations are the remainders of sum f^eq = rho and
// sum h^eq = rho Es (Eqs. 19a/19b make this an identity), Es being the
// node's own specific energy.
template <class C, bool TOTAL>
__device__ __forceinline__ void equilibria3(C rho, C ux, C uy, C uz, C th, C es, C feq[Q19],
                                            C heq[Q19]) {
  const C usq = ux * ux + uy * uy + uz * uz;
  const C A0 = C(1) - C(1.5) * usq;
  const C lin1 = C(6) - C(3) * th, lin2 = C(1.5) + C(1.5) * th;
  const C base2 = A0 + C(1.5) * (th - C(1));
  const C p = rho * th * (C(1) / C(3));
  const C hu = C(-3) * usq;
  C sf = 0, sh = 0;
#pragma unroll
  for (int a = 1; a < Q19; a += 2) {
    const C eu = C(e3x(a)) * ux + C(e3y(a)) * uy + C(e3z(a)) * uz;
    const bool axis = a <= 6;
    const C w = w3<C>(a);
    const C even = (axis ? A0 : base2) + C(4.5) * eu * eu;
    const C odd = (axis ? lin1 : lin2) * eu;
    feq[a] = rho * w * (even + odd);
    feq[a + 1] = rho * w * (even - odd);
    if constexpr (TOTAL) {
      const C he = hu + C(9) * eu * eu + (axis ? C(0) : C(1.5) * th);
      const C ho = C(3) * eu;
      heq[a] = es * feq[a] + w * p * (he + ho);
      heq[a + 1] = es * feq[a + 1] + w * p * (he - ho);
    } else {
      heq[a] = es * feq[a];
      heq[a + 1] = es * feq[a + 1];
    }
    sf += feq[a] + feq[a + 1];
    sh += heq[a] + heq[a + 1];
  }
  feq[0] = rho - sf;
  heq[0] = rho * es - sh;
}

// C_a from the gradients dq[k][j] = dQ_j/dx_k (closed form above).
template <class C>
__device__ __forceinline__ void correction3(const C dq[3][3], C cc[Q19]) {
  const C gxx = dq[0][0] + (dq[1][1] + dq[2][2]) * C(1.0 / 6.0);
  const C gyy = dq[1][1] + (dq[0][0] + dq[2][2]) * C(1.0 / 6.0);
  const C gzz = dq[2][2] + (dq[0][0] + dq[1][1]) * C(1.0 / 6.0);
  const C gxy = (dq[0][1] + dq[1][0]) * C(1.0 / 6.0);
  const C gxz = (dq[0][2] + dq[2][0]) * C(1.0 / 6.0);
  const C gyz = (dq[1][2] + dq[2][1]) * C(1.0 / 6.0);
  const C tr = gxx + gyy + gzz;
  const C c0 = tr * C(-5.0 / 21.0);
  const C t47 = tr * C(4.0 / 7.0);
  const C axx = (gxx + t47) * C(1.0 / 6.0), ayy = (gyy + t47) * C(1.0 / 6.0),
          azz = (gzz + t47) * C(1.0 / 6.0);
  cc[0] = c0;
  cc[1] = cc[2] = axx + c0;
  cc[3] = cc[4] = ayy + c0;
  cc[5] = cc[6] = azz + c0;
  const C dxy = axx + ayy + c0, dxz = axx + azz + c0, dyz = ayy + azz + c0;
  const C oxy = gxy * C(0.25), oxz = gxz * C(0.25), oyz = gyz * C(0.25);
  cc[7] = cc[8] = dxy + oxy;    // e_x e_y = +1
  cc[9] = cc[10] = dxy - oxy;   // e_x e_y = -1
  cc[11] = cc[12] = dxz + oxz;  // e_x e_z = +1
  cc[13] = cc[14] = dxz - oxz;  // e_x e_z = -1
  cc[15] = cc[16] = dyz + oyz;  // e_y e_z = +1
  cc[17] = cc[18] = dyz - oyz;  // e_y e_z = -1
}

// f^eq and h^eq of one direction a at (rho, u, theta) with the specific
// energy es (the expressions of equilibria3 for that direction).
template <class C, bool TOTAL>
__device__ __forceinline__ void eq_one3(int a, C rho, C ux, C uy, C uz, C th, C es, C& f, C& h) {
  const C usq = ux * ux + uy * uy + uz * uz;
  const C A0 = C(1) - C(1.5) * usq;
  const C eu = C(e3x(a)) * ux + C(e3y(a)) * uy + C(e3z(a)) * uz;
  const bool axis = e3sq(a) == 1;
  const C w = axis ? w3<C>(1) : w3<C>(7);
  const C even = (axis ? A0 : A0 + C(1.5) * (th - C(1))) + C(4.5) * eu * eu;
  const C odd = (axis ? C(6) - C(3) * th : C(1.5) + C(1.5) * th) * eu;
  f = rho * w * (even + odd);
  if constexpr (TOTAL) {
    const C p = rho * th * (C(1) / C(3));
    const C he = C(-3) * usq + C(9) * eu * eu + (axis ? C(0) : C(1.5) * th);
    h = es * f + w * p * (he + C(3) * eu);
  } else {
    h = es * f;
  }
}

// The populations of node (x, y, z) that leave through a wall come back
// into the node as their opposites (halfway walls at x = -1/2 and nx - 1/2,
// likewise in y and z; a population leaving through an edge of two walled
// sides takes the first of x, y, z): with b the opposite of a,
// f_b = f*_a - 2 (odd part of f^eq_a at the node's rho and theta and the
// wall velocity); h on an isothermal wall h_b = h^eq_b(ghost) +
// (h*_b - h^eq_b), the ghost one spacing outside at u_g = 2 u_w - u,
// theta_g = max(2 theta_w - theta, theta_w / 2), rho_g theta_g =
// rho (theta - 3 g n_z) (the node's pressure carried across by hydrostatic
// balance, n_z the z component of the outward normal); h on an adiabatic
// wall h_b = h*_a - 2 (odd part of h^eq_a at (rho, u_w, theta)), for total
// energy plus the wall's work on the pair u_w . (f_b e_b - f*_a e_a) =
// -(e_a . u_w)(f_b + f*_a) (no heat crosses a moving adiabatic wall; its
// work does).  Each goes to the slot from which the node pulls b:
// x - e_b = x + e_a, a ghost slot.  Sides and directions are compile-time
// after unrolling, so every index into the parameters is a constant.
__device__ __forceinline__ int axis_coord3(int ax, int x, int y, int z) {
  return ax == 0 ? x : (ax == 1 ? y : z);
}
__device__ __forceinline__ int axis_n3(const Grid3& g, int ax) {
  return ax == 0 ? g.nx : (ax == 1 ? g.ny : g.nz);
}
__host__ __device__ constexpr int e3ax(int a, int ax) {
  return ax == 0 ? e3x(a) : (ax == 1 ? e3y(a) : e3z(a));
}
// Side (2 axis + high end) through which population a leaves node
// (x, y, z) if that side is a wall, x before y before z; -1 otherwise.
__device__ __forceinline__ int wall_side3(const Grid3& g, int a, int x, int y, int z) {
#pragma unroll
  for (int ax = 0; ax < 3; ++ax) {
    const int e = e3ax(a, ax);
    if (e == 0) continue;
    const int c = axis_coord3(ax, x, y, z) + e;
    const int s = 2 * ax + (e > 0 ? 1 : 0);
    if ((e < 0 ? c < 0 : c >= axis_n3(g, ax)) && g.bc[s] != BC3_PERIODIC) return s;
  }
  return -1;
}

template <class S, bool TOTAL, int SIDE>
__device__ __forceinline__ void wall_writes_side3(const Grid3& g, S* __restrict__ dst, int x,
                                                  int y, int z,
                                                  const typename Io<S>::C v[NP3],
                                                  const typename Io<S>::C heq[Q19],
                                                  typename Io<S>::C rho, typename Io<S>::C ux,
                                                  typename Io<S>::C uy, typename Io<S>::C uz,
                                                  typename Io<S>::C th) {
  using C = typename Io<S>::C;
  constexpr int AX = SIDE >> 1, DIR = (SIDE & 1) ? 1 : -1;
  const Phys3<C>& k = phys3<C>(g);
  const int c = axis_coord3(AX, x, y, z);
  if (g.bc[SIDE] == BC3_PERIODIC || c != (DIR > 0 ? axis_n3(g, AX) - 1 : 0)) return;
#pragma unroll
  for (int a = 1; a < Q19; ++a) {
    if (e3ax(a, AX) != DIR) continue;
    // an earlier axis's wall takes the populations leaving through an edge
    bool earlier = false;
#pragma unroll
    for (int ax = 0; ax < AX; ++ax) {
      const int e = e3ax(a, ax);
      if (e == 0) continue;
      const int ce = axis_coord3(ax, x, y, z) + e;
      if ((e < 0 ? ce < 0 : ce >= axis_n3(g, ax)) && g.bc[2 * ax + (e > 0 ? 1 : 0)] != BC3_PERIODIC)
        earlier = true;
    }
    if (earlier) continue;
    const int b = (a & 1) ? a + 1 : a - 1;  // opposite
    const C uwx = k.uw[SIDE][0], uwy = k.uw[SIDE][1], uwz = k.uw[SIDE][2];
    const C euw = C(e3x(a)) * uwx + C(e3y(a)) * uwy + C(e3z(a)) * uwz;
    const bool axis = e3sq(a) == 1;
    const C w = axis ? w3<C>(1) : w3<C>(7);
    const C fodd = rho * w * (axis ? C(6) - C(3) * th : C(1.5) + C(1.5) * th) * euw;
    const long long o = slot3(g, 0, x + e3x(a), y + e3y(a), z + e3z(a));
    const C fb = v[a] - C(2) * fodd;
    dst[o + (long long)b * g.pitch] = Io<S>::from(fb);
    C hin;
    if (g.bc[SIDE] == BC3_ISO) {
      const C thg = fmax(C(2) * k.thw[SIDE] - th, C(0.5) * k.thw[SIDE]);
      const C ugx = C(2) * uwx - ux, ugy = C(2) * uwy - uy, ugz = C(2) * uwz - uz;
      const C esg = TOTAL ? k.b6 * thg + C(0.5) * (ugx * ugx + ugy * ugy + ugz * ugz) : k.b6 * thg;
      // the node's pressure carried to the ghost by hydrostatic balance:
      // rho_g theta_g = rho (theta - 3 g n_z), n_z the outward normal's z
      // component (gravity acts along -z)
      C rg;
      if constexpr (AX == 2)
        rg = rho * (th - C(3) * k.g * C(DIR)) / thg;
      else
        rg = rho * th / thg;
      C fg, hg;
      eq_one3<C, TOTAL>(b, rg, ugx, ugy, ugz, thg, esg, fg, hg);
      hin = hg + (v[Q19 + b] - heq[b]);
    } else {
      C hodd;
      if constexpr (TOTAL) {
        const C E = k.b6 * th + C(0.5) * (uwx * uwx + uwy * uwy + uwz * uwz);
        hodd = E * fodd + w * (rho * th * (C(1) / C(3))) * C(3) * euw;
      } else {
        hodd = k.b6 * th * fodd;
      }
      hin = v[Q19 + a] - C(2) * hodd;
      // total energy: the wall's work on the pair, u_w . (f_b e_b - f*_a e_a)
      if constexpr (TOTAL) hin -= euw * (fb + v[a]);
    }
    dst[o + (long long)(Q19 + b) * g.pitch] = Io<S>::from(hin);
  }
}

template <class S, bool TOTAL>
__device__ __forceinline__ void wall_writes3(const Grid3& g, S* __restrict__ dst, int x, int y,
                                             int z, const typename Io<S>::C v[NP3],
                                             const typename Io<S>::C heq[Q19],
                                             typename Io<S>::C rho, typename Io<S>::C ux,
                                             typename Io<S>::C uy, typename Io<S>::C uz,
                                             typename Io<S>::C th) {
  wall_writes_side3<S, TOTAL, 0>(g, dst, x, y, z, v, heq, rho, ux, uy, uz, th);
  wall_writes_side3<S, TOTAL, 1>(g, dst, x, y, z, v, heq, rho, ux, uy, uz, th);
  wall_writes_side3<S, TOTAL, 2>(g, dst, x, y, z, v, heq, rho, ux, uy, uz, th);
  wall_writes_side3<S, TOTAL, 3>(g, dst, x, y, z, v, heq, rho, ux, uy, uz, th);
  wall_writes_side3<S, TOTAL, 4>(g, dst, x, y, z, v, heq, rho, ux, uy, uz, th);
  wall_writes_side3<S, TOTAL, 5>(g, dst, x, y, z, v, heq, rho, ux, uy, uz, th);
}

// Store of the 38 post-collision values of node (x, y, z) at its own slots,
// and for a node on a face the periodic copies into the ghost slots: the
// node at w = wrap(x + e_a) pulls population a from w - e_a.
template <class S>
__device__ __forceinline__ void store3(const Grid3& g, S* __restrict__ dst, int x, int y, int z,
                                       const typename Io<S>::C v[NP3]) {
  S* p = dst + slot3(g, 0, x, y, z);
#pragma unroll
  for (int a = 0; a < NP3; ++a) p[(long long)a * g.pitch] = Io<S>::from(v[a]);
  const bool face = x == 0 || y == 0 || z == 0 || x == g.nx - 1 || y == g.ny - 1 || z == g.nz - 1;
  if (!face) return;
#pragma unroll
  for (int q = 1; q < Q19; ++q) {
    const int dx = x + e3x(q), dy = y + e3y(q), dz = z + e3z(q);
    if (dx >= 0 && dx < g.nx && dy >= 0 && dy < g.ny && dz >= 0 && dz < g.nz) continue;
    // through a wall: wall_writes3 takes it
    if (wall_side3(g, q, x, y, z) >= 0) continue;
    const int sx = wrap3(dx, g.nx) - e3x(q), sy = wrap3(dy, g.ny) - e3y(q),
              sz = wrap3(dz, g.nz) - e3z(q);
    dst[slot3(g, q, sx, sy, sz)] = Io<S>::from(v[q]);
    dst[slot3(g, Q19 + q, sx, sy, sz)] = Io<S>::from(v[Q19 + q]);
  }
}

// The mirror ghost of Eq. 50 across wall side SIDE of a node with rho and
// theta: component j of 2 Q_w - q0, Q_w = rho u_w (1 - theta_w), theta_w
// the wall's on an isothermal wall and the node's own on an adiabatic one.
template <class C, int SIDE>
__device__ __forceinline__ C mirror_q3(const Grid3& g, C rho, C th, int j, C q0) {
  const Phys3<C>& k = phys3<C>(g);
  const C thw = g.bc[SIDE] == BC3_ISO ? k.thw[SIDE] : th;
  return C(2) * rho * k.uw[SIDE][j] * (C(1) - thw) - q0;
}

constexpr int TX3 = 32;

// Cells of the one-node halo ring around a 32 x TY tile, and the threads of a
// block: one per tile cell, plus (SPLIT) whole warps of their own for the
// halo cells; otherwise the tile's first threads take a halo cell each too.
template <int TY>
__host__ __device__ constexpr int nhalo3() {
  return 2 * (TX3 + 2) + 2 * TY;
}
template <int TY, bool SPLIT>
__host__ __device__ constexpr int threads3() {
  return TX3 * TY + (SPLIT ? (nhalo3<TY>() + 31) / 32 * 32 : 0);
}

// Dynamic shared memory of the step kernel with tiles of TY rows: the parked
// populations of two planes, [2][38][tile cells], then the Q ring
// [4][3][halo tile].
template <class S, int TY>
__host__ __device__ constexpr size_t step3d_smem() {
  using C = typename Io<S>::C;
  return sizeof(C) * ((size_t)2 * NP3 * TX3 * TY + 12 * (TX3 + 2) * (TY + 2));
}

// Resident blocks per SM the register budget is sized for: two 256-thread
// blocks (8-row tiles), two 224-thread blocks (4-row tiles with halo warps)
// or one block otherwise; FP64 one.
template <class S, int TY, bool SPLIT>
__host__ __device__ constexpr int step3d_min_blocks() {
  return sizeof(S) == 8 ? 1 : ((SPLIT ? TY <= 4 : TY == 8) ? 2 : 1);
}

// One time step of every node of the block's 32 x TY tile over z in
// [z0, z0 + zrows).  Per plane r: pull the populations of plane r (each
// tile cell: parked in shared memory for the collision a plane later) and
// form Q = rho u (1 - theta) of the tile and its halo ring into a 4-plane
// ring; one barrier; collide plane r - 1.  With four planes in the ring the
// slot written at plane r + 1 was last read by the collision of plane r - 2,
// which every thread finished before the barrier of plane r, so one barrier
// per plane suffices (and threads that are done with the collision go on
// pulling the next plane while the others collide).
template <class S, int M, int TY, bool SPLIT>
__global__ void __launch_bounds__(threads3<TY, SPLIT>(), (step3d_min_blocks<S, TY, SPLIT>()))
    step3d_kernel(const Grid3 g, int zrows) {
  using C = typename Io<S>::C;
  constexpr int HX = TX3 + 2, HY = TY + 2, HN = HX * HY, NT = TX3 * TY;
  constexpr int NHALO = HN - NT;
  static_assert(NHALO == nhalo3<TY>(), "halo ring");
  static_assert(SPLIT || NHALO <= NT, "one halo cell per thread at most");
  extern __shared__ __align__(16) unsigned char smem3[];
  C* park = reinterpret_cast<C*>(smem3);  // [2][NP3][NT]
  C(*qs)[3][HN] = reinterpret_cast<C(*)[3][HN]>(park + 2 * NP3 * NT);  // [4][3][HN]

  const int t = threadIdx.x;
  const bool interior = !SPLIT || t < NT;  // owns a tile cell
  const int hk = SPLIT ? t - NT : t;      // halo cell index, if in [0, NHALO)
  const int tx = t % TX3, ty = t / TX3;
  const int nx = g.nx, ny = g.ny, nz = g.nz;
  const int x0 = blockIdx.x * TX3, y0 = blockIdx.y * TY, z0 = blockIdx.z * zrows;
  if (z0 >= nz) return;
  const int z1 = min(z0 + zrows, nz);
  const S* __restrict__ src = static_cast<const S*>(g.src);
  S* __restrict__ dst = static_cast<S*>(g.dst);

  // this thread's interior cell and node
  const int cell = (ty + 1) * HX + tx + 1;
  const int x = x0 + tx, y = y0 + ty;
  const bool mine = interior && x < nx && y < ny;
  const int wx = wrap3(x % nx, nx), wy = wrap3(y % ny, ny);  // wrapped (ragged tiles)
  // this thread's node on a walled x or y side
  const bool wxl = x == 0 && g.bc[0] != BC3_PERIODIC, wxh = x == nx - 1 && g.bc[1] != BC3_PERIODIC;
  const bool wyl = y == 0 && g.bc[2] != BC3_PERIODIC, wyh = y == ny - 1 && g.bc[3] != BC3_PERIODIC;
  const bool wxy = wxl || wxh || wyl || wyh;
  // halo cell of this thread: the ring around the tile
  int hcell = -1, hx = 0, hy = 0;
  if (hk >= 0 && hk < NHALO) {
    int cx, cy;
    if (hk < HX) {
      cx = hk;
      cy = 0;
    } else if (hk < 2 * HX) {
      cx = hk - HX;
      cy = HY - 1;
    } else {
      const int k = hk - 2 * HX;  // the side columns, rows 1 .. HY - 2
      cx = (k & 1) ? HX - 1 : 0;
      cy = 1 + (k >> 1);
    }
    hcell = cy * HX + cx;
    hx = wrap3(((x0 + cx - 1) % nx + nx) % nx, nx);
    hy = wrap3(((y0 + cy - 1) % ny + ny) % ny, ny);
  }

  C prho = 1, pux = 0, puy = 0, puz = 0, pth = 1, pes = 0;
  for (int r = z0 - 1; r <= z1; ++r) {
    const int s = (r - z0 + 1) & 3;
    const int zr = wrap3(r, nz);
    // moments of plane r: this thread's cell (wrapped), and its halo cell
    C crho = 1, cux = 0, cuy = 0, cuz = 0, cth = 1, ces = 0;
    if (interior) {
      C d[NP3];
      pull3<S>(g, src, wx, wy, zr, d);
      C* pk = park + (r & 1) * NP3 * NT + t;
#pragma unroll
      for (int a = 0; a < NP3; ++a) pk[a * NT] = d[a];
      moments3<C, M>(g, d, crho, cux, cuy, cuz, cth, ces);
      const C f = crho * (C(1) - cth);
      qs[s][0][cell] = f * cux;
      qs[s][1][cell] = f * cuy;
      qs[s][2][cell] = f * cuz;
    }
    if (hcell >= 0) {
      C d[NP3], hr, hu, hv, hw, ht, he;
      pull3<S>(g, src, hx, hy, zr, d);
      moments3<C, M>(g, d, hr, hu, hv, hw, ht, he);
      const C f = hr * (C(1) - ht);
      qs[s][0][hcell] = f * hu;
      qs[s][1][hcell] = f * hv;
      qs[s][2][hcell] = f * hw;
    }
    __syncthreads();
    const int zc = r - 1;  // plane to collide
    if (zc >= z0 && mine) {
      const int sm = (s + 2) & 3, s0 = (s + 3) & 3;  // planes r - 2 and r - 1
      C dq[3][3];  // dq[k][j] = dQ_j / dx_k
      // across a wall Eq. 50 takes the mirror ghost 2 Q_w - Q(node),
      // Q_w = rho u_w (1 - theta_w) (theta_w: the node's own on an adiabatic
      // wall)
      const bool wb = zc == 0 && g.bc[4] != BC3_PERIODIC;
      const bool wt = zc == nz - 1 && g.bc[5] != BC3_PERIODIC;
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        C xp = qs[s0][j][cell + 1], xm = qs[s0][j][cell - 1];
        C yp = qs[s0][j][cell + HX], ym = qs[s0][j][cell - HX];
        C up = qs[s][j][cell], dn = qs[sm][j][cell];
        if (wxy || wb || wt) {
          const C q0 = qs[s0][j][cell];
          if (wxl) xm = mirror_q3<C, 0>(g, prho, pth, j, q0);
          if (wxh) xp = mirror_q3<C, 1>(g, prho, pth, j, q0);
          if (wyl) ym = mirror_q3<C, 2>(g, prho, pth, j, q0);
          if (wyh) yp = mirror_q3<C, 3>(g, prho, pth, j, q0);
          if (wb) dn = mirror_q3<C, 4>(g, prho, pth, j, q0);
          if (wt) up = mirror_q3<C, 5>(g, prho, pth, j, q0);
        }
        dq[0][j] = C(0.5) * (xp - xm);
        dq[1][j] = C(0.5) * (yp - ym);
        dq[2][j] = C(0.5) * (up - dn);
      }
      C cc[Q19];
      if constexpr ((M & M3_CORR) != 0) {
        correction3<C>(dq, cc);
      } else {
#pragma unroll
        for (int a = 0; a < Q19; ++a) cc[a] = C(0);
      }
      if constexpr ((M & M3_FORCE) != 0) {
        // Guo's force term beside C (Eq. 51 with D = 3), a = (0, 0, -rho g):
        // F_a = w_a [3 (e_a - u).a + 9 (e_a.u)(e_a.a)]
        const C az = -prho * phys3<C>(g).g;
#pragma unroll
        for (int a = 0; a < Q19; ++a) {
          const C eu = C(e3x(a)) * pux + C(e3y(a)) * puy + C(e3z(a)) * puz;
          const C ea = C(e3z(a)) * az;
          cc[a] += w3<C>(a) * (C(3) * (ea - puz * az) + C(9) * eu * ea);
        }
      }
      C d[NP3];
      const C* pk = park + (zc & 1) * NP3 * NT + t;  // parked by this thread at plane zc
#pragma unroll
      for (int a = 0; a < NP3; ++a) d[a] = pk[a * NT];
      C feq[Q19], heq[Q19];
      equilibria3<C, (M & M3_TOTAL) != 0>(prho, pux, puy, puz, pth, pes, feq, heq);
      const Phys3<C>& k = phys3<C>(g);
      const C wf = k.omega_f, wh = k.omega_h, kc = C(1) - C(0.5) * wf;
      const C zc2 = (M & M3_ZFULL) ? C(0.5) * (pux * pux + puy * puy + puz * puz) : C(0);
      C v[NP3];
#pragma unroll
      for (int a = 0; a < Q19; ++a) {
        const C fneq = d[a] - feq[a];
        v[a] = d[a] - wf * fneq + kc * cc[a];  // Eq. 34 with +(1 - w_f/2) C
        C hs = d[Q19 + a] - wh * (d[Q19 + a] - heq[a]);
        if constexpr ((M & M3_TOTAL) != 0) {  // Eq. 36
          const C eu = C(e3x(a)) * pux + C(e3y(a)) * puy + C(e3z(a)) * puz;
          hs += k.kz * (eu - zc2) * (fneq + C(0.5) * cc[a]);
        }
        v[Q19 + a] = hs;
      }
      store3<S>(g, dst, x, y, zc, v);
      if (wxy || wb || wt)
        wall_writes3<S, (M & M3_TOTAL) != 0>(g, dst, x, y, zc, v, heq, prho, pux, puy, puz, pth);
    }
    prho = crho;
    pux = cux;
    puy = cuy;
    puz = cuz;
    pth = cth;
    pes = ces;
  }
}

// ---- initialisation, export, reductions -----------------------------------

// Equilibrium state (FP64) of node i at the given fields, scattered into the
// slots the next pull reads: buf_a(x - e_a).
template <class S, bool TOTAL>
__global__ void init3d_kernel(const Grid3 g, S* buf, const double* __restrict__ rho,
                              const double* __restrict__ ux, const double* __restrict__ uy,
                              const double* __restrict__ uz, const double* __restrict__ T,
                              double invT0) {
  const long long n = (long long)g.nx * g.ny * g.nz;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(i % g.nx), y = (int)((i / g.nx) % g.ny), z = (int)(i / g.nx / g.ny);
    const double th = T[i] * invT0;
    const double es = TOTAL ? g.pd.b6 * th + 0.5 * (ux[i] * ux[i] + uy[i] * uy[i] + uz[i] * uz[i])
                            : g.pd.b6 * th;
    double feq[Q19], heq[Q19];
    equilibria3<double, TOTAL>(rho[i], ux[i], uy[i], uz[i], th, es, feq, heq);
    for (int a = 0; a < Q19; ++a) {
      const long long o = slot3(g, a, x - e3x(a), y - e3y(a), z - e3z(a));
      buf[o] = Io<S>::from((typename Io<S>::C)feq[a]);
      buf[o + (long long)Q19 * g.pitch] = Io<S>::from((typename Io<S>::C)heq[a]);
    }
  }
}

// Canonical populations (FP64) of node (x, y, z).
template <class S>
__device__ __forceinline__ void pull3_fp64(const Grid3& g, const S* __restrict__ buf, int x,
                                           int y, int z, double p[NP3]) {
  for (int a = 0; a < NP3; ++a) {
    const int q = a % Q19;
    p[a] = (double)Io<S>::to(buf[slot3(g, a, x - e3x(q), y - e3y(q), z - e3z(q))]);
  }
}

// rho, u, T (FP64) and optionally the canonical populations [38][nz][ny][nx];
// *nonfinite set to 1 if a moment is NaN or infinite.
template <class S>
__global__ void export3d_kernel(const Grid3 g, const S* __restrict__ buf, double* rho, double* ux,
                                double* uy, double* uz, double* T, double T0, double* pops,
                                int* nonfinite) {
  const long long n = (long long)g.nx * g.ny * g.nz;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(i % g.nx), y = (int)((i / g.nx) % g.ny), z = (int)(i / g.nx / g.ny);
    double p[NP3];
    pull3_fp64<S>(g, buf, x, y, z, p);
    if (pops)
      for (int a = 0; a < NP3; ++a) pops[(long long)a * n + i] = p[a];
    if (rho) {
      double r = 0, jx = 0, jy = 0, jz = 0, sh = 0;
      for (int a = 0; a < Q19; ++a) {
        r += p[a];
        jx += e3x(a) * p[a];
        jy += e3y(a) * p[a];
        jz += e3z(a) * p[a];
        sh += p[Q19 + a];
      }
      const double vx = jx / r, vy = jy / r, vz = (jz - 0.5 * r * g.pd.g) / r;
      const double th = g.energy_model == 0
                            ? g.pd.six_b * (sh / r - 0.5 * (vx * vx + vy * vy + vz * vz))
                            : g.pd.six_b * sh / r;
      rho[i] = r;
      ux[i] = vx;
      uy[i] = vy;
      uz[i] = vz;
      T[i] = th * T0;
      if (nonfinite && !(isfinite(r) && isfinite(vx) && isfinite(vy) && isfinite(vz) &&
                         isfinite(th)))
        *nonfinite = 1;
    }
  }
}

// Per-block FP64 partial sums of rho, rho u (3) and hbar, fixed order.
constexpr int RED3 = 256;
template <class S>
__global__ void __launch_bounds__(RED3) conserved3d_kernel(const Grid3 g, const S* __restrict__ buf,
                                                           double* partial) {
  __shared__ double sm[5][RED3];
  const long long n = (long long)g.nx * g.ny * g.nz;
  double acc[5] = {0, 0, 0, 0, 0};
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(i % g.nx), y = (int)((i / g.nx) % g.ny), z = (int)(i / g.nx / g.ny);
    double p[NP3];
    pull3_fp64<S>(g, buf, x, y, z, p);
    for (int a = 0; a < Q19; ++a) {
      acc[0] += p[a];
      acc[1] += e3x(a) * p[a];
      acc[2] += e3y(a) * p[a];
      acc[3] += e3z(a) * p[a];
      acc[4] += p[Q19 + a];
    }
  }
  for (int k = 0; k < 5; ++k) sm[k][threadIdx.x] = acc[k];
  __syncthreads();
  for (int s = RED3 / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s)
      for (int k = 0; k < 5; ++k) sm[k][threadIdx.x] += sm[k][threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int k = 0; k < 5; ++k) partial[5 * blockIdx.x + k] = sm[k][0];
}

template <int UNUSED = 0>
__global__ void conserved3d_final_kernel(const double* __restrict__ partial, int nb, double* out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  for (int k = 0; k < 5; ++k) {
    double s = 0;
    for (int i = 0; i < nb; ++i) s += partial[5 * i + k];
    out[k] = s;
  }
}

}  // namespace lbm3
