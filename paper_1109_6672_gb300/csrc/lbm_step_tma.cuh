// Building blocks of the TMA-staged step kernel (lbm_step_pr.cuh): the
// compile-time physics mode, the per-node moments and collision written for
// one mode, and the mbarrier / bulk-tensor-copy primitives.
//
// The physics mode (total or internal energy, form of Z, correction, force)
// is a template parameter, so the per-direction code is straight-line.
#pragma once

#include <cuda.h>

#include "lbm_device.cuh"

namespace lbm {

// ---- compile-time physics mode ---------------------------------------------

enum { MODE_TOTAL = 1, MODE_ZFULL = 2, MODE_CORR = 4, MODE_FORCE = 8, MODE_MRT = 16,
       MODE_VARMU = 32 };

// The BGK modes mode_of() produces (total energy with the full or simple Z,
// internal energy with or without gravity; each with or without the
// correction); each has an MRT twin (| MODE_MRT), and each of those a twin
// with a temperature-dependent viscosity (| MODE_VARMU).
constexpr int NUM_BGK_MODES = 8;
constexpr int BGK_MODES[NUM_BGK_MODES] = {MODE_TOTAL | MODE_ZFULL | MODE_CORR,
                                          MODE_TOTAL | MODE_ZFULL,
                                          MODE_TOTAL | MODE_CORR,
                                          MODE_TOTAL,
                                          MODE_FORCE | MODE_CORR,
                                          MODE_FORCE,
                                          MODE_CORR,
                                          0};

template <int M>
struct Mode {
  static constexpr bool total = (M & MODE_TOTAL) != 0;
  static constexpr bool zfull = (M & MODE_ZFULL) != 0;
  static constexpr bool corr = (M & MODE_CORR) != 0;
  static constexpr bool force = (M & MODE_FORCE) != 0;
  static constexpr bool mrt = (M & MODE_MRT) != 0;
  static constexpr bool varmu = (M & MODE_VARMU) != 0;
};

// The eight modes the validated parameters can produce (Z only matters for
// total energy; gravity needs internal energy).
inline int mode_of(const Grid& g) {
  int m = 0;
  if (g.energy_model == E_TOTAL) {
    m |= MODE_TOTAL;
    if (g.z_full) m |= MODE_ZFULL;
  } else if (g.has_force) {
    m |= MODE_FORCE;
  }
  if (g.correction) m |= MODE_CORR;
  if (g.collision == COLL_MRT) m |= MODE_MRT;
  if (g.mu_law != MU_TAU) m |= MODE_VARMU;
  return m;
}

// Moments of the pulled populations d (Eq. 35 with the force shift under
// Eq. 51; Eq. 37 or the Eq. 38 form for theta).  Absolute storage returns
// r0 = rho, rth = theta, res = Es (= sum h / rho); deviation storage returns
// the deviations from the rest state, r0 = rho - 1, rth = theta - 1,
// res = Es - b/6, formed from the sums of the stored deviations so that
// nothing is rounded at the scale of the populations (the references' own
// sums are taken in FP64 on the host: dref).  The balance of internal
// energy, rho (Es - b/6) - rho u^2 / 2, is then one subtraction of two FP32
// numbers, and FP32's correctly rounded subtraction gives the value an FP64
// subtraction rounded back to FP32 would: the exact difference is an FP64
// number when the exponents differ by at most 28, and otherwise lies within
// 2^-28 of the larger operand, far from any FP32 rounding tie.
template <class S, int M>
__device__ __forceinline__ void moments_m(const Grid& g, const typename Io<S>::C d[NPOP],
                                          typename Io<S>::C& r0, typename Io<S>::C& ux,
                                          typename Io<S>::C& uy, typename Io<S>::C& rth,
                                          typename Io<S>::C& res) {
  using C = typename Io<S>::C;
  using MD = Mode<M>;
  const Phys<C>& k = phys<C>(g);
  const C sf = (d[0] + d[1]) + (d[2] + d[3]) + (d[4] + d[5]) + (d[6] + d[7]) + d[8];
  const C sh = (d[9] + d[10]) + (d[11] + d[12]) + (d[13] + d[14]) + (d[15] + d[16]) + d[17];
  const C jx = (d[1] - d[3]) + (d[5] - d[7]) + (d[8] - d[6]);
  C jy = (d[2] - d[4]) + (d[5] - d[7]) + (d[6] - d[8]);
  const C rho = Io<S>::dev ? C(1) + sf : sf;  // the f references sum to 1
  if constexpr (MD::force) jy -= C(0.5) * rho * k.g;
  C inv;
  if constexpr (sizeof(C) == 4)
    inv = __frcp_rn(rho);
  else
    inv = C(1) / rho;
  ux = jx * inv;
  uy = jy * inv;
  if constexpr (Io<S>::dev) {
    r0 = sf;
    if constexpr (sizeof(S) == 2) {
      const C e = k.dref + sh - k.b6 * sf;  // rho (Es - b/6): small terms only
      res = e * inv;
      if constexpr (MD::total) {
        const C kin = C(0.5) * (rho * (ux * ux + uy * uy));
        rth = k.six_b * __fsub_rn(e, kin) * inv;
      } else {
        rth = k.six_b * res;
      }
    } else {
      res = (k.dref + sh - k.b6 * sf) * inv;
      rth = k.six_b * (MD::total ? res - C(0.5) * (ux * ux + uy * uy) : res);
    }
  } else if constexpr (MD::total) {
    r0 = rho;
    res = sh * inv;
    rth = k.six_b * (res - C(0.5) * (ux * ux + uy * uy));
  } else {
    r0 = rho;
    res = sh * inv;
    rth = k.six_b * res;
  }
}

// Collision (Eq. 34 with +(1 - w_f/2) C', Eq. 36 or Eq. 38; C' = C_a of
// Eq. 49 plus the Guo force; MRT: Eq. 44) of one node and its 18 stores at p
// (node slot, population stride `pitch`).  (r0, rth, res) as moments_m
// returns them.  v receives f*, h*, h^eq for the wall rules: absolute values
// for absolute storage, deviations from the rest equilibria for deviation
// storage (whose arithmetic then runs on deviations throughout).
template <class S, int M>
__device__ __forceinline__ void collide_m(const Grid& g, S* __restrict__ p, int pitch, int x, int y,
                                          const typename Io<S>::C d[NPOP], typename Io<S>::C r0,
                                          typename Io<S>::C ux, typename Io<S>::C uy,
                                          typename Io<S>::C rth, typename Io<S>::C res,
                                          typename Io<S>::C dqx, typename Io<S>::C dqy,
                                          typename Io<S>::C v[27]) {
  using C = typename Io<S>::C;
  using MD = Mode<M>;
  constexpr bool DEV = Io<S>::dev;
  const Phys<C>& k = phys<C>(g);
  const C rho = DEV ? C(1) + r0 : r0;
  C wf = k.omega_f, wh = k.omega_h, kz = k.kz;
  if constexpr (MD::varmu) node_rates<C>(g, k, rho, DEV ? C(1) + rth : rth, MD::mrt, wf, wh, kz);
  C feq[9], heq[9];
  if constexpr (DEV) {
    const C sdh = (d[9] + d[10]) + (d[11] + d[12]) + (d[13] + d[14]) + (d[15] + d[16]) + d[17];
    equilibria_dev<C>(r0, ux, uy, rth, res, k.b6, MD::total, sdh, feq, heq);
  } else {
    collision_equilibria<C>(rho, ux, uy, rth, res, k.b6, MD::total, feq, heq);
  }

  C cc[9];
#pragma unroll
  for (int a = 0; a < 9; ++a) cc[a] = C(0);
  const C phx = C(3) * (dqx + dqy), phy = dqx - dqy;
  if constexpr (MD::corr) {
    const C c13 = phx * C(-1.0 / 36.0) + phy * C(0.25);
    const C c24 = phx * C(-1.0 / 36.0) - phy * C(0.25);
    const C cd = phx * C(1.0 / 18.0);
    cc[0] = phx * C(-1.0 / 9.0);
    cc[1] = c13;
    cc[3] = c13;
    cc[2] = c24;
    cc[4] = c24;
    cc[5] = cd;
    cc[6] = cd;
    cc[7] = cd;
    cc[8] = cd;
  }
  if constexpr (MD::force) {
    // F_a = w_a [3 e.a + 9 (e.u)(e.a) - 3 u.a], a = (0, ay)
    const C ay = -rho * k.g;
#pragma unroll
    for (int a = 0; a < 9; ++a) {
      const C ea = C(ey(a)) * ay;
      const C eu = C(ex(a)) * ux + C(ey(a)) * uy;
      cc[a] += wgt<C>(a) * (C(3) * ea + C(9) * eu * ea - C(3) * uy * ay);
    }
  }
  const C kc = C(1) - C(0.5) * wf;
  const C zc = MD::zfull ? C(0.5) * (ux * ux + uy * uy) : C(0);
  // fa, ha: the stored quantity (absolute value or deviation); the
  // non-equilibrium parts f - f^eq, h - h^eq are the same either way
  if constexpr (MD::mrt) {
    C fa[9], fneq[9], mc[9];
#pragma unroll
    for (int a = 0; a < 9; ++a) {
      fa[a] = d[a];
      fneq[a] = fa[a] - feq[a];
    }
    mrt_source<C>(MD::corr, phx, phy, MD::force, ux, uy, -rho * k.g, mc);
    mrt_collide<C>(k, wf, fa, fneq, mc, v);
  }
#pragma unroll
  for (int a = 0; a < 9; ++a) {
    const C fa = d[a], ha = d[9 + a];
    const C fneq = fa - feq[a];
    if constexpr (!MD::mrt) v[a] = fa - wf * fneq + kc * cc[a];
    C hs = ha - wh * (ha - heq[a]);
    if constexpr (MD::total) {
      const C eu = C(ex(a)) * ux + C(ey(a)) * uy;
      hs += kz * (eu - zc) * (fneq + C(0.5) * cc[a]);
    }
    v[9 + a] = hs;
    v[18 + a] = heq[a];
  }
  if constexpr (Io<S>::sr) {
    // stochastic rounding in hardware, two populations per conversion and
    // one random word per pair (non-finite values pass through unchanged)
    unsigned r = sr_hash(g, x, y);
#pragma unroll
    for (int a = 0; a < NPOP; a += 2) {
      r = lcg_next(r);
      S sa, sb;
      Io<S>::from_sr2(v[a], v[a + 1], r, sa, sb);
      p[plane(a) * pitch] = sa;
      p[plane(a + 1) * pitch] = sb;
    }
  } else {
#pragma unroll
    for (int a = 0; a < NPOP; ++a) p[plane(a) * pitch] = Io<S>::from(v[a]);
  }
}

// ---- TMA pipeline primitives ----------------------------------------------

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(unsigned bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(unsigned bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_test(unsigned bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Wait for phase `parity` of the barrier, giving up after `limit_ns`.
__device__ __forceinline__ bool mbar_wait(unsigned bar, unsigned parity,
                                          unsigned long long limit_ns) {
  if (mbar_test(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  while (!mbar_test(bar, parity)) {
    if (global_ns() - t0 > limit_ns) return false;
  }
  return true;
}

__device__ __forceinline__ void tma_load_box(unsigned dst, const CUtensorMap* map, unsigned bar,
                                             int cx, int ca, int cy) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
      "l"(reinterpret_cast<unsigned long long>(map)), "r"(cx), "r"(ca), "r"(cy), "r"(bar)
      : "memory");
}

}  // namespace lbm
