// Device side of the coupled DDF thermal lattice Boltzmann step (D2Q9), after
// Li, Luo, He, Gao & Tao, arXiv:1109.6672, BGK scheme of Sec. III.C.1.
//
// State layout (one buffer; two buffers ping-pong):
//   element (a, x, y), a = 0..17 (f_0..f_8, h_0..h_8), x in [-1, nx],
//   y in [-1, ny], lives at
//       base + (y + 1) * 18 * pitch + plane(a) * pitch + x + 32.
//   Rows of the 18 populations of one lattice row are adjacent ("row
//   interleaved SoA"); a warp reading 32 consecutive x of one population
//   reads 32 contiguous elements, and x = 0 starts a 32-element boundary, so
//   the stores of a block whose first column is a multiple of 32 are aligned.
//   pitch >= nx + 33 and is a multiple of 32; x = -1 and x = nx fall in
//   padding that no other element uses: that is the one-node ghost ring.
//   plane(a) groups the populations by e_y: planes 0-5 hold e_y = +1
//   (f2 f5 f6 h2 h5 h6), 6-11 e_y = 0 (f0 f1 f3 h0 h1 h3), 12-17 e_y = -1
//   (f4 f7 f8 h4 h7 h8), so the values one lattice row pulls from the row
//   below, the same row and the row above are three contiguous plane groups.
//
// Meaning of a buffer: it holds post-collision populations f*_a(s) at the
// slot s from which node s + e_a pulls them, so the canonical pre-collision
// state of node x is fbar_a(x) = buf_a(x - e_a) for every a (pull streaming,
// left-hand side of Eqs. 34 and 36).  Interior slots are written by the
// collision of the node itself; ghost slots are written at collision time by
// boundary nodes (periodic copies, or the wall rules), so the pull needs no
// boundary logic at all.
//
// The correction C_a (Eqs. 48-50) needs Q = rho u (1 - theta) of the four
// axis neighbours at the same time level.  A block owns a strip of
// blockDim.x - 2 columns and marches down its rows: each row's pulled
// populations and moments are computed once (plus one halo column on each
// side), Q_x is exchanged through shared memory, Q_y stays in the thread's
// registers for the row above and below, and the row is collided one
// iteration later, when the row above is known.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

namespace lbm {

constexpr int NPOP = 18;
constexpr int XOFF = 32;  // element offset of x = 0 within a population row

// BC_INLET / BC_OUTLET: open x sides (x- / x+ only, y periodic).  The step
// kernels treat them as walls; side_fixup_kernel (lbm_open.cuh) then rewrites
// their ghost slots.
enum { BC_PERIODIC = 0, BC_ISO = 1, BC_ADIA = 2, BC_INLET = 3, BC_OUTLET = 4 };
enum { E_TOTAL = 0, E_INTERNAL = 1 };

// D2Q9 velocities (Eq. 6 with c = 1) and weights (below Eq. 8).
__host__ __device__ constexpr int ex(int a) {
  return (a == 1 || a == 5 || a == 8) ? 1 : ((a == 3 || a == 6 || a == 7) ? -1 : 0);
}
__host__ __device__ constexpr int ey(int a) {
  return (a == 2 || a == 5 || a == 6) ? 1 : ((a == 4 || a == 7 || a == 8) ? -1 : 0);
}
__host__ __device__ constexpr int opp(int a) {
  return a == 0 ? 0 : (a <= 4 ? ((a + 1) % 4) + 1 : ((a - 3) % 4) + 5);
}
template <class C>
__host__ __device__ constexpr C wgt(int a) {
  return a == 0 ? C(4) / C(9) : (a <= 4 ? C(1) / C(9) : C(1) / C(36));
}

// Storage plane of population a (0..17): group by e_y (+1, 0, -1), then
// distribution (f, h), then velocity.
__host__ __device__ constexpr int pgroup(int a) {
  return ey(a % 9) > 0 ? 0 : (ey(a % 9) == 0 ? 1 : 2);
}
__host__ __device__ constexpr int pidx(int q) {
  return (q == 2 || q == 0 || q == 4) ? 0 : ((q == 5 || q == 1 || q == 7) ? 1 : 2);
}
__host__ __device__ constexpr int plane(int a) {
  return 6 * pgroup(a) + 3 * (a / 9) + pidx(a % 9);
}

// Physical constants in one arithmetic precision (lattice units, R T0 = 1/3).
enum { COLL_BGK = 0, COLL_MRT = 1 };
enum { MU_TAU = 0, MU_POWER = 1, MU_SUTHERLAND = 2 };

template <class C>
struct Phys {
  C omega_f, omega_h;  // 2 / (2 tau + 1)
  C g;                 // gravity, a = (0, -rho g)
  C b6, six_b;         // b / 6 and 6 / b
  C dref;              // sum of the h references - b/6 (deviation storage)
  C uw[4][2];          // wall velocities
  C thw[4];            // wall theta = T_w / T0
  C kz;                // coefficient of the Z coupling of h (Eq. 36 / Eq. 47)
  C se, seps, sq;      // MRT rates of e, epsilon, q (Eq. 40); 0: the node's omega_f
  C tau_f0, tau_ratio; // tau_f at rho = 1, T = T0 and tau_h / tau_f (viscosity laws)
  C mu_n, mu_s;        // power-law exponent, Sutherland S / T0
};

// Per-grid launch argument.
struct Grid {
  void* src;  // state at time t (pull layout)
  void* dst;  // state at time t + 1
  int nx, ny, pitch, rp;  // rp = 18 * pitch
  int bc[4];              // x-, x+, y-, y+
  int energy_model, correction, z_full, has_force;
  int collision;          // COLL_BGK or COLL_MRT
  int mu_law;             // MU_TAU, MU_POWER or MU_SUTHERLAND
  Phys<double> pd;
  Phys<float> pf;
  float fref[9], href[9];  // rest equilibria (deviation storage)
  double href_sum;         // sum of href in FP64
  double dref;             // href_sum - b/6 (rounding of the references)
  // inlet (x-, Eq. 53): rho = in_rho + in_drho s, u = uw[0] + (in_du s, 0),
  // theta = thw[0] + in_dth s, s = sin(in_omega t)
  double in_rho, in_drho, in_du, in_dth, in_omega;
  int nee;                 // sides (bit s) with walls of non-equilibrium extrapolation
  int* status;             // device error word (bounded waits), may be NULL
  unsigned t;              // time step being taken (stochastic rounding counter)
};

template <class C>
__host__ __device__ __forceinline__ const Phys<C>& phys(const Grid& g) {
  if constexpr (sizeof(C) == 8)
    return g.pd;
  else
    return g.pf;
}

// ---- storage <-> compute ---------------------------------------------------

template <class S>
struct Io;
// dev: the buffer holds deviations from the rest equilibria (pref); sr: the
// stores round stochastically (from_sr).
template <>
struct Io<double> {
  using C = double;
  static constexpr bool dev = false;
  static constexpr bool sr = false;
  __device__ static double ld(const double* p) { return __ldg(p); }
  __device__ static double to(double v) { return v; }
  __device__ static double from(double v) { return v; }
};
template <>
struct Io<float> {
  using C = float;
  static constexpr bool dev = false;
  static constexpr bool sr = false;
  __device__ static float ld(const float* p) { return __ldg(p); }
  __device__ static float to(float v) { return v; }
  __device__ static float from(float v) { return v; }
};
// 16-bit deviations.  FP16 holds 256 x the deviation (an exact scaling that
// moves deviations down to 2.4e-7 into the normal range; the largest, 255, is
// far above any population).  from_sr() rounds stochastically with the 32
// random bits r: up with probability equal to the dropped fraction of a
// spacing, so the rounding error has zero mean (non-finite values and FP16
// overflow round to nearest, so they stay non-finite).
template <>
struct Io<__half> {
  using C = float;
  static constexpr bool dev = true;
  static constexpr bool sr = true;
  __device__ static __half ld(const __half* p) { return __ldg(p); }
  __device__ static float to(__half v) { return __half2float(v) * (1.0f / 256.0f); }
  __device__ static __half from(float v) { return __float2half_rn(v * 256.0f); }
  // |256 v| below the FP16 maximum 65504 (false for NaN)
  __device__ static bool in_range(float v) { return fabsf(v) < 255.875f; }
  // stochastic rounding of an in-range value: FP32 -> FP16 keeps 10 of 23
  // mantissa bits, so add 13 random bits, cut them, and convert the now
  // exactly representable value
  __device__ static __half from_sr_in_range(float v, unsigned r) {
    const unsigned u = (__float_as_uint(v * 256.0f) + (r >> 19)) & 0xFFFFE000u;
    return __float2half_rz(__uint_as_float(u));
  }
  __device__ static __half from_sr(float v, unsigned r) {
    return in_range(v) ? from_sr_in_range(v, r) : __float2half_rn(v * 256.0f);
  }
  // two values in one stochastically rounding conversion (cvt.rs, sm_100
  // family): the random word r supplies the bits of both (bits 28-16 the
  // first value's, 12-0 the second's).  No saturation: non-finite values
  // stay non-finite, and a finite 256 v at or above 65536 becomes infinite
  // (in the last spacing below it, infinite or 65504 at random), so a
  // diverging state is still flagged
  __device__ static void from_sr2(float va, float vb, unsigned r, __half& sa, __half& sb) {
    unsigned d;
    asm("cvt.rs.f16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(va * 256.0f), "f"(vb * 256.0f), "r"(r));
    sa = __ushort_as_half((unsigned short)(d >> 16));
    sb = __ushort_as_half((unsigned short)(d & 0xFFFFu));
  }
};
template <>
struct Io<__nv_bfloat16> {
  using C = float;
  static constexpr bool dev = true;
  static constexpr bool sr = true;
  __device__ static __nv_bfloat16 ld(const __nv_bfloat16* p) { return __ldg(p); }
  __device__ static float to(__nv_bfloat16 v) { return __bfloat162float(v); }
  __device__ static __nv_bfloat16 from(float v) { return __float2bfloat16_rn(v); }
  // finite (false for infinities and NaN)
  __device__ static bool in_range(float v) { return fabsf(v) <= 3.40282347e38f; }
  // stochastic rounding of a finite value: BF16 is the upper half of FP32,
  // so add 16 random bits below it and cut
  __device__ static __nv_bfloat16 from_sr_in_range(float v, unsigned r) {
    return __ushort_as_bfloat16((unsigned short)((__float_as_uint(v) + (r >> 16)) >> 16));
  }
  __device__ static __nv_bfloat16 from_sr(float v, unsigned r) {
    return in_range(v) ? from_sr_in_range(v, r) : __float2bfloat16_rn(v);
  }
  // two values in one stochastically rounding conversion (cvt.rs, sm_100
  // family), as for FP16 (bits 31-16 round the first value, 15-0 the
  // second; a value rounded up past the largest finite one is infinite)
  __device__ static void from_sr2(float va, float vb, unsigned r, __nv_bfloat16& sa,
                                  __nv_bfloat16& sb) {
    unsigned d;
    asm("cvt.rs.bf16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(va), "f"(vb), "r"(r));
    sa = __ushort_as_bfloat16((unsigned short)(d >> 16));
    sb = __ushort_as_bfloat16((unsigned short)(d & 0xFFFFu));
  }
};

// ---- random bits of the stochastic rounding --------------------------------
// Round-to-nearest repeats the same rounding error at every step where the
// flow is (nearly) steady, and those errors add up in the conserved moments;
// stochastic rounding makes them cancel on average.  The random bits are a
// counter-based function of (step, node, population), so results depend
// neither on the launch shape nor on the other grids of a batch.
constexpr unsigned SR_SEED = 0x2545F491u;

__device__ __forceinline__ unsigned sr_hash(const Grid& g, int x, int y) {
  unsigned h = ((unsigned)x * 0x9E3779B1u) ^ ((unsigned)y * 0x85EBCA77u) ^ (g.t * 0xC2B2AE3Du) ^
               SR_SEED;
  h ^= h >> 16;  // 32-bit integer finaliser (xor-shift-multiply)
  h *= 0x7FEB352Du;
  h ^= h >> 15;
  h *= 0x846CA68Bu;
  h ^= h >> 16;
  return h;
}

// Random words of a node: the linear congruential sequence
// x -> 1664525 x + 1013904223 (mod 2^32) started at the node's hash h (the
// 32-bit generator published in Press et al., Numerical Recipes, ch. 7).
// Words 18 + a / 27 + a round the wall values of f_a / h_a that the node
// writes into ghost slots (stepping there directly); the node's own 18
// stores walk the sequence one multiply-add per word: in the pulled-row
// kernels word j + 1 rounds the pair of populations 2j, 2j + 1 in one
// hardware conversion (its two 16-bit halves: over the ensemble of nodes
// the word is uniform, the sequence being a bijection of the hash, so each
// half is too), in the register-pull kernel word k + 1 rounds population k.
__device__ __forceinline__ unsigned lcg_next(unsigned r) { return r * 1664525u + 1013904223u; }
__device__ __forceinline__ unsigned sr_bits(unsigned h, int k) {
  unsigned r = h;
  for (int i = 0; i <= k; ++i) r = lcg_next(r);
  return r;
}

// Store of one value (deviation for 16-bit storage, rounded stochastically
// with the random word r).
template <class S>
__device__ __forceinline__ S store_val(typename Io<S>::C v, unsigned r) {
  if constexpr (Io<S>::sr)
    return Io<S>::from_sr(v, r);
  else
    return Io<S>::from(v);
}

__device__ __forceinline__ long long slot(const Grid& g, int a, int x, int y) {
  return (long long)(y + 1) * g.rp + (long long)plane(a) * g.pitch + (x + XOFF);
}

// Reference value of population a (0 unless the storage holds deviations).
template <class S>
__device__ __forceinline__ typename Io<S>::C pref(const Grid& g, int a) {
  using C = typename Io<S>::C;
  if constexpr (Io<S>::dev) return C(a < 9 ? g.fref[a] : g.href[a - 9]);
  return C(0);
}

// Pull the 18 stored values of node (x, y): d[a] = buf_a(x - e_a).  For
// deviation storage these are deviations; pref() adds the reference back.
template <class S>
__device__ __forceinline__ void pull(const Grid& g, const S* __restrict__ src, int x, int y,
                                     typename Io<S>::C d[NPOP]) {
  const S* p = src + slot(g, 0, x, y);
#pragma unroll
  for (int a = 0; a < NPOP; ++a) {
    const int q = a % 9;
    d[a] = Io<S>::to(Io<S>::ld(p + (plane(a) - plane(0)) * g.pitch - ey(q) * g.rp - ex(q)));
  }
}

// Moments of the pulled state: Eq. 35 with the force shift (text under
// Eq. 51), and Eq. 37 (total energy) or 2 sum h / (rho b R) (Eq. 38 form).
// Deviation storage recovers rho and theta in FP64 from the FP32 sums of the
// deviations and the FP64 sum of the references.  Es = sum h / rho, the
// specific energy the collision's h^eq carries (collision_equilibria).
template <class S>
__device__ __forceinline__ void moments(const Grid& g, const typename Io<S>::C d[NPOP],
                                        typename Io<S>::C& rho, typename Io<S>::C& ux,
                                        typename Io<S>::C& uy, typename Io<S>::C& th,
                                        typename Io<S>::C& Es) {
  using C = typename Io<S>::C;
  C sf = 0, sh = 0;
#pragma unroll
  for (int a = 0; a < 9; ++a) {
    sf += d[a];
    sh += d[9 + a];
  }
  const C jx = (d[1] - d[3]) + (d[5] - d[7]) + (d[8] - d[6]);
  const C jy = (d[2] - d[4]) + (d[5] - d[7]) + (d[6] - d[8]);
  const Phys<C>& k = phys<C>(g);
  if constexpr (Io<S>::dev) {
    // rho = 1 + sum of f deviations (the f references sum to 1); the energy
    // balance rho E - rho u^2 / 2 is formed in FP64 from the FP64 sum of the
    // h references and the FP32 sum of the h deviations.
    rho = C(1) + sf;
    const C inv = C(1) / rho;
    ux = jx * inv;
    uy = (jy - C(0.5) * rho * k.g) * inv;
    double e = g.href_sum + (double)sh;
    Es = (C)e * inv;
    if (g.energy_model == E_TOTAL) e -= 0.5 * (double)(rho * (ux * ux + uy * uy));
    th = k.six_b * (C)e * inv;
  } else {
    rho = sf;
    const C inv = C(1) / rho;
    ux = jx * inv;
    uy = (jy - C(0.5) * rho * k.g) * inv;
    Es = sh * inv;
    if (g.energy_model == E_TOTAL)
      th = k.six_b * (Es - C(0.5) * (ux * ux + uy * uy));
    else
      th = k.six_b * Es;
  }
}

template <class S>
__device__ __forceinline__ void moments(const Grid& g, const typename Io<S>::C d[NPOP],
                                        typename Io<S>::C& rho, typename Io<S>::C& ux,
                                        typename Io<S>::C& uy, typename Io<S>::C& th) {
  typename Io<S>::C Es;
  moments<S>(g, d, rho, ux, uy, th, Es);
}

// f^eq (Eq. 18a, R T0 = 1/3, D = 2, third-order velocity term dropped) and
// h^eq (Eq. 18b or b R T f^eq / 2), evaluated per pair of opposite velocities:
//   f^eq_a = rho w_a [1 + 3 eu + 9/2 eu^2 - 3/2 u^2 + (th-1)(3 e^2 - 2)/2
//                     + 3/2 eu (th-1)(3 e^2 - 4)]
//   h^eq_a = E f^eq_a + w_a p [3 eu + 9 eu^2 - 3 u^2 + th (3 e^2 - 2)/2],
//   E = b th / 6 + u^2 / 2, p = rho th / 3.
// Es is the specific energy the h^eq moment carries: E (total-energy model)
// or b th / 6 (internal-energy model, h^eq = Es f^eq).
//
// The rest populations are formed as the remainders of the moment sums,
// f^eq_0 = rho - sum_{a>0} f^eq_a and h^eq_0 = rho Es - sum_{a>0} h^eq_a
// (Eq. 19a/19b make this an identity): with rounded weights the direct
// formula would miss sum f^eq = rho by a fixed amount (7e-9 relative in FP32,
// 1e-16 in FP64), which the collision would add to the mass (and energy) of
// every node at every step.
template <class C>
__device__ __forceinline__ void equilibria_es(C rho, C ux, C uy, C th, C Es, bool total, C feq[9],
                                              C heq[9]) {
  constexpr bool remainder = true;
  const C usq = ux * ux + uy * uy;
  const C tm1 = th - C(1);
  const C A0 = C(1) - C(1.5) * usq;
  const C p = rho * th * (C(1) / C(3));
  // axis shell (e^2 = 1) and diagonal shell (e^2 = 2)
  const C base1 = A0 + C(0.5) * tm1, lin1 = C(3) - C(1.5) * tm1;
  const C base2 = A0 + C(2) * tm1, lin2 = C(3) * th;
  const C hb1 = C(-3) * usq + C(0.5) * th, hb2 = C(-3) * usq + C(2) * th;
  const C eus[4] = {ux, uy, ux + uy, uy - ux};  // e.u for a = 1, 2, 5, 6
  const int ia[4] = {1, 2, 5, 6};
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int a = ia[k], o = opp(a);
    const C eu = eus[k];
    const C w = wgt<C>(a);
    const C even = (k < 2 ? base1 : base2) + C(4.5) * eu * eu;
    const C odd = (k < 2 ? lin1 : lin2) * eu;
    feq[a] = rho * w * (even + odd);
    feq[o] = rho * w * (even - odd);
    if (total) {
      const C he = (k < 2 ? hb1 : hb2) + C(9) * eu * eu;
      const C ho = C(3) * eu;
      heq[a] = Es * feq[a] + w * p * (he + ho);
      heq[o] = Es * feq[o] + w * p * (he - ho);
    } else {
      heq[a] = Es * feq[a];
      heq[o] = Es * feq[o];
    }
  }
  // rest population
  if constexpr (remainder) {
    const C sf = ((feq[1] + feq[2]) + (feq[3] + feq[4])) + ((feq[5] + feq[6]) + (feq[7] + feq[8]));
    const C sh = ((heq[1] + heq[2]) + (heq[3] + heq[4])) + ((heq[5] + heq[6]) + (heq[7] + heq[8]));
    feq[0] = rho - sf;
    heq[0] = rho * Es - sh;
  } else {
    feq[0] = rho * wgt<C>(0) * (A0 - tm1);
    const C pb = C(-3) * usq - th;  // bracket of h^eq at e = 0: -3u^2 + th(-2)/2
    heq[0] = total ? Es * feq[0] + wgt<C>(0) * p * pb : Es * feq[0];
  }
}

// Equilibria of deviation storage as deviations from the rest equilibria
// (rho = 1, u = 0, theta = 1, Es = b/6): fd_a = f^eq_a - w_a and
// hd_a = h^eq_a - href_a from drho = rho - 1, dth = theta - 1 and
// dEs = Es - b/6, so that only small quantities are rounded:
//   f^eq_a - w_a = w_a [drho + rho (even_a - 1 + odd_a)],
//   h^eq_a - href_a = Es (f^eq_a - w_a) + dEs w_a
//                     + w_a [p (9 eu^2 - 3 u^2 +- 3 eu) + (p th - 1/3)(3 e^2 - 2)/2]
// (the last line for the total-energy model; p th - 1/3 = (drho + rho dth
// (2 + dth))/3).  The rest populations are the remainders of the sums
// sum fd = drho and sum hd = sdh (the sum of the node's h deviations, since
// rho Es = sum href + sdh), as in equilibria_es.
template <class C>
__device__ __forceinline__ void equilibria_dev(C drho, C ux, C uy, C dth, C dEs, C b6, bool total,
                                               C sdh, C fd[9], C hd[9]) {
  const C rho = C(1) + drho;
  const C Es = b6 + dEs;
  const C usq = ux * ux + uy * uy;
  const C em1 = C(-1.5) * usq + C(0.5) * dth;  // even part - 1 without 9/2 eu^2: axis
  const C em2 = C(-1.5) * usq + C(2) * dth;    // diagonal
  const C lin1 = C(3) - C(1.5) * dth, lin2 = C(3) * (C(1) + dth);
  const C p = rho * (C(1) + dth) * (C(1) / C(3));
  const C pt = (drho + rho * dth * (C(2) + dth)) * (C(1) / C(3));  // p th - 1/3
  const C hu = C(-3) * usq;
  const C eus[4] = {ux, uy, ux + uy, uy - ux};  // e.u for a = 1, 2, 5, 6
  const int ia[4] = {1, 2, 5, 6};
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int a = ia[k], o = opp(a);
    const C eu = eus[k];
    const C w = wgt<C>(a);
    const C evenm = (k < 2 ? em1 : em2) + C(4.5) * eu * eu;
    const C odd = (k < 2 ? lin1 : lin2) * eu;
    fd[a] = w * (drho + rho * (evenm + odd));
    fd[o] = w * (drho + rho * (evenm - odd));
    if (total) {
      const C he = p * (hu + C(9) * eu * eu) + (k < 2 ? C(0.5) : C(2)) * pt;
      const C ho = p * C(3) * eu;
      hd[a] = Es * fd[a] + w * (dEs + he + ho);
      hd[o] = Es * fd[o] + w * (dEs + he - ho);
    } else {
      hd[a] = Es * fd[a] + w * dEs;
      hd[o] = Es * fd[o] + w * dEs;
    }
  }
  const C sf = ((fd[1] + fd[2]) + (fd[3] + fd[4])) + ((fd[5] + fd[6]) + (fd[7] + fd[8]));
  const C sh = ((hd[1] + hd[2]) + (hd[3] + hd[4])) + ((hd[5] + hd[6]) + (hd[7] + hd[8]));
  fd[0] = drho - sf;
  hd[0] = sdh - sh;
}

// The same from theta alone (Es from b / 6).
template <class C>
__device__ __forceinline__ void equilibria(C rho, C ux, C uy, C th, C b6, bool total, C feq[9],
                                           C heq[9]) {
  const C Es = total ? b6 * th + C(0.5) * (ux * ux + uy * uy) : b6 * th;
  equilibria_es<C>(rho, ux, uy, th, Es, total, feq, heq);
}

// Equilibria of the collision: h^eq carries the specific energy Es
// recovered from the node's own sum of h (rho Es = sum h, Eq. 37 or the
// Eq. 38 form), so that the relaxation conserves energy to rounding; forming
// it from theta through b / 6 and 6 / b (each rounded) would bias it by up to
// 2e-8 relative per step in FP32 (and 1e-16 in FP64).
template <class C>
__device__ __forceinline__ void collision_equilibria(C rho, C ux, C uy, C th, C Es, C b6,
                                                     bool total, C feq[9], C heq[9]) {
  (void)b6;
  equilibria_es<C>(rho, ux, uy, th, Es, total, feq, heq);
}

// Wall equilibria: f^eq at (rho, u_w, theta) (halfway bounce-back term) and
// h^eq at the ghost (isothermal) or wall (adiabatic) state.
template <class C>
__device__ void wall_equilibria(const Grid& g, int side, C rho, C ux, C uy, C th, C fw[9],
                                C hw[9]) {
  const bool total = g.energy_model == E_TOTAL;
  const Phys<C>& k = phys<C>(g);
  const C uwx = k.uw[side][0], uwy = k.uw[side][1];
  C tmp[9];
  equilibria<C>(rho, uwx, uwy, th, k.b6, total, fw, tmp);
  if (g.bc[side] == BC_ISO) {
    const C thg = fmax(C(2) * k.thw[side] - th, C(0.5) * k.thw[side]);  // floored: see xedge_one
    // the node's pressure carried to the ghost by hydrostatic balance
    // (rho_g theta_g = rho (theta - 3 g n_y), n_y the outward normal of a y
    // side; equal pressure across an x side)
    const int ny_out = side == 2 ? -1 : (side == 3 ? 1 : 0);
    const C rg = rho * (th - C(3) * k.g * C(ny_out)) / thg;
    equilibria<C>(rg, C(2) * uwx - ux, C(2) * uwy - uy, thg, k.b6, total, tmp, hw);
  } else {
    for (int a = 0; a < 9; ++a) hw[a] = tmp[a];
  }
}

template <class S>
__device__ __forceinline__ void put(const Grid& g, S* dst, int a, int x, int y,
                                    typename Io<S>::C v, unsigned h, int k) {
  dst[slot(g, a, x, y)] = store_val<S>(v - pref<S>(g, a), Io<S>::sr ? sr_bits(h, k) : 0u);
}

// Ghost-slot writes of a boundary node (x, y): periodic copies and the wall
// rules (adiabatic walls of the total-energy model add the wall's work on the
// bounced pair, u_w . (f_b e_b - f*_a e_a): no heat crosses a moving
// adiabatic wall, its work does).  v[0..8] = f*, v[9..17] = h*, v[18..26] = h^eq of the node.  A
// population leaving through a corner takes the x side's rule when that side
// is a wall, else the y side's.  SKIPX: the populations that leave through the
// x sides (x wall or periodic in both directions) are written by xedge_writes.
template <class S, bool SKIPX = false>
__device__ __noinline__ void boundary_writes(const Grid& g, S* __restrict__ dst, int x, int y,
                                             const typename Io<S>::C* v,
                                             typename Io<S>::C rho, typename Io<S>::C ux,
                                             typename Io<S>::C uy, typename Io<S>::C th) {
  using C = typename Io<S>::C;
  C fw[9], hw[9];
  int have = -1;
  const unsigned hs = Io<S>::sr ? sr_hash(g, x, y) : 0u;
  for (int a = 1; a < 9; ++a) {
    const int dx = x + ex(a), dy = y + ey(a);
    const int ox = dx < 0 ? 0 : (dx >= g.nx ? 1 : -1);
    const int oy = dy < 0 ? 2 : (dy >= g.ny ? 3 : -1);
    if (ox < 0 && oy < 0) continue;
    int side = -1;
    if (ox >= 0 && g.bc[ox] != BC_PERIODIC)
      side = ox;
    else if (oy >= 0 && g.bc[oy] != BC_PERIODIC)
      side = oy;
    if (SKIPX && ox >= 0 && (side == ox || side < 0)) continue;
    if (side < 0) {
      // periodic: the node at wrap(d) pulls population a from wrap(d) - e_a
      const int wx = (dx + g.nx) % g.nx, wy = (dy + g.ny) % g.ny;
      put<S>(g, dst, a, wx - ex(a), wy - ey(a), v[a], hs, a);
      put<S>(g, dst, 9 + a, wx - ex(a), wy - ey(a), v[9 + a], hs, 9 + a);
      continue;
    }
    if (have != side) {
      wall_equilibria<C>(g, side, rho, ux, uy, th, fw, hw);
      have = side;
    }
    const int b = opp(a);  // reflected direction; node (x, y) pulls it from d
    const C fb = v[a] + (fw[b] - fw[a]);
    put<S>(g, dst, b, dx, dy, fb, hs, 18 + b);
    C hin;
    if (g.bc[side] == BC_ISO) {
      hin = hw[b] + (v[9 + b] - v[18 + b]);
    } else {
      hin = v[9 + a] + (hw[b] - hw[a]);
      if (g.energy_model == E_TOTAL) {  // the wall's work u_w . (f_b e_b - f*_a e_a)
        const Phys<C>& k = phys<C>(g);
        hin -= (C(ex(a)) * k.uw[side][0] + C(ey(a)) * k.uw[side][1]) * (fb + v[a]);
      }
    }
    put<S>(g, dst, 9 + b, dx, dy, hin, hs, 27 + b);
  }
}

// f^eq and h^eq of one direction e = (EX, EY) (same expressions as
// `equilibria`).
template <class C, int EX, int EY>
__device__ __forceinline__ void eq_dir(C rho, C ux, C uy, C th, C b6, bool total, C& f, C& h) {
  constexpr int e2 = EX * EX + EY * EY;
  const C usq = ux * ux + uy * uy;
  const C tm1 = th - C(1);
  const C A0 = C(1) - C(1.5) * usq;
  const C eu = C(EX) * ux + C(EY) * uy;
  const C w = wgt<C>(e2 == 1 ? 1 : 5);
  const C even = (e2 == 1 ? A0 + C(0.5) * tm1 : A0 + C(2) * tm1) + C(4.5) * eu * eu;
  const C odd = (e2 == 1 ? C(3) - C(1.5) * tm1 : C(3) * th) * eu;
  f = rho * w * (even + odd);
  if (total) {
    const C E = b6 * th + C(0.5) * usq;
    const C p = rho * th * (C(1) / C(3));
    const C he = (e2 == 1 ? C(-3) * usq + C(0.5) * th : C(-3) * usq + C(2) * th) + C(9) * eu * eu;
    h = E * f + w * p * (he + C(3) * eu);
  } else {
    h = b6 * th * f;
  }
}

// One population a leaving an x-edge node (x, y) through x side XS.  Wall:
// f halfway bounce-back with the moving-wall term, h by the ghost-node
// equilibrium (isothermal) or bounce-back (adiabatic), as in boundary_writes
// but with the odd equilibrium parts written out for this direction alone.
// Periodic x: the copy into the opposite ghost column, unless the population
// also leaves through a y wall (boundary_writes takes it then).
template <class S, int XS, int A>
__device__ __forceinline__ void xedge_one(const Grid& g, S* __restrict__ dst, int x, int y,
                                          const typename Io<S>::C* v, typename Io<S>::C rho,
                                          typename Io<S>::C ux, typename Io<S>::C uy,
                                          typename Io<S>::C th) {
  using C = typename Io<S>::C;
  constexpr int B = opp(A), EX = ex(A), EY = ey(A);
  constexpr bool diag = EY != 0;
  const int dx = x + EX, dy = y + EY;
  if (g.bc[XS] != BC_PERIODIC) {
    const Phys<C>& k = phys<C>(g);
    const bool total = g.energy_model == E_TOTAL;
    const C uwx = k.uw[XS][0], uwy = k.uw[XS][1];
    const C euw = C(EX) * uwx + C(EY) * uwy;
    const C w = wgt<C>(A);
    const C lin = diag ? C(3) * th : C(3) - C(1.5) * (th - C(1));
    const C fodd = rho * w * lin * euw;  // odd part of f^eq_A at (rho, u_w, theta)
    const unsigned hs = Io<S>::sr ? sr_hash(g, x, y) : 0u;
    const C fb = v[A] - C(2) * fodd;
    put<S>(g, dst, B, dx, dy, fb, hs, 18 + B);
    C hin;
    if (g.bc[XS] == BC_ISO) {
      // ghost temperature linear through the wall value, floored at half of
      // it (the equal-pressure ghost density diverges as it vanishes)
      const C thg = fmax(C(2) * k.thw[XS] - th, C(0.5) * k.thw[XS]);
      C fg, hg;
      eq_dir<C, ex(B), ey(B)>(rho * th / thg, C(2) * uwx - ux, C(2) * uwy - uy, thg, k.b6, total,
                              fg, hg);
      hin = hg + (v[9 + B] - v[18 + B]);
    } else {
      C hodd;  // odd part of h^eq_A at (rho, u_w, theta)
      if (total) {
        const C E = k.b6 * th + C(0.5) * (uwx * uwx + uwy * uwy);
        hodd = E * fodd + w * (rho * th * (C(1) / C(3))) * C(3) * euw;
      } else {
        hodd = k.b6 * th * fodd;
      }
      hin = v[9 + A] - C(2) * hodd;
      if (total) hin -= euw * (fb + v[A]);  // the wall's work u_w . (f_b e_b - f*_a e_a)
    }
    put<S>(g, dst, 9 + B, dx, dy, hin, hs, 27 + B);
    return;
  }
  if (EY != 0 && (dy < 0 || dy >= g.ny) && g.bc[dy < 0 ? 2 : 3] != BC_PERIODIC) return;
  const int wx = (dx + g.nx) % g.nx, wy = (dy + g.ny) % g.ny;
  const unsigned hs = Io<S>::sr ? sr_hash(g, x, y) : 0u;
  put<S>(g, dst, A, wx - EX, wy - EY, v[A], hs, A);
  put<S>(g, dst, 9 + A, wx - EX, wy - EY, v[9 + A], hs, 9 + A);
}

// Ghost-slot writes of the populations leaving an x-edge node through x side
// XS (0: x = 0, populations 3, 6, 7; 1: x = nx - 1, populations 1, 5, 8).
template <class S, int XS>
__device__ __forceinline__ void xedge_writes(const Grid& g, S* __restrict__ dst, int x, int y,
                                             const typename Io<S>::C* v, typename Io<S>::C rho,
                                             typename Io<S>::C ux, typename Io<S>::C uy,
                                             typename Io<S>::C th) {
  if (XS == 0) {
    xedge_one<S, 0, 3>(g, dst, x, y, v, rho, ux, uy, th);
    xedge_one<S, 0, 6>(g, dst, x, y, v, rho, ux, uy, th);
    xedge_one<S, 0, 7>(g, dst, x, y, v, rho, ux, uy, th);
  } else {
    xedge_one<S, 1, 1>(g, dst, x, y, v, rho, ux, uy, th);
    xedge_one<S, 1, 5>(g, dst, x, y, v, rho, ux, uy, th);
    xedge_one<S, 1, 8>(g, dst, x, y, v, rho, ux, uy, th);
  }
}

// Moment-space source C-hat of the MRT collision: the correction of Eq. 48,
// (0, phi_x, 0, 0, 0, 0, 0, phi_y, 0), plus the force of Eq. 51 with
// a = (0, a_y) (its seventh entry read as 2 (u_x a_x - u_y a_y)).
template <class C>
__device__ __forceinline__ void mrt_source(bool corr, C phx, C phy, bool force, C ux, C uy, C ay,
                                           C mc[9]) {
#pragma unroll
  for (int q = 0; q < 9; ++q) mc[q] = C(0);
  if (corr) {
    mc[1] = phx;
    mc[7] = phy;
  }
  if (force) {
    const C uay = uy * ay;
    mc[1] += C(6) * uay;
    mc[2] = C(-6) * uay;
    mc[5] = ay;
    mc[6] = -ay;
    mc[7] -= C(2) * uay;
    mc[8] = ux * ay;
  }
}

// Relaxation rates of a node: the constants for constant tau; with a
// temperature-dependent viscosity mu(theta) (power law mu0 theta^n, the
// premise of Eq. 52, or Sutherland's law, Eq. 59 referred to T0) the BGK
// relation mu = tau_f p (Eq. 30) gives tau_f = tau_f0 (mu / mu0) / (rho theta)
// and tau_h = tau_f tau_h0 / tau_f0 (constant Pr).  kz: the Z coupling of h
// (w_h - w_f, Eq. 36; (1 - w_h/2)(Pr - 1)/(tau_f + 1/2), Eq. 47).
template <class C>
__device__ __forceinline__ void node_rates(const Grid& g, const Phys<C>& k, C rho, C th, bool mrt,
                                           C& wf, C& wh, C& kz) {
  if (g.mu_law == MU_TAU) {
    wf = k.omega_f;
    wh = k.omega_h;
    kz = k.kz;
    return;
  }
  C law;
  if (g.mu_law == MU_POWER)
    law = pow(th, k.mu_n);
  else
    law = th * sqrt(th) * (C(1) + k.mu_s) / (th + k.mu_s);
  const C tf = k.tau_f0 * law / (rho * th);
  const C tq = tf * k.tau_ratio;
  wf = C(2) / (C(2) * tf + C(1));
  wh = C(2) / (C(2) * tq + C(1));
  kz = mrt ? (C(1) - C(0.5) * wh) * (tf / tq - C(1)) / (tf + C(0.5)) : wh - wf;
}

// MRT collision of f (Eq. 44 with the Appendix B matrices): with n = f - f^eq
// and the moment-space source mc (mrt_source),
//   f* = f + M^-1 [ -S M n + (I - S/2) mc ],
// S = diag(1, s_e, s_eps, 1, s_q, 1, s_q, w_f, w_f) (Eq. 40; the rates of
// the conserved moments rho and j drop out of the result).
template <class C, bool NODE = true>
__device__ __forceinline__ void mrt_collide(const Phys<C>& k, C wf, const C f[9], const C n[9],
                                            const C mc[9], C out[9]) {
  // moments (e, eps, qx, qy, pxx, pxy) of n: rows of M.  For a node
  // (NODE) the conserved ones need no sums: rho of n is 0 (f^eq carries the
  // node's rho), jx of n is 0 and jy of n is -a_y/2 (u = (j + a/2)/rho,
  // a = (0, a_y)); with their rate 1 and the source mc (jy: a_y) their
  // relaxed changes are 0, 0, a_y.  A wall node of non-equilibrium
  // extrapolation borrows n from its neighbour, so it takes them in full.
  C mn[9];
  {
    const C* q = n;
    C* m = mn;
    const C sa = (q[1] + q[2]) + (q[3] + q[4]), sd = (q[5] + q[6]) + (q[7] + q[8]);
    const C dx1 = q[1] - q[3], dy1 = q[2] - q[4];
    const C dxd = (q[5] - q[6]) - (q[7] - q[8]), dyd = (q[5] + q[6]) - (q[7] + q[8]);
    m[0] = NODE ? C(0) : q[0] + sa + sd;
    m[1] = C(-4) * q[0] - sa + C(2) * sd;
    m[2] = C(4) * q[0] - C(2) * sa + sd;
    m[3] = NODE ? C(0) : dx1 + dxd;
    m[4] = C(-2) * dx1 + dxd;
    m[5] = NODE ? C(0) : dy1 + dyd;
    m[6] = C(-2) * dy1 + dyd;
    m[7] = (q[1] + q[3]) - (q[2] + q[4]);
    m[8] = (q[5] - q[6]) + (q[7] - q[8]);
  }
  const C se = k.se > C(0) ? k.se : wf, seps = k.seps > C(0) ? k.seps : wf;
  const C sq = k.sq > C(0) ? k.sq : wf;
  C dm[9];
  dm[1] = -se * mn[1] + (C(1) - C(0.5) * se) * mc[1];
  dm[2] = -seps * mn[2] + (C(1) - C(0.5) * seps) * mc[2];
  dm[4] = -sq * mn[4] + (C(1) - C(0.5) * sq) * mc[4];
  dm[0] = NODE ? C(0) : -mn[0] + C(0.5) * mc[0];
  dm[3] = NODE ? C(0) : -mn[3] + C(0.5) * mc[3];
  dm[5] = NODE ? mc[5] : -mn[5] + C(0.5) * mc[5];
  dm[6] = -sq * mn[6] + (C(1) - C(0.5) * sq) * mc[6];
  dm[7] = -wf * mn[7] + (C(1) - C(0.5) * wf) * mc[7];
  dm[8] = -wf * mn[8] + (C(1) - C(0.5) * wf) * mc[8];
  // M^-1 dm (Eq. B2), grouped by shell (for a node dm[0] = dm[3] = 0)
  const C r0 = dm[0] * C(1.0 / 9.0);
  const C ax = r0 - dm[1] * C(1.0 / 36.0) - dm[2] * C(1.0 / 18.0);
  const C dg = r0 + dm[1] * C(1.0 / 18.0) + dm[2] * C(1.0 / 36.0);
  const C x1 = (dm[3] - dm[4]) * C(1.0 / 6.0), y1 = (dm[5] - dm[6]) * C(1.0 / 6.0);
  const C x2 = dm[3] * C(1.0 / 6.0) + dm[4] * C(1.0 / 12.0);
  const C y2 = dm[5] * C(1.0 / 6.0) + dm[6] * C(1.0 / 12.0);
  const C pp = dm[7] * C(0.25), pq = dm[8] * C(0.25);
  out[0] = f[0] + (r0 + (dm[2] - dm[1]) * C(1.0 / 9.0));
  out[1] = f[1] + (ax + x1 + pp);
  out[2] = f[2] + (ax + y1 - pp);
  out[3] = f[3] + (ax - x1 + pp);
  out[4] = f[4] + (ax - y1 - pp);
  out[5] = f[5] + (dg + x2 + y2 + pq);
  out[6] = f[6] + (dg - x2 + y2 - pq);
  out[7] = f[7] + (dg - x2 - y2 + pq);
  out[8] = f[8] + (dg + x2 - y2 - pq);
}

// Collision of one node (Eq. 34 with +(1 - w_f/2) C, Eq. 36 or Eq. 38) with
// the correction C_a (Eq. 49) plus the Guo force F_a, then the stores.
template <class S>
__device__ __forceinline__ void collide_store(const Grid& g, S* __restrict__ dst, int x, int y,
                                              const typename Io<S>::C d[NPOP],
                                              typename Io<S>::C rho, typename Io<S>::C ux,
                                              typename Io<S>::C uy, typename Io<S>::C th,
                                              typename Io<S>::C Es, typename Io<S>::C dqx,
                                              typename Io<S>::C dqy) {
  using C = typename Io<S>::C;
  const bool total = g.energy_model == E_TOTAL;
  const Phys<C>& k = phys<C>(g);
  C wf, wh, kz;
  node_rates<C>(g, k, rho, th, g.collision == COLL_MRT, wf, wh, kz);
  C feq[9], heq[9];
  collision_equilibria<C>(rho, ux, uy, th, Es, k.b6, total, feq, heq);

  // C'_a = C_a + F_a
  C cc[9];
  if (g.correction) {
    const C phx = C(3) * (dqx + dqy), phy = dqx - dqy;
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
  } else {
#pragma unroll
    for (int a = 0; a < 9; ++a) cc[a] = C(0);
  }
  if (g.has_force) {
    // F_a = w_a [3 e.a + 9 (e.u)(e.a) - 3 u.a], a = (0, ay)
    const C ay = -rho * k.g;
#pragma unroll
    for (int a = 0; a < 9; ++a) {
      const C ea = C(ey(a)) * ay;
      const C eu = C(ex(a)) * ux + C(ey(a)) * uy;
      cc[a] += wgt<C>(a) * (C(3) * ea + C(9) * eu * ea - C(3) * uy * ay);
    }
  }

  const C usq = ux * ux + uy * uy;
  const C kc = C(1) - C(0.5) * wf;
  C v[27];
  if (g.collision == COLL_MRT) {
    C fa[9], fneq[9], mc[9];
#pragma unroll
    for (int a = 0; a < 9; ++a) {
      fa[a] = pref<S>(g, a) + d[a];
      fneq[a] = fa[a] - feq[a];
    }
    mrt_source<C>(g.correction != 0, C(3) * (dqx + dqy), dqx - dqy, g.has_force != 0, ux, uy,
                  -rho * k.g, mc);
    mrt_collide<C>(k, wf, fa, fneq, mc, v);
  }
#pragma unroll
  for (int a = 0; a < 9; ++a) {
    const C fa = pref<S>(g, a) + d[a];
    const C ha = pref<S>(g, 9 + a) + d[9 + a];
    const C fneq = fa - feq[a];
    if (g.collision != COLL_MRT) v[a] = fa - wf * fneq + kc * cc[a];
    C hs = ha - wh * (ha - heq[a]);
    if (total) {
      const C eu = C(ex(a)) * ux + C(ey(a)) * uy;
      const C Z = g.z_full ? eu - C(0.5) * usq : eu;
      hs += kz * Z * (fneq + C(0.5) * cc[a]);
    }
    v[9 + a] = hs;
    v[18 + a] = heq[a];
  }
  S* p = dst + slot(g, 0, x, y);
  unsigned r = Io<S>::sr ? sr_hash(g, x, y) : 0u;
#pragma unroll
  for (int a = 0; a < NPOP; ++a) {
    if constexpr (Io<S>::sr) r = lcg_next(r);
    p[(plane(a) - plane(0)) * g.pitch] = store_val<S>(v[a] - pref<S>(g, a), r);
  }
  if (x == 0 || y == 0 || x == g.nx - 1 || y == g.ny - 1) {
    C tmp[27];
#pragma unroll
    for (int a = 0; a < 27; ++a) tmp[a] = v[a];
    boundary_writes<S>(g, dst, x, y, tmp, rho, ux, uy, th);
  }
}

// Q of the mirror ghost across a wall side: 2 rho u_w (1 - theta_w) - Q.
template <class C>
__device__ __forceinline__ C ghost_q(const Grid& g, int side, int comp, C rho, C th, C q) {
  const Phys<C>& k = phys<C>(g);
  const C thw = g.bc[side] == BC_ISO ? k.thw[side] : th;
  return C(2) * rho * k.uw[side][comp] * (C(1) - thw) - q;
}

// One time step.  Block = strip of blockDim.x - 2 output columns (one halo
// column each side), rows [blockIdx.y * rows, +rows).  Dynamic shared memory:
// 3 * blockDim.x compute-precision words.
template <class S>
__global__ void __launch_bounds__(256) step_kernel(const Grid g, int rows) {
  using C = typename Io<S>::C;
  extern __shared__ unsigned char smem_raw[];
  C* qxs = reinterpret_cast<C*>(smem_raw);
  const int NT = blockDim.x, W = NT - 2, t = threadIdx.x;
  const int nx = g.nx, ny = g.ny;
  const int c = blockIdx.x * W - 1 + t;
  const int y0 = blockIdx.y * rows;
  if (y0 >= ny) return;  // whole block
  const int y1 = min(y0 + rows, ny);
  const S* __restrict__ src = static_cast<const S*>(g.src);
  S* __restrict__ dst = static_cast<S*>(g.dst);

  bool colv;
  int ncol;
  if (c >= 0 && c < nx) {
    colv = true;
    ncol = c;
  } else if (c == -1) {
    colv = g.bc[0] == BC_PERIODIC;
    ncol = nx - 1;
  } else if (c == nx) {
    colv = g.bc[1] == BC_PERIODIC;
    ncol = 0;
  } else {
    colv = false;
    ncol = 0;
  }
  const bool outc = t >= 1 && t <= W && c < nx;
  const bool wall_l = g.bc[0] != BC_PERIODIC, wall_r = g.bc[1] != BC_PERIODIC;
  const bool wall_b = g.bc[2] != BC_PERIODIC, wall_t = g.bc[3] != BC_PERIODIC;

  C pd[NPOP];
  C prho = 1, pux = 0, puy = 0, pth = 1, pes = 0, pqx = 0, pqy = 0, qymm = 0;
#pragma unroll
  for (int a = 0; a < NPOP; ++a) pd[a] = 0;

  int sl = 0;  // slot of row r in the 3-row ring
  for (int r = y0 - 1; r <= y1; ++r) {
    bool rowv;
    int nrow;
    if (r >= 0 && r < ny) {
      rowv = true;
      nrow = r;
    } else if (r < 0) {
      rowv = !wall_b;
      nrow = ny - 1;
    } else {
      rowv = !wall_t;
      nrow = 0;
    }
    C cd[NPOP];
    C crho = 1, cux = 0, cuy = 0, cth = 1, ces = 0, cqx = 0, cqy = 0;
    if (colv && rowv) {
      pull<S>(g, src, ncol, nrow, cd);
      moments<S>(g, cd, crho, cux, cuy, cth, ces);
      cqx = crho * cux * (C(1) - cth);
      cqy = crho * cuy * (C(1) - cth);
    } else {
#pragma unroll
      for (int a = 0; a < NPOP; ++a) cd[a] = 0;
    }
    qxs[sl * NT + t] = cqx;
    __syncthreads();
    const int ro = r - 1;
    if (ro >= y0 && outc) {
      const int ps = sl == 0 ? 2 : sl - 1;
      const C qxl = (c > 0 || !wall_l) ? qxs[ps * NT + t - 1] : ghost_q<C>(g, 0, 0, prho, pth, pqx);
      const C qxr =
          (c < nx - 1 || !wall_r) ? qxs[ps * NT + t + 1] : ghost_q<C>(g, 1, 0, prho, pth, pqx);
      const C qyu = (ro < ny - 1 || !wall_t) ? cqy : ghost_q<C>(g, 3, 1, prho, pth, pqy);
      const C qyd = (ro > 0 || !wall_b) ? qymm : ghost_q<C>(g, 2, 1, prho, pth, pqy);
      collide_store<S>(g, dst, c, ro, pd, prho, pux, puy, pth, pes, C(0.5) * (qxr - qxl),
                       C(0.5) * (qyu - qyd));
    }
#pragma unroll
    for (int a = 0; a < NPOP; ++a) pd[a] = cd[a];
    qymm = pqy;
    prho = crho;
    pux = cux;
    puy = cuy;
    pth = cth;
    pes = ces;
    pqx = cqx;
    pqy = cqy;
    sl = sl == 2 ? 0 : sl + 1;
  }
}

// ---- initialisation, state export, moments, reductions ---------------------

// Writes population values p[18] (full values, FP64) of node (x, y) into the
// slots the next pull reads: buf_a(x - e_a).
template <class S>
__device__ __forceinline__ void scatter_node(const Grid& g, S* __restrict__ buf, int x, int y,
                                             const double p[NPOP]) {
  for (int a = 0; a < NPOP; ++a) {
    const int q = a % 9;
    const double ref = Io<S>::dev ? (double)(a < 9 ? g.fref[a] : g.href[a - 9]) : 0.0;
    buf[slot(g, a, x - ex(q), y - ey(q))] =
        Io<S>::from((typename Io<S>::C)(Io<S>::dev ? (p[a] - ref) : p[a]));
  }
}

// FP64 equilibrium populations of (rho, u, T/T0) (initial state).
__device__ __forceinline__ void init_pops(const Grid& g, double rho, double ux, double uy,
                                          double th, double p[NPOP]) {
  double feq[9], heq[9];
  equilibria<double>(rho, ux, uy, th, g.pd.b6, g.energy_model == E_TOTAL, feq, heq);
  for (int a = 0; a < 9; ++a) {
    p[a] = feq[a];
    p[9 + a] = heq[a];
  }
}

// Nodes [i0, i1) (row-major index; i1 < 0: to the end), so that a caller can
// initialise a grid chunk by chunk as its fields arrive.
template <class S>
__global__ void init_kernel(const Grid g, S* buf, const double* __restrict__ rho,
                            const double* __restrict__ ux, const double* __restrict__ uy,
                            const double* __restrict__ T, double invT0, long long i0 = 0,
                            long long i1 = -1) {
  const long long n = i1 < 0 ? (long long)g.nx * g.ny : i1;
  for (long long i = i0 + blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(i % g.nx), y = (int)(i / g.nx);
    double p[NPOP];
    init_pops(g, rho[i], ux[i], uy[i], T[i] * invT0, p);
    scatter_node<S>(g, buf, x, y, p);
  }
}

template <class S>
__global__ void set_state_kernel(const Grid g, S* buf, const double* __restrict__ pops) {
  const long long n = (long long)g.nx * g.ny;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(i % g.nx), y = (int)(i / g.nx);
    double p[NPOP];
    for (int a = 0; a < NPOP; ++a) p[a] = pops[(long long)a * n + i];
    scatter_node<S>(g, buf, x, y, p);
  }
}

// FP64 pull of node (x, y) from buffer buf.
template <class S>
__device__ __forceinline__ void pull_fp64(const Grid& g, const S* __restrict__ buf, int x, int y,
                                          double p[NPOP]) {
  const S* q = buf + slot(g, 0, x, y);
  for (int a = 0; a < NPOP; ++a) {
    const int k = a % 9;
    const double ref = Io<S>::dev ? (double)(a < 9 ? g.fref[a] : g.href[a - 9]) : 0.0;
    p[a] = ref + (double)Io<S>::to(q[(plane(a) - plane(0)) * g.pitch - ey(k) * g.rp - ex(k)]);
  }
}

__device__ __forceinline__ void moments_fp64(const Grid& g, const double p[NPOP], double& rho,
                                             double& ux, double& uy, double& th, double& sh) {
  double r = 0, jx = 0, jy = 0;
  sh = 0;
  for (int a = 0; a < 9; ++a) {
    r += p[a];
    jx += ex(a) * p[a];
    jy += ey(a) * p[a];
    sh += p[9 + a];
  }
  rho = r;
  ux = jx / r;
  uy = (jy - 0.5 * r * g.pd.g) / r;
  if (g.energy_model == E_TOTAL)
    th = g.pd.six_b * (sh / r - 0.5 * (ux * ux + uy * uy));
  else
    th = g.pd.six_b * sh / r;
}

// rho, u, T (FP64) and optionally the canonical populations [18][ny][nx],
// of nodes [i0, i1) (i1 < 0: to the end).  nonfinite (may be NULL): set to 1
// when any exported moment is NaN or infinite, so the host need not scan the
// fields.
template <class S>
__global__ void export_kernel(const Grid g, const S* __restrict__ buf, double* rho, double* ux,
                              double* uy, double* T, double T0, double* pops,
                              int* nonfinite = nullptr, long long i0 = 0, long long i1 = -1) {
  const long long nn = (long long)g.nx * g.ny;
  const long long n = i1 < 0 ? nn : i1;
  for (long long i = i0 + blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(i % g.nx), y = (int)(i / g.nx);
    double p[NPOP];
    pull_fp64<S>(g, buf, x, y, p);
    if (pops) {
      for (int a = 0; a < NPOP; ++a) pops[(long long)a * nn + i] = p[a];
    }
    if (rho) {
      double r, vx, vy, th, sh;
      moments_fp64(g, p, r, vx, vy, th, sh);
      rho[i] = r;
      ux[i] = vx;
      uy[i] = vy;
      T[i] = th * T0;
      if (nonfinite && !(isfinite(r) && isfinite(vx) && isfinite(vy) && isfinite(th * T0)))
        *nonfinite = 1;
    }
  }
}

// Sums of rho, rho u_x, rho u_y, hbar: per-block partials in a fixed order.
constexpr int RED_THREADS = 256;
template <class S>
__global__ void __launch_bounds__(RED_THREADS) conserved_partial_kernel(const Grid g,
                                                                        const S* __restrict__ buf,
                                                                        double* partial) {
  __shared__ double sm[4][RED_THREADS];
  const long long n = (long long)g.nx * g.ny;
  double acc[4] = {0, 0, 0, 0};
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(i % g.nx), y = (int)(i / g.nx);
    double p[NPOP];
    pull_fp64<S>(g, buf, x, y, p);
    double r, vx, vy, th, sh;
    moments_fp64(g, p, r, vx, vy, th, sh);
    acc[0] += r;
    acc[1] += r * vx;
    acc[2] += r * vy;
    acc[3] += sh;
  }
  for (int k = 0; k < 4; ++k) sm[k][threadIdx.x] = acc[k];
  __syncthreads();
  for (int s = RED_THREADS / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s)
      for (int k = 0; k < 4; ++k) sm[k][threadIdx.x] += sm[k][threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int k = 0; k < 4; ++k) partial[4 * blockIdx.x + k] = sm[k][0];
}

// Final fixed-order sum of nb partial quadruples into out[4].  (A template
// only so that every translation unit including this header may define it.)
template <int UNUSED = 0>
__global__ void conserved_final_kernel(const double* __restrict__ partial, int nb, double* out) {
  __shared__ double sm[4][RED_THREADS];
  double acc[4] = {0, 0, 0, 0};
  for (int i = threadIdx.x; i < nb; i += blockDim.x)
    for (int k = 0; k < 4; ++k) acc[k] += partial[4 * i + k];
  for (int k = 0; k < 4; ++k) sm[k][threadIdx.x] = acc[k];
  __syncthreads();
  for (int s = RED_THREADS / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s)
      for (int k = 0; k < 4; ++k) sm[k][threadIdx.x] += sm[k][threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int k = 0; k < 4; ++k) out[k] = sm[k][0];
}

}  // namespace lbm
