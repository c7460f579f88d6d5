/*
 * Oracle: plain, slow, FP64 CPU statement of one time step of the coupled
 * double-distribution-function (DDF) thermal lattice Boltzmann method on D2Q9
 * (Li, Luo, He, Gao & Tao, arXiv:1109.6672), BGK scheme of Sec. III.C.1.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
 * load this file; only the tests, the smoke check and the benchmark's CPU
 * baseline do.  It shares no code, header, table or constant with the CUDA
 * library: every constant below is written out here from the paper.
 *
 * Parity unpinned, in part: the -u^2/2 part of Z_a in the coupling term of
 * Eq. 36 (the full Z form).  The paper notes that Z_a reduces to e_a.u at
 * the Navier-Stokes level, so no closed form, decay rate or table it fixes
 * depends on that part; it is checked only against the independent NumPy
 * restatement.  Q of the ghost node across a wall in the Eq. 50 differences
 * (the linear ghost 2 Q_w - Q, a reading: the paper does not say) is pinned
 * by consistency: at the boundary node the difference converges to the
 * derivative of any smooth field that takes Q_w at the wall
 * (orc_gradients).  The other pieces of the step tried so far are caught by
 * a pin the paper or the mathematics fixes when a plausible mistake is
 * planted in them (tests/test_oracle_mutants.py).
 *
 * Build: gcc -O2 -ffp-contract=off -fPIC -shared [-fopenmp] (no FMA
 * contraction, so every product and sum is rounded as written).
 *
 * State: the canonical pre-collision distributions fbar_a(x,t), hbar_a(x,t)
 * (Eqs. 33-36 variable change), stored as f[a][y*nx+x], h[a][y*nx+x].
 *
 * One step, in the order the paper defines it:
 *   phase 1, every node: rho, u (Eq. 35 with the force shift under Eq. 51),
 *            T from Eq. 37 (total energy) or from the internal-energy form
 *            under Eq. 38, theta = T/T0, Q = rho u (1 - theta) (Eq. 48);
 *   phase 2, every node: dQx/dx, dQy/dy by Eq. 50, phi (Eq. 48), C_a
 *            (Eq. 49), Guo force F_a (text above Eq. 51) added to C_a,
 *            equilibria (Eq. 18a/18b), collision (Eq. 34 with the sign of the
 *            C term read as +, Eq. 36 or Eq. 38), then push-streaming to
 *            x + e_a with periodic wrap or the wall rules below.
 *
 * Readings where the paper is silent (the wall rules are not in the paper,
 * which uses non-equilibrium extrapolation):
 *   - halfway bounce-back for f with the odd part of Eq. 18a at the wall
 *     state (moving wall);
 *   - f wall state: rho and theta of the boundary node itself and the wall
 *     velocity (the linear Couette profile is then reproduced exactly);
 *   - h on isothermal walls: non-equilibrium extrapolation (the paper's wall
 *     method, ref. [45]) from a ghost node one spacing outside the node, with
 *     u_g = 2 u_w - u, theta_g = 2 theta_w - theta (linear through the wall
 *     value at the halfway point), floored at theta_w / 2, and the node's
 *     pressure carried to the ghost by hydrostatic balance, rho_g theta_g =
 *     rho (theta - 3 g n_y), n_y the wall's outward normal (equal pressure
 *     across an x wall, or without gravity; without the hydrostatic term a
 *     floor or ceiling under gravity sat g / (2 R) off its temperature):
 *     h_in = h^eq(ghost) + (h* - h^eq)(node);
 *   - h on adiabatic walls: bounce-back plus twice the odd part of h^eq at
 *     (rho, u_w, theta) of the node (zero total-energy flux through a wall at
 *     rest), for total energy plus the work of the wall on the pair,
 *     u_w . (f_b e_b - f*_a e_a): the energy a moving wall gives the gas is
 *     its velocity times the momentum it gives, so heat, not work, is what
 *     the wall stops;
 *   - a population leaving through a corner across two walls takes the
 *     x-side wall's rule;
 *   - Eq. 50 across a wall uses the mirror ghost Q_g = 2 Q_w - Q(node),
 *     Q_w = rho(node) u_w (1 - theta_w).
 *
 * Open x sides for the acoustic set-up of Sec. IV.B (y must be periodic):
 *   - inlet (side x-): the ghost node one spacing outside (the source of
 *     the wave) is reset every step to the equilibria of the state of
 *     Eq. 53 at time t, rho = rho_in + d_rho sin(w t), u = u_wall[0] +
 *     (d_u sin(w t), 0), T = T_wall[0] + d_T sin(w t); it emits them into the
 *     first column (populations with e_x = +1), and what leaves the first
 *     column through that side is dropped;
 *   - outlet (side x+): zero-gradient extrapolation of (rho, u, T) into the
 *     ghost column, then non-equilibrium extrapolation; the ghost's
 *     equilibria equal the last column's, so its post-collision populations
 *     are those of the last column, which it emits back (e_x = -1);
 *   - Eq. 50 at the inlet uses the inlet node's Q = rho u (1 - theta), at the
 *     outlet the last column's own Q (zero gradient).
 *
 * Walls of non-equilibrium extrapolation (the paper's wall method, ref. [45];
 * a side whose bit is set in wall_nee): the wall sits on the ghost node G one
 * spacing outside the boundary node F.  G's state is the wall velocity,
 * theta_G (theta_w on an isothermal wall; on an adiabatic one zero normal
 * gradient at G to second order, (4 theta_F - theta_F2)/3 with F2 the next
 * node inward) and F's pressure carried to G by hydrostatic balance
 * (rho_G theta_G = rho_F (theta_F - 3 g n_y): p = rho R T, so equal density
 * would push mass through the wall, and so would gravity without the
 * hydrostatic term).  Its pre-collision
 * populations are its equilibria plus F's non-equilibrium part
 * fbar(F) - f^eq(F) (likewise for h; on an adiabatic wall without the normal
 * heat flux that part carries: the normal moment of h^neq - Z f^neq, Z the
 * coupling of Eq. 36 at the wall velocity, so that the viscous work Z f^neq
 * of a moving wall still passes), and it collides like any node, with
 * the Guo force of its own density and no correction term; G emits the
 * post-collision populations pointing into the domain, and what leaves
 * through the side is dropped.
 * Along an axis that is not periodic the corner ghost at the end of an x
 * side's column emits its one inward diagonal into the corner node from that
 * node's values (the x side wins, as for the halfway rules); a y side's
 * ghosts emit nothing across an x side that is not periodic.  Eq. 50 across
 * such a wall keeps the mirror ghost of the halfway rules.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* D2Q9 velocities and weights, Eq. 6 with c = 1 and the weights under Eq. 8. */
static const int EX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int EY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const int OPP[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
static const double W[9] = {4.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0, 1.0 / 9.0,
                            1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
static const double DIM = 2.0; /* D */

enum { ORC_PERIODIC = 0, ORC_WALL_ISOTHERMAL = 1, ORC_WALL_ADIABATIC = 2, ORC_INLET = 3,
       ORC_OUTLET = 4 };
enum { ORC_E_TOTAL = 0, ORC_E_INTERNAL = 1 };
enum { ORC_BGK = 0, ORC_MRT = 1 };
enum { ORC_MU_TAU = 0, ORC_MU_POWER = 1, ORC_MU_SUTHERLAND = 2 };

typedef struct {
  int32_t nx, ny;
  int32_t bc[4]; /* sides x-, x+, y-, y+ */
  double tau_f, tau_h;
  double R, T0, b;
  double u_wall[4][2];
  double T_wall[4];
  double g; /* gravity; force density a = (0, -rho g) */
  int32_t energy_model;
  int32_t correction;
  int32_t z_full;
  int32_t collision;        /* ORC_BGK: Eq. 34; ORC_MRT: Eqs. 43-45 */
  double s_e, s_eps, s_q;   /* MRT rates of e, epsilon, q in S (Eq. 40); 0: omega_f */
  int32_t mu_law;           /* ORC_MU_TAU: constant tau (mu = tau_f p, Eq. 30);
                               ORC_MU_POWER: mu = mu0 theta^n (Eq. 52 premise);
                               ORC_MU_SUTHERLAND: Eq. 59 referred to T0 */
  double mu_n;              /* power-law exponent n */
  double mu_S;              /* Sutherland constant S / T0 */
  /* inlet (side x-, Eq. 53): rho_in + d_rho sin(w t), u_wall[0] + (d_u sin(w t), 0),
     T_wall[0] + d_T sin(w t) */
  double in_rho, in_drho, in_du, in_dT, in_omega;
  /* bit s set: side s is a wall of non-equilibrium extrapolation on the
     ghost node one spacing outside (instead of the halfway rules) */
  int32_t wall_nee;
} orc_params;

typedef struct {
  orc_params p;
  long n;
  double *f[9], *h[9];   /* current state, pre-collision */
  double *fn[9], *hn[9]; /* next state */
  double *rho, *ux, *uy, *theta, *Qx, *Qy;
  double* es; /* specific energy sum(hbar)/rho: E (Eq. 37) or b R T / 2 (Eq. 38) */
  long t;     /* steps taken: the time of the current state */
} orc_state;

/* ---- pointwise pieces (exported so the tests can pin them one by one) ---- */

/* Eq. 18a: f^eq with the theta terms, third-order velocity term dropped. */
void orc_feq(double RT0, double rho, double ux, double uy, double theta, double out[9]) {
  double usq = ux * ux + uy * uy;
  for (int a = 0; a < 9; ++a) {
    double eu = EX[a] * ux + EY[a] * uy;
    double esq = (double)(EX[a] * EX[a] + EY[a] * EY[a]);
    double second = (eu / RT0) * (eu / RT0) - usq / RT0 + (theta - 1.0) * (esq / RT0 - DIM);
    double third = eu / (2.0 * RT0) * (theta - 1.0) * (esq / RT0 - DIM - 2.0);
    out[a] = rho * W[a] * (1.0 + eu / RT0 + 0.5 * second + third);
  }
}

/* Eq. 18b: h^eq = E f^eq + w p [...], p = rho R T = rho RT0 theta. */
void orc_heq(double RT0, double rho, double ux, double uy, double theta, double E,
             const double feq[9], double out[9]) {
  double usq = ux * ux + uy * uy;
  double p = rho * RT0 * theta;
  for (int a = 0; a < 9; ++a) {
    double eu = EX[a] * ux + EY[a] * uy;
    double esq = (double)(EX[a] * EX[a] + EY[a] * EY[a]);
    double br = eu / RT0 + (eu / RT0) * (eu / RT0) - usq / RT0 + 0.5 * theta * (esq / RT0 - DIM);
    out[a] = E * feq[a] + W[a] * p * br;
  }
}

/* Text under Eq. 38: internal-energy equilibrium h^eq = b R T f^eq / 2. */
void orc_heq_internal(double RT0, double b, double theta, const double feq[9], double out[9]) {
  double bRT = b * RT0 * theta;
  for (int a = 0; a < 9; ++a) out[a] = 0.5 * bRT * feq[a];
}

/* Eq. 48 and Eq. 49: C_a from the two divergence pieces of Q. */
void orc_correction(double dQx_dx, double dQy_dy, double out[9]) {
  double phx = 3.0 * (dQx_dx + dQy_dy);
  double phy = dQx_dx - dQy_dy;
  out[0] = -phx / 9.0;
  out[1] = -phx / 36.0 + phy / 4.0;
  out[2] = -phx / 36.0 - phy / 4.0;
  out[3] = out[1];
  out[4] = out[2];
  out[5] = phx / 18.0;
  out[6] = phx / 18.0;
  out[7] = phx / 18.0;
  out[8] = phx / 18.0;
}

/* Guo forcing term (the text above Eq. 51):
 * F_a = w_a [ (e.a)/RT0 + u a : (e e - RT0 I) / RT0^2 ]. */
void orc_force(double RT0, double ux, double uy, double ax, double ay, double out[9]) {
  for (int a = 0; a < 9; ++a) {
    double ea = EX[a] * ax + EY[a] * ay;
    double ua_ee = (EX[a] * ux + EY[a] * uy) * ea; /* (u.e)(e.a) */
    double ua = ux * ax + uy * ay;
    out[a] = W[a] * (ea / RT0 + (ua_ee - RT0 * ua) / (RT0 * RT0));
  }
}

/* Appendix B: the D2Q9 transformation matrix M (B1), moments in the order
 * (rho, e, epsilon, j_x, q_x, j_y, q_y, p_xx, p_xy), and its inverse (B2). */
static const double MRT_M[9][9] = {
    {1, 1, 1, 1, 1, 1, 1, 1, 1},       {-4, -1, -1, -1, -1, 2, 2, 2, 2},
    {4, -2, -2, -2, -2, 1, 1, 1, 1},   {0, 1, 0, -1, 0, 1, -1, -1, 1},
    {0, -2, 0, 2, 0, 1, -1, -1, 1},    {0, 0, 1, 0, -1, 1, 1, -1, -1},
    {0, 0, -2, 0, 2, 1, 1, -1, -1},    {0, 1, -1, 1, -1, 0, 0, 0, 0},
    {0, 0, 0, 0, 0, 1, -1, 1, -1}};
static const double MRT_MINV[9][9] = {
    {1. / 9, -1. / 9, 1. / 9, 0, 0, 0, 0, 0, 0},
    {1. / 9, -1. / 36, -1. / 18, 1. / 6, -1. / 6, 0, 0, 1. / 4, 0},
    {1. / 9, -1. / 36, -1. / 18, 0, 0, 1. / 6, -1. / 6, -1. / 4, 0},
    {1. / 9, -1. / 36, -1. / 18, -1. / 6, 1. / 6, 0, 0, 1. / 4, 0},
    {1. / 9, -1. / 36, -1. / 18, 0, 0, -1. / 6, 1. / 6, -1. / 4, 0},
    {1. / 9, 1. / 18, 1. / 36, 1. / 6, 1. / 12, 1. / 6, 1. / 12, 0, 1. / 4},
    {1. / 9, 1. / 18, 1. / 36, -1. / 6, -1. / 12, 1. / 6, 1. / 12, 0, -1. / 4},
    {1. / 9, 1. / 18, 1. / 36, -1. / 6, -1. / 12, -1. / 6, -1. / 12, 0, 1. / 4},
    {1. / 9, 1. / 18, 1. / 36, 1. / 6, 1. / 12, -1. / 6, -1. / 12, 0, -1. / 4}};

void orc_mrt_matrices(double M[81], double Minv[81]) {
  for (int r = 0; r < 9; ++r)
    for (int c = 0; c < 9; ++c) {
      M[9 * r + c] = MRT_M[r][c];
      Minv[9 * r + c] = MRT_MINV[r][c];
    }
}

/* Eq. 41: the moment-space equilibria of the coupled model. */
void orc_meq(double rho, double ux, double uy, double theta, double out[9]) {
  double usq = ux * ux + uy * uy;
  out[0] = rho;
  out[1] = rho * (-4.0 + 3.0 * usq + 2.0 * theta);
  out[2] = rho * (3.0 - 3.0 * usq - 2.0 * theta);
  out[3] = rho * ux;
  out[4] = rho * (-2.0 * ux + ux * theta);
  out[5] = rho * uy;
  out[6] = rho * (-2.0 * uy + uy * theta);
  out[7] = rho * (ux * ux - uy * uy);
  out[8] = rho * ux * uy;
}

static void matvec9(const double A[9][9], const double v[9], double out[9]) {
  for (int r = 0; r < 9; ++r) {
    double acc = 0.0;
    for (int c = 0; c < 9; ++c) acc += A[r][c] * v[c];
    out[r] = acc;
  }
}

/* ---- state ---- */

static long nodes(const orc_params* p) { return (long)p->nx * (long)p->ny; }

orc_state* orc_new(const orc_params* p) {
  orc_state* s = (orc_state*)calloc(1, sizeof(orc_state));
  if (!s) return NULL;
  s->p = *p;
  s->n = nodes(p);
  for (int a = 0; a < 9; ++a) {
    s->f[a] = (double*)calloc(s->n, sizeof(double));
    s->h[a] = (double*)calloc(s->n, sizeof(double));
    s->fn[a] = (double*)calloc(s->n, sizeof(double));
    s->hn[a] = (double*)calloc(s->n, sizeof(double));
  }
  s->rho = (double*)calloc(s->n, sizeof(double));
  s->ux = (double*)calloc(s->n, sizeof(double));
  s->uy = (double*)calloc(s->n, sizeof(double));
  s->theta = (double*)calloc(s->n, sizeof(double));
  s->Qx = (double*)calloc(s->n, sizeof(double));
  s->Qy = (double*)calloc(s->n, sizeof(double));
  s->es = (double*)calloc(s->n, sizeof(double));
  return s;
}

void orc_free(orc_state* s) {
  if (!s) return;
  for (int a = 0; a < 9; ++a) {
    free(s->f[a]);
    free(s->h[a]);
    free(s->fn[a]);
    free(s->hn[a]);
  }
  free(s->rho);
  free(s->ux);
  free(s->uy);
  free(s->theta);
  free(s->Qx);
  free(s->Qy);
  free(s->es);
  free(s);
}

/* Initial state (the paper is silent): fbar = f^eq(rho, u, T), hbar = h^eq. */
void orc_init(orc_state* s, const double* rho, const double* ux, const double* uy,
              const double* T) {
  const orc_params* p = &s->p;
  double RT0 = p->R * p->T0;
  s->t = 0;
  for (long i = 0; i < s->n; ++i) {
    double th = T[i] / p->T0;
    double feq[9], heq[9];
    orc_feq(RT0, rho[i], ux[i], uy[i], th, feq);
    if (p->energy_model == ORC_E_TOTAL) {
      double E = 0.5 * (p->b * p->R * T[i] + ux[i] * ux[i] + uy[i] * uy[i]);
      orc_heq(RT0, rho[i], ux[i], uy[i], th, E, feq, heq);
    } else {
      orc_heq_internal(RT0, p->b, th, feq, heq);
    }
    for (int a = 0; a < 9; ++a) {
      s->f[a][i] = feq[a];
      s->h[a][i] = heq[a];
    }
  }
}

/* Moments of the pre-collision state at node i: Eq. 35 with the force shift
 * (rho u = sum e fbar + a/2, a = (0, -rho g)), Eq. 37 or the internal-energy
 * temperature under Eq. 38. */
static void node_moments(const orc_state* s, long i, double* rho, double* ux, double* uy,
                         double* theta, double* es) {
  const orc_params* p = &s->p;
  double r = 0, jx = 0, jy = 0, sh = 0;
  for (int a = 0; a < 9; ++a) {
    r += s->f[a][i];
    jx += EX[a] * s->f[a][i];
    jy += EY[a] * s->f[a][i];
    sh += s->h[a][i];
  }
  double ax = 0.0, ay = -r * p->g;
  double vx = (jx + 0.5 * ax) / r;
  double vy = (jy + 0.5 * ay) / r;
  double T;
  if (p->energy_model == ORC_E_TOTAL)
    T = 2.0 / (p->b * p->R) * (sh / r - 0.5 * (vx * vx + vy * vy));
  else
    T = 2.0 * sh / (r * p->b * p->R);
  *rho = r;
  *ux = vx;
  *uy = vy;
  *theta = T / p->T0;
  *es = sh / r;
}

/* Wall temperature ratio for side `side` seen from node i. */
static double wall_theta(const orc_state* s, int side, long i) {
  const orc_params* p = &s->p;
  if (p->bc[side] == ORC_WALL_ISOTHERMAL) return p->T_wall[side] / p->T0;
  return s->theta[i];
}

/* State of the inlet node at time t, Eq. 53 (theta = T / T0). */
static void inlet_state(const orc_params* p, long t, double* rho, double* ux, double* uy,
                        double* theta) {
  double sn = sin(p->in_omega * (double)t);
  *rho = p->in_rho + p->in_drho * sn;
  *ux = p->u_wall[0][0] + p->in_du * sn;
  *uy = p->u_wall[0][1];
  *theta = (p->T_wall[0] + p->in_dT * sn) / p->T0;
}

/* Q of the neighbour across one side of node i (Eq. 50 stencil). */
static double neighbour_Q(const orc_state* s, int x, int y, int side, int comp) {
  const orc_params* p = &s->p;
  int nx = p->nx, ny = p->ny;
  int xx = x + (side == 0 ? -1 : side == 1 ? 1 : 0);
  int yy = y + (side == 2 ? -1 : side == 3 ? 1 : 0);
  const double* Q = comp == 0 ? s->Qx : s->Qy;
  long i = (long)y * nx + x;
  int outside = xx < 0 || xx >= nx || yy < 0 || yy >= ny;
  if (!outside) return Q[(long)yy * nx + xx];
  if (p->bc[side] == ORC_PERIODIC) {
    xx = (xx + nx) % nx;
    yy = (yy + ny) % ny;
    return Q[(long)yy * nx + xx];
  }
  if (p->bc[side] == ORC_OUTLET) return Q[i]; /* zero gradient */
  if (p->bc[side] == ORC_INLET) {
    double r, vx, vy, th;
    inlet_state(p, s->t, &r, &vx, &vy, &th);
    return r * (comp == 0 ? vx : vy) * (1.0 - th);
  }
  /* mirror ghost across the wall: Q_g = 2 Q_w - Q(node) */
  double Qw = s->rho[i] * p->u_wall[side][comp] * (1.0 - wall_theta(s, side, i));
  return 2.0 * Qw - Q[i];
}

/* Eq. 50: the central differences dQx/dx, dQy/dy at node (x, y), from the Q
 * of phase 1 and, across a side, the neighbour_Q stand-ins above. */
static void node_dQ(const orc_state* s, int x, int y, double* dQx, double* dQy) {
  *dQx = 0.5 * (neighbour_Q(s, x, y, 1, 0) - neighbour_Q(s, x, y, 0, 0));
  *dQy = 0.5 * (neighbour_Q(s, x, y, 3, 1) - neighbour_Q(s, x, y, 2, 1));
}

static void phase1(orc_state* s, int nthreads) {
  const orc_params* p = &s->p;
  (void)nthreads;
#pragma omp parallel for num_threads(nthreads) schedule(static)
  for (int y = 0; y < p->ny; ++y) {
    for (int x = 0; x < p->nx; ++x) {
      long i = (long)y * p->nx + x;
      node_moments(s, i, &s->rho[i], &s->ux[i], &s->uy[i], &s->theta[i], &s->es[i]);
      s->Qx[i] = s->rho[i] * s->ux[i] * (1.0 - s->theta[i]);
      s->Qy[i] = s->rho[i] * s->uy[i] * (1.0 - s->theta[i]);
    }
  }
}

/* Relaxation times of a node.  Constant: the given tau_f, tau_h.  With a
 * temperature-dependent viscosity mu(T) (power law mu0 theta^n, the premise
 * of Eq. 52; or Sutherland's law, Eq. 59, written relative to T0:
 * mu = mu0 theta^{3/2} (1 + S/T0)/(theta + S/T0)), mu0 = tau_f R T0 is the
 * viscosity at rho = 1, T = T0, the BGK relation mu = tau_f p (Eq. 30) gives
 * tau_f = mu / (rho R T), and the Prandtl number stays tau_f / tau_h. */
static void node_taus(const orc_params* p, double rho, double th, double* tf, double* tq) {
  if (p->mu_law == ORC_MU_TAU) {
    *tf = p->tau_f;
    *tq = p->tau_h;
    return;
  }
  const double RT0 = p->R * p->T0;
  const double mu0 = p->tau_f * RT0;
  double mu;
  if (p->mu_law == ORC_MU_POWER)
    mu = mu0 * pow(th, p->mu_n);
  else
    mu = mu0 * pow(th, 1.5) * (1.0 + p->mu_S) / (th + p->mu_S);
  *tf = mu / (rho * RT0 * th);
  *tq = *tf * (p->tau_h / p->tau_f);
}

/* Equilibria a node relaxes to: Eq. 18a and Eq. 18b with the specific
 * energy es (or es f^eq, Eq. 38), rest populations from the moment sums. */
static void node_equilibria(const orc_params* p, double rho, double ux, double uy, double th,
                            double es, double feq[9], double heq[9]) {
  const double RT0 = p->R * p->T0;
  orc_feq(RT0, rho, ux, uy, th, feq);
  if (p->energy_model == ORC_E_TOTAL) {
    orc_heq(RT0, rho, ux, uy, th, es, feq, heq);
  } else {
    for (int a = 0; a < 9; ++a) heq[a] = es * feq[a];
  }
  double sf = 0.0, sh = 0.0;
  for (int a = 1; a < 9; ++a) {
    sf += feq[a];
    sh += heq[a];
  }
  feq[0] = rho - sf;
  heq[0] = rho * es - sh;
}

/* Collision of one node (phase 2 below): from its pre-collision fbar, hbar,
 * moments (rho, u, theta, es = sum(hbar)/rho) and source C (correction plus
 * force), the equilibria feq, heq it relaxes to and its post-collision fs, hs. */
static void collide(const orc_params* p, double rho, double ux, double uy, double th, double es,
                    const double fb[9], const double hb[9], const double C[9], double feq[9],
                    double heq[9], double fs[9], double hs[9]) {
  double usq = ux * ux + uy * uy;
  double tau_f, tau_h;
  node_taus(p, rho, th, &tau_f, &tau_h);
  const double wf = 2.0 / (2.0 * tau_f + 1.0); /* omega_f below Eq. 34, dt = 1 */
  const double wh = 2.0 / (2.0 * tau_h + 1.0); /* omega_h below Eq. 36 */

  /* Equilibria at the node's moments.  The energy they carry is the one
   * recovered from hbar: E = sum(hbar)/rho (Eq. 37) in Eq. 18b, and
   * b R T / 2 = sum(hbar)/rho (Eq. 38) for the internal-energy model, so
   * that the relaxation returns exactly the energy it was given; the rest
   * populations follow from the moment sums of Eqs. 19a/19b,
   * sum f^eq = rho and sum h^eq = rho E, so that no rounding of the
   * weights biases mass or energy step after step. */
  node_equilibria(p, rho, ux, uy, th, es, feq, heq);

  /* Collision of f.  BGK: Eq. 34 ("+(1 - w_f/2) C" from Eqs. 32-33).  MRT:
   * Eq. 44 in moment space with m = M f (the stored f is f-hat of
   * Eq. 43), m^eq of Eq. 41, C-hat = M C and S of Eq. 40; the shear rate
   * 1/tau_f of Eq. 40 is omega_f (the discrete MRT time is the
   * continuous tau_f plus 1/2, mu = (tau - 1/2) p), tau_rho = tau_j = 1
   * (the rates of conserved moments drop out); then f* = M^-1 m*. */
  if (p->collision == ORC_MRT) {
    double fh[9], m[9], meq[9], Ch[9], ms[9];
    double S[9] = {1.0, p->s_e > 0 ? p->s_e : wf, p->s_eps > 0 ? p->s_eps : wf, 1.0,
                   p->s_q > 0 ? p->s_q : wf, 1.0, p->s_q > 0 ? p->s_q : wf, wf, wf};
    for (int a = 0; a < 9; ++a) fh[a] = fb[a];
    matvec9(MRT_M, fh, m);
    orc_meq(rho, ux, uy, th, meq);
    matvec9(MRT_M, C, Ch);
    for (int k = 0; k < 9; ++k) ms[k] = m[k] - S[k] * (m[k] - meq[k]) + (1.0 - 0.5 * S[k]) * Ch[k];
    matvec9(MRT_MINV, ms, fs);
  } else {
    for (int a = 0; a < 9; ++a) {
      double fa = fb[a];
      fs[a] = fa - wf * (fa - feq[a]) + (1.0 - 0.5 * wf) * C[a];
    }
  }
  /* Collision of h: Eq. 36 (BGK) or Eq. 47 (MRT), or Eq. 38 (internal
   * energy, no coupling).  The Eq. 47 coupling (1 - w_h/2) Z / tau_hf
   * with tau_hf = tau/(Pr - 1), tau = tau_f + 1/2 the discrete MRT time
   * and Pr = (tau - 1/2)/tau_h. */
  const double kz = p->collision == ORC_MRT
                        ? (1.0 - 0.5 * wh) * (tau_f / tau_h - 1.0) / (tau_f + 0.5)
                        : wh - wf;
  for (int a = 0; a < 9; ++a) {
    double fa = fb[a], ha = hb[a];
    hs[a] = ha - wh * (ha - heq[a]);
    if (p->energy_model == ORC_E_TOTAL) {
      double eu = EX[a] * ux + EY[a] * uy;
      double Z = p->z_full ? eu - 0.5 * usq : eu;
      hs[a] += kz * Z * (fa - feq[a] + 0.5 * C[a]);
    }
  }
}

static void phase2(orc_state* s, int nthreads) {
  const orc_params* p = &s->p;
  const int nx = p->nx, ny = p->ny;
  const double RT0 = p->R * p->T0;
  /* equilibria of the inlet node at this step's time (Eq. 53) */
  double fin[9], hin[9];
  if (p->bc[0] == ORC_INLET) {
    double r, vx, vy, th;
    inlet_state(p, s->t, &r, &vx, &vy, &th);
    orc_feq(RT0, r, vx, vy, th, fin);
    if (p->energy_model == ORC_E_TOTAL)
      orc_heq(RT0, r, vx, vy, th, 0.5 * (p->b * RT0 * th + vx * vx + vy * vy), fin, hin);
    else
      orc_heq_internal(RT0, p->b, th, fin, hin);
  }
  (void)nthreads;
#pragma omp parallel for num_threads(nthreads) schedule(static)
  for (int y = 0; y < ny; ++y) {
    for (int x = 0; x < nx; ++x) {
      long i = (long)y * nx + x;
      double rho = s->rho[i], ux = s->ux[i], uy = s->uy[i], th = s->theta[i];
      /* Eq. 50: central differences of Q; Eq. 48-49: C_a. */
      double C[9] = {0};
      if (p->correction) {
        double dQx, dQy;
        node_dQ(s, x, y, &dQx, &dQy);
        orc_correction(dQx, dQy, C);
      }
      /* Force absorbed into C (text under Eq. 51). */
      double F[9];
      orc_force(RT0, ux, uy, 0.0, -rho * p->g, F);
      for (int a = 0; a < 9; ++a) C[a] += F[a];

      /* equilibria and collision of the node */
      double fb[9], hb[9], feq[9], heq[9], fs[9], hs[9];
      for (int a = 0; a < 9; ++a) {
        fb[a] = s->f[a][i];
        hb[a] = s->h[a][i];
      }
      collide(p, rho, ux, uy, th, s->es[i], fb, hb, C, feq, heq, fs, hs);

      /* Wall (f, adiabatic h) and ghost (isothermal h) equilibria for the up
       * to two sides this node touches. */
      double fw[4][9], hw[4][9];
      int have[4] = {0, 0, 0, 0};

      /* Streaming (LHS of Eqs. 34 and 36: x + e_a at t + 1). */
      for (int a = 0; a < 9; ++a) {
        /* open x sides: the inlet node emits its equilibria into the first
         * column, the outlet ghost (a copy of the last column) emits the
         * last column's own post-collision values back into it */
        if (x == 0 && EX[a] == 1 && p->bc[0] == ORC_INLET) {
          s->fn[a][i] = fin[a];
          s->hn[a][i] = hin[a];
        }
        if (x == nx - 1 && EX[a] == -1 && p->bc[1] == ORC_OUTLET) {
          long j = (long)((y + EY[a] + ny) % ny) * nx + x;
          s->fn[a][j] = fs[a];
          s->hn[a][j] = hs[a];
        }
        int dx = x + EX[a], dy = y + EY[a];
        int ox = dx < 0 ? 0 : (dx >= nx ? 1 : -1);
        int oy = dy < 0 ? 2 : (dy >= ny ? 3 : -1);
        int side = -1;
        if (ox >= 0 && p->bc[ox] != ORC_PERIODIC)
          side = ox;
        else if (oy >= 0 && p->bc[oy] != ORC_PERIODIC)
          side = oy;
        if (side < 0) {
          long j = (long)((dy + ny) % ny) * nx + (long)((dx + nx) % nx);
          s->fn[a][j] = fs[a];
          s->hn[a][j] = hs[a];
          continue;
        }
        if (p->bc[side] == ORC_INLET || p->bc[side] == ORC_OUTLET) continue; /* leaves */
        if (p->wall_nee >> side & 1) continue; /* leaves; the ghost node emits below */
        double uwx = p->u_wall[side][0], uwy = p->u_wall[side][1];
        int iso = p->bc[side] == ORC_WALL_ISOTHERMAL;
        if (!have[side]) {
          double thw = wall_theta(s, side, i);
          orc_feq(RT0, rho, uwx, uwy, th, fw[side]);
          /* h: ghost state for isothermal walls, wall state for adiabatic. */
          /* linear through the wall value, floored at half of it: a node
           * more than 1.5 times hotter than the wall would otherwise give
           * the ghost a vanishing or negative temperature, where the
           * equal-pressure ghost density diverges */
          double thg = iso ? fmax(2.0 * thw - th, 0.5 * thw) : th;
          const int nyo = side == 2 ? -1 : (side == 3 ? 1 : 0);
          double rg = iso ? rho * (th - 3.0 * p->g * nyo) / thg : rho;
          double ugx = iso ? 2.0 * uwx - ux : uwx;
          double ugy = iso ? 2.0 * uwy - uy : uwy;
          double fg[9];
          orc_feq(RT0, rg, ugx, ugy, thg, fg);
          if (p->energy_model == ORC_E_TOTAL) {
            double Eg = 0.5 * (p->b * RT0 * thg + ugx * ugx + ugy * ugy);
            orc_heq(RT0, rg, ugx, ugy, thg, Eg, fg, hw[side]);
          } else {
            orc_heq_internal(RT0, p->b, thg, fg, hw[side]);
          }
          have[side] = 1;
        }
        int b = OPP[a]; /* reflected direction, points back into the fluid */
        double A = 0.5 * (fw[side][b] - fw[side][a]);   /* odd part of f^eq along e_b */
        s->fn[b][i] = fs[a] + 2.0 * A;
        if (iso) {
          s->hn[b][i] = hw[side][b] + (hs[b] - heq[b]);
        } else {
          double B = 0.5 * (hw[side][b] - hw[side][a]); /* odd part of h^eq */
          s->hn[b][i] = hs[a] + 2.0 * B;
          if (p->energy_model == ORC_E_TOTAL)
            s->hn[b][i] += uwx * (s->fn[b][i] * EX[b] - fs[a] * EX[a]) +
                           uwy * (s->fn[b][i] * EY[b] - fs[a] * EY[a]);
        }
      }

      /* Walls of non-equilibrium extrapolation touching this node. */
      for (int side = 0; side < 4; ++side) {
        if (!(p->wall_nee >> side & 1)) continue;
        const int on = side == 0 ? x == 0 : side == 1 ? x == nx - 1 : side == 2 ? y == 0 : y == ny - 1;
        if (!on) continue;
        const int nxo = side == 0 ? -1 : side == 1 ? 1 : 0; /* outward normal */
        const int nyo = side == 2 ? -1 : side == 3 ? 1 : 0;
        /* wall temperature: given (isothermal), or zero normal gradient at
         * the wall node to second order, from F and the next node inward */
        double thG;
        if (p->bc[side] == ORC_WALL_ISOTHERMAL) {
          thG = p->T_wall[side] / p->T0;
        } else {
          const long i2 = (long)(y - nyo) * nx + (x - nxo);
          thG = fmax((4.0 * th - s->theta[i2]) / 3.0, 0.5 * th); /* floored: rho_G = rho theta / theta_G */
        }
        const double uwx = p->u_wall[side][0], uwy = p->u_wall[side][1];
        /* the wall node: F's pressure, the wall's velocity, theta_G; its
         * pre-collision populations are its equilibria plus F's
         * non-equilibrium part, and it collides like any node, with the
         * force of its own density (no correction term) */
        /* F's pressure carried one spacing outward by hydrostatic balance,
         * p_G = p_F - rho_F g n_y (a = (0, -rho g), R T0 = 1/3) */
        const double rG = rho * (th - 3.0 * p->g * nyo) / thG;
        const double esG = 0.5 * (p->b * RT0 * thG +
                                  (p->energy_model == ORC_E_TOTAL ? uwx * uwx + uwy * uwy : 0.0));
        double eqfG[9], eqhG[9], fbG[9], hbG[9], CG[9], fG[9], hG[9], dummyf[9], dummyh[9];
        node_equilibria(p, rG, uwx, uwy, thG, esG, eqfG, eqhG);
        for (int a = 0; a < 9; ++a) {
          fbG[a] = eqfG[a] + (fb[a] - feq[a]);
          hbG[a] = eqhG[a] + (hb[a] - heq[a]);
        }
        if (p->bc[side] == ORC_WALL_ADIABATIC) {
          /* an adiabatic wall node carries no normal heat flux: the normal
           * moment of the borrowed h non-equilibrium part, less the viscous
           * work Z f^neq it carries at the wall velocity (h - Z f relaxes at
           * the thermal rate in Eq. 36), is taken out (its energy and
           * tangential moments are untouched) */
          double qn = 0.0, wn = 0.0;
          for (int a = 0; a < 9; ++a) {
            const double en = EX[a] * nxo + EY[a] * nyo;
            double Zw = 0.0;
            if (p->energy_model == ORC_E_TOTAL)
              Zw = EX[a] * uwx + EY[a] * uwy - (p->z_full ? 0.5 * (uwx * uwx + uwy * uwy) : 0.0);
            qn += en * ((hb[a] - heq[a]) - Zw * (fb[a] - feq[a]));
            wn += W[a] * en * en;
          }
          for (int a = 0; a < 9; ++a) hbG[a] -= W[a] * (EX[a] * nxo + EY[a] * nyo) * qn / wn;
        }
        orc_force(RT0, uwx, uwy, 0.0, -rG * p->g, CG);
        collide(p, rG, uwx, uwy, thG, esG, fbG, hbG, CG, dummyf, dummyh, fG, hG);
        /* ghosts emitting into the domain: G = F - n (every inward a), and
         * for an x side along a walled y axis the corner ghost beyond F */
        for (int k = 0; k < 3; ++k) {
          const int gx = x + nxo, gy = y + nyo + (k == 1 ? -1 : k == 2 ? 1 : 0) * (side < 2);
          if (k > 0 && side >= 2) break;
          for (int a = 1; a < 9; ++a) {
            if (EX[a] * nxo + EY[a] * nyo >= 0) continue; /* not inward */
            int dx = gx + EX[a], dy = gy + EY[a];
            if (k > 0) {
              /* corner ghost: only its diagonal into F, and only across a
               * walled y side */
              if (dx != x || dy != y) continue;
              const int ys = gy < 0 ? 2 : 3;
              if ((gy >= 0 && gy < ny) || p->bc[ys] == ORC_PERIODIC) continue;
            } else {
              if (dx < 0 || dx >= nx) {
                if (p->bc[dx < 0 ? 0 : 1] != ORC_PERIODIC) continue;
                dx = (dx + nx) % nx;
              }
              if (dy < 0 || dy >= ny) {
                if (p->bc[dy < 0 ? 2 : 3] != ORC_PERIODIC) continue;
                dy = (dy + ny) % ny;
              }
            }
            const long j = (long)dy * nx + dx;
            s->fn[a][j] = fG[a];
            s->hn[a][j] = hG[a];
          }
        }
      }
    }
  }
}

void orc_step(orc_state* s, long nsteps, int nthreads) {
  if (nthreads < 1) nthreads = 1;
  for (long t = 0; t < nsteps; ++t) {
    phase1(s, nthreads);
    phase2(s, nthreads);
    ++s->t;
    for (int a = 0; a < 9; ++a) {
      double* tf = s->f[a];
      s->f[a] = s->fn[a];
      s->fn[a] = tf;
      double* th = s->h[a];
      s->h[a] = s->hn[a];
      s->hn[a] = th;
    }
  }
}

/* Macroscopic output of the current state: rho, u, T (T = theta T0). */
void orc_moments(const orc_state* s, double* rho, double* ux, double* uy, double* T) {
  for (long i = 0; i < s->n; ++i) {
    double r, vx, vy, th, es;
    node_moments(s, i, &r, &vx, &vy, &th, &es);
    rho[i] = r;
    ux[i] = vx;
    uy[i] = vy;
    T[i] = th * s->p.T0;
  }
}

/* Sums of rho, rho u (with the force shift), and of hbar (= sum rho E). */
void orc_conserved(const orc_state* s, double out[4]) {
  double m = 0, px = 0, py = 0, e = 0;
  for (long i = 0; i < s->n; ++i) {
    double r, vx, vy, th, es;
    node_moments(s, i, &r, &vx, &vy, &th, &es);
    m += r;
    px += r * vx;
    py += r * vy;
    for (int a = 0; a < 9; ++a) e += s->h[a][i];
  }
  out[0] = m;
  out[1] = px;
  out[2] = py;
  out[3] = e;
}

/* Populations as [18][ny][nx]: f_0..f_8 then h_0..h_8. */
void orc_get_pops(const orc_state* s, double* out) {
  for (int a = 0; a < 9; ++a) {
    memcpy(out + (long)a * s->n, s->f[a], sizeof(double) * s->n);
    memcpy(out + (long)(9 + a) * s->n, s->h[a], sizeof(double) * s->n);
  }
}

void orc_set_pops(orc_state* s, const double* in) {
  for (int a = 0; a < 9; ++a) {
    memcpy(s->f[a], in + (long)a * s->n, sizeof(double) * s->n);
    memcpy(s->h[a], in + (long)(9 + a) * s->n, sizeof(double) * s->n);
  }
}

/* The Eq. 50 differences of the current state at every node, as phase 2 of
 * the next step takes them (phase 1 recomputes the moments and Q first):
 * dqx[y*nx+x] = dQx/dx, dqy[y*nx+x] = dQy/dy.  Does not advance the state. */
void orc_gradients(orc_state* s, double* dqx, double* dqy) {
  phase1(s, 1);
  for (int y = 0; y < s->p.ny; ++y)
    for (int x = 0; x < s->p.nx; ++x) {
      long i = (long)y * s->p.nx + x;
      node_dQ(s, x, y, &dqx[i], &dqy[i]);
    }
}

int orc_param_size(void) { return (int)sizeof(orc_params); }

/* Time of the current state (steps taken), and setting it (resume). */
long orc_time(const orc_state* s) { return s->t; }
void orc_set_time(orc_state* s, long t) { s->t = t; }
