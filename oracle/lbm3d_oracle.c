/*
 * Oracle of the three-dimensional extension: plain, slow, FP64 CPU statement
 * of one time step of the coupled double-distribution-function thermal
 * lattice Boltzmann method (Li, Luo, He, Gao & Tao, arXiv:1109.6672) on the
 * D3Q19 lattice, BGK scheme.  The paper derives the model for D2Q9 and
 * states (Sec. V) that its formulation extends to 3-D; this file is that
 * extension written from the paper's own construction:
 *   - equilibria: Eq. 18a and Eq. 18b with D = 3 (the Hermite expansions of
 *     Eqs. 13 and 17 discretised on D3Q19, c = 1, R T0 = 1/3);
 *   - correction term: Eq. 22 with the constraints of Eq. 26 and, as Eq. 28
 *     is obtained from Eq. 27, a second moment that removes the deviation of
 *     the third-order moment of f^eq from Eq. 10d:
 *        sum_a e_ai e_aj C_a = sum_k d/dx_k D_ijk,
 *        D_ijk = sum_a f^eq_a e_ai e_aj e_ak - rho R T (u_i d_jk + u_j d_ik + u_k d_ij)
 *     (on D2Q9 this is exactly Eq. 20/28; on D3Q19 the deviation also has
 *     entries D_iik, i != k, besides the diagonal D_iii).  D is evaluated
 *     here by summing the lattice, node by node, and differentiated by the
 *     central differences of Eq. 50 along each axis.  C_a itself is the
 *     lattice analogue of Eqs. 48-49: an even quadratic polynomial of e_a
 *     without weights, C_a = sum_ij A_ij (e_ai e_aj - kappa d_ij) with
 *     kappa = sum_a e_ax^2 / 19 (so sum C = 0), the symmetric A solved from
 *     the six second-moment conditions (on D2Q9 this construction gives
 *     Eq. 49 exactly: only the second-order moments of the orthogonal basis
 *     are non-zero);
 *   - time discretisation: Eqs. 33-36 (BGK, omega = 2/(2 tau + 1), the sign
 *     of the C term read as + as in the D2Q9 oracle), or Eq. 38 with the
 *     internal-energy h^eq = b R T f^eq / 2; moments Eq. 35, Eq. 37.
 * Each side of the box is periodic or a halfway wall (at x = -1/2 and
 * nx - 1/2, likewise in y and z; a population leaving through an edge of
 * two walls takes the rule of the first of x, y, z, as the D2Q9 oracle's
 * corners take the x side's), with the D2Q9 oracle's wall rules carried
 * to D3Q19: for a population a leaving through the wall, with b its
 * opposite, f_b(node, t+1) = f*_a - 2 (odd part of f^eq_a at the node's rho
 * and theta and the wall velocity); h on an isothermal wall by the
 * equilibrium of a ghost node one spacing outside (u_g = 2 u_w - u,
 * theta_g = max(2 theta_w - theta, theta_w / 2), rho_g theta_g =
 * rho (theta - 3 g n_z), the node's pressure carried across by hydrostatic
 * balance, n_z the wall's outward normal) plus the node's own
 * non-equilibrium part, h_b = h^eq_b(ghost) +
 * (h*_b - h^eq_b)(node); h on an adiabatic wall h_b = h*_a - 2 (odd part of
 * h^eq_a at (rho, u_w, theta)), for total energy plus the work of the wall
 * on the pair, u_w . (f_b e_b - f*_a e_a) (the energy a moving wall gives
 * the gas is its velocity times the momentum it gives; without this term
 * a moving adiabatic wall would hold the total energy flux, not the heat
 * flux, at zero, and the gas under it would cool).  Across a wall the
 * derivative of D in the correction takes the ghost D_g = 2 D_w - D(node),
 * D_w = D at the node's rho and the wall's u_w, theta_w (theta of the node
 * on an adiabatic wall): D is linear in Q = rho u (1 - theta), so this is
 * the D2Q9 oracle's mirror ghost Q_g = 2 Q_w - Q.
 *
 * Gravity along -z (g > 0, the internal-energy model, as the paper's cavity
 * runs it): Guo's force term of Eq. 51 carried to D = 3 enters beside C_a,
 * and the velocity carries the half-force shift of the text under Eq. 51.
 *
 * Parity unpinned, in part: the -u^2/2 part of Z_a in the Eq. 36 coupling
 * (the full Z form).  No closed form or decay rate the paper fixes depends
 * on it (Z_a reduces to e_a.u at the Navier-Stokes level); it is checked
 * only against an independent NumPy restatement of the step
 * (tests/brute_lbm3d.py), which also restates the z walls.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
 * load this file; only the tests, the smoke check and the benchmark's CPU
 * baseline do.  It shares no code, header, table or constant with the CUDA
 * library or with the D2Q9 oracle.
 *
 * Build: gcc -O2 -ffp-contract=off -fPIC -shared [-fopenmp].
 *
 * State: the canonical pre-collision distributions fbar_a(x,t), hbar_a(x,t),
 * stored as f[a][(z*ny + y)*nx + x].
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define Q3 19

/* D3Q19 velocities: rest, the six axis directions, the twelve face
 * diagonals; weights 1/3, 1/18, 1/36. */
static const int E3[Q3][3] = {
    {0, 0, 0},  {1, 0, 0},   {-1, 0, 0}, {0, 1, 0},  {0, -1, 0}, {0, 0, 1},  {0, 0, -1},
    {1, 1, 0},  {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0}, {1, 0, 1},  {-1, 0, -1}, {1, 0, -1},
    {-1, 0, 1}, {0, 1, 1},   {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};

static double weight3(int a) {
  int s = abs(E3[a][0]) + abs(E3[a][1]) + abs(E3[a][2]);
  return s == 0 ? 1.0 / 3.0 : (s == 1 ? 1.0 / 18.0 : 1.0 / 36.0);
}

enum { O3_E_TOTAL = 0, O3_E_INTERNAL = 1 };
enum { O3_PERIODIC = 0, O3_WALL_ISOTHERMAL = 1, O3_WALL_ADIABATIC = 2 };

typedef struct {
  int32_t nx, ny, nz;
  int32_t energy_model; /* O3_E_TOTAL (Eq. 36) or O3_E_INTERNAL (Eq. 38 form) */
  int32_t correction;   /* 1: C_a as above; 0: omitted */
  int32_t z_full;       /* 1: Z = e.u - u^2/2; 0: Z = e.u */
  double tau_f, tau_h;  /* continuous-time relaxation times */
  double R, T0, b;      /* R T0 = 1/3; b degrees of freedom */
  int32_t bc_z[2];      /* sides z- and z+: O3_PERIODIC or a wall */
  double u_wall_z[2][3];
  double T_wall_z[2];
  double g;             /* gravity along -z: force density a = (0, 0, -rho g) */
  int32_t bc_x[2], bc_y[2]; /* sides x-, x+ and y-, y+, as bc_z */
  double u_wall_x[2][3], u_wall_y[2][3];
  double T_wall_x[2], T_wall_y[2];
} o3_params;

/* Side s = 2 axis + (0: low end, 1: high end) of the box: its boundary
 * kind, wall velocity and wall temperature. */
static int side_bc(const o3_params* p, int s) {
  return s < 2 ? p->bc_x[s] : (s < 4 ? p->bc_y[s - 2] : p->bc_z[s - 4]);
}
static const double* side_uw(const o3_params* p, int s) {
  return s < 2 ? p->u_wall_x[s] : (s < 4 ? p->u_wall_y[s - 2] : p->u_wall_z[s - 4]);
}
static double side_Tw(const o3_params* p, int s) {
  return s < 2 ? p->T_wall_x[s] : (s < 4 ? p->T_wall_y[s - 2] : p->T_wall_z[s - 4]);
}

typedef struct {
  o3_params p;
  long n;
  double *f[Q3], *h[Q3], *fn[Q3], *hn[Q3];
  double *rho, *ux, *uy, *uz, *theta, *es;
  double* D; /* 27 per node: the third-moment deviation D_ijk */
} o3_state;

/* ---- pointwise pieces ---------------------------------------------------- */

/* Eq. 18a with D = 3. */
void o3_feq(double RT0, double rho, const double u[3], double theta, double out[Q3]) {
  const double usq = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  for (int a = 0; a < Q3; ++a) {
    double eu = E3[a][0] * u[0] + E3[a][1] * u[1] + E3[a][2] * u[2];
    double esq = (double)(E3[a][0] * E3[a][0] + E3[a][1] * E3[a][1] + E3[a][2] * E3[a][2]);
    double t = 1.0 + eu / RT0 +
               0.5 * ((eu / RT0) * (eu / RT0) - usq / RT0 + (theta - 1.0) * (esq / RT0 - 3.0)) +
               eu / (2.0 * RT0) * (theta - 1.0) * (esq / RT0 - 3.0 - 2.0);
    out[a] = rho * weight3(a) * t;
  }
}

/* Eq. 18b with D = 3 (p = rho R T = rho RT0 theta). */
void o3_heq(double RT0, double rho, const double u[3], double theta, double E,
            const double feq[Q3], double out[Q3]) {
  const double usq = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  const double p = rho * RT0 * theta;
  for (int a = 0; a < Q3; ++a) {
    double eu = E3[a][0] * u[0] + E3[a][1] * u[1] + E3[a][2] * u[2];
    double esq = (double)(E3[a][0] * E3[a][0] + E3[a][1] * E3[a][1] + E3[a][2] * E3[a][2]);
    double br = eu / RT0 + (eu / RT0) * (eu / RT0) - usq / RT0 + 0.5 * theta * (esq / RT0 - 3.0);
    out[a] = E * feq[a] + weight3(a) * p * br;
  }
}

/* Internal-energy form under Eq. 38: h^eq = b R T f^eq / 2. */
void o3_heq_internal(double RT0, double b, double theta, const double feq[Q3], double out[Q3]) {
  for (int a = 0; a < Q3; ++a) out[a] = 0.5 * b * RT0 * theta * feq[a];
}

/* Deviation of the third-order moment of f^eq from Eq. 10d without its
 * cubic velocity term (which the model neglects): D[9i+3j+k]. */
void o3_defect(double RT0, double rho, const double u[3], double theta, double D[27]) {
  double feq[Q3];
  o3_feq(RT0, rho, u, theta, feq);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      for (int k = 0; k < 3; ++k) {
        double m = 0.0;
        for (int a = 0; a < Q3; ++a) m += feq[a] * E3[a][i] * E3[a][j] * E3[a][k];
        double req = rho * RT0 * theta *
                     (u[i] * (j == k) + u[j] * (i == k) + u[k] * (i == j));
        D[9 * i + 3 * j + k] = m - req;
      }
}

/* Solve the n x n system M x = r in place (Gaussian elimination with
 * partial pivoting); n <= 6. */
static void solve(int n, double M[6][6], double r[6], double x[6]) {
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int i = c + 1; i < n; ++i)
      if (fabs(M[i][c]) > fabs(M[piv][c])) piv = i;
    if (piv != c) {
      for (int j = 0; j < n; ++j) {
        double t = M[c][j];
        M[c][j] = M[piv][j];
        M[piv][j] = t;
      }
      double t = r[c];
      r[c] = r[piv];
      r[piv] = t;
    }
    for (int i = c + 1; i < n; ++i) {
      double f = M[i][c] / M[c][c];
      for (int j = c; j < n; ++j) M[i][j] -= f * M[c][j];
      r[i] -= f * r[c];
    }
  }
  for (int i = n - 1; i >= 0; --i) {
    double s = r[i];
    for (int j = i + 1; j < n; ++j) s -= M[i][j] * x[j];
    x[i] = s / M[i][i];
  }
}

/* The correction term whose second moments are G (G[3i+j], symmetrised):
 * C_a = sum_ij A_ij (e_ai e_aj - kappa d_ij), zero mass and momentum. */
void o3_correction(const double G[9], double out[Q3]) {
  static const int P[6][2] = {{0, 0}, {1, 1}, {2, 2}, {0, 1}, {0, 2}, {1, 2}};
  double kappa = 0.0;
  for (int a = 0; a < Q3; ++a) kappa += E3[a][0] * E3[a][0];
  kappa /= Q3;
  /* basis polynomial m of the unknown A_m at velocity a (off-diagonal
   * entries appear twice in the double sum) */
  double phi[6][Q3];
  for (int m = 0; m < 6; ++m) {
    int i = P[m][0], j = P[m][1];
    for (int a = 0; a < Q3; ++a)
      phi[m][a] = i == j ? E3[a][i] * E3[a][i] - kappa : 2.0 * E3[a][i] * E3[a][j];
  }
  double M[6][6], r[6], A[6];
  for (int row = 0; row < 6; ++row) {
    int k = P[row][0], l = P[row][1];
    for (int m = 0; m < 6; ++m) {
      double s = 0.0;
      for (int a = 0; a < Q3; ++a) s += E3[a][k] * E3[a][l] * phi[m][a];
      M[row][m] = s;
    }
    r[row] = 0.5 * (G[3 * k + l] + G[3 * l + k]);
  }
  solve(6, M, r, A);
  for (int a = 0; a < Q3; ++a) {
    double c = 0.0;
    for (int m = 0; m < 6; ++m) c += A[m] * phi[m][a];
    out[a] = c;
  }
}

/* ---- grid state ------------------------------------------------------------ */

static long idx3(const o3_params* p, int x, int y, int z) {
  x = (x % p->nx + p->nx) % p->nx;
  y = (y % p->ny + p->ny) % p->ny;
  z = (z % p->nz + p->nz) % p->nz;
  return ((long)z * p->ny + y) * p->nx + x;
}

o3_state* o3_new(const o3_params* p) {
  o3_state* s = (o3_state*)calloc(1, sizeof(o3_state));
  if (!s) return NULL;
  s->p = *p;
  s->n = (long)p->nx * p->ny * p->nz;
  for (int a = 0; a < Q3; ++a) {
    s->f[a] = (double*)calloc(s->n, sizeof(double));
    s->h[a] = (double*)calloc(s->n, sizeof(double));
    s->fn[a] = (double*)calloc(s->n, sizeof(double));
    s->hn[a] = (double*)calloc(s->n, sizeof(double));
  }
  s->rho = (double*)calloc(s->n, sizeof(double));
  s->ux = (double*)calloc(s->n, sizeof(double));
  s->uy = (double*)calloc(s->n, sizeof(double));
  s->uz = (double*)calloc(s->n, sizeof(double));
  s->theta = (double*)calloc(s->n, sizeof(double));
  s->es = (double*)calloc(s->n, sizeof(double));
  s->D = (double*)calloc(27 * s->n, sizeof(double));
  return s;
}

void o3_free(o3_state* s) {
  if (!s) return;
  for (int a = 0; a < Q3; ++a) {
    free(s->f[a]);
    free(s->h[a]);
    free(s->fn[a]);
    free(s->hn[a]);
  }
  free(s->rho);
  free(s->ux);
  free(s->uy);
  free(s->uz);
  free(s->theta);
  free(s->es);
  free(s->D);
  free(s);
}

static void equilibria(const o3_params* p, double rho, const double u[3], double th, double E,
                       double feq[Q3], double heq[Q3]) {
  const double RT0 = p->R * p->T0;
  o3_feq(RT0, rho, u, th, feq);
  if (p->energy_model == O3_E_TOTAL)
    o3_heq(RT0, rho, u, th, E, feq, heq);
  else
    o3_heq_internal(RT0, p->b, th, feq, heq);
}

/* Initial state: fbar = f^eq, hbar = h^eq at the given fields (T in units
 * of T0's temperature scale). */
void o3_init(o3_state* s, const double* rho, const double* ux, const double* uy,
             const double* uz, const double* T) {
  const o3_params* p = &s->p;
  const double RT0 = p->R * p->T0;
  for (long i = 0; i < s->n; ++i) {
    double u[3] = {ux[i], uy[i], uz[i]};
    double th = T[i] / p->T0;
    double E = 0.5 * (p->b * RT0 * th + u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    double feq[Q3], heq[Q3];
    equilibria(p, rho[i], u, th, E, feq, heq);
    for (int a = 0; a < Q3; ++a) {
      s->f[a][i] = feq[a];
      s->h[a][i] = heq[a];
    }
  }
}

/* Eq. 35 and Eq. 37 (or the internal-energy temperature under Eq. 38). */
static void node_moments(const o3_state* s, long i, double* rho, double u[3], double* th,
                         double* es) {
  const o3_params* p = &s->p;
  double r = 0, j[3] = {0, 0, 0}, sh = 0;
  for (int a = 0; a < Q3; ++a) {
    r += s->f[a][i];
    for (int d = 0; d < 3; ++d) j[d] += E3[a][d] * s->f[a][i];
    sh += s->h[a][i];
  }
  /* Eq. 35 with the half-force shift (under Eq. 51): rho u = sum e f + a / 2 */
  j[2] -= 0.5 * r * p->g;
  for (int d = 0; d < 3; ++d) u[d] = j[d] / r;
  double T;
  if (p->energy_model == O3_E_TOTAL)
    T = 2.0 / (p->b * p->R) * (sh / r - 0.5 * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]));
  else
    T = 2.0 * sh / (r * p->b * p->R);
  *rho = r;
  *th = T / p->T0;
  *es = sh / r;
}

static void phase1(o3_state* s, int nthreads) {
  const o3_params* p = &s->p;
  const double RT0 = p->R * p->T0;
  (void)nthreads;
#pragma omp parallel for num_threads(nthreads) schedule(static)
  for (long i = 0; i < s->n; ++i) {
    double u[3];
    node_moments(s, i, &s->rho[i], u, &s->theta[i], &s->es[i]);
    s->ux[i] = u[0];
    s->uy[i] = u[1];
    s->uz[i] = u[2];
    o3_defect(RT0, s->rho[i], u, s->theta[i], &s->D[27 * i]);
  }
}

/* D of the ghost node across wall side `side` (2 axis + high end) of node i. */
static void wall_ghost_D(const o3_state* s, long i, int side, double Dg[27]) {
  const o3_params* p = &s->p;
  const double RT0 = p->R * p->T0;
  double thw = side_bc(p, side) == O3_WALL_ISOTHERMAL ? side_Tw(p, side) / p->T0 : s->theta[i];
  double Dw[27];
  o3_defect(RT0, s->rho[i], side_uw(p, side), thw, Dw);
  for (int m = 0; m < 27; ++m) Dg[m] = 2.0 * Dw[m] - s->D[27 * i + m];
}

/* G_ij = sum_k dD_ijk/dx_k by the central differences of Eq. 50 (the ghost D
 * across a wall). */
static void node_G(const o3_state* s, int x, int y, int z, double G[9]) {
  const o3_params* p = &s->p;
  const long i = idx3(p, x, y, z);
  const int c[3] = {x, y, z}, n[3] = {p->nx, p->ny, p->nz};
  for (int ij = 0; ij < 9; ++ij) G[ij] = 0.0;
  for (int k = 0; k < 3; ++k) {
    int dx = k == 0, dy = k == 1, dz = k == 2;
    double gp[27], gm[27];
    const double* Dp = &s->D[27 * idx3(p, x + dx, y + dy, z + dz)];
    const double* Dm = &s->D[27 * idx3(p, x - dx, y - dy, z - dz)];
    if (c[k] == n[k] - 1 && side_bc(p, 2 * k + 1) != O3_PERIODIC) {
      wall_ghost_D(s, i, 2 * k + 1, gp);
      Dp = gp;
    }
    if (c[k] == 0 && side_bc(p, 2 * k) != O3_PERIODIC) {
      wall_ghost_D(s, i, 2 * k, gm);
      Dm = gm;
    }
    for (int ij = 0; ij < 9; ++ij) G[ij] += 0.5 * (Dp[3 * ij + k] - Dm[3 * ij + k]);
  }
}

/* Index of the opposite velocity. */
static int opp3(int a) {
  for (int b = 0; b < Q3; ++b)
    if (E3[b][0] == -E3[a][0] && E3[b][1] == -E3[a][1] && E3[b][2] == -E3[a][2]) return b;
  return a;
}

/* Population a leaving node i through wall side `side` comes back into
 * node i as the opposite population b (the rules in the header).  fs, hs:
 * the node's post-collision populations; heq: its h^eq. */
static void wall_bounce(const o3_params* p, int side, int a, double rho, const double u[3],
                        double th, const double fs[Q3], const double hs[Q3],
                        const double heq[Q3], double* fn[Q3], double* hn[Q3], long i) {
  const double RT0 = p->R * p->T0;
  const int b = opp3(a);
  const double* uw = side_uw(p, side);
  /* equilibria at the node's rho and theta and the wall velocity */
  double fw[Q3], hw[Q3];
  double Ew = 0.5 * (p->b * RT0 * th + uw[0] * uw[0] + uw[1] * uw[1] + uw[2] * uw[2]);
  o3_feq(RT0, rho, uw, th, fw);
  if (p->energy_model == O3_E_TOTAL)
    o3_heq(RT0, rho, uw, th, Ew, fw, hw);
  else
    o3_heq_internal(RT0, p->b, th, fw, hw);
  fn[b][i] = fs[a] + (fw[b] - fw[a]); /* f*_a - 2 (odd part of f^eq_a) */
  if (side_bc(p, side) == O3_WALL_ISOTHERMAL) {
    const double thw = side_Tw(p, side) / p->T0;
    double thg = 2.0 * thw - th;
    if (thg < 0.5 * thw) thg = 0.5 * thw;
    /* the node's pressure carried to the ghost by hydrostatic balance
     * (gravity along -z: only the z sides) */
    const double nz_out = side == 4 ? -1.0 : (side == 5 ? 1.0 : 0.0);
    const double rg = rho * (th - 3.0 * p->g * nz_out) / thg;
    double ug[3], fg[Q3], hg[Q3];
    for (int d = 0; d < 3; ++d) ug[d] = 2.0 * uw[d] - u[d];
    double Eg = 0.5 * (p->b * RT0 * thg + ug[0] * ug[0] + ug[1] * ug[1] + ug[2] * ug[2]);
    o3_feq(RT0, rg, ug, thg, fg);
    if (p->energy_model == O3_E_TOTAL)
      o3_heq(RT0, rg, ug, thg, Eg, fg, hg);
    else
      o3_heq_internal(RT0, p->b, thg, fg, hg);
    hn[b][i] = hg[b] + (hs[b] - heq[b]); /* the ghost's equilibrium + the node's h*_b - h^eq_b */
  } else {
    hn[b][i] = hs[a] + (hw[b] - hw[a]); /* h*_a - 2 (odd part of h^eq_a) */
    if (p->energy_model == O3_E_TOTAL) {
      /* total energy: plus the wall's work on the pair, u_w . (f_b e_b -
       * f*_a e_a), so that no heat crosses a moving wall */
      double work = 0.0;
      for (int d = 0; d < 3; ++d) work += uw[d] * (fn[b][i] * E3[b][d] - fs[a] * E3[a][d]);
      hn[b][i] += work;
    }
  }
}

static void phase2(o3_state* s, int nthreads) {
  const o3_params* p = &s->p;
  const double RT0 = p->R * p->T0;
  const double wf = 2.0 / (2.0 * p->tau_f + 1.0);
  const double wh = 2.0 / (2.0 * p->tau_h + 1.0);
  (void)nthreads;
#pragma omp parallel for num_threads(nthreads) schedule(static)
  for (int z = 0; z < p->nz; ++z)
    for (int y = 0; y < p->ny; ++y)
      for (int x = 0; x < p->nx; ++x) {
        long i = idx3(p, x, y, z);
        double rho = s->rho[i], th = s->theta[i];
        double u[3] = {s->ux[i], s->uy[i], s->uz[i]};
        double usq = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
        double C[Q3] = {0};
        if (p->correction) {
          double G[9];
          node_G(s, x, y, z, G);
          o3_correction(G, C);
        }
        if (p->g != 0.0) {
          /* Guo's force term, entering with C (Eq. 51 carried to D = 3):
           * F_a = w_a [(e_a - u).a / RT0 + (e_a.u)(e_a.a) / RT0^2] */
          const double az = -rho * p->g;
          for (int a = 0; a < Q3; ++a) {
            const double eu = E3[a][0] * u[0] + E3[a][1] * u[1] + E3[a][2] * u[2];
            const double ea = E3[a][2] * az;
            C[a] += weight3(a) * ((ea - u[2] * az) / RT0 + eu * ea / (RT0 * RT0));
          }
        }
        double feq[Q3], heq[Q3], fs[Q3], hs[Q3];
        equilibria(p, rho, u, th, s->es[i], feq, heq);
        for (int a = 0; a < Q3; ++a) {
          double fb = s->f[a][i], hb = s->h[a][i];
          double fneq = fb - feq[a];
          /* Eq. 34 (+ (1 - w_f/2) C) */
          fs[a] = fb - wf * fneq + (1.0 - 0.5 * wf) * C[a];
          /* Eq. 36 or Eq. 38 */
          hs[a] = hb - wh * (hb - heq[a]);
          if (p->energy_model == O3_E_TOTAL) {
            double eu = E3[a][0] * u[0] + E3[a][1] * u[1] + E3[a][2] * u[2];
            double Z = p->z_full ? eu - 0.5 * usq : eu;
            hs[a] += (wh - wf) * Z * (fneq + 0.5 * C[a]);
          }
        }
        for (int a = 0; a < Q3; ++a) {
          /* a halfway wall crossed (x before y before z when a leaves
           * through an edge): back into this node as the opposite */
          const int t[3] = {x + E3[a][0], y + E3[a][1], z + E3[a][2]};
          const int n[3] = {p->nx, p->ny, p->nz};
          int side = -1;
          for (int k = 0; k < 3 && side < 0; ++k) {
            const int sk = t[k] < 0 ? 2 * k : (t[k] >= n[k] ? 2 * k + 1 : -1);
            if (sk >= 0 && side_bc(p, sk) != O3_PERIODIC) side = sk;
          }
          if (side >= 0) {
            wall_bounce(p, side, a, rho, u, th, fs, hs, heq, s->fn, s->hn, i);
            continue;
          }
          /* streaming to x + e_a (periodic) */
          long j = idx3(p, t[0], t[1], t[2]);
          s->fn[a][j] = fs[a];
          s->hn[a][j] = hs[a];
        }
      }
}

void o3_step(o3_state* s, long nsteps, int nthreads) {
  if (nthreads < 1) nthreads = 1;
  for (long t = 0; t < nsteps; ++t) {
    phase1(s, nthreads);
    phase2(s, nthreads);
    for (int a = 0; a < Q3; ++a) {
      double* tf = s->f[a];
      s->f[a] = s->fn[a];
      s->fn[a] = tf;
      double* th = s->h[a];
      s->h[a] = s->hn[a];
      s->hn[a] = th;
    }
  }
}

void o3_moments(const o3_state* s, double* rho, double* ux, double* uy, double* uz,
                double* T) {
  for (long i = 0; i < s->n; ++i) {
    double u[3], th, es;
    node_moments(s, i, &rho[i], u, &th, &es);
    ux[i] = u[0];
    uy[i] = u[1];
    uz[i] = u[2];
    T[i] = th * s->p.T0;
  }
}

/* G_ij = sum_k dD_ijk/dx_k of the current state at every node, the
 * argument of the correction term, into G[n][9] (row-major i, j). */
void o3_gradients(o3_state* s, double* G) {
  const o3_params* p = &s->p;
  phase1(s, 1);
  for (int z = 0; z < p->nz; ++z)
    for (int y = 0; y < p->ny; ++y)
      for (int x = 0; x < p->nx; ++x) node_G(s, x, y, z, &G[9 * idx3(p, x, y, z)]);
}

/* Sums of rho, rho u (3) and hbar over the grid. */
void o3_conserved(const o3_state* s, double out[5]) {
  for (int k = 0; k < 5; ++k) out[k] = 0.0;
  for (long i = 0; i < s->n; ++i) {
    for (int a = 0; a < Q3; ++a) {
      out[0] += s->f[a][i];
      for (int d = 0; d < 3; ++d) out[1 + d] += E3[a][d] * s->f[a][i];
      out[4] += s->h[a][i];
    }
  }
}

/* Populations [38][nz][ny][nx]: f_0..f_18, then h_0..h_18. */
void o3_get_pops(const o3_state* s, double* out) {
  for (int a = 0; a < Q3; ++a) {
    memcpy(out + (long)a * s->n, s->f[a], s->n * sizeof(double));
    memcpy(out + (long)(Q3 + a) * s->n, s->h[a], s->n * sizeof(double));
  }
}

void o3_set_pops(o3_state* s, const double* in) {
  for (int a = 0; a < Q3; ++a) {
    memcpy(s->f[a], in + (long)a * s->n, s->n * sizeof(double));
    memcpy(s->h[a], in + (long)(Q3 + a) * s->n, s->n * sizeof(double));
  }
}

/* The lattice as the oracle uses it: e[3a+d] and w[a]. */
void o3_lattice(int* e, double* w) {
  for (int a = 0; a < Q3; ++a) {
    for (int d = 0; d < 3; ++d) e[3 * a + d] = E3[a][d];
    w[a] = weight3(a);
  }
}

int o3_param_size(void) { return (int)sizeof(o3_params); }
