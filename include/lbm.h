/*
 * lbm.h -- C ABI of the GB300 library for the coupled double-distribution-
 * function (DDF) thermal lattice Boltzmann method on D2Q9 of Li, Luo, He, Gao
 * and Tao, "Coupling lattice Boltzmann model for simulation of thermal flows
 * on standard lattices" (arXiv:1109.6672), BGK scheme of Sec. III.C.1.
 *
 * One time step advances, for every node x, the density distribution f
 * (Eq. 34, equilibrium Eq. 18a with p = rho R T) and the total-energy
 * distribution h (Eq. 36, equilibrium Eq. 18b; or the internal-energy form of
 * Eq. 38), with the third-moment correction C_a (Eqs. 48-50) and the Guo
 * gravity force (text around Eq. 51), followed by streaming and the wall rules.
 *
 * Conventions shared by every entry point:
 *  - Every function returns an int status: LBM_OK (0) or a negative LBM_ERR_*
 *    code; no C++ exception crosses this boundary.  lbm_last_error() gives a
 *    one-line message for the last failure on a handle.
 *  - Host arrays are caller-owned, row-major [ny][nx] doubles (node (x, y) at
 *    index y * nx + x), unless stated otherwise.  The library never keeps a
 *    pointer to a caller array after the call returns.
 *  - Device memory for the state is owned by the handle unless it was created
 *    with lbm_create_in(), in which case the caller owns the buffer and must
 *    keep it alive until lbm_destroy().
 *  - Work is enqueued on the CUDA stream given at creation (NULL: the legacy
 *    default stream).  Calls that return host data synchronise that stream.
 *    lbm_step() is asynchronous: a kernel failure is reported by the next
 *    call that synchronises.
 *  - Lattice units: dx = dt = 1, c = sqrt(3 R T0) = 1 (Eq. 6 and Eq. 28), so
 *    R * T0 must equal 1/3.  Sides are ordered x-, x+, y-, y+.
 *  - Walls sit halfway between the boundary node and the first node outside
 *    (at x = -1/2, x = nx - 1/2, y = -1/2, y = ny - 1/2).  The paper uses
 *    non-equilibrium extrapolation walls; this library uses:
 *      f: halfway bounce-back plus twice the odd part of Eq. 18a evaluated at
 *         the boundary node's rho and theta and the wall velocity;
 *      h, isothermal wall: non-equilibrium extrapolation from a ghost node one
 *         spacing outside, with u_g = 2 u_w - u, theta_g = max(2 theta_w - theta,
 *         theta_w / 2) and the node's pressure carried to the ghost by
 *         hydrostatic balance, rho_g theta_g = rho (theta - 3 g n_y), n_y the
 *         wall's outward normal (0 on x walls);
 *      h, adiabatic wall: bounce-back plus twice the odd part of h^eq at the
 *         boundary node's (rho, theta) and the wall velocity, for total energy
 *         plus the wall's work on the bounced pair u_w . (f_b e_b - f*_a e_a)
 *         (a moving adiabatic wall passes its work, not heat);
 *      corners: a population leaving across two walls uses the x-side wall;
 *      Eq. 50 across a wall: mirror ghost Q_g = 2 rho u_w (1 - theta_w) - Q.
 *  - Open x sides, for the attenuation-driven acoustic streaming of Sec. IV.B
 *    (y must then be periodic, and correction = 0, as the paper runs it):
 *      LBM_BC_INLET (x- only): the node one spacing outside the first column
 *         is reset every step to the equilibria (Eq. 18a, Eq. 18b or the
 *         Eq. 38 form) of the state of Eq. 53 at the current step t:
 *         rho = in_rho + in_drho s, u = u_wall[0] + (in_du s, 0),
 *         T = T_wall[0] + in_dT s, s = sin(in_omega t); it feeds the first
 *         column, and what leaves the first column through x- is dropped;
 *      LBM_BC_OUTLET (x+ only): zero-gradient extrapolation of (rho, u, T)
 *         into the ghost column, then non-equilibrium extrapolation; the
 *         ghost's equilibria equal the last column's, so the ghost emits the
 *         last column's own post-collision populations back.
 *    Each step that touches them ends with a second, small kernel that
 *    writes these ghost slots.
 *  - Walls of non-equilibrium extrapolation (wall_nee): the wall node G sits
 *    one spacing outside the boundary node F.  Its state is the wall
 *    velocity, theta_G (the wall's; adiabatic: zero slope at G to second
 *    order, (4 theta_F - theta_F2)/3, F2 the next node inward, floored at
 *    theta_F / 2) and F's
 *    pressure carried to G by hydrostatic balance (rho_G theta_G =
 *    rho_F (theta_F - 3 g n_y), since p = rho R T); its
 *    pre-collision populations are its equilibria plus F's non-equilibrium
 *    part (for h on an adiabatic wall, without that part's normal heat
 *    flux: the normal moment of h^neq - Z f^neq, Z = e.u_w - |u_w|^2/2 the
 *    Eq. 36 coupling at the wall velocity, so that a moving wall's viscous
 *    work passes); it collides like a fluid node (force of its own density, no
 *    correction term) and sends its populations into the domain.  A corner
 *    ghost at the end of an x side's column feeds the corner node (the x side
 *    wins); Eq. 50 across such a wall keeps the mirror ghost above.  Written
 *    by the same second kernel.
 */
#ifndef LBM_H_
#define LBM_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  LBM_OK = 0,
  LBM_ERR_PARAM = -1,     /* invalid argument; the handle is unchanged        */
  LBM_ERR_OOM = -2,       /* device or host allocation failed / does not fit  */
  LBM_ERR_CUDA = -3,      /* a CUDA call or kernel failed                     */
  LBM_ERR_NONFINITE = -4, /* a moment or population is NaN/Inf (state kept)   */
  LBM_ERR_TIMEOUT = -5,   /* a bounded device-side wait ran out               */
  LBM_ERR_STATE = -6      /* call out of order (e.g. lbm_step before lbm_init) */
};

enum {
  LBM_BC_PERIODIC = 0,
  LBM_BC_WALL_ISOTHERMAL = 1,
  LBM_BC_WALL_ADIABATIC = 2,
  LBM_BC_INLET = 3, /* x- only, see above */
  LBM_BC_OUTLET = 4 /* x+ only, see above */
};
/* LBM_E_TOTAL: total-energy h, Eq. 18b and Eq. 36 (viscous heating and
 * compression work, Z = e.u - u^2/2 or e.u).  LBM_E_INTERNAL: internal-energy
 * h of Eq. 38 with h^eq = b R T f^eq / 2 and T = 2 sum h / (rho b R). */
enum { LBM_E_TOTAL = 0, LBM_E_INTERNAL = 1 };
/* Storage / arithmetic: FP64 everywhere; FP32 everywhere; FP32 arithmetic with
 * populations stored as FP16 or BF16 deviations from the rest equilibrium
 * (rho = 1, u = 0, T = T0; the step computed on deviations), T recovered from
 * deviation sums and FP64 reference sums (its last subtraction, of two FP32
 * numbers, rounds as in FP64), reductions accumulated in FP64.
 * The 16-bit stores of a time step round stochastically (zero-mean error;
 * the random bits are a function of step, node and population only, see
 * lbm_set_steps_done); FP16 holds 256 x the deviation. */
enum { LBM_P_FP64 = 0, LBM_P_FP32 = 1, LBM_P_FP32_FP16 = 2, LBM_P_FP32_BF16 = 3 };
/* Collision of f: LBM_COLL_BGK, Eq. 34; LBM_COLL_MRT, Eqs. 43-45: relaxation in
 * the moment space of Appendix B with S of Eq. 40 and m^eq of Eq. 41 (h keeps
 * its BGK relaxation with the Eq. 47 coupling, which has the same coefficient
 * as Eq. 36). */
enum { LBM_COLL_BGK = 0, LBM_COLL_MRT = 1 };
enum { LBM_MU_TAU = 0, LBM_MU_POWER = 1, LBM_MU_SUTHERLAND = 2 };

typedef struct {
  int32_t nx, ny;           /* fluid nodes per axis, >= 1 (>= 3 on a walled axis)  */
  int32_t bc[4];            /* LBM_BC_* per side x-, x+, y-, y+; a periodic side
                               needs its opposite side periodic too             */
  double tau_f, tau_h;      /* continuous relaxation times (Eq. 30: mu = tau_f p,
                               lambda = tau_h (b+2)/2 p R); omega = 2/(2 tau + 1),
                               text below Eqs. 34 and 36; both > 0             */
  double Pr;                /* <= 0: ignored; > 0: must equal tau_f / tau_h     */
  double R, T0;             /* gas constant and reference temperature, R T0 = 1/3 */
  double b;                 /* degrees of freedom, gamma = (b + 2)/b (Eq. 37), b >= 2 */
  double u_wall[4][2];      /* wall velocity per side (tangential in practice)  */
  double T_wall[4];         /* wall temperature per isothermal side, > 0        */
  double g;                 /* gravity; force density a = (0, -rho g), text under
                               Eq. 51; needs energy_model = LBM_E_INTERNAL      */
  int32_t energy_model;     /* LBM_E_TOTAL or LBM_E_INTERNAL                    */
  int32_t correction;       /* 1: C_a of Eqs. 48-50; 0: omitted                 */
  int32_t z_full;           /* 1: Z = e.u - u^2/2 (Eq. 7b); 0: Z = e.u           */
  int32_t precision;        /* LBM_P_*                                          */
  int32_t collision;        /* LBM_COLL_BGK (0) or LBM_COLL_MRT                 */
  double s_e, s_eps, s_q;   /* MRT rates of the moments e, epsilon, q_x / q_y
                               (Eq. 40: 1/tau_e, 1/tau_eps, 1/tau_q), each in
                               (0, 2); 0 selects omega_f (the paper's cavity:
                               s_e = s_eps = omega_f, s_q = 1.5).  The shear
                               rate is omega_f (the discrete MRT time is tau_f
                               + 1/2: mu = tau_f p as for BGK); conserved
                               moments relax at rate 1.  Ignored for BGK.     */
  int32_t mu_law;           /* viscosity: LBM_MU_TAU (0): constant tau_f, tau_h
                               (mu = tau_f p, Eq. 30); LBM_MU_POWER: mu = mu0
                               theta^mu_n (the premise of Eq. 52); LBM_MU_SUTHERLAND:
                               Eq. 59 referred to T0, mu = mu0 theta^(3/2)
                               (1 + mu_S)/(theta + mu_S).  mu0 = tau_f R T0 (tau_f
                               is the value at rho = 1, T = T0); per node
                               tau_f = mu / (rho R T) and tau_h = tau_f / Pr with
                               Pr = tau_f / tau_h fixed (text before Eq. 52).   */
  double mu_n;              /* power-law exponent (finite)                      */
  double mu_S;              /* Sutherland constant S / T0 (> 0 for that law)    */
  double in_rho;            /* LBM_BC_INLET: mean density (> in_drho)           */
  double in_drho, in_du;    /* density and x-velocity amplitudes (Eq. 53, Eq. 54) */
  double in_dT;             /* temperature amplitude (< T_wall[0] in magnitude) */
  double in_omega;          /* angular frequency per step; the phase is taken
                               from the step count modulo 2^32              */
  int32_t wall_nee;         /* bit s (side s): that wall (isothermal or
                               adiabatic) is one of non-equilibrium
                               extrapolation, the paper's wall method (ref.
                               [45]), sitting ON the ghost node one spacing
                               outside the boundary node (so H = n + 1
                               between two of them) instead of halfway; see
                               the conventions above.  0: halfway walls.    */
} lbm_params;

typedef struct lbm_handle lbm_handle;

/* Bytes of device memory the state of one grid occupies (two population
 * buffers in the layout described in lbm_create_in()).  Returns a negative
 * LBM_ERR_* code for invalid parameters. */
int64_t lbm_state_bytes(const lbm_params* p);

/* Validates *p, allocates the device state and creates a handle bound to the
 * current CUDA device and to cuda_stream (a cudaStream_t; NULL = default).
 * Also allocates the staging of host transfers (4 nx ny doubles), so that
 * lbm_init() and lbm_moments() allocate nothing (lbm_get_state() and
 * lbm_set_state() grow it to 18 nx ny doubles on first use).
 * On error *out is NULL.  Errors: LBM_ERR_PARAM (see lbm_params), LBM_ERR_OOM,
 * LBM_ERR_CUDA. */
int lbm_create(const lbm_params* p, void* cuda_stream, lbm_handle** out);

/* Same as lbm_create() but places the state in caller-owned device memory
 * (the staging of host transfers is still the library's own)
 * (for example a buffer from a caching allocator): device_buffer must be
 * 256-byte aligned and at least lbm_state_bytes(p) long.  Layout (opaque to
 * callers): two buffers, each 18 planes per row, row-interleaved
 * [y + 1][population][x + 1] with a one-node ghost ring. */
int lbm_create_in(const lbm_params* p, void* cuda_stream, void* device_buffer, int64_t bytes,
                  lbm_handle** out);

/* Sets the state to equilibrium (Eq. 18a, Eq. 18b or the Eq. 38 form) at the
 * given host fields (nx*ny doubles each; T in the units of T0; the paper
 * leaves the initial state free).  Resets the step counter.  Synchronous.
 * The fields travel in row chunks on a transfer stream of the handle while
 * earlier chunks are initialised on its own stream (pinned host memory lets
 * the two overlap). */
int lbm_init(lbm_handle* h, const double* rho, const double* ux, const double* uy,
             const double* T);

/* Same as lbm_init() with device pointers (nx*ny doubles each, on the handle's
 * device); asynchronous on the handle's stream. */
int lbm_init_device(lbm_handle* h, const double* d_rho, const double* d_ux, const double* d_uy,
                    const double* d_T);

/* Advances n >= 0 time steps (one fused stream-and-collide kernel per step).
 * Asynchronous; returns LBM_ERR_CUDA if a launch fails, LBM_ERR_STATE before
 * lbm_init(). */
int lbm_step(lbm_handle* h, int64_t n);

/* Macroscopic fields of the current state: rho, u = (sum e fbar + a/2)/rho
 * (Eq. 35 and text under Eq. 51) and T (Eq. 37, or 2 sum hbar/(rho b R)),
 * computed in FP64 from the stored populations.  Host outputs, nx*ny each;
 * synchronous.  LBM_ERR_NONFINITE if any value is NaN/Inf (arrays still
 * filled; the export kernel raises a device flag, the host scans nothing).
 * LBM_ERR_STATE before lbm_init() or after a lost state (lbm_sync()). */
int lbm_moments(lbm_handle* h, double* rho, double* ux, double* uy, double* T);

/* Same as lbm_moments() into device arrays, asynchronous, no finite check. */
int lbm_moments_device(lbm_handle* h, double* d_rho, double* d_ux, double* d_uy, double* d_T);

/* FP64 sums over all nodes of rho, rho u_x, rho u_y and hbar (sum rho E for
 * LBM_E_TOTAL, internal energy for LBM_E_INTERNAL), reduced in a fixed order
 * (bitwise reproducible).  out: host, 4 doubles; synchronous. */
int lbm_conserved(lbm_handle* h, double out[4]);

/* Canonical pre-collision populations fbar_a(x, t), hbar_a(x, t) as
 * host [18][ny][nx] doubles (f_0..f_8 then h_0..h_8, velocities
 * e = (0,0),(1,0),(0,1),(-1,0),(0,-1),(1,1),(-1,1),(-1,-1),(1,-1)).
 * Synchronous.  lbm_set_state() writes them back (rounded to the storage
 * precision); together they checkpoint and resume a run. */
int lbm_get_state(lbm_handle* h, double* pops);
int lbm_set_state(lbm_handle* h, const double* pops);

/* Allocation-free form of lbm_conserved() for callers that cannot allocate
 * device memory when they need the sums: code inside CUDA stream capture,
 * serving loops whose device memory belongs to a pool that forbids outside
 * allocations, and latency-bound paths that cannot afford cudaMalloc's
 * implicit synchronisation.  (The paper has no counterpart; this is a
 * property of the library, not of the method.)
 *   p        parameters of the grid (validated as in lbm_create()).
 *   d_state  device pointer to one state buffer in the library's layout: for a
 *            handle made by lbm_create_in() on buffer B, the state after k
 *            steps since lbm_init()/lbm_set_state() starts at
 *            B + (k % 2) * lbm_state_bytes(p) / 2 (256-byte aligned).
 *   d_out    device pointer to 4 doubles (8-byte aligned): sums of rho,
 *            rho u_x, rho u_y and hbar, the same values lbm_conserved()
 *            returns.
 *   cuda_stream  stream to enqueue on (NULL = default stream); asynchronous.
 * Calls no cudaMalloc, cudaFree or allocating routine: the per-block partial
 * sums live in a file-scope device array of 1024 quadruples of doubles
 * (32 KiB) that every device loading the library keeps until process exit;
 * grids needing more partial slots are rejected with LBM_ERR_PARAM (with the
 * library's node limit of 2^31 none does).  The first call on a device looks
 * the array up on that device (make it, with that device current, before any
 * stream capture); every later call outside stream capture looks it up again
 * (a host-side lookup that allocates nothing), so that a context recreated
 * after cudaDeviceReset() is followed, and calls inside a capture use the
 * address of the last call outside one (after a device reset, make one call
 * outside capture first again).  All calls share the array: calls that overlap on the GPU
 * (different streams, or devices sharing nothing but the host thread's
 * current device) race and must be ordered by the caller.  Returns
 * LBM_ERR_PARAM for invalid arguments, LBM_ERR_CUDA if the lookup or a launch
 * fails. */
int lbm_conserved_noalloc(const lbm_params* p, const void* d_state, double* d_out,
                          void* cuda_stream);

/* ---- Batched grids ---------------------------------------------------------
 * Many independent grids (any sizes, physics modes and boundary conditions, one
 * storage precision) advance together: one kernel launch per time step covers
 * every grid, k steps are replayed from a CUDA graph captured once per k, and
 * the per-grid work is split into items (128 columns x rows of one grid) that a
 * persistent grid of blocks takes in turn.  Results do not depend on which other
 * grids are in the batch, nor on the schedule.  Grids are placed in one device
 * pool (first fit, 256-byte aligned); lbm_batch_add() admits a grid only if a
 * slot and lbm_state_bytes(p) of contiguous pool space are free. */
typedef struct lbm_batch lbm_batch;

/* Creates a batch for `precision` (LBM_P_*) with up to max_grids slots and a
 * device pool of pool_bytes (allocated here; lbm_batch_create_in() takes a
 * caller-owned, 256-byte aligned pool instead).  cuda_stream NULL: the batch
 * creates its own non-blocking stream (graph capture needs one). */
int lbm_batch_create(int32_t precision, int32_t max_grids, int64_t pool_bytes, void* cuda_stream,
                     lbm_batch** out);
int lbm_batch_create_in(int32_t precision, int32_t max_grids, void* device_pool,
                        int64_t pool_bytes, void* cuda_stream, lbm_batch** out);

/* Admits a grid (params as for lbm_create(), precision equal to the batch's),
 * initialises it to equilibrium at the host fields (as lbm_init()) and gives it
 * a budget of `steps` time steps.  *slot receives its slot.  LBM_ERR_OOM if no
 * slot or no pool space is free (the batch is unchanged).  Synchronous. */
int lbm_batch_add(lbm_batch* b, const lbm_params* p, const double* rho, const double* ux,
                  const double* uy, const double* T, int64_t steps, int32_t* slot);

/* Advances every admitted grid by min(k, its remaining budget) steps, k in
 * [0, 4096], with one graph launch; synchronous. */
int lbm_batch_run(lbm_batch* b, int64_t k);

/* Remaining step budget of a slot (negative LBM_ERR_* for a free slot). */
int64_t lbm_batch_remaining(const lbm_batch* b, int32_t slot);

/* Moments (as lbm_moments()) and canonical populations (as lbm_get_state())
 * of a slot's current state into host arrays; synchronous. */
int lbm_batch_moments(lbm_batch* b, int32_t slot, double* rho, double* ux, double* uy,
                      double* T);
int lbm_batch_get_state(lbm_batch* b, int32_t slot, double* pops);

/* Releases a slot and its pool space. */
int lbm_batch_remove(lbm_batch* b, int32_t slot);

/* Autotuner: times `reps` launches of one step of the admitted grids (without
 * advancing them) for each candidate schedule -- rows per work item in
 * {4, 6, 8, 12, 16, 24} x atomic or round-robin item assignment -- and keeps
 * the fastest.  out_best (may be NULL): rows, dynamic (1 atomic, 0 round
 * robin), microseconds per step. */
int lbm_batch_autotune(lbm_batch* b, int32_t reps, int64_t out_best[3]);

/* Sets the schedule by hand (rows 0 = default). */
int lbm_batch_set_schedule(lbm_batch* b, int32_t rows, int32_t dynamic);

/* out: admitted grids, their total nodes, free pool bytes, largest free range,
 * rows per item, dynamic flag. */
int lbm_batch_info(const lbm_batch* b, int64_t out[6]);

void lbm_batch_destroy(lbm_batch* b); /* NULL-safe */
const char* lbm_batch_last_error(const lbm_batch* b);

/* Waits for all work enqueued on the handle's stream; reports a pending
 * kernel error as LBM_ERR_CUDA.  LBM_ERR_TIMEOUT if a step kernel gave up a
 * bounded wait for a staged row (2 s; the handle stays usable).  If such a
 * kernel also ran out of time draining its own copies, a copy may have landed
 * in shared memory after it left: the state is then treated as lost, and
 * lbm_step(), lbm_moments(), lbm_conserved() and lbm_get_state() return
 * LBM_ERR_STATE until lbm_init(), lbm_init_device() or lbm_set_state()
 * reloads it.  (A batch in that case refuses further runs and reads until it
 * is destroyed.) */
int lbm_sync(lbm_handle* h);

/* Time steps taken since the last lbm_init() / lbm_set_state(). */
int64_t lbm_steps_done(const lbm_handle* h);

/* Self-test of the bounded device-side waits (no counterpart in the paper).
 * Launches one block on the current device that arms a shared-memory barrier
 * for a transfer no copy ever completes and waits on it with the same bounded
 * wait the step kernels use (limit_ns nanoseconds, 1e3 .. 2e9); the block then
 * records the timeout in a status word and returns, as a step kernel does.
 * Synchronous.  Returns LBM_ERR_TIMEOUT when the wait ran out (the expected
 * result), LBM_OK if it did not, LBM_ERR_PARAM for a limit out of range (no
 * device call is made then), LBM_ERR_OOM / LBM_ERR_CUDA on CUDA failures. */
int lbm_selftest_wait(int64_t limit_ns);

/* Sets the step counter (no counterpart in the paper).  The 16-bit storage
 * precisions round every stored deviation stochastically with random bits
 * drawn from (step counter, node, population), so a run resumed from a
 * state saved with lbm_get_state() after t steps reproduces the
 * uninterrupted run bit for bit only if the counter is set back to t after
 * lbm_set_state().  Other precisions do not read it.  t < 0:
 * LBM_ERR_PARAM. */
int lbm_set_steps_done(lbm_handle* h, int64_t t);

/* Step kernel and launch shape.  variant 0 or 1 (default): pulled-row
 * staging by the tensor memory accelerator (TMA), 128 columns per block;
 * 2: the same with 256 columns per block (two per thread); 64..256, a
 * multiple of 32: the register-pull kernel, each block owning variant - 2
 * columns.  rows_per_block >= 1, or 0 for the default (6 rows for FP32
 * storage, 12 otherwise, for the TMA kernel; about one wave of blocks for the
 * register-pull kernel).  rows_per_block (and the block width of the
 * register-pull kernel) never changes a bit of the result; different variants
 * agree to rounding (different FMA contraction).  Variant 2 is built for the
 * BGK collision with constant relaxation times only (LBM_ERR_PARAM with
 * LBM_COLL_MRT or a viscosity law). */
int lbm_set_launch(lbm_handle* h, int32_t variant, int32_t rows_per_block);

/* Frees the handle and the device memory it owns.  NULL-safe. */
void lbm_destroy(lbm_handle* h);

/* Message of the last failure on h (or of the last failed lbm_create on this
 * thread when h is NULL).  Never NULL; valid until the next call on h. */
const char* lbm_last_error(const lbm_handle* h);

/* Static name of a status code. */
const char* lbm_status_string(int status);

#ifdef __cplusplus
}
#endif

#endif /* LBM_H_ */
