/*
 * lbm3d.h -- C ABI of the three-dimensional (D3Q19) extension of the coupled
 * double-distribution-function thermal lattice Boltzmann method of Li, Luo,
 * He, Gao and Tao (arXiv:1109.6672).  The paper builds the model on D2Q9 and
 * states that its formulation extends to three dimensions (Sec. V); this is
 * that extension, BGK scheme (Sec. III.C.1), each side of the box periodic
 * or a halfway wall:
 *
 *   - f^eq: Eq. 18a with D = 3; h^eq: Eq. 18b with D = 3 (total energy,
 *     Eq. 36 with the (omega_h - omega_f) Z_a coupling), or the internal-
 *     energy form h^eq = b R T f^eq / 2 of Eq. 38;
 *   - correction term C_a (Eq. 22): zero mass and momentum (Eq. 26) and the
 *     second moments that remove the deviation of the third-order moment of
 *     f^eq (the argument of Eqs. 27-28), which on D3Q19 has, besides Eq. 20's
 *     diagonal D_iii = 3 rho R T0 u_i (1 - theta), the entries
 *     D_iik = rho R T0 u_k (1 - theta) / 2 (i != k):
 *        sum_a e_ai e_aj C_a = sum_k dD_ijk / dx_k,
 *     by the central differences of Eq. 50 along each axis; C_a is the even
 *     quadratic polynomial of e_a with no constant moment (the counterpart of
 *     Eq. 49);
 *   - time step: Eq. 34 (with +(1 - omega_f/2) C_a) and Eq. 36 / Eq. 38;
 *     moments Eq. 35 and Eq. 37;
 *   - gravity along -z (g, internal-energy model): Guo's force term of
 *     Eq. 51 with D = 3 beside C_a and the half-force shift of u;
 *   - walls (not in the paper, which uses non-equilibrium extrapolation;
 *     the rules of lbm.h carried to D3Q19), halfway at x = -1/2 and
 *     nx - 1/2, likewise in y and z; a population leaving through an edge
 *     where two walled sides meet takes the rule of the first of x, y, z
 *     (as the D2Q9 corners take the x side's); a population a leaving
 *     through the wall comes back as its
 *     opposite b with f_b = f*_a - 2 (odd part of Eq. 18a at the node's rho
 *     and theta and the wall velocity); h on an isothermal wall
 *     h_b = h^eq_b(ghost) + (h*_b - h^eq_b) with the ghost one spacing
 *     outside at u_g = 2 u_w - u, theta_g = max(2 theta_w - theta,
 *     theta_w / 2), rho_g theta_g = rho (theta - 3 g n_z) (the node's
 *     pressure carried across by hydrostatic balance, n_z the z component
 *     of the outward normal: 0 on the x and y sides); h on an adiabatic
 *     wall
 *     h_b = h*_a - 2 (odd part of h^eq_a at (rho, u_w, theta)), for total
 *     energy plus the wall's work on the pair u_w . (f_b e_b - f*_a e_a)
 *     (a moving adiabatic wall passes its work, not heat); Eq. 50 across a
 *     wall takes the mirror ghost Q_g = 2 rho u_w (1 - theta_w) - Q.
 *
 * Velocity set (index a: e_a), weights 1/3 (a = 0), 1/18 (1-6), 1/36 (7-18):
 *   0 (0,0,0)  1 (1,0,0)  2 (-1,0,0)  3 (0,1,0)   4 (0,-1,0)   5 (0,0,1)
 *   6 (0,0,-1) 7 (1,1,0)  8 (-1,-1,0) 9 (1,-1,0) 10 (-1,1,0)  11 (1,0,1)
 *  12 (-1,0,-1) 13 (1,0,-1) 14 (-1,0,1) 15 (0,1,1) 16 (0,-1,-1) 17 (0,1,-1)
 *  18 (0,-1,1)
 *
 * Conventions: as in lbm.h (status codes LBM_OK / LBM_ERR_*, caller-owned
 * host arrays, the handle's stream, lattice units with R T0 = 1/3).  Host
 * fields are [nz][ny][nx] doubles, node (x, y, z) at (z ny + y) nx + x.
 * Storage precision: LBM_P_FP64 or LBM_P_FP32 (the 16-bit deviation storage
 * of the D2Q9 path is not built for D3Q19).  The node count must stay below
 * 2^31.
 */
#ifndef LBM3D_H
#define LBM3D_H

#include <stdint.h>

#include "lbm.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  int32_t nx, ny, nz;   /* nodes per axis, >= 1 each                          */
  double tau_f, tau_h;  /* continuous-time relaxation times, > 0:             */
                        /* omega = 2 / (2 tau + 1), nu = tau_f R T,           */
                        /* chi = tau_h R T, Pr = tau_f / tau_h                */
  double R, T0, b;      /* R T0 = 1/3; b >= 3 degrees of freedom, gamma =     */
                        /* (b + 2) / b                                        */
  int32_t energy_model; /* LBM_E_TOTAL (Eq. 36) or LBM_E_INTERNAL (Eq. 38)    */
  int32_t correction;   /* 1: C_a as above; 0: omitted                        */
  int32_t z_full;       /* total energy: 1 Z = e.u - u^2/2, 0 Z = e.u         */
  int32_t precision;    /* LBM_P_FP64 or LBM_P_FP32                           */
  int32_t bc_z[2];      /* z- and z+ sides: LBM_BC_PERIODIC,                  */
                        /* LBM_BC_WALL_ISOTHERMAL or                          */
                        /* LBM_BC_WALL_ADIABATIC (halfway walls, see above);  */
                        /* both periodic or both walls                        */
  double u_wall_z[2][3];  /* wall velocities of the z sides                   */
  double T_wall_z[2];     /* wall temperatures, > 0 on an isothermal wall      */
  double g;               /* gravity along -z, a = (0, 0, -rho g): Guo's force */
                          /* term beside C_a (Eq. 51 with D = 3) and the half- */
                          /* force velocity shift; LBM_E_INTERNAL only, else 0 */
  int32_t bc_x[2], bc_y[2]; /* x-, x+ and y-, y+ sides, as bc_z (zeroed: all  */
                            /* periodic)                                       */
  double u_wall_x[2][3], u_wall_y[2][3]; /* wall velocities of those sides    */
  double T_wall_x[2], T_wall_y[2];       /* their wall temperatures, > 0 on   */
                                         /* an isothermal wall               */
} lbm3d_params;

typedef struct lbm3d_handle lbm3d_handle;

/* Bytes of device memory of the two population buffers of a grid:
 * 2 (nz + 2)(ny + 2) 38 pitch elements, pitch = the smallest multiple of 32
 * >= nx + 33.  Negative LBM_ERR_* for invalid parameters. */
int64_t lbm3d_state_bytes(const lbm3d_params* p);

/* Validates *p and allocates the state and the staging of host transfers
 * (5 nx ny nz doubles) on the current device; binds the handle to
 * cuda_stream (NULL: the legacy default stream).  Errors: LBM_ERR_PARAM
 * (nx, ny or nz < 1, tau <= 0, R T0 != 1/3, b < 3, an unknown model,
 * precision or side kind, one side of an axis periodic and the other a
 * wall, a non-finite wall velocity, an isothermal wall's temperature <= 0,
 * a non-finite g or g != 0 with total energy, 2^31 nodes or more),
 * LBM_ERR_OOM, LBM_ERR_CUDA.  *out is NULL
 * on error. */
int lbm3d_create(const lbm3d_params* p, void* cuda_stream, lbm3d_handle** out);

/* Sets the state to equilibrium (Eq. 18a, Eq. 18b or the Eq. 38 form) at the
 * host fields rho, u = (ux, uy, uz), T (T in the units of T0), nx ny nz each;
 * resets the step counter.  Synchronous. */
int lbm3d_init(lbm3d_handle* h, const double* rho, const double* ux, const double* uy,
               const double* uz, const double* T);

/* Same with device arrays on the handle's device; asynchronous. */
int lbm3d_init_device(lbm3d_handle* h, const double* d_rho, const double* d_ux,
                      const double* d_uy, const double* d_uz, const double* d_T);

/* Advances n >= 0 time steps, one fused stream-and-collide kernel per step.
 * Asynchronous; LBM_ERR_STATE before an init, LBM_ERR_CUDA if a launch fails. */
int lbm3d_step(lbm3d_handle* h, int64_t n);

/* rho, u and T of the current state (Eq. 35, Eq. 37 or the Eq. 38 form) in
 * FP64 into host arrays of nx ny nz; synchronous.  LBM_ERR_NONFINITE if any
 * value is NaN or infinite (the arrays are still filled). */
int lbm3d_moments(lbm3d_handle* h, double* rho, double* ux, double* uy, double* uz, double* T);

/* The canonical pre-collision populations (FP64) into a host array
 * [38][nz][ny][nx]: f_0..f_18 then h_0..h_18 in the order of the velocity
 * table above.  Synchronous. */
int lbm3d_get_state(lbm3d_handle* h, double* pops);

/* FP64 sums over the grid of rho, rho u_x, rho u_y, rho u_z and hbar (rho E
 * for LBM_E_TOTAL), in a fixed order; synchronous. */
int lbm3d_conserved(lbm3d_handle* h, double out[5]);

/* Waits for the handle's stream; LBM_ERR_CUDA on a pending kernel error. */
int lbm3d_sync(lbm3d_handle* h);

/* Steps taken since the last init. */
int64_t lbm3d_steps_done(const lbm3d_handle* h);

/* Launch shape of the step kernel (no counterpart in the paper; results do
 * not depend on it beyond FP32 rounding): a block owns 32 x tile_rows nodes
 * of (x, y) and marches along z.  tile_rows = 8 or 16 (16 for LBM_P_FP32
 * only), with the halo ring on the tile's first threads; 0 = automatic
 * (LBM_P_FP64: 8 rows; LBM_P_FP32: 4 rows with halo warps, see
 * lbm3d_set_launch).  LBM_ERR_PARAM for other values. */
int lbm3d_set_tile(lbm3d_handle* h, int32_t tile_rows);

/* Launch shape of the step kernel with the halo option (no counterpart in
 * the paper; results do not depend on it): tile_rows as above (0 =
 * automatic, halo_warps then ignored) and halo_warps = 1 to give the tile's
 * one-node halo ring warps of its own instead of a second pull on the
 * tile's first threads.  Shapes (tile_rows, halo_warps): (8, 0); for
 * LBM_P_FP32 also (16, 0), (4, 1) and (8, 1).  LBM_ERR_PARAM otherwise. */
int lbm3d_set_launch(lbm3d_handle* h, int32_t tile_rows, int32_t halo_warps);

/* Frees the device state and the handle; NULL-safe. */
void lbm3d_destroy(lbm3d_handle* h);

/* Message of the last failure on h (or of the last failed lbm3d_create on
 * this thread when h is NULL). */
const char* lbm3d_last_error(const lbm3d_handle* h);

#ifdef __cplusplus
}
#endif

#endif /* LBM3D_H */
