// Host side of the D3Q19 C ABI declared in include/lbm3d.h: validation,
// device state, launches of the kernels in lbm3d.cuh.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>

#include "lbm3d.h"
#include "lbm3d_launch.h"

using namespace lbm3;

struct lbm3d_handle {
  lbm3d_params p{};
  cudaStream_t stream = nullptr;
  int device = 0, num_sms = 0;
  void* base = nullptr;  // two state buffers
  size_t buf_bytes = 0;
  int cur = 0;
  int64_t steps = 0;
  bool ready = false;
  Grid3 grid{};
  dim3 launch{};
  int zrows = 0;
  int tile = 0;       // tile rows asked for: 0 (automatic), 4, 8 or 16
  int tile_split = 0;  // separate halo warps asked for (tile != 0)
  int tile_rows = 8;   // tile rows in use
  int split = 0;       // separate halo warps in use
  double* staging = nullptr;  // 5 n doubles (host transfers), later 38 n (get_state)
  size_t staging_bytes = 0;
  double* partial = nullptr;  // reduction partials + result + flag
  std::string err;
};

namespace {

constexpr int RED_BLOCKS3 = 512;
thread_local std::string g_create_err3;

int fail3(lbm3d_handle* h, int code, const std::string& msg) {
  if (h)
    h->err = msg;
  else
    g_create_err3 = msg;
  return code;
}

int cuda_fail3(lbm3d_handle* h, cudaError_t e, const char* what) {
  return fail3(h, LBM_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

// Side s = 2 axis + (0: low end, 1: high end) of the box.
int side_bc3(const lbm3d_params* p, int s) {
  return s < 2 ? p->bc_x[s] : (s < 4 ? p->bc_y[s - 2] : p->bc_z[s - 4]);
}
const double* side_uw3(const lbm3d_params* p, int s) {
  return s < 2 ? p->u_wall_x[s] : (s < 4 ? p->u_wall_y[s - 2] : p->u_wall_z[s - 4]);
}
double side_Tw3(const lbm3d_params* p, int s) {
  return s < 2 ? p->T_wall_x[s] : (s < 4 ? p->T_wall_y[s - 2] : p->T_wall_z[s - 4]);
}

int validate3(const lbm3d_params* p, std::string& why) {
  if (!p) {
    why = "params is NULL";
    return LBM_ERR_PARAM;
  }
  if (p->nx < 1 || p->ny < 1 || p->nz < 1) {
    why = "nx, ny and nz must be >= 1";
    return LBM_ERR_PARAM;
  }
  if ((long long)p->nx * p->ny * p->nz >= (1ll << 31)) {
    why = "the node count must be below 2^31";
    return LBM_ERR_PARAM;
  }
  if (!(p->tau_f > 0.0) || !(p->tau_h > 0.0) || !std::isfinite(p->tau_f) ||
      !std::isfinite(p->tau_h)) {
    why = "tau_f and tau_h must be finite and > 0";
    return LBM_ERR_PARAM;
  }
  if (!(std::fabs(p->R * p->T0 - 1.0 / 3.0) <= 1e-12)) {
    why = "R * T0 must equal 1/3 (lattice speed c = 1)";
    return LBM_ERR_PARAM;
  }
  if (!(p->b >= 3.0) || !std::isfinite(p->b)) {
    why = "b must be >= 3 in three dimensions (the translational degrees of freedom)";
    return LBM_ERR_PARAM;
  }
  if (p->energy_model != LBM_E_TOTAL && p->energy_model != LBM_E_INTERNAL) {
    why = "energy_model must be LBM_E_TOTAL or LBM_E_INTERNAL";
    return LBM_ERR_PARAM;
  }
  if ((p->correction != 0 && p->correction != 1) || (p->z_full != 0 && p->z_full != 1)) {
    why = "correction and z_full must be 0 or 1";
    return LBM_ERR_PARAM;
  }
  if (p->precision != LBM_P_FP64 && p->precision != LBM_P_FP32) {
    why = "precision must be LBM_P_FP64 or LBM_P_FP32";
    return LBM_ERR_PARAM;
  }
  for (int s = 0; s < 6; ++s) {
    const char* ax = s < 2 ? "x" : (s < 4 ? "y" : "z");
    const int bc = side_bc3(p, s);
    if (bc != LBM_BC_PERIODIC && bc != LBM_BC_WALL_ISOTHERMAL && bc != LBM_BC_WALL_ADIABATIC) {
      why = std::string("bc_") + ax + " must be LBM_BC_PERIODIC or a wall";
      return LBM_ERR_PARAM;
    }
    for (int d = 0; d < 3; ++d)
      if (!std::isfinite(side_uw3(p, s)[d])) {
        why = std::string("u_wall_") + ax + " must be finite";
        return LBM_ERR_PARAM;
      }
    // a wall temperature is read on isothermal walls only
    const double Tw = side_Tw3(p, s);
    if (bc == LBM_BC_WALL_ISOTHERMAL && (!(Tw > 0.0) || !std::isfinite(Tw))) {
      why = std::string("T_wall_") + ax + " must be finite and > 0";
      return LBM_ERR_PARAM;
    }
    if ((s & 1) && (side_bc3(p, s - 1) == LBM_BC_PERIODIC) != (bc == LBM_BC_PERIODIC)) {
      why = std::string("the ") + ax + " sides are both periodic or both walls";
      return LBM_ERR_PARAM;
    }
  }
  if (!std::isfinite(p->g) || (p->g != 0.0 && p->energy_model != LBM_E_INTERNAL)) {
    why = "g must be finite, and 0 unless energy_model is LBM_E_INTERNAL";
    return LBM_ERR_PARAM;
  }
  return LBM_OK;
}

int pitch3(int nx) { return (nx + 33 + 31) / 32 * 32; }

size_t buffer_bytes3(const lbm3d_params* p) {
  const size_t es = p->precision == LBM_P_FP64 ? 8 : 4;
  return (size_t)(p->nz + 2) * (p->ny + 2) * NP3 * pitch3(p->nx) * es;
}

void fill_grid3(const lbm3d_params* p, Grid3& g) {
  g = Grid3{};
  g.nx = p->nx;
  g.ny = p->ny;
  g.nz = p->nz;
  g.pitch = pitch3(p->nx);
  g.lp = (long long)NP3 * g.pitch;
  g.zs = (long long)(p->ny + 2) * g.lp;
  g.energy_model = p->energy_model;
  g.correction = p->correction;
  g.z_full = p->z_full;
  const double wf = 2.0 / (2.0 * p->tau_f + 1.0), wh = 2.0 / (2.0 * p->tau_h + 1.0);
  g.pd = Phys3<double>{};
  g.pf = Phys3<float>{};
  g.pd.omega_f = wf;
  g.pd.omega_h = wh;
  g.pd.kz = wh - wf;
  g.pd.b6 = p->b / 6.0;
  g.pd.six_b = 6.0 / p->b;
  g.pf.omega_f = (float)wf;
  g.pf.omega_h = (float)wh;
  g.pf.kz = (float)(wh - wf);
  g.pf.b6 = (float)(p->b / 6.0);
  g.pf.six_b = (float)(6.0 / p->b);
  g.pd.g = p->g;
  g.pf.g = (float)p->g;
  for (int k = 0; k < 6; ++k) {
    g.bc[k] = side_bc3(p, k);
    g.pd.thw[k] = side_Tw3(p, k) / p->T0;
    g.pf.thw[k] = (float)g.pd.thw[k];
    for (int d = 0; d < 3; ++d) {
      g.pd.uw[k][d] = side_uw3(p, k)[d];
      g.pf.uw[k][d] = (float)side_uw3(p, k)[d];
    }
  }
}

void* buf_ptr3(const lbm3d_handle* h, int b) {
  return static_cast<char*>(h->base) + (size_t)b * h->buf_bytes;
}

int ensure_staging3(lbm3d_handle* h, size_t bytes) {
  if (h->staging_bytes >= bytes) return LBM_OK;
  if (h->staging) cudaFree(h->staging);
  h->staging = nullptr;
  h->staging_bytes = 0;
  if (cudaMalloc(&h->staging, bytes) != cudaSuccess) {
    cudaGetLastError();
    return fail3(h, LBM_ERR_OOM, "device staging allocation failed");
  }
  h->staging_bytes = bytes;
  return LBM_OK;
}

int aux_blocks(long long n) {
  return (int)std::max<long long>(1, std::min<long long>(4096, (n + 255) / 256));
}

cudaError_t aux(lbm3d_handle* h, int what, void* buf, const double* const* in, double* const* out,
                double* pops, int* flag, int blocks) {
  Grid3 g = h->grid;
  if (h->p.precision == LBM_P_FP64)
    return launch_aux3d_f64(what, g, buf, in, out, h->p.T0, pops, flag, h->partial, blocks,
                            h->stream);
  return launch_aux3d_f32(what, g, buf, in, out, h->p.T0, pops, flag, h->partial, blocks,
                          h->stream);
}

// Launch shape: 32 x TY tiles of (x, y).  Automatic: FP64 8 rows; FP32 4
// rows with separate halo warps (two 224-thread blocks per SM), which at
// 256^3 ran at 11.1 GLUPS against 10.3 for 8 rows with the halo ring on the
// tile's first threads (those threads pulled twice per plane while the rest
// of the block waited), 9.2 for 8 rows with halo warps (one 352-thread block
// per SM by registers) and 9.0 for 16 rows (one 512-thread block).  The z
// range of a block is chosen so that the grid is about four waves of
// resident blocks.
size_t smem3(bool f64, int ty) {
  if (f64) return step3d_smem<double, 8>();
  return ty == 16 ? step3d_smem<float, 16>()
                  : (ty == 4 ? step3d_smem<float, 4>() : step3d_smem<float, 8>());
}
int threads_of3(int ty, int split) {
  if (!split) return TX3 * ty;
  return ty == 4 ? threads3<4, true>() : threads3<8, true>();
}
void choose_launch(lbm3d_handle* h) {
  const bool f64 = h->p.precision == LBM_P_FP64;
  h->tile_rows = f64 ? 8 : (h->tile ? h->tile : 4);
  h->split = f64 ? 0 : (h->tile ? h->tile_split : 1);
  const int TYr = h->tile_rows;
  const int tx = (h->p.nx + TX3 - 1) / TX3, ty = (h->p.ny + TYr - 1) / TYr;
  cudaFuncAttributes a{};
  const int mode = mode3_of(h->grid);
  const cudaError_t e = f64 ? step3d_attributes_f64(mode, TYr, h->split, &a)
                            : step3d_attributes_f32(mode, TYr, h->split, &a);
  int per_sm = 1;
  if (e == cudaSuccess && a.numRegs > 0)
    per_sm = std::max(1, 65536 / (a.numRegs * threads_of3(TYr, h->split)));
  // and by shared memory (the parked populations and the Q ring, plus the
  // 1 KB the hardware reserves per block, of 228 KB per SM)
  const size_t smem = smem3(f64, TYr);
  per_sm = std::max(1, std::min(per_sm, (int)(233472 / (smem + 1024))));
  const long long resident = (long long)per_sm * std::max(1, h->num_sms);
  const long long chunks =
      std::max<long long>(1, std::min<long long>(h->p.nz, (4 * resident + tx * ty - 1) / (tx * ty)));
  h->zrows = (int)((h->p.nz + chunks - 1) / chunks);
  h->launch = dim3(tx, ty, (h->p.nz + h->zrows - 1) / h->zrows);
}

}  // namespace

extern "C" {

int64_t lbm3d_state_bytes(const lbm3d_params* p) {
  std::string why;
  const int rc = validate3(p, why);
  if (rc != LBM_OK) return rc;
  return (int64_t)(2 * buffer_bytes3(p));
}

int lbm3d_create(const lbm3d_params* p, void* stream, lbm3d_handle** out) {
  if (!out) return fail3(nullptr, LBM_ERR_PARAM, "out is NULL");
  *out = nullptr;
  std::string why;
  const int rc = validate3(p, why);
  if (rc != LBM_OK) return fail3(nullptr, rc, why);
  lbm3d_handle* h = new lbm3d_handle();
  h->p = *p;
  h->stream = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaGetDevice(&h->device);
  if (e != cudaSuccess) {
    delete h;
    return fail3(nullptr, LBM_ERR_CUDA, std::string("no CUDA device: ") + cudaGetErrorString(e));
  }
  cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device);
  h->buf_bytes = buffer_bytes3(p);
  const size_t n = (size_t)p->nx * p->ny * p->nz;
  if (cudaMalloc(&h->base, 2 * h->buf_bytes) != cudaSuccess ||
      cudaMalloc(&h->partial, sizeof(double) * (5 * RED_BLOCKS3 + 8)) != cudaSuccess ||
      ensure_staging3(h, 5 * n * sizeof(double)) != LBM_OK) {
    cudaGetLastError();
    lbm3d_destroy(h);
    return fail3(nullptr, LBM_ERR_OOM, "device allocation of the state failed");
  }
  // slots no rule writes are never read; zero everything once
  e = cudaMemsetAsync(h->base, 0, 2 * h->buf_bytes, h->stream);
  if (e != cudaSuccess) {
    lbm3d_destroy(h);
    return fail3(nullptr, LBM_ERR_CUDA, std::string("memset: ") + cudaGetErrorString(e));
  }
  fill_grid3(p, h->grid);
  choose_launch(h);
  *out = h;
  return LBM_OK;
}

int lbm3d_init_device(lbm3d_handle* h, const double* rho, const double* ux, const double* uy,
                      const double* uz, const double* T) {
  if (!h) return LBM_ERR_PARAM;
  if (!rho || !ux || !uy || !uz || !T) return fail3(h, LBM_ERR_PARAM, "NULL field pointer");
  const long long n = (long long)h->p.nx * h->p.ny * h->p.nz;
  h->cur = 0;
  const double* in[5] = {rho, ux, uy, uz, T};
  const cudaError_t e = aux(h, AUX3_INIT, buf_ptr3(h, 0), in, nullptr, nullptr, nullptr,
                            aux_blocks(n));
  if (e != cudaSuccess) return cuda_fail3(h, e, "init kernel launch");
  h->steps = 0;
  h->ready = true;
  return LBM_OK;
}

int lbm3d_init(lbm3d_handle* h, const double* rho, const double* ux, const double* uy,
               const double* uz, const double* T) {
  if (!h) return LBM_ERR_PARAM;
  if (!rho || !ux || !uy || !uz || !T) return fail3(h, LBM_ERR_PARAM, "NULL field pointer");
  const size_t n = (size_t)h->p.nx * h->p.ny * h->p.nz;
  int rc = ensure_staging3(h, 5 * n * sizeof(double));
  if (rc) return rc;
  const double* src[5] = {rho, ux, uy, uz, T};
  for (int k = 0; k < 5; ++k) {
    const cudaError_t e = cudaMemcpyAsync(h->staging + k * n, src[k], n * sizeof(double),
                                          cudaMemcpyHostToDevice, h->stream);
    if (e != cudaSuccess) return cuda_fail3(h, e, "host-to-device copy");
  }
  rc = lbm3d_init_device(h, h->staging, h->staging + n, h->staging + 2 * n, h->staging + 3 * n,
                         h->staging + 4 * n);
  if (rc) return rc;
  return lbm3d_sync(h);
}

int lbm3d_step(lbm3d_handle* h, int64_t n) {
  if (!h) return LBM_ERR_PARAM;
  if (!h->ready) return fail3(h, LBM_ERR_STATE, "lbm3d_step before lbm3d_init");
  if (n < 0) return fail3(h, LBM_ERR_PARAM, "n must be >= 0");
  for (int64_t k = 0; k < n; ++k) {
    Grid3 g = h->grid;
    g.src = buf_ptr3(h, h->cur);
    g.dst = buf_ptr3(h, h->cur ^ 1);
    const cudaError_t e = h->p.precision == LBM_P_FP64
                              ? launch_step3d_f64(g, h->launch, h->zrows, 8, 0, h->stream)
                              : launch_step3d_f32(g, h->launch, h->zrows, h->tile_rows,
                                                  h->split, h->stream);
    if (e != cudaSuccess) return cuda_fail3(h, e, "step kernel launch");
    h->cur ^= 1;
    ++h->steps;
  }
  return LBM_OK;
}

int lbm3d_moments(lbm3d_handle* h, double* rho, double* ux, double* uy, double* uz, double* T) {
  if (!h) return LBM_ERR_PARAM;
  if (!h->ready) return fail3(h, LBM_ERR_STATE, "lbm3d_moments before lbm3d_init");
  if (!rho || !ux || !uy || !uz || !T) return fail3(h, LBM_ERR_PARAM, "NULL output pointer");
  const size_t n = (size_t)h->p.nx * h->p.ny * h->p.nz;
  int rc = ensure_staging3(h, 5 * n * sizeof(double));
  if (rc) return rc;
  int* flag = reinterpret_cast<int*>(h->partial + 5 * RED_BLOCKS3 + 6);
  cudaError_t e = cudaMemsetAsync(flag, 0, sizeof(int), h->stream);
  double* out[5] = {h->staging, h->staging + n, h->staging + 2 * n, h->staging + 3 * n,
                    h->staging + 4 * n};
  if (e == cudaSuccess)
    e = aux(h, AUX3_EXPORT, buf_ptr3(h, h->cur), nullptr, out, nullptr, flag, aux_blocks(n));
  double* dst[5] = {rho, ux, uy, uz, T};
  for (int k = 0; k < 5 && e == cudaSuccess; ++k)
    e = cudaMemcpyAsync(dst[k], out[k], n * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
  int bad = 0;
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&bad, flag, sizeof(int), cudaMemcpyDeviceToHost, h->stream);
  if (e != cudaSuccess) return cuda_fail3(h, e, "moments");
  rc = lbm3d_sync(h);
  if (rc) return rc;
  if (bad) return fail3(h, LBM_ERR_NONFINITE, "non-finite moment");
  return LBM_OK;
}

int lbm3d_get_state(lbm3d_handle* h, double* pops) {
  if (!h) return LBM_ERR_PARAM;
  if (!h->ready) return fail3(h, LBM_ERR_STATE, "lbm3d_get_state before lbm3d_init");
  if (!pops) return fail3(h, LBM_ERR_PARAM, "pops is NULL");
  const size_t n = (size_t)h->p.nx * h->p.ny * h->p.nz;
  int rc = ensure_staging3(h, NP3 * n * sizeof(double));
  if (rc) return rc;
  cudaError_t e =
      aux(h, AUX3_EXPORT, buf_ptr3(h, h->cur), nullptr, nullptr, h->staging, nullptr,
          aux_blocks(n));
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(pops, h->staging, NP3 * n * sizeof(double), cudaMemcpyDeviceToHost,
                        h->stream);
  if (e != cudaSuccess) return cuda_fail3(h, e, "get_state");
  return lbm3d_sync(h);
}

int lbm3d_conserved(lbm3d_handle* h, double out[5]) {
  if (!h) return LBM_ERR_PARAM;
  if (!h->ready) return fail3(h, LBM_ERR_STATE, "lbm3d_conserved before lbm3d_init");
  if (!out) return fail3(h, LBM_ERR_PARAM, "out is NULL");
  const long long n = (long long)h->p.nx * h->p.ny * h->p.nz;
  const int nb = (int)std::min<long long>(RED_BLOCKS3, (n + RED3 - 1) / RED3);
  cudaError_t e = aux(h, AUX3_CONSERVED, buf_ptr3(h, h->cur), nullptr, nullptr, nullptr, nullptr,
                      nb);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(out, h->partial + 5 * nb, 5 * sizeof(double), cudaMemcpyDeviceToHost,
                        h->stream);
  if (e != cudaSuccess) return cuda_fail3(h, e, "conserved");
  const int rc = lbm3d_sync(h);
  if (rc) return rc;
  for (int k = 0; k < 5; ++k)
    if (!std::isfinite(out[k])) return fail3(h, LBM_ERR_NONFINITE, "non-finite sum");
  return LBM_OK;
}

int lbm3d_sync(lbm3d_handle* h) {
  if (!h) return LBM_ERR_PARAM;
  const cudaError_t e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail3(h, e, "stream synchronize");
  return LBM_OK;
}

int64_t lbm3d_steps_done(const lbm3d_handle* h) { return h ? h->steps : LBM_ERR_PARAM; }

int lbm3d_set_launch(lbm3d_handle* h, int32_t tile_rows, int32_t halo_warps) {
  if (!h) return LBM_ERR_PARAM;
  if (tile_rows != 0) {
    const bool f32 = h->p.precision == LBM_P_FP32;
    const bool ok = (tile_rows == 8 && halo_warps == 0) ||
                    (f32 && ((tile_rows == 16 && halo_warps == 0) ||
                             ((tile_rows == 4 || tile_rows == 8) && halo_warps == 1)));
    if (!ok)
      return fail3(h, LBM_ERR_PARAM,
                   "launch shapes: (8, 0); for FP32 storage also (16, 0), (4, 1), (8, 1)");
  }
  h->tile = tile_rows;
  h->tile_split = tile_rows ? halo_warps : 0;
  choose_launch(h);
  return LBM_OK;
}

int lbm3d_set_tile(lbm3d_handle* h, int32_t tile_rows) {
  if (!h) return LBM_ERR_PARAM;
  if (tile_rows != 0 && tile_rows != 8 && tile_rows != 16)
    return fail3(h, LBM_ERR_PARAM, "tile_rows must be 0 (automatic), 8 or 16");
  if (tile_rows == 16 && h->p.precision == LBM_P_FP64)
    return fail3(h, LBM_ERR_PARAM, "16-row tiles are built for FP32 storage only");
  return lbm3d_set_launch(h, tile_rows, 0);
}

void lbm3d_destroy(lbm3d_handle* h) {
  if (!h) return;
  if (h->stream || h->base) cudaStreamSynchronize(h->stream);
  if (h->base) cudaFree(h->base);
  if (h->partial) cudaFree(h->partial);
  if (h->staging) cudaFree(h->staging);
  delete h;
}

const char* lbm3d_last_error(const lbm3d_handle* h) {
  return h ? h->err.c_str() : g_create_err3.c_str();
}

}  // extern "C"
