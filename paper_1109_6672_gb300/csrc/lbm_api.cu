// Host side of the single-grid C ABI declared in include/lbm.h: parameter
// validation, device state, launches of the kernels in lbm_device.cuh.
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "lbm.h"
#include "lbm_device.cuh"
#include "lbm_host.h"
#include "lbm_launch.h"
#include "lbm_open.cuh"

using namespace lbm;

struct lbm_handle {
  lbm_params p{};
  cudaStream_t stream = nullptr;
  int device = 0;
  int num_sms = 0;
  void* base = nullptr;  // start of the two state buffers
  bool owns = false;
  size_t buf_bytes = 0;
  int cur = 0;  // buffer holding the state at the current time
  int64_t steps = 0;
  bool ready = false;
  bool lost = false;  // a step kernel left with copies in flight: reload the state
  Grid grid{};
  int variant = TMA_PR_1, rows = 0;  // 1, 2: pulled-row TMA kernel; 64..256: register pull
  int auto_rows = 0;                 // rows chosen for (variant, rows = 0); 0: not yet
  cudaGraphExec_t graph[2] = {nullptr, nullptr};  // GRAPH_STEPS steps from buffer 0 / 1
  CUtensorMap maps[2][2];            // TMA descriptors [buffer][columns per thread - 1]
  double* partial = nullptr;  // reduction scratch: RED_BLOCKS x 4
  double* out4 = nullptr;     // reduction result
  int* status = nullptr;      // device error word of the step kernels
  int* nonfinite = nullptr;   // device flag of export_kernel (lbm_moments)
  // host transfers in row chunks: copies on `xfer`, kernels on `stream`,
  // linked by one event per chunk, so each chunk's kernel overlaps the next
  // chunk's copies
  cudaStream_t xfer = nullptr;
  cudaEvent_t chunk_ev[8] = {};
  double* staging = nullptr;  // device staging for host transfers
  size_t staging_bytes = 0;
  std::string err;
};

namespace {

thread_local std::string g_create_error;

int fail(lbm_handle* h, int code, const std::string& msg) {
  if (h)
    h->err = msg;
  else
    g_create_error = msg;
  return code;
}

int cuda_fail(lbm_handle* h, cudaError_t e, const char* what) {
  return fail(h, LBM_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

constexpr int RED_BLOCKS = 1024;

size_t elem_size(int precision) {
  switch (precision) {
    case LBM_P_FP64: return 8;
    case LBM_P_FP32: return 4;
    default: return 2;
  }
}

}  // namespace

namespace lbm_host {

int validate(const lbm_params* p, std::string& why) {
  if (!p) {
    why = "params is NULL";
    return LBM_ERR_PARAM;
  }
  if (p->nx < 1 || p->ny < 1) {
    why = "nx and ny must be >= 1";
    return LBM_ERR_PARAM;
  }
  for (int s = 0; s < 4; ++s) {
    if (p->bc[s] < 0 || p->bc[s] > LBM_BC_OUTLET) {
      why = "bc values must be one of LBM_BC_*";
      return LBM_ERR_PARAM;
    }
  }
  const bool inlet = p->bc[0] == LBM_BC_INLET, outlet = p->bc[1] == LBM_BC_OUTLET;
  if (p->bc[1] == LBM_BC_INLET || p->bc[0] == LBM_BC_OUTLET || p->bc[2] >= LBM_BC_INLET ||
      p->bc[3] >= LBM_BC_INLET) {
    why = "LBM_BC_INLET is an x- side only, LBM_BC_OUTLET an x+ side only";
    return LBM_ERR_PARAM;
  }
  if ((inlet || outlet) && p->bc[2] != LBM_BC_PERIODIC) {
    why = "open x sides (inlet / outlet) need a periodic y axis";
    return LBM_ERR_PARAM;
  }
  if (p->wall_nee < 0 || p->wall_nee > 15) {
    why = "wall_nee is a bit mask of the four sides";
    return LBM_ERR_PARAM;
  }
  for (int s = 0; s < 4; ++s) {
    if ((p->wall_nee >> s & 1) && p->bc[s] != LBM_BC_WALL_ISOTHERMAL &&
        p->bc[s] != LBM_BC_WALL_ADIABATIC) {
      why = "wall_nee flags only isothermal or adiabatic wall sides";
      return LBM_ERR_PARAM;
    }
  }
  if ((inlet || outlet) && p->correction != 0) {
    why = "open x sides (inlet / outlet) need correction = 0 (as the paper runs them)";
    return LBM_ERR_PARAM;
  }
  if (inlet) {
    for (double v : {p->in_rho, p->in_drho, p->in_du, p->in_dT, p->in_omega}) {
      if (!std::isfinite(v)) {
        why = "inlet parameters must be finite";
        return LBM_ERR_PARAM;
      }
    }
    if (!(p->in_rho - std::fabs(p->in_drho) > 0.0) ||
        !(p->T_wall[0] - std::fabs(p->in_dT) > 0.0)) {
      why = "inlet density and temperature must stay > 0 (in_rho > |in_drho|, T_wall[0] > |in_dT|)";
      return LBM_ERR_PARAM;
    }
  }
  if ((p->bc[0] == LBM_BC_PERIODIC) != (p->bc[1] == LBM_BC_PERIODIC) ||
      (p->bc[2] == LBM_BC_PERIODIC) != (p->bc[3] == LBM_BC_PERIODIC)) {
    why = "a periodic side needs its opposite side periodic";
    return LBM_ERR_PARAM;
  }
  if ((p->bc[0] != LBM_BC_PERIODIC && p->nx < 3) || (p->bc[2] != LBM_BC_PERIODIC && p->ny < 3)) {
    why = "a walled axis needs at least 3 nodes";
    return LBM_ERR_PARAM;
  }
  if ((int64_t)p->nx * (int64_t)p->ny > (int64_t)1 << 31 || p->nx > (1 << 20) ||
      p->ny > (1 << 20)) {
    why = "grid too large (nx * ny must be <= 2^31)";
    return LBM_ERR_PARAM;
  }
  if (!(p->tau_f > 0.0) || !(p->tau_h > 0.0) || !std::isfinite(p->tau_f) ||
      !std::isfinite(p->tau_h)) {
    why = "tau_f and tau_h must be finite and > 0 (omega in (0, 2))";
    return LBM_ERR_PARAM;
  }
  if (p->Pr > 0.0 && std::fabs(p->Pr - p->tau_f / p->tau_h) > 1e-9 * p->Pr) {
    why = "Pr must equal tau_f / tau_h (or be <= 0)";
    return LBM_ERR_PARAM;
  }
  if (!(p->R > 0.0) || !(p->T0 > 0.0) || std::fabs(p->R * p->T0 * 3.0 - 1.0) > 1e-12) {
    why = "R * T0 must equal 1/3 (lattice speed c = sqrt(3 R T0) = 1)";
    return LBM_ERR_PARAM;
  }
  if (!(p->b >= 2.0) || !std::isfinite(p->b)) {
    why = "b (degrees of freedom) must be >= 2";
    return LBM_ERR_PARAM;
  }
  for (int s = 0; s < 4; ++s) {
    if (p->bc[s] == LBM_BC_WALL_ISOTHERMAL && !(p->T_wall[s] > 0.0)) {
      why = "T_wall must be > 0 on isothermal walls";
      return LBM_ERR_PARAM;
    }
    if (!std::isfinite(p->u_wall[s][0]) || !std::isfinite(p->u_wall[s][1])) {
      why = "u_wall must be finite";
      return LBM_ERR_PARAM;
    }
  }
  if (p->energy_model != LBM_E_TOTAL && p->energy_model != LBM_E_INTERNAL) {
    why = "energy_model must be LBM_E_TOTAL or LBM_E_INTERNAL";
    return LBM_ERR_PARAM;
  }
  if (p->g != 0.0 && p->energy_model == LBM_E_TOTAL) {
    why = "gravity needs energy_model = LBM_E_INTERNAL (the paper gives no work term for h)";
    return LBM_ERR_PARAM;
  }
  if (!std::isfinite(p->g)) {
    why = "g must be finite";
    return LBM_ERR_PARAM;
  }
  if (p->correction != 0 && p->correction != 1) {
    why = "correction must be 0 or 1";
    return LBM_ERR_PARAM;
  }
  if (p->z_full != 0 && p->z_full != 1) {
    why = "z_full must be 0 or 1";
    return LBM_ERR_PARAM;
  }
  if (p->precision < LBM_P_FP64 || p->precision > LBM_P_FP32_BF16) {
    why = "precision must be one of LBM_P_*";
    return LBM_ERR_PARAM;
  }
  if (p->collision != LBM_COLL_BGK && p->collision != LBM_COLL_MRT) {
    why = "collision must be LBM_COLL_BGK or LBM_COLL_MRT";
    return LBM_ERR_PARAM;
  }
  if (p->mu_law < LBM_MU_TAU || p->mu_law > LBM_MU_SUTHERLAND || !std::isfinite(p->mu_n) ||
      (p->mu_law == LBM_MU_SUTHERLAND && !(p->mu_S > 0.0 && std::isfinite(p->mu_S)))) {
    why = "mu_law must be LBM_MU_* with a finite mu_n (and mu_S > 0 for Sutherland)";
    return LBM_ERR_PARAM;
  }
  if (p->collision == LBM_COLL_MRT) {
    for (double r : {p->s_e, p->s_eps, p->s_q}) {
      if (!(r >= 0.0 && r < 2.0)) {
        why = "MRT rates s_e, s_eps, s_q must be in (0, 2), or 0 for omega_f";
        return LBM_ERR_PARAM;
      }
    }
  }
  return LBM_OK;
}

int pitch_of(int nx) { return ((nx + XOFF + 1 + 31) / 32) * 32; }

size_t buffer_elems(const lbm_params* p) {
  const size_t pitch = (size_t)pitch_of(p->nx);
  size_t n = (size_t)(p->ny + 2) * NPOP * pitch;
  return (n + 127) / 128 * 128;
}

size_t buffer_bytes(const lbm_params* p) { return buffer_elems(p) * elem_size(p->precision); }

void fill_grid(const lbm_params* p, Grid& g) {
  std::memset(&g, 0, sizeof(g));
  g.nx = p->nx;
  g.ny = p->ny;
  g.pitch = pitch_of(p->nx);
  g.rp = NPOP * g.pitch;
  Phys<double>& k = g.pd;
  for (int s = 0; s < 4; ++s) {
    g.bc[s] = p->bc[s];
    k.uw[s][0] = p->u_wall[s][0];
    k.uw[s][1] = p->u_wall[s][1];
    k.thw[s] = p->T_wall[s] / p->T0;
  }
  g.energy_model = p->energy_model;
  g.correction = p->correction;
  g.z_full = p->z_full;
  g.has_force = p->g != 0.0;
  g.collision = p->collision;
  k.omega_f = 2.0 / (2.0 * p->tau_f + 1.0);
  k.omega_h = 2.0 / (2.0 * p->tau_h + 1.0);
  // Z coupling of h: w_h - w_f (Eq. 36); for MRT (Eq. 47) (1 - w_h/2) / tau_hf
  // with tau_hf = tau/(Pr - 1), tau = tau_f + 1/2, Pr = (tau - 1/2)/tau_h
  k.kz = p->collision == LBM_COLL_MRT
             ? (1.0 - 0.5 * k.omega_h) * (p->tau_f / p->tau_h - 1.0) / (p->tau_f + 0.5)
             : k.omega_h - k.omega_f;
  k.se = p->s_e;
  k.seps = p->s_eps;
  k.sq = p->s_q;
  g.mu_law = p->mu_law;
  k.tau_f0 = p->tau_f;
  k.tau_ratio = p->tau_h / p->tau_f;
  k.mu_n = p->mu_n;
  k.mu_s = p->mu_S;
  k.g = p->g;
  k.b6 = p->b / 6.0;
  k.six_b = 6.0 / p->b;
  Phys<float>& f = g.pf;
  f.omega_f = (float)k.omega_f;
  f.omega_h = (float)k.omega_h;
  f.g = (float)k.g;
  f.b6 = (float)k.b6;
  f.six_b = (float)k.six_b;
  f.kz = (float)k.kz;
  f.se = (float)k.se;
  f.seps = (float)k.seps;
  f.sq = (float)k.sq;
  f.tau_f0 = (float)k.tau_f0;
  f.tau_ratio = (float)k.tau_ratio;
  f.mu_n = (float)k.mu_n;
  f.mu_s = (float)k.mu_s;
  for (int s = 0; s < 4; ++s) {
    f.uw[s][0] = (float)k.uw[s][0];
    f.uw[s][1] = (float)k.uw[s][1];
    f.thw[s] = (float)k.thw[s];
  }
  g.status = nullptr;
  // rest equilibria rho = 1, u = 0, theta = 1: f = w, h = w (b + 3 e^2 - 2)/6
  // (total energy) or w b / 6 (internal energy)
  double hs = 0.0;
  for (int a = 0; a < 9; ++a) {
    const double w = wgt<double>(a);
    const double e2 = (double)(ex(a) * ex(a) + ey(a) * ey(a));
    const double h = p->energy_model == LBM_E_TOTAL ? w * (p->b + 3.0 * e2 - 2.0) / 6.0
                                                    : w * p->b / 6.0;
    g.fref[a] = (float)w;
    g.href[a] = (float)h;
    hs += (double)g.href[a];
  }
  g.href_sum = hs;
  g.dref = hs - p->b / 6.0;
  g.pd.dref = g.dref;
  g.pf.dref = (float)g.dref;
  g.in_rho = p->in_rho;
  g.in_drho = p->in_drho;
  g.in_du = p->in_du;
  g.in_dth = p->in_dT / p->T0;
  g.in_omega = p->in_omega;
  g.nee = p->wall_nee;
}

}  // namespace lbm_host

using namespace lbm_host;

namespace {

template <class F>
int dispatch(int precision, F&& f) {
  switch (precision) {
    case LBM_P_FP64: return f((double*)nullptr);
    case LBM_P_FP32: return f((float*)nullptr);
    case LBM_P_FP32_FP16: return f((__half*)nullptr);
    default: return f((__nv_bfloat16*)nullptr);
  }
}

void* buf_ptr(lbm_handle* h, int which) {
  return static_cast<unsigned char*>(h->base) + (size_t)which * h->buf_bytes;
}

int ensure_staging(lbm_handle* h, size_t bytes) {
  if (h->staging_bytes >= bytes) return LBM_OK;
  if (h->staging) cudaFree(h->staging);
  h->staging = nullptr;
  h->staging_bytes = 0;
  cudaError_t e = cudaMalloc(&h->staging, bytes);
  if (e != cudaSuccess) return fail(h, LBM_ERR_OOM, "device staging allocation failed");
  h->staging_bytes = bytes;
  return LBM_OK;
}

int grid_blocks(long long n) { return (int)std::max(1LL, std::min(4096LL, (n + 255) / 256)); }

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

}  // namespace

namespace lbm_host {

// 3-D view of one state buffer for the TMA row loads: (x + 32, population,
// y + 1) with a box of one lattice row, all 18 populations, box_cols columns.
// The x extent ends at the ghost column x = nx: a box reaching past it (the
// last strip of a grid, narrow grids) is filled by the TMA unit without
// reading the row's padding up to the pitch; nothing reads those columns.
int make_tensor_map(CUtensorMap* map, void* buffer, const lbm_params& p, const Grid& g,
                    int box_cols, int box_planes) {
  auto fn = encode_fn();
  if (!fn) return LBM_ERR_CUDA;
  const size_t es = elem_size(p.precision);
  CUtensorMapDataType dt = p.precision == LBM_P_FP64   ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64
                           : p.precision == LBM_P_FP32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                           : p.precision == LBM_P_FP32_FP16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                                             : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
  cuuint64_t dims[3] = {(cuuint64_t)(XOFF + g.nx + 1), (cuuint64_t)NPOP, (cuuint64_t)(g.ny + 2)};
  cuuint64_t strides[2] = {(cuuint64_t)g.pitch * es, (cuuint64_t)g.rp * es};
  cuuint32_t box[3] = {(cuuint32_t)box_cols, (cuuint32_t)box_planes, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = fn(map, dt, 3, buffer, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? LBM_OK : LBM_ERR_CUDA;
}

}  // namespace lbm_host

namespace {

int create_impl(const lbm_params* p, void* stream, void* ext, int64_t ext_bytes, lbm_handle** out) {
  if (!out) return fail(nullptr, LBM_ERR_PARAM, "out is NULL");
  *out = nullptr;
  std::string why;
  int rc = validate(p, why);
  if (rc != LBM_OK) return fail(nullptr, rc, why);
  lbm_handle* h = new lbm_handle();
  h->p = *p;
  h->stream = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaGetDevice(&h->device);
  if (e != cudaSuccess) {
    delete h;
    return fail(nullptr, LBM_ERR_CUDA, std::string("no CUDA device: ") + cudaGetErrorString(e));
  }
  cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device);
  h->buf_bytes = buffer_bytes(p);
  const size_t need = 2 * h->buf_bytes;
  if (ext) {
    if ((int64_t)need > ext_bytes || (reinterpret_cast<uintptr_t>(ext) & 255u)) {
      delete h;
      return fail(nullptr, LBM_ERR_PARAM,
                  "device_buffer too small or not 256-byte aligned (need lbm_state_bytes)");
    }
    h->base = ext;
    h->owns = false;
  } else {
    e = cudaMalloc(&h->base, need);
    if (e != cudaSuccess) {
      cudaGetLastError();
      delete h;
      return fail(nullptr, LBM_ERR_OOM, "cudaMalloc of the state failed");
    }
    h->owns = true;
  }
  e = cudaMalloc(&h->partial, sizeof(double) * (RED_BLOCKS * 4 + 4) + 64);
  if (e != cudaSuccess) {
    cudaGetLastError();
    if (h->owns) cudaFree(h->base);
    delete h;
    return fail(nullptr, LBM_ERR_OOM, "cudaMalloc of the reduction scratch failed");
  }
  h->out4 = h->partial + RED_BLOCKS * 4;
  h->status = reinterpret_cast<int*>(h->out4 + 4);
  h->nonfinite = h->status + 1;
  cudaMemsetAsync(h->status, 0, 2 * sizeof(int), h->stream);
  // staging of the host fields (lbm_init, lbm_moments), allocated here so
  // that no transfer call allocates
  rc = ensure_staging(h, 4 * (size_t)p->nx * p->ny * sizeof(double));
  if (rc != LBM_OK) {
    cudaGetLastError();
    if (h->owns) cudaFree(h->base);
    cudaFree(h->partial);
    delete h;
    return fail(nullptr, LBM_ERR_OOM, "cudaMalloc of the host-transfer staging failed");
  }
  e = cudaStreamCreateWithFlags(&h->xfer, cudaStreamNonBlocking);
  for (int k = 0; k < 8 && e == cudaSuccess; ++k)
    e = cudaEventCreateWithFlags(&h->chunk_ev[k], cudaEventDisableTiming);
  if (e != cudaSuccess) {
    lbm_destroy(h);
    return fail(nullptr, LBM_ERR_CUDA, std::string("transfer stream: ") + cudaGetErrorString(e));
  }
  // ghost slots that no rule writes are never read; zero everything once so
  // the buffers hold defined values
  e = cudaMemsetAsync(h->base, 0, need, h->stream);
  if (e != cudaSuccess) {
    lbm_destroy(h);
    return fail(nullptr, LBM_ERR_CUDA, std::string("memset: ") + cudaGetErrorString(e));
  }
  fill_grid(p, h->grid);
  h->grid.status = h->status;
  for (int b = 0; b < 2; ++b) {
    for (int k = 0; k < 2; ++k) {
      rc = make_tensor_map(&h->maps[b][k], buf_ptr(h, b), h->p, h->grid, tma_box(k + 1), 6);
      if (rc != LBM_OK) {
        lbm_destroy(h);
        return fail(nullptr, rc, "cuTensorMapEncodeTiled failed");
      }
    }
  }
  *out = h;
  return LBM_OK;
}

// Columns a block of the selected kernel owns.
int block_cols(int variant) { return variant >= 64 ? variant - 2 : tma_cols(variant); }

// Rows per block so that the step launches about one wave of blocks.
// Rows per block of the pulled-row kernel.  Large grids keep the default
// (6 rows, 12 for 16-bit storage; many waves of blocks); a grid that needs
// fewer than 3 waves at the default takes the row count that minimises
// waves x (rows + 2) (the 2: a block's fixed cost of staging its halo rows
// and starting up, in rows), so that a mid-size grid runs in one full wave of
// taller blocks instead of a wave and a fraction.
int tma_rows(const lbm_handle* h, int variant) {
  const int r0 = std::min(h->p.ny, tma_default_rows(elem_size(h->p.precision)));
  const int bx = (h->p.nx + block_cols(variant) - 1) / block_cols(variant);
  int occ = 0;
  dispatch(h->p.precision, [&](auto* tag) {
    using S = std::remove_pointer_t<decltype(tag)>;
    occ = occupancy_step_tma<S>(h->grid, variant);
    return 0;
  });
  const long long slots = (long long)std::max(occ, 1) * std::max(1, h->num_sms);
  auto waves = [&](int r) { return ((long long)bx * ((h->p.ny + r - 1) / r) + slots - 1) / slots; };
  if (waves(r0) >= 3) return r0;
  int best = r0;
  long long cost = waves(r0) * (r0 + 2);
  for (int r = 2; r <= std::min(h->p.ny, 64); ++r) {
    const long long c = waves(r) * (r + 2);
    if (c < cost) {
      cost = c;
      best = r;
    }
  }
  return best;
}

int auto_rows(const lbm_handle* h, int variant) {
  const int W = block_cols(variant);
  const int bx = (h->p.nx + W - 1) / W;
  int occ = 0;
  dispatch(h->p.precision, [&](auto* tag) {
    using S = std::remove_pointer_t<decltype(tag)>;
    if (variant >= 64) {
      const size_t smem = 3 * (size_t)variant * sizeof(typename Io<S>::C);
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, step_kernel<S>, variant, smem);
    } else {
      occ = occupancy_step_tma<S>(h->grid, variant);
    }
    return 0;
  });
  if (occ < 1) occ = 1;
  const long long slots = (long long)occ * std::max(1, h->num_sms);
  long long by = std::max(1LL, slots / bx);
  int rows = (int)((h->p.ny + by - 1) / by);
  rows = std::max(rows, 8);
  return std::min(rows, h->p.ny);
}

}  // namespace

extern "C" {

int64_t lbm_state_bytes(const lbm_params* p) {
  std::string why;
  int rc = validate(p, why);
  if (rc != LBM_OK) return rc;
  return (int64_t)(2 * buffer_bytes(p));
}

int lbm_create(const lbm_params* p, void* cuda_stream, lbm_handle** out) {
  return create_impl(p, cuda_stream, nullptr, 0, out);
}

int lbm_create_in(const lbm_params* p, void* cuda_stream, void* device_buffer, int64_t bytes,
                  lbm_handle** out) {
  if (!device_buffer) return fail(nullptr, LBM_ERR_PARAM, "device_buffer is NULL");
  return create_impl(p, cuda_stream, device_buffer, bytes, out);
}

int lbm_init_device(lbm_handle* h, const double* rho, const double* ux, const double* uy,
                    const double* T) {
  if (!h) return LBM_ERR_PARAM;
  if (!rho || !ux || !uy || !T) return fail(h, LBM_ERR_PARAM, "NULL field pointer");
  const long long n = (long long)h->p.nx * h->p.ny;
  h->cur = 0;
  Grid g = h->grid;
  void* dst = buf_ptr(h, 0);
  const double invT0 = 1.0 / h->p.T0;
  dispatch(h->p.precision, [&](auto* tag) {
    using S = std::remove_pointer_t<decltype(tag)>;
    init_kernel<S><<<grid_blocks(n), 256, 0, h->stream>>>(g, static_cast<S*>(dst), rho, ux, uy,
                                                           T, invT0);
    return 0;
  });
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(h, e, "init kernel launch");
  h->steps = 0;
  h->ready = true;
  h->lost = false;
  return LBM_OK;
}

namespace {

// Row chunks of the host transfers: [y0, y1) of chunk k of kc.
constexpr int XFER_CHUNKS = 8;
void chunk_rows(int ny, int k, int kc, int& y0, int& y1) {
  const int per = (ny + kc - 1) / kc;
  y0 = std::min(ny, k * per);
  y1 = std::min(ny, y0 + per);
}

}  // namespace

int lbm_init(lbm_handle* h, const double* rho, const double* ux, const double* uy,
             const double* T) {
  if (!h) return LBM_ERR_PARAM;
  if (!rho || !ux || !uy || !T) return fail(h, LBM_ERR_PARAM, "NULL field pointer");
  const size_t n = (size_t)h->p.nx * h->p.ny;
  int rc = ensure_staging(h, 4 * n * sizeof(double));
  if (rc) return rc;
  // row chunks: the four fields' rows of chunk k are copied on the transfer
  // stream, then chunk k is initialised on the handle's stream while chunk
  // k + 1 is copied.  The transfer stream first waits for the work already
  // on the handle's stream (which may still read the staging).
  cudaError_t e = cudaEventRecord(h->chunk_ev[0], h->stream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(h->xfer, h->chunk_ev[0], 0);
  const double* src[4] = {rho, ux, uy, T};
  Grid g = h->grid;
  void* dst = buf_ptr(h, 0);
  const double invT0 = 1.0 / h->p.T0;
  const int kc = std::min(XFER_CHUNKS, h->p.ny);
  for (int k = 0; k < kc && e == cudaSuccess; ++k) {
    int y0, y1;
    chunk_rows(h->p.ny, k, kc, y0, y1);
    if (y1 <= y0) continue;
    const long long i0 = (long long)y0 * h->p.nx, i1 = (long long)y1 * h->p.nx;
    for (int f = 0; f < 4 && e == cudaSuccess; ++f)
      e = cudaMemcpyAsync(h->staging + f * n + i0, src[f] + i0, (i1 - i0) * sizeof(double),
                          cudaMemcpyHostToDevice, h->xfer);
    if (e == cudaSuccess) e = cudaEventRecord(h->chunk_ev[k], h->xfer);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(h->stream, h->chunk_ev[k], 0);
    if (e != cudaSuccess) break;
    const double* st = h->staging;
    dispatch(h->p.precision, [&](auto* tag) {
      using S = std::remove_pointer_t<decltype(tag)>;
      init_kernel<S><<<grid_blocks(i1 - i0), 256, 0, h->stream>>>(
          g, static_cast<S*>(dst), st, st + n, st + 2 * n, st + 3 * n, invT0, i0, i1);
      return 0;
    });
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) {
    cudaStreamSynchronize(h->xfer);
    return cuda_fail(h, e, "host-to-device transfer or init kernel");
  }
  h->cur = 0;
  h->steps = 0;
  h->ready = true;
  h->lost = false;
  return lbm_sync(h);
}

namespace {

// Steps that a cached CUDA graph replays at once (even: the buffer parity is
// the same after it).
constexpr int GRAPH_STEPS = 32;

int step_rows(lbm_handle* h) {
  if (h->rows <= 0 && h->auto_rows == 0)
    h->auto_rows = h->variant >= 64 ? auto_rows(h, h->variant) : tma_rows(h, h->variant);
  return h->rows > 0 ? h->rows : h->auto_rows;
}

// Enqueue n steps on `stream` (the step kernel, then the second pass of the
// open sides and of the walls of non-equilibrium extrapolation).
cudaError_t enqueue_steps(lbm_handle* h, int64_t n, cudaStream_t stream) {
  const int variant = h->variant;
  const int rows = step_rows(h);
  const int W = block_cols(variant);
  const int npt = variant >= 64 ? 1 : tma_npt(variant);
  dim3 grid((h->p.nx + W - 1) / W, (h->p.ny + rows - 1) / rows);
  for (int64_t s = 0; s < n; ++s) {
    Grid g = h->grid;
    g.src = buf_ptr(h, h->cur);
    g.dst = buf_ptr(h, 1 - h->cur);
    g.t = (unsigned)h->steps;
    const CUtensorMap& map = h->maps[h->cur][npt - 1];
    cudaError_t e = cudaSuccess;
    dispatch(h->p.precision, [&](auto* tag) {
      using S = std::remove_pointer_t<decltype(tag)>;
      if (variant >= 64) {
        const size_t smem = 3 * (size_t)variant * sizeof(typename Io<S>::C);
        step_kernel<S><<<grid, variant, smem, stream>>>(g, rows);
        e = cudaGetLastError();
      } else {
        e = launch_step_tma<S>(g, map, variant, rows, grid, stream);
      }
      if (e == cudaSuccess && (g.bc[0] == BC_INLET || g.bc[1] == BC_OUTLET || g.nee)) {
        // open sides and walls of NEE: their ghost slots of the state just
        // written
        const int units = std::max(h->p.ny, g.nee ? nee_ghosts(g) : 0);
        const int blocks = std::min((units + 127) / 128, 1024);
        side_fixup_kernel<S><<<blocks, 128, 0, stream>>>(g, static_cast<const S*>(g.src),
                                                         static_cast<S*>(g.dst));
        e = cudaGetLastError();
      }
      return 0;
    });
    if (e != cudaSuccess) return e;
    h->cur = 1 - h->cur;
    ++h->steps;
  }
  return cudaSuccess;
}

// Replaying a graph is exact where the launches of a step do not depend on
// the step count: FP32 and FP64 storage (no stochastic rounding) without an
// inlet (whose phase follows the step count).
bool graphable(const lbm_handle* h) {
  return (h->p.precision == LBM_P_FP64 || h->p.precision == LBM_P_FP32) &&
         h->p.bc[0] != LBM_BC_INLET && h->p.bc[1] != LBM_BC_OUTLET;
}

void drop_step_graphs(lbm_handle* h) {
  for (auto& gx : h->graph) {
    if (gx) cudaGraphExecDestroy(gx);
    gx = nullptr;
  }
}

// The graph of GRAPH_STEPS steps from the current buffer, captured on a
// private stream (the handle's may be the legacy default stream).
cudaError_t step_graph(lbm_handle* h, cudaGraphExec_t* out) {
  cudaGraphExec_t& gx = h->graph[h->cur];
  if (!gx) {
    cudaStream_t cs;
    cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e != cudaSuccess) return e;
    const int cur = h->cur;
    const int64_t steps = h->steps;
    cudaGraph_t graph = nullptr;
    e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      const cudaError_t e1 = enqueue_steps(h, GRAPH_STEPS, cs);
      const cudaError_t e2 = cudaStreamEndCapture(cs, &graph);
      e = e1 != cudaSuccess ? e1 : e2;
    }
    h->cur = cur;
    h->steps = steps;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&gx, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    cudaStreamDestroy(cs);
    if (e != cudaSuccess) {
      gx = nullptr;
      return e;
    }
  }
  *out = gx;
  return cudaSuccess;
}

}  // namespace

int lbm_step(lbm_handle* h, int64_t n) {
  if (!h) return LBM_ERR_PARAM;
  if (n < 0) return fail(h, LBM_ERR_PARAM, "n must be >= 0");
  if (!h->ready) return fail(h, LBM_ERR_STATE, "lbm_step before lbm_init");
  if (h->lost) return fail(h, LBM_ERR_STATE, "state lost after a timeout: reload it");
  // long runs of identical launches: replay a captured graph of
  // GRAPH_STEPS steps (it saves the host most of a launch per step)
  while (n >= GRAPH_STEPS && graphable(h)) {
    cudaGraphExec_t gx;
    cudaError_t e = step_graph(h, &gx);
    if (e == cudaSuccess) e = cudaGraphLaunch(gx, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "step graph");
    h->steps += GRAPH_STEPS;
    n -= GRAPH_STEPS;
  }
  const cudaError_t e = enqueue_steps(h, n, h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "step kernel launch");
  return LBM_OK;
}

static int export_impl(lbm_handle* h, double* rho, double* ux, double* uy, double* T,
                       double* pops, int* nonfinite = nullptr) {
  const long long n = (long long)h->p.nx * h->p.ny;
  Grid g = h->grid;
  const void* src = buf_ptr(h, h->cur);
  const double T0 = h->p.T0;
  dispatch(h->p.precision, [&](auto* tag) {
    using S = std::remove_pointer_t<decltype(tag)>;
    export_kernel<S><<<grid_blocks(n), 256, 0, h->stream>>>(g, static_cast<const S*>(src), rho,
                                                             ux, uy, T, T0, pops, nonfinite);
    return 0;
  });
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(h, e, "export kernel launch");
  return LBM_OK;
}

int lbm_moments_device(lbm_handle* h, double* rho, double* ux, double* uy, double* T) {
  if (!h) return LBM_ERR_PARAM;
  if (!h->ready) return fail(h, LBM_ERR_STATE, "lbm_moments before lbm_init");
  if (h->lost) return fail(h, LBM_ERR_STATE, "state lost after a timeout: reload it");
  if (!rho || !ux || !uy || !T) return fail(h, LBM_ERR_PARAM, "NULL output pointer");
  return export_impl(h, rho, ux, uy, T, nullptr);
}

int lbm_moments(lbm_handle* h, double* rho, double* ux, double* uy, double* T) {
  if (!h) return LBM_ERR_PARAM;
  if (!h->ready) return fail(h, LBM_ERR_STATE, "lbm_moments before lbm_init");
  if (h->lost) return fail(h, LBM_ERR_STATE, "state lost after a timeout: reload it");
  if (!rho || !ux || !uy || !T) return fail(h, LBM_ERR_PARAM, "NULL output pointer");
  const size_t n = (size_t)h->p.nx * h->p.ny;
  int rc = ensure_staging(h, 4 * n * sizeof(double));
  if (rc) return rc;
  // row chunks: chunk k is exported on the handle's stream (after the steps
  // enqueued there), then copied to the host on the transfer stream while
  // chunk k + 1 is exported
  cudaError_t e = cudaMemsetAsync(h->nonfinite, 0, sizeof(int), h->stream);
  double* dst[4] = {rho, ux, uy, T};
  Grid g = h->grid;
  const void* src = buf_ptr(h, h->cur);
  const double T0 = h->p.T0;
  const int kc = std::min(XFER_CHUNKS, h->p.ny);
  for (int k = 0; k < kc && e == cudaSuccess; ++k) {
    int y0, y1;
    chunk_rows(h->p.ny, k, kc, y0, y1);
    if (y1 <= y0) continue;
    const long long i0 = (long long)y0 * h->p.nx, i1 = (long long)y1 * h->p.nx;
    double* st = h->staging;
    int* flag = h->nonfinite;
    dispatch(h->p.precision, [&](auto* tag) {
      using S = std::remove_pointer_t<decltype(tag)>;
      export_kernel<S><<<grid_blocks(i1 - i0), 256, 0, h->stream>>>(
          g, static_cast<const S*>(src), st, st + n, st + 2 * n, st + 3 * n, T0, nullptr, flag,
          i0, i1);
      return 0;
    });
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventRecord(h->chunk_ev[k], h->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(h->xfer, h->chunk_ev[k], 0);
    for (int f = 0; f < 4 && e == cudaSuccess; ++f)
      e = cudaMemcpyAsync(dst[f] + i0, h->staging + f * n + i0, (i1 - i0) * sizeof(double),
                          cudaMemcpyDeviceToHost, h->xfer);
  }
  int bad = 0;
  if (e == cudaSuccess)  // the last chunk's event orders the flag after every export
    e = cudaMemcpyAsync(&bad, h->nonfinite, sizeof(int), cudaMemcpyDeviceToHost, h->xfer);
  const cudaError_t es = cudaStreamSynchronize(h->xfer);
  if (e == cudaSuccess) e = es;
  if (e != cudaSuccess) return cuda_fail(h, e, "export kernel or device-to-host transfer");
  rc = lbm_sync(h);
  if (rc) return rc;
  if (bad) return fail(h, LBM_ERR_NONFINITE, "non-finite moment");
  return LBM_OK;
}

int lbm_conserved(lbm_handle* h, double out[4]) {
  if (!h) return LBM_ERR_PARAM;
  if (!h->ready) return fail(h, LBM_ERR_STATE, "lbm_conserved before lbm_init");
  if (h->lost) return fail(h, LBM_ERR_STATE, "state lost after a timeout: reload it");
  if (!out) return fail(h, LBM_ERR_PARAM, "out is NULL");
  const long long n = (long long)h->p.nx * h->p.ny;
  const int nb = (int)std::min<long long>(RED_BLOCKS, (n + RED_THREADS - 1) / RED_THREADS);
  Grid g = h->grid;
  const void* src = buf_ptr(h, h->cur);
  dispatch(h->p.precision, [&](auto* tag) {
    using S = std::remove_pointer_t<decltype(tag)>;
    conserved_partial_kernel<S><<<nb, RED_THREADS, 0, h->stream>>>(
        g, static_cast<const S*>(src), h->partial);
    return 0;
  });
  conserved_final_kernel<><<<1, RED_THREADS, 0, h->stream>>>(h->partial, nb, h->out4);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(h, e, "reduction launch");
  e = cudaMemcpyAsync(out, h->out4, 4 * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "device-to-host copy");
  int rc = lbm_sync(h);
  if (rc) return rc;
  for (int k = 0; k < 4; ++k)
    if (!std::isfinite(out[k])) return fail(h, LBM_ERR_NONFINITE, "non-finite sum");
  return LBM_OK;
}

int lbm_get_state(lbm_handle* h, double* pops) {
  if (!h) return LBM_ERR_PARAM;
  if (!h->ready) return fail(h, LBM_ERR_STATE, "lbm_get_state before lbm_init");
  if (h->lost) return fail(h, LBM_ERR_STATE, "state lost after a timeout: reload it");
  if (!pops) return fail(h, LBM_ERR_PARAM, "pops is NULL");
  const size_t n = (size_t)h->p.nx * h->p.ny;
  int rc = ensure_staging(h, NPOP * n * sizeof(double));
  if (rc) return rc;
  rc = export_impl(h, nullptr, nullptr, nullptr, nullptr, h->staging);
  if (rc) return rc;
  cudaError_t e = cudaMemcpyAsync(pops, h->staging, NPOP * n * sizeof(double),
                                  cudaMemcpyDeviceToHost, h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "device-to-host copy");
  return lbm_sync(h);
}

int lbm_set_state(lbm_handle* h, const double* pops) {
  if (!h) return LBM_ERR_PARAM;
  if (!pops) return fail(h, LBM_ERR_PARAM, "pops is NULL");
  const long long n = (long long)h->p.nx * h->p.ny;
  int rc = ensure_staging(h, NPOP * (size_t)n * sizeof(double));
  if (rc) return rc;
  cudaError_t e = cudaMemcpyAsync(h->staging, pops, NPOP * (size_t)n * sizeof(double),
                                  cudaMemcpyHostToDevice, h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "host-to-device copy");
  h->cur = 0;
  Grid g = h->grid;
  void* dst = buf_ptr(h, 0);
  const double* staged = h->staging;
  dispatch(h->p.precision, [&](auto* tag) {
    using S = std::remove_pointer_t<decltype(tag)>;
    set_state_kernel<S><<<grid_blocks(n), 256, 0, h->stream>>>(g, static_cast<S*>(dst), staged);
    return 0;
  });
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(h, e, "set-state launch");
  h->steps = 0;
  h->ready = true;
  h->lost = false;
  return lbm_sync(h);
}

int lbm_sync(lbm_handle* h) {
  if (!h) return LBM_ERR_PARAM;
  int st = 0;
  cudaError_t e = cudaMemcpyAsync(&st, h->status, sizeof(int), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "stream synchronize");
  if (st != 0) {
    cudaMemsetAsync(h->status, 0, sizeof(int), h->stream);
    cudaStreamSynchronize(h->stream);
    if (st & 2) {
      h->lost = true;
      return fail(h, LBM_ERR_TIMEOUT,
                  "a step kernel gave up waiting for a staged row and left with copies in "
                  "flight; the state is lost until lbm_init/lbm_set_state reloads it");
    }
    return fail(h, LBM_ERR_TIMEOUT, "a step kernel gave up waiting for a staged row");
  }
  return LBM_OK;
}

int64_t lbm_steps_done(const lbm_handle* h) { return h ? h->steps : LBM_ERR_PARAM; }

int lbm_set_steps_done(lbm_handle* h, int64_t t) {
  if (!h) return LBM_ERR_PARAM;
  if (t < 0) return fail(h, LBM_ERR_PARAM, "step count must be >= 0");
  h->steps = t;
  return LBM_OK;
}

int lbm_set_launch(lbm_handle* h, int32_t variant, int32_t rows_per_block) {
  if (!h) return LBM_ERR_PARAM;
  if ((variant > 2 && (variant < 64 || variant > 256 || variant % 32 != 0)) || variant < 0 ||
      rows_per_block < 0)
    return fail(h, LBM_ERR_PARAM,
                "variant must be 0, 1, 2 or a multiple of 32 in [64, 256]; rows >= 0");
  if (variant == TMA_PR_2 && (h->p.collision == LBM_COLL_MRT || h->p.mu_law != LBM_MU_TAU))
    return fail(h, LBM_ERR_PARAM,
                "variant 2 (two nodes per thread) is built for BGK with constant tau only");
  h->variant = variant == 0 ? TMA_PR_1 : variant;
  h->rows = rows_per_block;
  h->auto_rows = 0;
  drop_step_graphs(h);
  return LBM_OK;
}

void lbm_destroy(lbm_handle* h) {
  if (!h) return;
  cudaStreamSynchronize(h->stream);
  drop_step_graphs(h);
  if (h->owns && h->base) cudaFree(h->base);
  if (h->partial) cudaFree(h->partial);
  if (h->xfer) {
    cudaStreamSynchronize(h->xfer);
    cudaStreamDestroy(h->xfer);
  }
  for (int k = 0; k < 8; ++k)
    if (h->chunk_ev[k]) cudaEventDestroy(h->chunk_ev[k]);
  if (h->staging) cudaFree(h->staging);
  delete h;
}

const char* lbm_last_error(const lbm_handle* h) {
  if (!h) return g_create_error.c_str();
  return h->err.c_str();
}

const char* lbm_status_string(int status) {
  switch (status) {
    case LBM_OK: return "LBM_OK";
    case LBM_ERR_PARAM: return "LBM_ERR_PARAM";
    case LBM_ERR_OOM: return "LBM_ERR_OOM";
    case LBM_ERR_CUDA: return "LBM_ERR_CUDA";
    case LBM_ERR_NONFINITE: return "LBM_ERR_NONFINITE";
    case LBM_ERR_TIMEOUT: return "LBM_ERR_TIMEOUT";
    case LBM_ERR_STATE: return "LBM_ERR_STATE";
    default: return "LBM_ERR_UNKNOWN";
  }
}

}  // extern "C"
