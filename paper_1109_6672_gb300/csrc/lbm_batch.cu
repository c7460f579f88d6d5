// Host side of the batched C ABI (include/lbm.h, lbm_batch_*): a device pool
// with first-fit placement (admission by footprint), slot bookkeeping, the work
// list, CUDA-graph segments and the autotuner of the launch schedule.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "lbm.h"
#include "lbm_batch.cuh"
#include "lbm_open.cuh"
#include "lbm_host.h"
#include "lbm_launch.h"

using namespace lbm;

struct lbm_batch {
  int precision = LBM_P_FP32_BF16;
  int max_grids = 0;
  cudaStream_t stream = nullptr;
  bool owns_stream = false;
  int device = 0, num_sms = 0;
  // pool: [offset -> size] of free ranges
  void* pool = nullptr;
  size_t pool_bytes = 0;
  bool owns_pool = false;
  std::map<size_t, size_t> free_ranges;
  struct Slot {
    bool used = false;
    lbm_params p{};
    size_t off = 0, bytes = 0;
    long long steps = 0, remaining = 0;
  };
  std::vector<Slot> slots;
  std::vector<BatchGrid> h_grids;
  std::vector<WorkItem> h_items;
  BatchGrid* d_grids = nullptr;
  WorkItem* d_items = nullptr;
  size_t item_cap = 0;
  BatchCtl* d_ctl = nullptr;
  int* d_status = nullptr;
  bool lost = false;  // a step left with copies in flight: every state is suspect
  double* staging = nullptr;
  size_t staging_bytes = 0;
  bool items_dirty = true;
  // launch schedule (autotuned)
  int rows = 0;      // 0: per-precision default
  int dynamic = 1;   // atomic work queue
  std::vector<int> modes;        // physics modes present in the work list
  bool has_fix = false;          // a grid with an open side or a wall of NEE is active
  int occ_mode[BATCH_MODE_SLOTS] = {0};  // resident blocks per SM per mode (0: not queried)
  std::map<std::pair<int64_t, std::vector<int>>, cudaGraphExec_t> graphs;
  std::string err;
};

namespace {

// A batch at step j of its segment: block b takes grid b if it has an open
// side or a wall of NEE and steps at j (it read buffer (t0 + j) mod 2 and
// wrote the other).
template <class S>
__global__ void __launch_bounds__(128)
    batch_side_fixup_kernel(const BatchGrid* __restrict__ grids, int j) {
  __shared__ Grid s_grid;
  const BatchGrid& bg = grids[blockIdx.x];
  if (j >= bg.seg_steps || (bg.g.bc[0] != BC_INLET && bg.g.bc[1] != BC_OUTLET && !bg.g.nee))
    return;
  const int* gsrc = reinterpret_cast<const int*>(&bg.g);
  int* gdst = reinterpret_cast<int*>(&s_grid);
  for (int i = threadIdx.x; i < (int)(sizeof(Grid) / sizeof(int)); i += blockDim.x)
    gdst[i] = gsrc[i];
  __syncthreads();
  if (threadIdx.x == 0) s_grid.t = (unsigned)(bg.t0 + j);
  __syncthreads();
  const int par = (int)((bg.t0 + j) & 1);
  fixup_grid<S>(s_grid, static_cast<const S*>(bg.buf[par]), static_cast<S*>(bg.buf[par ^ 1]),
                threadIdx.x, blockDim.x);
}


thread_local std::string g_batch_create_error;

int bfail(lbm_batch* b, int code, const std::string& msg) {
  if (b)
    b->err = msg;
  else
    g_batch_create_error = msg;
  return code;
}

size_t elem_bytes(int precision) {
  return precision == LBM_P_FP64 ? 8 : (precision == LBM_P_FP32 ? 4 : 2);
}

template <class F>
cudaError_t by_precision(int precision, F&& f) {
  switch (precision) {
    case LBM_P_FP64: return f((double*)nullptr);
    case LBM_P_FP32: return f((float*)nullptr);
    case LBM_P_FP32_FP16: return f((__half*)nullptr);
    default: return f((__nv_bfloat16*)nullptr);
  }
}

bool pool_alloc(lbm_batch* b, size_t bytes, size_t* off) {
  bytes = (bytes + 255) / 256 * 256;
  for (auto it = b->free_ranges.begin(); it != b->free_ranges.end(); ++it) {
    if (it->second >= bytes) {
      *off = it->first;
      const size_t rest = it->second - bytes;
      const size_t next = it->first + bytes;
      b->free_ranges.erase(it);
      if (rest) b->free_ranges[next] = rest;
      return true;
    }
  }
  return false;
}

void pool_free(lbm_batch* b, size_t off, size_t bytes) {
  bytes = (bytes + 255) / 256 * 256;
  auto it = b->free_ranges.emplace(off, bytes).first;
  auto nx = std::next(it);
  if (nx != b->free_ranges.end() && it->first + it->second == nx->first) {
    it->second += nx->second;
    b->free_ranges.erase(nx);
  }
  if (it != b->free_ranges.begin()) {
    auto pv = std::prev(it);
    if (pv->first + pv->second == it->first) {
      pv->second += it->second;
      b->free_ranges.erase(it);
    }
  }
}

int rows_of(const lbm_batch* b) {
  return b->rows > 0 ? b->rows : tma_default_rows(elem_bytes(b->precision));
}

// Work list: every (grid, strip, row block) of the active grids, largest grids
// first so that the long items start early.
int rebuild_items(lbm_batch* b) {
  std::vector<int> order;
  for (int s = 0; s < (int)b->slots.size(); ++s)
    if (b->slots[s].used) order.push_back(s);
  std::sort(order.begin(), order.end(), [&](int a, int c) {
    const int ma = mode_slot(b->h_grids[a].mode), mc = mode_slot(b->h_grids[c].mode);
    if (ma != mc) return ma < mc;
    const long long na = (long long)b->slots[a].p.nx * b->slots[a].p.ny;
    const long long nc = (long long)b->slots[c].p.nx * b->slots[c].p.ny;
    return na != nc ? na > nc : a < c;
  });
  const int rows = rows_of(b);
  b->h_items.clear();
  int begin[BATCH_MODE_SLOTS], end[BATCH_MODE_SLOTS];
  for (int m = 0; m < BATCH_MODE_SLOTS; ++m) begin[m] = end[m] = 0;
  b->modes.clear();
  b->has_fix = false;
  for (int s : order) {
    b->has_fix |= b->slots[s].p.bc[0] == LBM_BC_INLET || b->slots[s].p.bc[1] == LBM_BC_OUTLET ||
                  b->slots[s].p.wall_nee != 0;
    const lbm_params& p = b->slots[s].p;
    const int mode = b->h_grids[s].mode, ms = mode_slot(mode);
    if (b->modes.empty() || b->modes.back() != mode) {
      b->modes.push_back(mode);
      begin[ms] = (int)b->h_items.size();
    }
    for (int y0 = 0; y0 < p.ny; y0 += rows)
      for (int x0 = 0; x0 < p.nx; x0 += tma_cols(TMA_PR_1))
        b->h_items.push_back(WorkItem{s, x0, y0, std::min(rows, p.ny - y0)});
    end[ms] = (int)b->h_items.size();
  }
  if (b->h_items.size() > b->item_cap) {
    if (b->d_items) cudaFree(b->d_items);
    b->item_cap = std::max<size_t>(b->h_items.size() * 2, 1024);
    if (cudaMalloc(&b->d_items, b->item_cap * sizeof(WorkItem)) != cudaSuccess) {
      b->d_items = nullptr;
      b->item_cap = 0;
      return bfail(b, LBM_ERR_OOM, "work list allocation failed");
    }
  }
  if (!b->h_items.empty() &&
      cudaMemcpyAsync(b->d_items, b->h_items.data(), b->h_items.size() * sizeof(WorkItem),
                      cudaMemcpyHostToDevice, b->stream) != cudaSuccess)
    return bfail(b, LBM_ERR_CUDA, "work list upload failed");
  int hdr[2 * BATCH_MODE_SLOTS + 1];
  for (int m = 0; m < BATCH_MODE_SLOTS; ++m) {
    hdr[m] = begin[m];
    hdr[BATCH_MODE_SLOTS + m] = end[m];
  }
  hdr[2 * BATCH_MODE_SLOTS] = b->dynamic;
  static_assert(offsetof(BatchCtl, dynamic) == 2 * BATCH_MODE_SLOTS * sizeof(int),
                "control header layout");
  if (cudaMemcpyAsync(b->d_ctl, hdr, sizeof(hdr), cudaMemcpyHostToDevice, b->stream) !=
      cudaSuccess)
    return bfail(b, LBM_ERR_CUDA, "control upload failed");
  // the host vectors must outlive the copies
  if (cudaStreamSynchronize(b->stream) != cudaSuccess)
    return bfail(b, LBM_ERR_CUDA, "work list upload failed");
  b->items_dirty = false;
  return LBM_OK;
}

int upload_grids(lbm_batch* b) {
  if (cudaMemcpyAsync(b->d_grids, b->h_grids.data(), b->h_grids.size() * sizeof(BatchGrid),
                      cudaMemcpyHostToDevice, b->stream) != cudaSuccess)
    return bfail(b, LBM_ERR_CUDA, "descriptor upload failed");
  return cudaStreamSynchronize(b->stream) == cudaSuccess
             ? LBM_OK
             : bfail(b, LBM_ERR_CUDA, "descriptor upload failed");
}

int blocks_of(lbm_batch* b, int mode) {
  int& occ = b->occ_mode[mode_slot(mode)];
  if (!occ) {
    by_precision(b->precision, [&](auto* tag) {
      using S = std::remove_pointer_t<decltype(tag)>;
      occ = std::max(1, occupancy_batch<S>(mode));
      return cudaSuccess;
    });
  }
  return std::max(1, occ * b->num_sms);
}

// One step j of every mode group on the batch's stream.
cudaError_t launch_all_modes(lbm_batch* b, int j) {
  cudaError_t e = cudaSuccess;
  for (int mode : b->modes) {
    const int blocks = blocks_of(b, mode);
    e = by_precision(b->precision, [&](auto* tag) {
      using S = std::remove_pointer_t<decltype(tag)>;
      return launch_batch_step<S>(b->d_grids, b->d_items, b->d_ctl, j, mode, blocks, b->stream);
    });
    if (e != cudaSuccess) break;
  }
  if (e == cudaSuccess && b->has_fix) {
    // open sides and walls of NEE: their ghost slots, once every grid has
    // taken step j
    e = by_precision(b->precision, [&](auto* tag) {
      using S = std::remove_pointer_t<decltype(tag)>;
      batch_side_fixup_kernel<S><<<b->max_grids, 128, 0, b->stream>>>(b->d_grids, j);
      return cudaGetLastError();
    });
  }
  return e;
}

int* counters_of(lbm_batch* b) {
  return reinterpret_cast<int*>(reinterpret_cast<char*>(b->d_ctl) + offsetof(BatchCtl, counters));
}

// Graph of k steps (j = 0 .. k-1; one launch per physics mode present, plus
// the open-side fix-up when a grid has one) preceded by a reset of the
// counters.  Cached per (k, modes present, open sides present).
int graph_for(lbm_batch* b, int64_t k, cudaGraphExec_t* out) {
  auto key = std::make_pair(k, b->modes);
  if (b->has_fix) key.second.push_back(-1);
  auto it = b->graphs.find(key);
  if (it != b->graphs.end()) {
    *out = it->second;
    return LBM_OK;
  }
  for (int mode : b->modes) blocks_of(b, mode);  // occupancy queries before capture
  cudaGraph_t graph;
  if (cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
    return bfail(b, LBM_ERR_CUDA, "stream capture failed to start");
  const size_t counter_bytes = sizeof(int) * BATCH_MODE_SLOTS * BATCH_MAX_SEG;
  cudaError_t e = cudaMemsetAsync(counters_of(b), 0, counter_bytes, b->stream);
  for (int64_t j = 0; j < k && e == cudaSuccess; ++j) e = launch_all_modes(b, (int)j);
  cudaError_t e2 = cudaStreamEndCapture(b->stream, &graph);
  if (e != cudaSuccess || e2 != cudaSuccess)
    return bfail(b, LBM_ERR_CUDA, std::string("graph capture failed: ") +
                                      cudaGetErrorString(e != cudaSuccess ? e : e2));
  cudaGraphExec_t exec;
  e = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return bfail(b, LBM_ERR_CUDA, "graph instantiation failed");
  b->graphs[key] = exec;
  *out = exec;
  return LBM_OK;
}

void drop_graphs(lbm_batch* b) {
  for (auto& kv : b->graphs) cudaGraphExecDestroy(kv.second);
  b->graphs.clear();
}

int check_status(lbm_batch* b) {
  int st = 0;
  if (cudaMemcpy(&st, b->d_status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
    return bfail(b, LBM_ERR_CUDA, "status read failed");
  if (st) {
    cudaMemset(b->d_status, 0, sizeof(int));
    if (st & 2) {
      b->lost = true;
      return bfail(b, LBM_ERR_TIMEOUT,
                   "a batched step gave up waiting for a staged row and left with copies in "
                   "flight; the batch's states are lost (destroy the batch)");
    }
    return bfail(b, LBM_ERR_TIMEOUT, "a batched step gave up waiting for a staged row");
  }
  return LBM_OK;
}

int ensure_staging(lbm_batch* b, size_t bytes) {
  if (b->staging_bytes >= bytes) return LBM_OK;
  if (b->staging) cudaFree(b->staging);
  b->staging = nullptr;
  b->staging_bytes = 0;
  if (cudaMalloc(&b->staging, bytes) != cudaSuccess)
    return bfail(b, LBM_ERR_OOM, "staging allocation failed");
  b->staging_bytes = bytes;
  return LBM_OK;
}

int create_impl(int precision, int max_grids, void* pool, int64_t pool_bytes, void* stream,
                lbm_batch** out) {
  if (!out) return bfail(nullptr, LBM_ERR_PARAM, "out is NULL");
  *out = nullptr;
  if (precision < LBM_P_FP64 || precision > LBM_P_FP32_BF16 || max_grids < 1 ||
      max_grids > (1 << 20) || pool_bytes <= 0)
    return bfail(nullptr, LBM_ERR_PARAM, "invalid precision, max_grids or pool size");
  lbm_batch* b = new lbm_batch();
  b->precision = precision;
  b->max_grids = max_grids;
  cudaGetDevice(&b->device);
  cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, b->device);
  if (stream) {
    b->stream = static_cast<cudaStream_t>(stream);
  } else {
    if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete b;
      return bfail(nullptr, LBM_ERR_CUDA, "stream creation failed");
    }
    b->owns_stream = true;
  }
  b->pool_bytes = (size_t)pool_bytes / 256 * 256;
  if (pool) {
    if (reinterpret_cast<uintptr_t>(pool) & 255u) {
      lbm_batch_destroy(b);
      return bfail(nullptr, LBM_ERR_PARAM, "device_pool must be 256-byte aligned");
    }
    b->pool = pool;
  } else {
    if (cudaMalloc(&b->pool, b->pool_bytes) != cudaSuccess) {
      cudaGetLastError();
      b->pool = nullptr;
      lbm_batch_destroy(b);
      return bfail(nullptr, LBM_ERR_OOM, "pool allocation failed");
    }
    b->owns_pool = true;
  }
  b->free_ranges[0] = b->pool_bytes;
  b->slots.resize(max_grids);
  b->h_grids.resize(max_grids);
  std::memset(b->h_grids.data(), 0, sizeof(BatchGrid) * max_grids);
  if (cudaMalloc(&b->d_grids, sizeof(BatchGrid) * max_grids) != cudaSuccess ||
      cudaMalloc(&b->d_ctl, sizeof(BatchCtl)) != cudaSuccess ||
      cudaMalloc(&b->d_status, sizeof(int)) != cudaSuccess) {
    lbm_batch_destroy(b);
    return bfail(nullptr, LBM_ERR_OOM, "descriptor allocation failed");
  }
  cudaMemset(b->d_ctl, 0, sizeof(BatchCtl));
  cudaMemset(b->d_status, 0, sizeof(int));
  *out = b;
  return LBM_OK;
}

}  // namespace

extern "C" {

int lbm_batch_create(int32_t precision, int32_t max_grids, int64_t pool_bytes, void* cuda_stream,
                     lbm_batch** out) {
  return create_impl(precision, max_grids, nullptr, pool_bytes, cuda_stream, out);
}

int lbm_batch_create_in(int32_t precision, int32_t max_grids, void* device_pool, int64_t pool_bytes,
                        void* cuda_stream, lbm_batch** out) {
  if (!device_pool) return bfail(nullptr, LBM_ERR_PARAM, "device_pool is NULL");
  return create_impl(precision, max_grids, device_pool, pool_bytes, cuda_stream, out);
}

int lbm_batch_add(lbm_batch* b, const lbm_params* p, const double* rho, const double* ux,
                  const double* uy, const double* T, int64_t steps, int32_t* slot) {
  if (!b || !slot) return LBM_ERR_PARAM;
  *slot = -1;
  std::string why;
  int rc = lbm_host::validate(p, why);
  if (rc != LBM_OK) return bfail(b, rc, why);
  if (p->precision != b->precision) return bfail(b, LBM_ERR_PARAM, "precision differs from batch");
  if (steps < 0) return bfail(b, LBM_ERR_PARAM, "steps must be >= 0");
  if (!rho || !ux || !uy || !T) return bfail(b, LBM_ERR_PARAM, "NULL field pointer");
  int s = -1;
  for (int i = 0; i < b->max_grids; ++i)
    if (!b->slots[i].used) {
      s = i;
      break;
    }
  if (s < 0) return bfail(b, LBM_ERR_OOM, "no free slot");
  const size_t buf = lbm_host::buffer_bytes(p);
  size_t off = 0;
  if (!pool_alloc(b, 2 * buf, &off)) return bfail(b, LBM_ERR_OOM, "pool has no room for this grid");
  const size_t n = (size_t)p->nx * p->ny;
  rc = ensure_staging(b, 4 * n * sizeof(double));
  if (rc) {
    pool_free(b, off, 2 * buf);
    return rc;
  }
  BatchGrid& bg = b->h_grids[s];
  std::memset(&bg, 0, sizeof(bg));
  lbm_host::fill_grid(p, bg.g);
  bg.g.status = b->d_status;
  bg.buf[0] = static_cast<unsigned char*>(b->pool) + off;
  bg.buf[1] = static_cast<unsigned char*>(b->pool) + off + buf;
  bg.mode = mode_of(bg.g);
  for (int k = 0; k < 2; ++k) {
    rc = lbm_host::make_tensor_map(&bg.maps[k], bg.buf[k], *p, bg.g, tma_box(1), 6);
    if (rc) {
      pool_free(b, off, 2 * buf);
      return bfail(b, rc, "tensor map encoding failed");
    }
  }
  // zero both buffers (defined ghost slots), then equilibrium into buffer 0
  cudaError_t e = cudaMemsetAsync(bg.buf[0], 0, 2 * buf, b->stream);
  const double* src[4] = {rho, ux, uy, T};
  for (int k = 0; k < 4 && e == cudaSuccess; ++k)
    e = cudaMemcpyAsync(b->staging + k * n, src[k], n * sizeof(double), cudaMemcpyHostToDevice,
                        b->stream);
  if (e == cudaSuccess) {
    Grid g = bg.g;
    const double invT0 = 1.0 / p->T0;
    const int blocks = (int)std::max<size_t>(1, std::min<size_t>(4096, (n + 255) / 256));
    e = by_precision(b->precision, [&](auto* tag) {
      using S = std::remove_pointer_t<decltype(tag)>;
      init_kernel<S><<<blocks, 256, 0, b->stream>>>(g, static_cast<S*>(bg.buf[0]), b->staging,
                                                    b->staging + n, b->staging + 2 * n,
                                                    b->staging + 3 * n, invT0);
      return cudaGetLastError();
    });
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) {
    pool_free(b, off, 2 * buf);
    return bfail(b, LBM_ERR_CUDA,
                 std::string("grid initialisation failed: ") + cudaGetErrorString(e));
  }
  lbm_batch::Slot& sl = b->slots[s];
  sl.used = true;
  sl.p = *p;
  sl.off = off;
  sl.bytes = 2 * buf;
  sl.steps = 0;
  sl.remaining = steps;
  b->items_dirty = true;
  *slot = s;
  return LBM_OK;
}

int lbm_batch_run(lbm_batch* b, int64_t k) {
  if (!b) return LBM_ERR_PARAM;
  if (k < 0 || k > BATCH_MAX_SEG) return bfail(b, LBM_ERR_PARAM, "k must be in [0, 4096]");
  if (b->lost) return bfail(b, LBM_ERR_STATE, "states lost after a timeout: destroy the batch");
  if (k == 0) return LBM_OK;
  int rc;
  if (b->items_dirty && (rc = rebuild_items(b))) return rc;
  bool any = false;
  for (int s = 0; s < b->max_grids; ++s) {
    BatchGrid& bg = b->h_grids[s];
    const lbm_batch::Slot& sl = b->slots[s];
    bg.t0 = sl.steps;
    bg.seg_steps = sl.used ? (int)std::min<long long>(k, sl.remaining) : 0;
    any |= bg.seg_steps > 0;
  }
  if (!any) return LBM_OK;
  if ((rc = upload_grids(b))) return rc;
  cudaGraphExec_t exec;
  if ((rc = graph_for(b, k, &exec))) return rc;
  if (cudaGraphLaunch(exec, b->stream) != cudaSuccess)
    return bfail(b, LBM_ERR_CUDA, "graph launch failed");
  if (cudaStreamSynchronize(b->stream) != cudaSuccess)
    return bfail(b, LBM_ERR_CUDA, std::string("batched step failed: ") +
                                      cudaGetErrorString(cudaGetLastError()));
  if ((rc = check_status(b))) return rc;
  for (int s = 0; s < b->max_grids; ++s) {
    lbm_batch::Slot& sl = b->slots[s];
    if (!sl.used) continue;
    const int d = b->h_grids[s].seg_steps;
    sl.steps += d;
    sl.remaining -= d;
  }
  return LBM_OK;
}

int64_t lbm_batch_remaining(const lbm_batch* b, int32_t slot) {
  if (!b || slot < 0 || slot >= b->max_grids || !b->slots[slot].used) return LBM_ERR_PARAM;
  return b->slots[slot].remaining;
}

int lbm_batch_moments(lbm_batch* b, int32_t slot, double* rho, double* ux, double* uy,
                      double* T) {
  if (!b || slot < 0 || slot >= b->max_grids || !b->slots[slot].used)
    return bfail(b, LBM_ERR_PARAM, "no such slot");
  if (!rho || !ux || !uy || !T) return bfail(b, LBM_ERR_PARAM, "NULL output pointer");
  if (b->lost) return bfail(b, LBM_ERR_STATE, "states lost after a timeout: destroy the batch");
  const lbm_batch::Slot& sl = b->slots[slot];
  const size_t n = (size_t)sl.p.nx * sl.p.ny;
  // the four fields, then the non-finite flag of export_kernel
  int rc = ensure_staging(b, 4 * n * sizeof(double) + 16);
  if (rc) return rc;
  int* flag = reinterpret_cast<int*>(b->staging + 4 * n);
  const BatchGrid& bg = b->h_grids[slot];
  Grid g = bg.g;
  const void* cur = bg.buf[sl.steps & 1];
  const double T0 = sl.p.T0;
  const int blocks = (int)std::max<size_t>(1, std::min<size_t>(4096, (n + 255) / 256));
  cudaError_t e = cudaMemsetAsync(flag, 0, sizeof(int), b->stream);
  if (e == cudaSuccess)
    e = by_precision(b->precision, [&](auto* tag) {
      using S = std::remove_pointer_t<decltype(tag)>;
      export_kernel<S><<<blocks, 256, 0, b->stream>>>(g, static_cast<const S*>(cur), b->staging,
                                                      b->staging + n, b->staging + 2 * n,
                                                      b->staging + 3 * n, T0, nullptr, flag);
      return cudaGetLastError();
    });
  double* dst[4] = {rho, ux, uy, T};
  for (int k = 0; k < 4 && e == cudaSuccess; ++k)
    e = cudaMemcpyAsync(dst[k], b->staging + k * n, n * sizeof(double), cudaMemcpyDeviceToHost,
                        b->stream);
  int bad = 0;
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&bad, flag, sizeof(int), cudaMemcpyDeviceToHost, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return bfail(b, LBM_ERR_CUDA, "moments failed");
  if (bad) return bfail(b, LBM_ERR_NONFINITE, "non-finite moment");
  return LBM_OK;
}

int lbm_batch_get_state(lbm_batch* b, int32_t slot, double* pops) {
  if (!b || slot < 0 || slot >= b->max_grids || !b->slots[slot].used || !pops)
    return bfail(b, LBM_ERR_PARAM, "no such slot or NULL output");
  if (b->lost) return bfail(b, LBM_ERR_STATE, "states lost after a timeout: destroy the batch");
  const lbm_batch::Slot& sl = b->slots[slot];
  const size_t n = (size_t)sl.p.nx * sl.p.ny;
  int rc = ensure_staging(b, NPOP * n * sizeof(double));
  if (rc) return rc;
  const BatchGrid& bg = b->h_grids[slot];
  Grid g = bg.g;
  const void* cur = bg.buf[sl.steps & 1];
  const int blocks = (int)std::max<size_t>(1, std::min<size_t>(4096, (n + 255) / 256));
  cudaError_t e = by_precision(b->precision, [&](auto* tag) {
    using S = std::remove_pointer_t<decltype(tag)>;
    export_kernel<S><<<blocks, 256, 0, b->stream>>>(g, static_cast<const S*>(cur), nullptr,
                                                    nullptr, nullptr, nullptr, 1.0, b->staging);
    return cudaGetLastError();
  });
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(pops, b->staging, NPOP * n * sizeof(double), cudaMemcpyDeviceToHost,
                        b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  return e == cudaSuccess ? LBM_OK : bfail(b, LBM_ERR_CUDA, "state export failed");
}

int lbm_batch_remove(lbm_batch* b, int32_t slot) {
  if (!b || slot < 0 || slot >= b->max_grids || !b->slots[slot].used)
    return bfail(b, LBM_ERR_PARAM, "no such slot");
  cudaStreamSynchronize(b->stream);
  lbm_batch::Slot& sl = b->slots[slot];
  pool_free(b, sl.off, sl.bytes);
  sl = lbm_batch::Slot();
  std::memset(&b->h_grids[slot], 0, sizeof(BatchGrid));
  b->items_dirty = true;
  return LBM_OK;
}

// Time one step of the current grids (without advancing them: the step reads
// the current buffers and writes the other ones, which the next real step
// overwrites) for each candidate schedule; keep the fastest.
int lbm_batch_autotune(lbm_batch* b, int32_t reps, int64_t out_best[3]) {
  if (!b || reps < 1) return LBM_ERR_PARAM;
  const int cand_rows[] = {4, 6, 8, 12, 16, 24};
  const int cand_dyn[] = {1, 0};
  float best = 1e30f;
  int best_rows = rows_of(b), best_dyn = b->dynamic;
  bool any = false;
  for (int s = 0; s < b->max_grids; ++s) {
    BatchGrid& bg = b->h_grids[s];
    bg.t0 = b->slots[s].steps;
    bg.seg_steps = b->slots[s].used ? 1 : 0;
    any |= bg.seg_steps > 0;
  }
  if (!any) return bfail(b, LBM_ERR_STATE, "no grids to tune on");
  int rc = upload_grids(b);
  if (rc) return rc;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  for (int rows : cand_rows) {
    for (int dyn : cand_dyn) {
      b->rows = rows;
      b->dynamic = dyn;
      if ((rc = rebuild_items(b))) break;
      cudaError_t e = cudaSuccess;
      for (int mode : b->modes) blocks_of(b, mode);
      for (int r = 0; r <= reps && e == cudaSuccess; ++r) {
        if (r == 1) cudaEventRecord(e0, b->stream);
        e = cudaMemsetAsync(counters_of(b), 0, sizeof(int) * BATCH_MODE_SLOTS * BATCH_MAX_SEG,
                            b->stream);
        if (e == cudaSuccess) e = launch_all_modes(b, 0);
      }
      cudaEventRecord(e1, b->stream);
      if (e != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
        rc = bfail(b, LBM_ERR_CUDA, "autotune launch failed");
        break;
      }
      float ms = 0;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best) {
        best = ms;
        best_rows = rows;
        best_dyn = dyn;
      }
    }
    if (rc) break;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  b->rows = best_rows;
  b->dynamic = best_dyn;
  b->items_dirty = true;
  drop_graphs(b);
  if (rc) return rc;
  if ((rc = check_status(b))) return rc;
  if (out_best) {
    out_best[0] = best_rows;
    out_best[1] = best_dyn;
    out_best[2] = (int64_t)std::llround(1e3 * best / reps);  // microseconds per step
  }
  return LBM_OK;
}

int lbm_batch_set_schedule(lbm_batch* b, int32_t rows, int32_t dynamic) {
  if (!b || rows < 0 || (dynamic != 0 && dynamic != 1)) return LBM_ERR_PARAM;
  b->rows = rows;
  b->dynamic = dynamic;
  b->items_dirty = true;
  drop_graphs(b);
  return LBM_OK;
}

int lbm_batch_info(const lbm_batch* b, int64_t out[6]) {
  if (!b || !out) return LBM_ERR_PARAM;
  int64_t active = 0, nodes = 0;
  for (const auto& s : b->slots)
    if (s.used) {
      ++active;
      nodes += (int64_t)s.p.nx * s.p.ny;
    }
  int64_t free_bytes = 0, largest = 0;
  for (const auto& kv : b->free_ranges) {
    free_bytes += kv.second;
    largest = std::max<int64_t>(largest, kv.second);
  }
  out[0] = active;
  out[1] = nodes;
  out[2] = free_bytes;
  out[3] = largest;
  out[4] = rows_of(b);
  out[5] = b->dynamic;
  return LBM_OK;
}

void lbm_batch_destroy(lbm_batch* b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  drop_graphs(b);
  if (b->owns_pool && b->pool) cudaFree(b->pool);
  if (b->d_grids) cudaFree(b->d_grids);
  if (b->d_items) cudaFree(b->d_items);
  if (b->d_ctl) cudaFree(b->d_ctl);
  if (b->d_status) cudaFree(b->d_status);
  if (b->staging) cudaFree(b->staging);
  if (b->owns_stream && b->stream) cudaStreamDestroy(b->stream);
  delete b;
}

const char* lbm_batch_last_error(const lbm_batch* b) {
  return b ? b->err.c_str() : g_batch_create_error.c_str();
}

}  // extern "C"
