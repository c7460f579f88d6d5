// Allocation-free variant of the conserved-sums reduction (lbm_conserved).
//
// Some callers cannot allocate device memory at the point where they need the
// sums: code running inside CUDA stream capture, serving loops whose device
// memory is owned by a pool that forbids outside allocations, and latency-
// bound paths where cudaMalloc's implicit synchronisation is not acceptable.
// This entry point takes the state buffer and the output location from the
// caller and keeps its per-block partial sums in a file-scope device array, so
// it calls no cudaMalloc, cudaFree or allocating library routine.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <mutex>
#include <string>

#include "lbm.h"
#include "lbm_device.cuh"
#include "lbm_host.h"

using namespace lbm;

namespace {

// Partial-sum slots: one quadruple (sum rho, rho u_x, rho u_y, hbar) per block
// of the first reduction pass.  32 KiB; every device that loads the library
// holds it until the process exits.
constexpr int kNoallocPartials = 1024;
static __device__ __align__(256) double g_noalloc_partials[kNoallocPartials * 4];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_partials_ptr[kMaxDevices] = {};

// Device address of the partial-sum array on `dev` (the current device).
// Looked up with that device current on the first call, and again on every
// call made outside stream capture (a host-side lookup that allocates
// nothing), so that a context recreated after cudaDeviceReset() is followed;
// a call inside a capture uses the address of the last call outside one.
cudaError_t partials_on(int dev, cudaStream_t st, double** out) {
  std::lock_guard<std::mutex> lock(g_mu);
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  const bool capturing =
      cudaStreamIsCapturing(st, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone;
  if (!capturing || !g_partials_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_partials);
    if (e != cudaSuccess) return e;
    g_partials_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_partials_ptr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" int lbm_conserved_noalloc(const lbm_params* p, const void* d_state, double* d_out,
                                     void* cuda_stream) {
  std::string why;
  int rc = lbm_host::validate(p, why);
  if (rc != LBM_OK) return rc;
  if (!d_state || (reinterpret_cast<uintptr_t>(d_state) & 255u) || !d_out ||
      (reinterpret_cast<uintptr_t>(d_out) & 7u))
    return LBM_ERR_PARAM;
  const long long n = (long long)p->nx * p->ny;
  // one partial quadruple per block of RED_THREADS nodes, at most kNoallocPartials
  // blocks (grid-stride beyond that); refuse anything that would need more
  const long long nb = std::min<long long>(kNoallocPartials, (n + RED_THREADS - 1) / RED_THREADS);
  if (nb < 1 || nb > kNoallocPartials) return LBM_ERR_PARAM;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) return LBM_ERR_CUDA;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  double* partials = nullptr;
  e = partials_on(dev, st, &partials);
  if (e != cudaSuccess) return LBM_ERR_CUDA;
  Grid g;
  lbm_host::fill_grid(p, g);
  // every slot the final pass reads is written by this call's first pass, so
  // nothing left over from an earlier call is used and nothing needs clearing
  switch (p->precision) {
    case LBM_P_FP64:
      conserved_partial_kernel<double><<<(int)nb, RED_THREADS, 0, st>>>(
          g, static_cast<const double*>(d_state), partials);
      break;
    case LBM_P_FP32:
      conserved_partial_kernel<float><<<(int)nb, RED_THREADS, 0, st>>>(
          g, static_cast<const float*>(d_state), partials);
      break;
    case LBM_P_FP32_FP16:
      conserved_partial_kernel<__half><<<(int)nb, RED_THREADS, 0, st>>>(
          g, static_cast<const __half*>(d_state), partials);
      break;
    default:
      conserved_partial_kernel<__nv_bfloat16><<<(int)nb, RED_THREADS, 0, st>>>(
          g, static_cast<const __nv_bfloat16*>(d_state), partials);
      break;
  }
  conserved_final_kernel<><<<1, RED_THREADS, 0, st>>>(partials, (int)nb, d_out);
  e = cudaGetLastError();
  return e == cudaSuccess ? LBM_OK : LBM_ERR_CUDA;
}
