// Self-test of the bounded device-side wait: one block arms an mbarrier for a
// transaction that no copy ever completes and waits on it with the bounded
// wait of the step kernels, then records the timeout in a status word the way
// they do.  The wait ends by itself; nothing faults or hangs.
#include <cuda_runtime.h>

#include <cstdint>

#include "lbm.h"
#include "lbm_step_tma.cuh"

namespace lbm {

__global__ void selftest_wait_kernel(unsigned long long limit_ns, int* status) {
  __shared__ __align__(8) unsigned long long bar;
  const unsigned b = smem_u32(&bar);
  if (threadIdx.x == 0) {
    mbar_init(b, 1);
    mbar_fence_init();
  }
  __syncthreads();
  // the one expected arrival, with 128 bytes that no copy will deliver
  if (threadIdx.x == 0) mbar_expect_tx(b, 128);
  __syncthreads();
  const bool ok = mbar_wait(b, 0, limit_ns);
  if (__syncthreads_or(!ok) && threadIdx.x == 0) atomicOr(status, 1);
}

}  // namespace lbm

extern "C" int lbm_selftest_wait(int64_t limit_ns) {
  if (limit_ns < 1000 || limit_ns > 2000000000LL) return LBM_ERR_PARAM;
  int* d_status = nullptr;
  if (cudaMalloc(&d_status, sizeof(int)) != cudaSuccess) return LBM_ERR_OOM;
  int st = 0;
  cudaError_t e = cudaMemset(d_status, 0, sizeof(int));
  if (e == cudaSuccess) {
    lbm::selftest_wait_kernel<<<1, 32>>>((unsigned long long)limit_ns, d_status);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(&st, d_status, sizeof(int), cudaMemcpyDeviceToHost);
  cudaFree(d_status);
  if (e != cudaSuccess) return LBM_ERR_CUDA;
  return st ? LBM_ERR_TIMEOUT : LBM_OK;
}
