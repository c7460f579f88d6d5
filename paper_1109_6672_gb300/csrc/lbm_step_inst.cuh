// Definitions of the launchers declared in lbm_launch.h; included by the four
// per-precision translation units.
#pragma once

#include "lbm_launch.h"
#include "lbm_batch.cuh"
#include "lbm_step_pr.cuh"

namespace lbm {

// Kernel pointer, block size and shared memory of one configuration.
template <class S, int NPT, int M>
struct Cfg {
  static constexpr int threads = PR_THREADS;
  static size_t smem() { return PrGeom<S, NPT>::smem_bytes(); }
  static auto kernel() { return step_pr_kernel<S, NPT, M>; }
};

template <class S, int NPT, int M>
cudaError_t launch_one(const Grid& g, const CUtensorMap& map, int rows, dim3 grid,
                       cudaStream_t stream, int* occ) {
  using K = Cfg<S, NPT, M>;
  static bool configured = false;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(K::kernel(), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)K::smem());
    if (e != cudaSuccess) return e;
    configured = true;
  }
  if (occ) {
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, K::kernel(), K::threads,
                                                         K::smem());
  }
  K::kernel()<<<grid, K::threads, K::smem(), stream>>>(g, map, rows);
  return cudaGetLastError();
}

template <class S, int NPT>
cudaError_t launch_mode(const Grid& g, const CUtensorMap& map, int rows, dim3 grid,
                        cudaStream_t stream, int* occ) {
  switch (mode_of(g)) {
    case MODE_TOTAL | MODE_ZFULL | MODE_CORR:
      return launch_one<S, NPT, MODE_TOTAL | MODE_ZFULL | MODE_CORR>(g, map, rows, grid,
                                                                         stream, occ);
    case MODE_TOTAL | MODE_ZFULL:
      return launch_one<S, NPT, MODE_TOTAL | MODE_ZFULL>(g, map, rows, grid, stream, occ);
    case MODE_TOTAL | MODE_CORR:
      return launch_one<S, NPT, MODE_TOTAL | MODE_CORR>(g, map, rows, grid, stream, occ);
    case MODE_TOTAL:
      return launch_one<S, NPT, MODE_TOTAL>(g, map, rows, grid, stream, occ);
    case MODE_FORCE | MODE_CORR:
      return launch_one<S, NPT, MODE_FORCE | MODE_CORR>(g, map, rows, grid, stream, occ);
    case MODE_FORCE:
      return launch_one<S, NPT, MODE_FORCE>(g, map, rows, grid, stream, occ);
    case MODE_CORR:
      return launch_one<S, NPT, MODE_CORR>(g, map, rows, grid, stream, occ);
    default:
      return launch_one<S, NPT, 0>(g, map, rows, grid, stream, occ);
  }
}

template <class S>
cudaError_t dispatch_variant(const Grid& g, const CUtensorMap& map, int variant, int rows,
                             dim3 grid, cudaStream_t stream, int* occ) {
  if (variant == TMA_PR_2) return launch_mode<S, 2>(g, map, rows, grid, stream, occ);
  return launch_mode<S, 1>(g, map, rows, grid, stream, occ);
}

template <class S>
cudaError_t launch_step_tma(const Grid& g, const CUtensorMap& map, int variant, int rows,
                            dim3 grid, cudaStream_t stream) {
  return dispatch_variant<S>(g, map, variant, rows, grid, stream, nullptr);
}

template <class S, int M>
cudaError_t batch_one(const BatchGrid* grids, const WorkItem* items, BatchCtl* ctl, int j,
                      int blocks, cudaStream_t stream, int* occ) {
  static bool configured = false;
  const size_t smem = PrGeom<S, 1, batch_depth<S>()>::smem_bytes();
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(batch_step_kernel<S, M>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  if (occ)
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, batch_step_kernel<S, M>, PR_THREADS,
                                                         smem);
  batch_step_kernel<S, M><<<blocks, PR_THREADS, smem, stream>>>(grids, items, ctl, j);
  return cudaGetLastError();
}

template <class S>
cudaError_t batch_mode(const BatchGrid* grids, const WorkItem* items, BatchCtl* ctl, int j,
                       int mode, int blocks, cudaStream_t stream, int* occ) {
  switch (mode) {
    case MODE_TOTAL | MODE_ZFULL | MODE_CORR:
      return batch_one<S, MODE_TOTAL | MODE_ZFULL | MODE_CORR>(grids, items, ctl, j, blocks,
                                                                stream, occ);
    case MODE_TOTAL | MODE_ZFULL:
      return batch_one<S, MODE_TOTAL | MODE_ZFULL>(grids, items, ctl, j, blocks, stream, occ);
    case MODE_TOTAL | MODE_CORR:
      return batch_one<S, MODE_TOTAL | MODE_CORR>(grids, items, ctl, j, blocks, stream, occ);
    case MODE_TOTAL:
      return batch_one<S, MODE_TOTAL>(grids, items, ctl, j, blocks, stream, occ);
    case MODE_FORCE | MODE_CORR:
      return batch_one<S, MODE_FORCE | MODE_CORR>(grids, items, ctl, j, blocks, stream, occ);
    case MODE_FORCE:
      return batch_one<S, MODE_FORCE>(grids, items, ctl, j, blocks, stream, occ);
    case MODE_CORR:
      return batch_one<S, MODE_CORR>(grids, items, ctl, j, blocks, stream, occ);
    default:
      return batch_one<S, 0>(grids, items, ctl, j, blocks, stream, occ);
  }
}

template <class S>
cudaError_t launch_batch_step(const BatchGrid* grids, const WorkItem* items, BatchCtl* ctl, int j,
                              int mode, int blocks, cudaStream_t stream) {
  return batch_mode<S>(grids, items, ctl, j, mode, blocks, stream, nullptr);
}

template <class S>
int occupancy_batch(int mode) {
  int occ = 0;
  batch_mode<S>(nullptr, nullptr, nullptr, 0, mode, 1, nullptr, &occ);
  return occ;
}

template <class S>
int occupancy_step_tma(const Grid& g, int variant) {
  int occ = 0;
  dispatch_variant<S>(g, CUtensorMap{}, variant, 1, dim3(1), nullptr, &occ);
  return occ;
}

}  // namespace lbm
