// Definitions of the launchers declared in lbm_launch.h; included by the four
// per-precision translation units.
#pragma once

#include "lbm_launch.h"
#include "lbm_batch.cuh"
#include "lbm_step_pr.cuh"

#include <type_traits>

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

// Calls fn(std::integral_constant<int, M>{}) for the kernel of physics mode
// `mode` (one of the BGK modes of mode_of, or with MRT_OK also their MRT
// twins); cudaErrorInvalidValue for a mode without a kernel.
template <int I, int OFF, class Fn>
cudaError_t dispatch_from(int mode, Fn& fn) {
  if constexpr (I == NUM_BGK_MODES) {
    return cudaErrorInvalidValue;
  } else {
    constexpr int M = BGK_MODES[I] | OFF;
    if (mode == M) return fn(std::integral_constant<int, M>{});
    return dispatch_from<I + 1, OFF>(mode, fn);
  }
}

template <bool ALL, class Fn>
cudaError_t dispatch_mode(int mode, Fn&& fn) {
  const int twin = mode & (MODE_MRT | MODE_VARMU);
  if (twin == 0) return dispatch_from<0, 0>(mode, fn);
  if constexpr (ALL) {
    if (twin == MODE_MRT) return dispatch_from<0, MODE_MRT>(mode, fn);
    if (twin == MODE_VARMU) return dispatch_from<0, MODE_VARMU>(mode, fn);
    return dispatch_from<0, MODE_MRT | MODE_VARMU>(mode, fn);
  }
  return cudaErrorInvalidValue;
}

// The two-node-per-thread variant is built for BGK with constant tau only.
template <class S, int NPT>
cudaError_t launch_mode(const Grid& g, const CUtensorMap& map, int rows, dim3 grid,
                        cudaStream_t stream, int* occ) {
  return dispatch_mode<NPT == 1>(mode_of(g), [&](auto m) {
    return launch_one<S, NPT, decltype(m)::value>(g, map, rows, grid, stream, occ);
  });
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
  const size_t smem = PrGeom<S, 1, batch_depth<S>(), 1>::smem_bytes();
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
  return dispatch_mode<true>(mode, [&](auto m) {
    return batch_one<S, decltype(m)::value>(grids, items, ctl, j, blocks, stream, occ);
  });
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
