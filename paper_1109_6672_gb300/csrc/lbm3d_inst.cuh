// Instantiation of the D3Q19 kernels for one storage precision S (included
// by lbm3d_f64.cu and lbm3d_f32.cu with LBM3_S and LBM3_NAME defined).
#pragma once

#include "lbm3d_launch.h"

namespace lbm3 {

template <class S, int M, int TY, bool SPLIT>
cudaError_t launch_tile3(const Grid3& g, dim3 grid, int zrows, cudaStream_t st) {
  constexpr size_t SM = step3d_smem<S, TY>();
  static bool attr_set = false;  // per process and instantiation (one device attribute)
  if (!attr_set) {
    const cudaError_t e = cudaFuncSetAttribute(
        step3d_kernel<S, M, TY, SPLIT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SM);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  step3d_kernel<S, M, TY, SPLIT><<<grid, threads3<TY, SPLIT>(), SM, st>>>(g, zrows);
  return cudaGetLastError();
}

// Launch shapes (tile rows, separate halo warps): (8, no) for both
// precisions; for FP32 storage also (16, no), (4, yes) and (8, yes).
template <class S, int M>
cudaError_t launch_mode3(const Grid3& g, dim3 grid, int zrows, int ty, int split,
                         cudaStream_t st) {
  if constexpr (sizeof(S) == 4) {
    if (ty == 16) return launch_tile3<S, M, 16, false>(g, grid, zrows, st);
    if (ty == 4 && split) return launch_tile3<S, M, 4, true>(g, grid, zrows, st);
    if (ty == 8 && split) return launch_tile3<S, M, 8, true>(g, grid, zrows, st);
  }
  return launch_tile3<S, M, 8, false>(g, grid, zrows, st);
}

template <class S>
cudaError_t launch_step3d(const Grid3& g, dim3 grid, int zrows, int ty, int split,
                          cudaStream_t st) {
  switch (mode3_of(g)) {
    case M3_TOTAL | M3_ZFULL | M3_CORR:
      return launch_mode3<S, M3_TOTAL | M3_ZFULL | M3_CORR>(g, grid, zrows, ty, split, st);
    case M3_TOTAL | M3_ZFULL:
      return launch_mode3<S, M3_TOTAL | M3_ZFULL>(g, grid, zrows, ty, split, st);
    case M3_TOTAL | M3_CORR:
      return launch_mode3<S, M3_TOTAL | M3_CORR>(g, grid, zrows, ty, split, st);
    case M3_TOTAL:
      return launch_mode3<S, M3_TOTAL>(g, grid, zrows, ty, split, st);
    case M3_CORR:
      return launch_mode3<S, M3_CORR>(g, grid, zrows, ty, split, st);
    case M3_FORCE | M3_CORR:
      return launch_mode3<S, M3_FORCE | M3_CORR>(g, grid, zrows, ty, split, st);
    case M3_FORCE:
      return launch_mode3<S, M3_FORCE>(g, grid, zrows, ty, split, st);
    default:
      return launch_mode3<S, 0>(g, grid, zrows, ty, split, st);
  }
}

template <class S, int TY, bool SPLIT>
cudaError_t attributes3d_tile(int mode, cudaFuncAttributes* a) {
  switch (mode) {
    case M3_TOTAL | M3_ZFULL | M3_CORR:
      return cudaFuncGetAttributes(a, step3d_kernel<S, M3_TOTAL | M3_ZFULL | M3_CORR, TY, SPLIT>);
    case M3_TOTAL | M3_ZFULL:
      return cudaFuncGetAttributes(a, step3d_kernel<S, M3_TOTAL | M3_ZFULL, TY, SPLIT>);
    case M3_TOTAL | M3_CORR:
      return cudaFuncGetAttributes(a, step3d_kernel<S, M3_TOTAL | M3_CORR, TY, SPLIT>);
    case M3_TOTAL:
      return cudaFuncGetAttributes(a, step3d_kernel<S, M3_TOTAL, TY, SPLIT>);
    case M3_CORR:
      return cudaFuncGetAttributes(a, step3d_kernel<S, M3_CORR, TY, SPLIT>);
    case M3_FORCE | M3_CORR:
      return cudaFuncGetAttributes(a, step3d_kernel<S, M3_FORCE | M3_CORR, TY, SPLIT>);
    case M3_FORCE:
      return cudaFuncGetAttributes(a, step3d_kernel<S, M3_FORCE, TY, SPLIT>);
    default:
      return cudaFuncGetAttributes(a, step3d_kernel<S, 0, TY, SPLIT>);
  }
}

template <class S>
cudaError_t attributes3d(int mode, int ty, int split, cudaFuncAttributes* a) {
  if constexpr (sizeof(S) == 4) {
    if (ty == 16) return attributes3d_tile<S, 16, false>(mode, a);
    if (ty == 4 && split) return attributes3d_tile<S, 4, true>(mode, a);
    if (ty == 8 && split) return attributes3d_tile<S, 8, true>(mode, a);
  }
  return attributes3d_tile<S, 8, false>(mode, a);
}

template <class S>
cudaError_t launch_aux3d(int what, const Grid3& g, void* buf, const double* const* in,
                         double* const* out, double T0, double* pops, int* flag, double* partial,
                         int blocks, cudaStream_t st) {
  if (what == AUX3_INIT) {
    if (g.energy_model == 0)
      init3d_kernel<S, true><<<blocks, 256, 0, st>>>(g, static_cast<S*>(buf), in[0], in[1],
                                                      in[2], in[3], in[4], 1.0 / T0);
    else
      init3d_kernel<S, false><<<blocks, 256, 0, st>>>(g, static_cast<S*>(buf), in[0], in[1],
                                                       in[2], in[3], in[4], 1.0 / T0);
  } else if (what == AUX3_EXPORT) {
    export3d_kernel<S><<<blocks, 256, 0, st>>>(
        g, static_cast<const S*>(buf), out ? out[0] : nullptr, out ? out[1] : nullptr,
        out ? out[2] : nullptr, out ? out[3] : nullptr, out ? out[4] : nullptr, T0, pops, flag);
  } else {
    conserved3d_kernel<S><<<blocks, RED3, 0, st>>>(g, static_cast<const S*>(buf), partial);
    conserved3d_final_kernel<><<<1, 32, 0, st>>>(partial, blocks, partial + 5 * blocks);
  }
  return cudaGetLastError();
}

}  // namespace lbm3
