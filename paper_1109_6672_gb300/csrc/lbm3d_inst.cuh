// Instantiation of the D3Q19 kernels for one storage precision S (included
// by lbm3d_f64.cu and lbm3d_f32.cu with LBM3_S and LBM3_NAME defined).
#pragma once

#include "lbm3d_launch.h"

namespace lbm3 {

template <class S>
cudaError_t launch_step3d(const Grid3& g, dim3 grid, int zrows, cudaStream_t st) {
  constexpr int NT = TX3 * ty3<S>();
  switch (mode3_of(g)) {
    case M3_TOTAL | M3_ZFULL | M3_CORR:
      step3d_kernel<S, M3_TOTAL | M3_ZFULL | M3_CORR><<<grid, NT, 0, st>>>(g, zrows);
      break;
    case M3_TOTAL | M3_ZFULL:
      step3d_kernel<S, M3_TOTAL | M3_ZFULL><<<grid, NT, 0, st>>>(g, zrows);
      break;
    case M3_TOTAL | M3_CORR:
      step3d_kernel<S, M3_TOTAL | M3_CORR><<<grid, NT, 0, st>>>(g, zrows);
      break;
    case M3_TOTAL:
      step3d_kernel<S, M3_TOTAL><<<grid, NT, 0, st>>>(g, zrows);
      break;
    case M3_CORR:
      step3d_kernel<S, M3_CORR><<<grid, NT, 0, st>>>(g, zrows);
      break;
    default:
      step3d_kernel<S, 0><<<grid, NT, 0, st>>>(g, zrows);
      break;
  }
  return cudaGetLastError();
}

template <class S>
cudaError_t attributes3d(int mode, cudaFuncAttributes* a) {
  switch (mode) {
    case M3_TOTAL | M3_ZFULL | M3_CORR:
      return cudaFuncGetAttributes(a, step3d_kernel<S, M3_TOTAL | M3_ZFULL | M3_CORR>);
    case M3_TOTAL | M3_ZFULL:
      return cudaFuncGetAttributes(a, step3d_kernel<S, M3_TOTAL | M3_ZFULL>);
    case M3_TOTAL | M3_CORR:
      return cudaFuncGetAttributes(a, step3d_kernel<S, M3_TOTAL | M3_CORR>);
    case M3_TOTAL:
      return cudaFuncGetAttributes(a, step3d_kernel<S, M3_TOTAL>);
    case M3_CORR:
      return cudaFuncGetAttributes(a, step3d_kernel<S, M3_CORR>);
    default:
      return cudaFuncGetAttributes(a, step3d_kernel<S, 0>);
  }
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
