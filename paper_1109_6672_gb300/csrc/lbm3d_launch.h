// Host launchers of the D3Q19 kernels, one translation unit per storage
// precision (lbm3d_f64.cu, lbm3d_f32.cu).
#pragma once

#include <cuda_runtime.h>

#include "lbm3d.cuh"

namespace lbm3 {

// Physics modes the validated parameters can produce.
inline int mode3_of(const Grid3& g) {
  int m = 0;
  if (g.energy_model == 0) {
    m |= M3_TOTAL;
    if (g.z_full) m |= M3_ZFULL;
  }
  if (g.correction) m |= M3_CORR;
  if (g.pd.g != 0.0) m |= M3_FORCE;  // internal energy only (validated)
  return m;
}

// ty: tile rows; split: separate halo warps (launch_mode3 lists the shapes)
cudaError_t launch_step3d_f64(const Grid3& g, dim3 grid, int zrows, int ty, int split,
                              cudaStream_t st);
cudaError_t launch_step3d_f32(const Grid3& g, dim3 grid, int zrows, int ty, int split,
                              cudaStream_t st);
cudaError_t launch_aux3d_f64(int what, const Grid3& g, void* buf, const double* const* in,
                             double* const* out, double T0, double* pops, int* flag,
                             double* partial, int blocks, cudaStream_t st);
cudaError_t launch_aux3d_f32(int what, const Grid3& g, void* buf, const double* const* in,
                             double* const* out, double T0, double* pops, int* flag,
                             double* partial, int blocks, cudaStream_t st);
// step kernel attributes (registers, for the resident-block count)
cudaError_t step3d_attributes_f64(int mode, int ty, int split, cudaFuncAttributes* attr);
cudaError_t step3d_attributes_f32(int mode, int ty, int split, cudaFuncAttributes* attr);

enum { AUX3_INIT = 0, AUX3_EXPORT = 1, AUX3_CONSERVED = 2 };

}  // namespace lbm3
