// D3Q19 kernels with FP32 storage and arithmetic.
#include "lbm3d_inst.cuh"

namespace lbm3 {
cudaError_t launch_step3d_f32(const Grid3& g, dim3 grid, int zrows, int ty, int split,
                              cudaStream_t st) {
  return launch_step3d<float>(g, grid, zrows, ty, split, st);
}
cudaError_t launch_aux3d_f32(int what, const Grid3& g, void* buf, const double* const* in,
                             double* const* out, double T0, double* pops, int* flag,
                             double* partial, int blocks, cudaStream_t st) {
  return launch_aux3d<float>(what, g, buf, in, out, T0, pops, flag, partial, blocks, st);
}
cudaError_t step3d_attributes_f32(int mode, int ty, int split, cudaFuncAttributes* a) {
  return attributes3d<float>(mode, ty, split, a);
}
}  // namespace lbm3
