// Instantiation of the TMA-staged step kernel for float storage.
#include "lbm_step_inst.cuh"

namespace lbm {
template cudaError_t launch_step_tma<float>(const Grid&, const CUtensorMap&, int, int, dim3,
                                            cudaStream_t);
template int occupancy_step_tma<float>(const Grid&, int);
}  // namespace lbm
