// Instantiation of the TMA-staged step kernel for double storage.
#include "lbm_step_inst.cuh"

namespace lbm {
template cudaError_t launch_step_tma<double>(const Grid&, const CUtensorMap&, int, int, dim3,
                                             cudaStream_t);
template int occupancy_step_tma<double>(const Grid&, int);
}  // namespace lbm
