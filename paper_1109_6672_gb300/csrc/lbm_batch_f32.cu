// Instantiation of the batched step kernels for float storage (a translation
// unit of its own, so that the step and the batch kernels compile in parallel).
#include "lbm_step_inst.cuh"

namespace lbm {
template cudaError_t launch_batch_step<float>(const BatchGrid*, const WorkItem*, BatchCtl*,
                                           int, int, int, cudaStream_t);
template int occupancy_batch<float>(int);
}  // namespace lbm
