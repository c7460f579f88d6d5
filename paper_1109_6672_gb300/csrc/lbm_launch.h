// Host launchers of the TMA-staged step kernel, one translation unit per
// storage type (lbm_step_f64.cu, lbm_step_f32.cu, lbm_step_f16.cu,
// lbm_step_bf16.cu) so the instantiations compile in parallel.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include "lbm_device.cuh"

namespace lbm {

// Pulled-row TMA step kernel (lbm_step_pr.cuh) with 128 (variant 1) or 256
// (variant 2) columns per block; box width (columns) of one TMA copy.
enum { TMA_PR_1 = 1, TMA_PR_2 = 2 };
constexpr int tma_npt(int variant) { return variant == TMA_PR_2 ? 2 : 1; }
constexpr int tma_cols(int variant) { return 128 * tma_npt(variant); }
constexpr int tma_box(int npt) { return npt == 1 ? 144 : 136; }
// Default rows per block of the pulled-row kernel: small blocks, many waves,
// dynamically balanced across SMs (measured on GB300 at 4096^2).
inline int tma_default_rows(size_t elem_bytes) { return elem_bytes == 4 ? 6 : 12; }

// Launch one step on `stream`; grid.x covers nx in tma_cols(variant)
// columns, grid.y covers ny in `rows` rows.  Returns the launch error.
template <class S>
cudaError_t launch_step_tma(const Grid& g, const CUtensorMap& map, int variant, int rows,
                            dim3 grid, cudaStream_t stream);

// Resident blocks per SM of that kernel (0 if it cannot launch).
template <class S>
int occupancy_step_tma(const Grid& g, int variant);

struct BatchGrid;
struct WorkItem;
struct BatchCtl;

// One step of the batched kernel (lbm_batch.cuh) for the items of physics
// mode `mode` over `blocks` persistent blocks, and its resident blocks per SM.
template <class S>
cudaError_t launch_batch_step(const BatchGrid* grids, const WorkItem* items, BatchCtl* ctl, int j,
                              int mode, int blocks, cudaStream_t stream);
template <class S>
int occupancy_batch(int mode);

}  // namespace lbm
