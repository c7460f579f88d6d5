// Host helpers shared by the single-grid and batched entry points.
#pragma once

#include <cuda.h>
#include <stddef.h>

#include <string>

#include "lbm.h"
#include "lbm_device.cuh"

namespace lbm_host {

// LBM_OK or LBM_ERR_PARAM with the reason in `why`.
int validate(const lbm_params* p, std::string& why);
// Row pitch in elements: >= nx + 2 (ghost columns), multiple of 32.
int pitch_of(int nx);
// Elements and bytes of one population buffer of a grid.
size_t buffer_elems(const lbm_params* p);
size_t buffer_bytes(const lbm_params* p);
// Fill the kernel argument (everything but the buffer pointers).
void fill_grid(const lbm_params* p, lbm::Grid& g);
// TMA descriptor of one state buffer for the row-staged step kernel.
int make_tensor_map(CUtensorMap* map, void* buffer, const lbm_params& p, const lbm::Grid& g,
                    int box_cols, int box_planes);

}  // namespace lbm_host
