// Batched step: many independent grids of different sizes and physics modes
// advance together.  One launch per time step covers every grid: a persistent
// grid of blocks (one per resident slot) takes work items from a list -- each
// item is the share of one block of the single-grid pulled-row kernel
// (pr_block: 128 columns x `rows` rows of one grid) -- either round-robin or
// from an atomic counter.  Per-grid descriptors (buffers, TMA descriptors of
// both buffers, step parity, steps left in the segment) live in device memory,
// so a CUDA graph of k launches is captured once per k and replayed while the
// host edits the descriptors between segments.
#pragma once

#include "lbm_step_pr.cuh"

namespace lbm {

constexpr int BATCH_MAX_SEG = 4096;  // steps per captured segment (counter slots)

struct alignas(64) BatchGrid {
  CUtensorMap maps[2];  // TMA descriptors of buffer 0 and 1 (box: 144 columns x 6 planes)
  Grid g;               // geometry and physics (src/dst unused)
  void* buf[2];         // the two state buffers
  long long t0;         // steps taken before this segment
  int seg_steps;        // steps this grid takes in the segment
  int mode;             // physics mode (mode_of)
};

struct WorkItem {
  int grid, x0, y0, rows;
};

// Items are grouped by physics mode; group m (0 .. 7, see mode_slot) holds
// items [begin[m], end[m]) and is advanced by the kernel instantiated for it.
struct BatchCtl {
  int begin[8], end[8];
  int dynamic;  // 1: atomic work queue, 0: round-robin
  int counters[8][BATCH_MAX_SEG];
};

// Compact index of the eight physics modes.
__host__ __device__ constexpr int mode_slot(int m) {
  return m == (MODE_TOTAL | MODE_ZFULL | MODE_CORR)   ? 0
         : m == (MODE_TOTAL | MODE_ZFULL)             ? 1
         : m == (MODE_TOTAL | MODE_CORR)              ? 2
         : m == MODE_TOTAL                            ? 3
         : m == (MODE_FORCE | MODE_CORR)              ? 4
         : m == MODE_FORCE                            ? 5
         : m == MODE_CORR                             ? 6
                                                      : 7;
}

template <class S, int M>
__global__ void __launch_bounds__(PR_THREADS, 4) batch_step_kernel(const BatchGrid* __restrict__ grids,
                                                                const WorkItem* __restrict__ items,
                                                                BatchCtl* ctl, int j) {
  constexpr int MS = mode_slot(M);
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ int s_item;
  __shared__ Grid s_grid;
  pr_init<S, 1>(smem);
  const int b0 = ctl->begin[MS], b1 = ctl->end[MS];
  const bool dyn = ctl->dynamic != 0;
  int kbase = 0;
  int it = b0 + blockIdx.x;
  for (;;) {
    if (dyn) {
      if (threadIdx.x == 0) s_item = b0 + atomicAdd(&ctl->counters[MS][j], 1);
      __syncthreads();
      it = s_item;
    }
    if (it >= b1) break;
    const WorkItem w = items[it];
    const BatchGrid& bg = grids[w.grid];
    if (j < bg.seg_steps) {
      // the grid descriptor in shared memory: uniform reads for the whole item
      const int* gsrc = reinterpret_cast<const int*>(&bg.g);
      int* gdst = reinterpret_cast<int*>(&s_grid);
      for (int i = threadIdx.x; i < (int)(sizeof(Grid) / sizeof(int)); i += blockDim.x)
        gdst[i] = gsrc[i];
      __syncthreads();
      const int par = (int)((bg.t0 + j) & 1);
      const int st = pr_block<S, 1, M>(s_grid, &bg.maps[par], bg.buf[par], bg.buf[par ^ 1], w.x0,
                                       w.y0, w.rows, smem, kbase);
      kbase += pr_staged_rows(s_grid, w.y0, w.rows);
      if (st) return;  // timeout recorded in the grid's status word
    }
    if (dyn)
      __syncthreads();  // everyone has read s_item (and s_grid) before they change
    else
      it += gridDim.x;
  }
}

}  // namespace lbm
