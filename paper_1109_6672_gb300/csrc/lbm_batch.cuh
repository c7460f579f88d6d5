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

// Items are grouped by physics mode; group m (0 .. 31, see mode_slot) holds
// items [begin[m], end[m]) and is advanced by the kernel instantiated for it.
constexpr int BATCH_MODE_SLOTS = 4 * NUM_BGK_MODES;
struct BatchCtl {
  int begin[BATCH_MODE_SLOTS], end[BATCH_MODE_SLOTS];
  int dynamic;  // 1: atomic work queue, 0: round-robin
  int counters[BATCH_MODE_SLOTS][BATCH_MAX_SEG];
};

// Compact index of the physics modes: position in BGK_MODES, + 8 for MRT,
// + 16 for a temperature-dependent viscosity.
__host__ __device__ constexpr int bgk_index(int m) {
  return m == (MODE_TOTAL | MODE_ZFULL | MODE_CORR) ? 0
         : m == (MODE_TOTAL | MODE_ZFULL)           ? 1
         : m == (MODE_TOTAL | MODE_CORR)            ? 2
         : m == MODE_TOTAL                          ? 3
         : m == (MODE_FORCE | MODE_CORR)            ? 4
         : m == MODE_FORCE                          ? 5
         : m == MODE_CORR                           ? 6
                                                    : 7;
}
__host__ __device__ constexpr int mode_slot(int m) {
  return bgk_index(m & ~(MODE_MRT | MODE_VARMU)) + ((m & MODE_MRT) ? NUM_BGK_MODES : 0) +
         ((m & MODE_VARMU) ? 2 * NUM_BGK_MODES : 0);
}
static_assert(bgk_index(BGK_MODES[0]) == 0 && bgk_index(BGK_MODES[3]) == 3 &&
                  bgk_index(BGK_MODES[5]) == 5 && bgk_index(BGK_MODES[7]) == 7,
              "mode slots follow BGK_MODES");

// Ring depth (0: as the single-grid kernel) and resident blocks per SM that
// the register budget of the batched kernel is sized for.
template <class S>
__host__ __device__ constexpr int batch_depth() {
  return 0;
}
template <class S>
__host__ __device__ constexpr int batch_min_blocks() {
  return sizeof(S) == 8 ? 3 : 4;
}
template <class S, int M>
__global__ void __launch_bounds__(PR_THREADS, (batch_min_blocks<S>()))
    batch_step_kernel(const BatchGrid* __restrict__ grids, const WorkItem* __restrict__ items,
                      BatchCtl* ctl, int j) {
  constexpr int MS = mode_slot(M);
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ int s_item;
  __shared__ Grid s_grid;
  constexpr int DD = batch_depth<S>();
  pr_init<S, 1, DD>(smem);
  const int b0 = ctl->begin[MS], b1 = ctl->end[MS];
  const bool dyn = ctl->dynamic != 0;
  // helper lane 0 issues the copies; it also takes the items from the queue,
  // one ahead, so that the next item's first rows are staged early
  const bool fetcher = threadIdx.x == PR_COMPUTE;
  int rr = b0 + blockIdx.x;  // round-robin cursor
  auto fetch = [&]() {       // next item of a grid that steps at j
    for (;;) {
      int it;
      if (dyn) {
        it = b0 + atomicAdd(&ctl->counters[MS][j], 1);
      } else {
        it = rr;
        rr += gridDim.x;
      }
      if (it >= b1) return b1;
      if (j < grids[items[it].grid].seg_steps) return it;
    }
  };
  int nxt = b1, pre = 0, kbase = 0;
  if (fetcher) {
    s_item = fetch();
    nxt = s_item < b1 ? fetch() : b1;
  }
  __syncthreads();
  for (;;) {
    const int it = s_item;
    if (it >= b1) break;
    const WorkItem w = items[it];
    const BatchGrid& bg = grids[w.grid];
    // the grid descriptor in shared memory: uniform reads for the whole item
    const int* gsrc = reinterpret_cast<const int*>(&bg.g);
    int* gdst = reinterpret_cast<int*>(&s_grid);
    for (int i = threadIdx.x; i < (int)(sizeof(Grid) / sizeof(int)); i += blockDim.x)
      gdst[i] = gsrc[i];
    __syncthreads();
    if (threadIdx.x == 0) s_grid.t = (unsigned)(bg.t0 + j);
    PrNext next{nullptr, 0, 0, 0, 0};
    if (fetcher && nxt < b1) {
      const WorkItem wn = items[nxt];
      const BatchGrid& gn = grids[wn.grid];
      next.map = &gn.maps[(int)((gn.t0 + j) & 1)];
      next.x0 = wn.x0;
      next.ny = gn.g.ny;
      next.nq = pr_span(gn.g.ny, gn.g.bc[2] == BC_PERIODIC, gn.g.bc[3] == BC_PERIODIC, wn.y0,
                        wn.rows, next.rs);
    }
    __syncthreads();
    const int par = (int)((bg.t0 + j) & 1);
    int pre_out = 0;
    const int st = pr_block<S, 1, M, DD, 1>(s_grid, &bg.maps[par], bg.buf[par], bg.buf[par ^ 1], w.x0,
                                     w.y0, w.rows, smem, kbase, pre, next, &pre_out);
    if (st) return;  // timeout recorded in the grid's status word
    kbase += pr_staged_rows(s_grid, w.y0, w.rows);
    // every thread passed the share's last barrier: s_item and s_grid are free
    if (fetcher) {
      s_item = nxt;
      pre = pre_out;
      nxt = nxt < b1 ? fetch() : b1;
    }
    __syncthreads();
  }
}

}  // namespace lbm
