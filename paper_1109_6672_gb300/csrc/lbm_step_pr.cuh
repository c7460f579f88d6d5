// Pulled-row TMA step kernel.
//
// The population planes are stored grouped by e_y (lbm_device.cuh), so the 18
// values that lattice row r pulls are three contiguous plane groups: the
// e_y = +1 group of row r - 1, the e_y = 0 group of row r and the e_y = -1
// group of row r + 1.  One ring slot in shared memory holds one such "pulled
// row" (3 groups x NB boxes of the tensor map, columns x0 - 8 .. x0 + TWC + 7),
// delivered by cp.async.bulk.tensor and guarded by an mbarrier with
// transaction-count completion.  The moments of row r and the collision of row
// r - 1 each read one slot, so a ring of D slots keeps D - 2 rows in flight.
// Rows across a periodic y boundary are staged the same way (their node row
// wraps; the ghost rows supply the wrapped neighbours).
//
// Block = 4 compute warps (each thread NPT columns, 128 apart) + 1 helper
// warp.  The helper warp computes Q_x of the two halo columns (x0 - 1 and
// x0 + TWC) and issues the copies, so the compute warps do identical work per
// row; one block barrier per row publishes Q_x and frees the slot of row r - 1.
//
// Waits on mbarriers are bounded by the global timer; on timeout the block
// sets *g.status, drains its own copies (bounded) and returns.
#pragma once

#include "lbm_step_tma.cuh"

namespace lbm {

constexpr int PR_COMPUTE = 128;              // compute threads per block
constexpr int PR_THREADS = PR_COMPUTE + 32;  // plus the helper warp

// DD: ring depth (0: 3 slots for FP64 storage, else 4).  XD: the walled x
// sides' ghost-slot writes are deferred (batched kernel, below).
template <class S, int NPT, int DD = 0, int XD = 0>
struct PrGeom {
  static constexpr int TWC = PR_COMPUTE * NPT;  // output columns per block
  static constexpr int NB = NPT == 1 ? 1 : 2;   // boxes per plane group
  static constexpr int BW = (TWC + 16) / NB;    // columns per box
  static constexpr int GB =                     // elements per box (128 B aligned)
      (int)(((size_t)6 * BW * sizeof(S) + 127) / 128 * 128 / sizeof(S));
  static constexpr int SLOT = 3 * NB * GB;  // elements per pulled row
  static constexpr int D = DD ? DD : (sizeof(S) == 8 ? 3 : 4);
  static constexpr unsigned BOX_BYTES = 6 * BW * sizeof(S);
  // x-edge records (XD, one thread per node): the walled x sides'
  // ghost-slot writes of XREC_ROWS rows are deferred and done together
  // (pr_block), in two banks of 2 XREC_ROWS records of XREC_VALS values
  static constexpr int XREC_ROWS = (XD && NPT == 1) ? 8 : 0;
  static constexpr int XREC_VALS = 16;
  static constexpr size_t smem_bytes() {
    return (size_t)D * SLOT * sizeof(S) + 2 * (TWC + 2) * sizeof(typename Io<S>::C) + D * 8 +
           (size_t)4 * XREC_ROWS * XREC_VALS * sizeof(typename Io<S>::C);
  }
  static_assert(BW % 8 == 0, "box starts must stay 16-byte aligned");
  static_assert((GB * sizeof(S)) % 128 == 0, "boxes must start on 128-byte boundaries");
};

// Offset inside a plane-group block of staged column sc (local column + 8).
template <class S, int NPT>
__device__ __forceinline__ int pr_col(int sc) {
  using G = PrGeom<S, NPT>;
  const int b = sc >= G::BW ? 1 : 0;
  return b * G::GB + (sc - b * G::BW);
}

// Pulled populations of a node from a slot; co[e_x + 1] = column offsets.
template <class S, int NPT>
__device__ __forceinline__ void pull_pr(const S* slot, const int co[3],
                                        typename Io<S>::C d[NPOP]) {
  using G = PrGeom<S, NPT>;
#pragma unroll
  for (int a = 0; a < NPOP; ++a) {
    const int grp = pgroup(a), lp = plane(a) - 6 * grp;
    d[a] = Io<S>::to(slot[grp * G::NB * G::GB + lp * G::BW + co[ex(a % 9) + 1]]);
  }
}

// Shared-memory layout of a block: ring slots, Q_x rows, mbarriers, x-edge
// records (XD).
template <class S, int NPT, int DD = 0, int XD = 0>
struct PrSmem {
  using C = typename Io<S>::C;
  using G = PrGeom<S, NPT, DD, XD>;
  __device__ static S* ring(unsigned char* smem) { return reinterpret_cast<S*>(smem); }
  __device__ static C* qxs(unsigned char* smem) {
    return reinterpret_cast<C*>(smem + (size_t)G::D * G::SLOT * sizeof(S));
  }
  __device__ static unsigned bars(unsigned char* smem) {
    return smem_u32(qxs(smem) + 2 * (G::TWC + 2));
  }
  __device__ static C* xrec(unsigned char* smem) {
    return reinterpret_cast<C*>(reinterpret_cast<unsigned char*>(qxs(smem) + 2 * (G::TWC + 2)) +
                                G::D * 8);
  }
};

// The values the x-edge writes of side XS (xedge_writes) read from a node:
// for each population A leaving through the side (B its opposite) f*_A,
// h*_A, h*_B and h^eq_B, then rho, u_x, u_y, theta.
template <int XS>
__host__ __device__ constexpr int xrec_pop(int k) {
  return XS == 0 ? (k == 0 ? 3 : (k == 1 ? 6 : 7)) : (k == 0 ? 1 : (k == 1 ? 5 : 8));
}
template <class C, int XS>
__device__ __forceinline__ void xrec_put(C* r, const C* v, C rho, C ux, C uy, C th) {
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const int A = xrec_pop<XS>(k), B = opp(A);
    r[4 * k] = v[A];
    r[4 * k + 1] = v[9 + A];
    r[4 * k + 2] = v[9 + B];
    r[4 * k + 3] = v[18 + B];
  }
  r[12] = rho;
  r[13] = ux;
  r[14] = uy;
  r[15] = th;
}
template <class S, int XS>
__device__ __forceinline__ void xrec_flush(const Grid& g, S* __restrict__ dst, int x, int y,
                                           const typename Io<S>::C* r) {
  using C = typename Io<S>::C;
  C v[27];
#pragma unroll
  for (int a = 0; a < 27; ++a) v[a] = C(0);
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const int A = xrec_pop<XS>(k), B = opp(A);
    v[A] = r[4 * k];
    v[9 + A] = r[4 * k + 1];
    v[9 + B] = r[4 * k + 2];
    v[18 + B] = r[4 * k + 3];
  }
  xedge_writes<S, XS>(g, dst, x, y, v, r[12], r[13], r[14], r[15]);
}

// Initialise the ring's mbarriers (once per kernel, all threads call).
template <class S, int NPT, int DD = 0>
__device__ __forceinline__ void pr_init(unsigned char* smem) {
  if (threadIdx.x == 0) {
    const unsigned bar_s = PrSmem<S, NPT, DD>::bars(smem);
    for (int i = 0; i < PrGeom<S, NPT, DD>::D; ++i) mbar_init(bar_s + 8 * i, 1);
    mbar_fence_init();
  }
  __syncthreads();
}

// Pulled rows staged by a block that owns rows [y0, y0 + rows) of a grid with
// ny rows: rs .. rs + count - 1 (halo rows only where they hold nodes).
__device__ __forceinline__ int pr_span(int ny, bool periodic_b, bool periodic_t, int y0, int rows,
                                       int& rs) {
  const int y1 = min(y0 + rows, ny);
  rs = (y0 >= 1 || periodic_b) ? y0 - 1 : y0;
  const int re = (y1 < ny || periodic_t) ? y1 : y1 - 1;
  return re - rs + 1;
}

__device__ __forceinline__ int pr_staged_rows(const Grid& g, int y0, int rows) {
  int rs;
  return pr_span(g.ny, g.bc[2] == BC_PERIODIC, g.bc[3] == BC_PERIODIC, y0, rows, rs);
}

// The share a block takes after the current one (persistent kernels): its
// first pulled rows are staged while the current share finishes.  nq = 0:
// no next share.
struct PrNext {
  const CUtensorMap* map;
  int x0, rs, nq, ny;
};

// One block's share of a step: columns [x0, x0 + TWC), rows [y0, y0 + rows)
// of grid g, reading the state at src through the tensor map `map` and
// writing the next state to dst.  kbase counts the rows this block staged
// before (ring slot and mbarrier phase continue across calls); `pre` of this
// share's rows were already issued by the previous call, and once this share's
// rows are all issued the copies run on into `next` (*pre_out: how many).
// Only helper lane 0 issues copies, so pre / *pre_out matter in that thread
// alone.  Returns 0, or 1 if a staged row never arrived (after draining its own
// copies).
template <class S, int NPT, int M, int DD = 0, int XD = 0>
__device__ __forceinline__ int pr_block(const Grid& g, const CUtensorMap* map, const void* src_v,
                                        void* dst_v, int x0, int y0, int rows, unsigned char* smem,
                                        int kbase, int pre = 0,
                                        PrNext next = PrNext{nullptr, 0, 0, 0, 0},
                                        int* pre_out = nullptr) {
  using C = typename Io<S>::C;
  using G = PrGeom<S, NPT, DD, XD>;
  using SM = PrSmem<S, NPT, DD, XD>;
  constexpr bool DEV = Io<S>::dev;  // moments carried as deviations (moments_m)
  constexpr int D = G::D, TWC = G::TWC;
  constexpr unsigned long long WAIT_NS = 2000000000ull;  // 2 s
  S* ring = SM::ring(smem);
  C* qxs = SM::qxs(smem);
  constexpr int XR = G::XREC_ROWS, XV = G::XREC_VALS;
  C* xrec = SM::xrec(smem);
  const unsigned ring_s = smem_u32(ring), bar_s = SM::bars(smem);

  const int t = threadIdx.x, nx = g.nx, ny = g.ny;
  const int y1 = min(y0 + rows, ny);
  const bool wall_l = g.bc[0] != BC_PERIODIC, wall_r = g.bc[1] != BC_PERIODIC;
  const bool wall_b = g.bc[2] != BC_PERIODIC, wall_t = g.bc[3] != BC_PERIODIC;
  // this share holds a node of a walled x side (recorded x-edge writes)
  const bool xl = wall_l && x0 == 0, xr = wall_r && x0 <= nx - 1 && nx - 1 < x0 + G::TWC;
  // staged pulled rows rs .. re (halo rows only where they hold nodes)
  const int rs = (y0 >= 1 || !wall_b) ? y0 - 1 : y0;
  const int re = (y1 < ny || !wall_t) ? y1 : y1 - 1;
  const int nq = re - rs + 1;
  const S* __restrict__ src = static_cast<const S*>(src_v);
  S* __restrict__ dst = static_cast<S*>(dst_v);
  const int pitch = g.pitch;
  const bool helper = t >= PR_COMPUTE;
  const int hl = t - PR_COMPUTE;  // helper lane

  // staged rows issued so far (helper lane 0), counted from this share's
  // first row; indices >= nq are rows of the next share
  int issued = pre;
  auto issue_upto = [&](int kmax) {
    kmax = min(kmax, nq + next.nq - 1);
    for (; issued <= kmax; ++issued) {
      const int s = (kbase + issued) % D;
      const unsigned bar = bar_s + 8 * s;
      const bool own = issued < nq;
      const CUtensorMap* m = own ? map : next.map;
      const int xs = own ? x0 : next.x0, yn = own ? ny : next.ny;
      int nr = own ? rs + issued : next.rs + (issued - nq);  // node row of this pulled row
      nr = nr < 0 ? nr + yn : (nr >= yn ? nr - yn : nr);
      mbar_expect_tx(bar, 3 * G::NB * G::BOX_BYTES);
#pragma unroll
      for (int grp = 0; grp < 3; ++grp)
#pragma unroll
        for (int b = 0; b < G::NB; ++b)
          tma_load_box(ring_s + (unsigned)((s * G::SLOT + (grp * G::NB + b) * G::GB) * sizeof(S)),
                       m, bar, xs - 8 + b * G::BW + XOFF, 6 * grp, nr + grp);  // row nr-1+grp, +1
    }
  };
  if (helper && hl == 0) issue_upto(D - 2);

  // columns handled by this thread and their staged-column offsets
  int cols[NPT], co[NPT][3];
#pragma unroll
  for (int i = 0; i < NPT; ++i) {
    const int lc = helper ? (hl == 0 ? -1 : TWC) : t + PR_COMPUTE * i;
    cols[i] = x0 + lc;
    co[i][0] = pr_col<S, NPT>(lc + 9);  // e_x = -1 pulls from x + 1
    co[i][1] = pr_col<S, NPT>(lc + 8);
    co[i][2] = pr_col<S, NPT>(lc + 7);  // e_x = +1 pulls from x - 1
  }
  // where the (first) node of this thread comes from: 0 idle, 1 ring, 2 global
  int src0 = 0, gx0 = 0;
  {
    const int c = cols[0];
    if (helper && hl > 1) {
      src0 = 0;
    } else if (c >= 0 && c < nx) {
      src0 = 1;
      gx0 = c;
    } else if (c == -1 && !wall_l) {
      src0 = 2;
      gx0 = nx - 1;
    } else if (c == nx && !wall_r) {
      src0 = 2;
      gx0 = 0;
    }
  }

  C prho[NPT], pux[NPT], puy[NPT], pth[NPT], pes[NPT], pqx[NPT], pqy[NPT], qymm[NPT];
#pragma unroll
  for (int i = 0; i < NPT; ++i) {
    prho[i] = DEV ? C(0) : C(1);
    pux[i] = puy[i] = pqx[i] = pqy[i] = qymm[i] = pes[i] = 0;
    pth[i] = DEV ? C(0) : C(1);
  }
  int qs = 0;  // Q_x slot of the current row
  for (int r = y0 - 1; r <= y1; ++r) {
    C crho[NPT], cux[NPT], cuy[NPT], cth[NPT], ces[NPT], cqx[NPT], cqy[NPT];
#pragma unroll
    for (int i = 0; i < NPT; ++i) {
      crho[i] = DEV ? C(0) : C(1);
      cux[i] = cuy[i] = cqx[i] = cqy[i] = ces[i] = 0;
      cth[i] = DEV ? C(0) : C(1);
    }
    bool ok = true;
    const int k = r - rs;
    if (k >= 0 && k < nq) {
      ok = mbar_wait(bar_s + 8 * ((kbase + k) % D), ((kbase + k) / D) & 1, WAIT_NS);
      const S* slot = ring + ((kbase + k) % D) * G::SLOT;
      int nr = r < 0 ? r + ny : (r >= ny ? r - ny : r);
#pragma unroll
      for (int i = 0; i < NPT; ++i) {
        if (helper && i > 0) break;
        int how;
        int gx;
        if (i == 0) {
          how = src0;
          gx = gx0;
        } else {
          const int c = cols[i];
          how = c < nx ? 1 : ((c == nx && !wall_r) ? 2 : 0);
          gx = c < nx ? c : 0;
        }
        if (!how) continue;
        C d[NPOP];
        if (how == 1)
          pull_pr<S, NPT>(slot, co[i], d);
        else
          pull<S>(g, src, gx, nr, d);
        moments_m<S, M>(g, d, crho[i], cux[i], cuy[i], cth[i], ces[i]);
        // Q = rho u (1 - theta) (Eq. 48); deviation storage carries rho - 1
        // and theta - 1 instead of rho and theta
        const C rq = DEV ? C(1) + crho[i] : crho[i];
        const C om = DEV ? -cth[i] : C(1) - cth[i];
        cqx[i] = rq * cux[i] * om;
        cqy[i] = rq * cuy[i] * om;
      }
    }
    C* qrow = qxs + qs * (TWC + 2);
    if (!helper) {
#pragma unroll
      for (int i = 0; i < NPT; ++i) qrow[t + PR_COMPUTE * i + 1] = cqx[i];
    } else if (hl == 0) {
      qrow[0] = cqx[0];
    } else if (hl == 1) {
      qrow[TWC + 1] = cqx[0];
    }
    const int ro = r - 1;
    if (!helper && ro >= y0) {
      const S* slot = ring + ((kbase + k - 1) % D) * G::SLOT;  // pulled row ro (k - 1 >= 0)
      const C* qprev = qxs + (qs ^ 1) * (TWC + 2);
      S* prow = dst + (long long)(ro + 1) * g.rp + XOFF;
#pragma unroll
      for (int i = 0; i < NPT; ++i) {
        const int c = cols[i];
        if (c >= nx) continue;
        C d[NPOP];
        pull_pr<S, NPT>(slot, co[i], d);
        const int lq = t + PR_COMPUTE * i + 1;
        const C rho_n = DEV ? C(1) + prho[i] : prho[i];
        const C th_n = DEV ? C(1) + pth[i] : pth[i];
        const C qxl =
            (c > 0 || !wall_l) ? qprev[lq - 1] : ghost_q<C>(g, 0, 0, rho_n, th_n, pqx[i]);
        const C qxr = (c < nx - 1 || !wall_r) ? qprev[lq + 1]
                                              : ghost_q<C>(g, 1, 0, rho_n, th_n, pqx[i]);
        const C qyu =
            (ro < ny - 1 || !wall_t) ? cqy[i] : ghost_q<C>(g, 3, 1, rho_n, th_n, pqy[i]);
        const C qyd =
            (ro > 0 || !wall_b) ? qymm[i] : ghost_q<C>(g, 2, 1, rho_n, th_n, pqy[i]);
        C v[27];
        collide_m<S, M>(g, prow + c, pitch, c, ro, d, prho[i], pux[i], puy[i], pth[i], pes[i],
                        C(0.5) * (qxr - qxl), C(0.5) * (qyu - qyd), v);
        // ghost-slot writes (from absolute values): x edges inline (one
        // thread of a warp), the edge rows (every thread of the row) through
        // the general routine
        const bool xedge = c == 0 || c == nx - 1, yedge = ro == 0 || ro == ny - 1;
        if (xedge || yedge) {
          if constexpr (DEV) {
#pragma unroll
            for (int a = 0; a < 27; ++a) v[a] += pref<S>(g, a < 18 ? a : a - 9);
          }
          // a walled x side's writes are recorded and done XREC_ROWS rows at
          // a time by a whole warp (below), so that the row barrier does not
          // wait on one lane's wall rules; periodic copies are cheap inline
          if constexpr (XR > 0) {
            C* rec = xrec + (((ro - y0) / XR) & 1) * (2 * XR * XV) + ((ro - y0) % XR) * 2 * XV;
            if (c == 0) {
              if (wall_l)
                xrec_put<C, 0>(rec, v, rho_n, pux[i], puy[i], th_n);
              else
                xedge_writes<S, 0>(g, dst, c, ro, v, rho_n, pux[i], puy[i], th_n);
            }
            if (c == nx - 1) {
              if (wall_r)
                xrec_put<C, 1>(rec + XV, v, rho_n, pux[i], puy[i], th_n);
              else
                xedge_writes<S, 1>(g, dst, c, ro, v, rho_n, pux[i], puy[i], th_n);
            }
          } else {
            if (c == 0) xedge_writes<S, 0>(g, dst, c, ro, v, rho_n, pux[i], puy[i], th_n);
            if (c == nx - 1) xedge_writes<S, 1>(g, dst, c, ro, v, rho_n, pux[i], puy[i], th_n);
          }
          if (yedge) {
            C tmp[27];
#pragma unroll
            for (int a = 0; a < 27; ++a) tmp[a] = v[a];
            boundary_writes<S, true>(g, dst, c, ro, tmp, rho_n, pux[i], puy[i], th_n);
          }
        }
      }
    }
    if (__syncthreads_or(!ok)) {
      // a staged row never arrived: record, drain what is in flight, leave.
      // Bit 2: the drain itself ran out, so a copy may still land in shared
      // memory after the block has left; the host then treats the state as
      // lost until it is reloaded.
      if (helper && hl == 0) {
        bool drained = true;
        for (int j = max(k, 0); j < issued; ++j)
          drained = mbar_wait(bar_s + 8 * ((kbase + j) % D), ((kbase + j) / D) & 1,
                              WAIT_NS / 4) && drained;
        if (g.status) atomicOr(g.status, drained ? 1 : 3);
      }
      return 1;
    }
    // everyone is done with pulled row r - 1: refill its slot
    if (helper && hl == 0) issue_upto(k + D - 1);
    // the recorded x-edge writes of the chunk that row ro completes: lane l
    // of warp 0 takes side l & 1 of chunk row l >> 1.  The other bank fills
    // meanwhile; this one is refilled only after the next chunk's last
    // barrier, which warp 0 reaches after this.
    if constexpr (XR > 0) {
      if (ro >= y0 && (xl || xr) && t < 2 * XR && ((ro - y0 + 1) % XR == 0 || ro == y1 - 1)) {
        const int c0 = ((ro - y0) / XR) * XR;  // first row of the chunk, from y0
        const int row = y0 + c0 + (t >> 1);
        const C* rec = xrec + ((c0 / XR) & 1) * (2 * XR * XV) + (t >> 1) * 2 * XV;
        if (row <= ro) {
          if ((t & 1) == 0 && xl) xrec_flush<S, 0>(g, dst, 0, row, rec);
          if ((t & 1) == 1 && xr) xrec_flush<S, 1>(g, dst, nx - 1, row, rec + XV);
        }
      }
    }
#pragma unroll
    for (int i = 0; i < NPT; ++i) {
      qymm[i] = pqy[i];
      prho[i] = crho[i];
      pux[i] = cux[i];
      puy[i] = cuy[i];
      pth[i] = cth[i];
      pes[i] = ces[i];
      pqx[i] = cqx[i];
      pqy[i] = cqy[i];
    }
    qs ^= 1;
  }
  if (pre_out) *pre_out = max(issued - nq, 0);
  return 0;
}

// Resident blocks per SM that the register budget is sized for (the shared
// memory of the ring allows as many): the rare wall branches may spill.  The
// MRT collision (moment vectors) and the per-node relaxation times of a
// viscosity law get a larger budget.
template <class S, int NPT, int M = 0>
__host__ __device__ constexpr int pr_min_blocks() {
  return NPT != 1 ? 1 : (sizeof(S) == 8 ? 3 : ((M & (MODE_MRT | MODE_VARMU)) ? 4 : 5));
}

template <class S, int NPT, int M>
__global__ void __launch_bounds__(PR_THREADS, (pr_min_blocks<S, NPT, M>())) step_pr_kernel(
    const Grid g, const __grid_constant__ CUtensorMap map, int rows) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const int y0 = blockIdx.y * rows;
  if (y0 >= g.ny) return;  // whole block
  pr_init<S, NPT>(smem);
  pr_block<S, NPT, M>(g, &map, g.src, g.dst, blockIdx.x * PrGeom<S, NPT>::TWC, y0, rows, smem, 0);
}

}  // namespace lbm
