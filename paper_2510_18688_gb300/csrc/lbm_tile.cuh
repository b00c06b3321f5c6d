// lbm_tile.cuh -- the fused time step of float states (FP32 and FP16
// storage) as a persistent kernel whose tiles are staged by TMA, for sm_103a.
//
// The arithmetic is that of step_tile (lbm_step.cuh, well-balanced storage);
// what differs is how a tile's inputs arrive.  Each CTA owns a sequence of
// 32 x 8 tiles (blockIdx.x, blockIdx.x + gridDim.x, ...).  One thread issues
// the TMA copies of the next tile's inputs into the free one of two
// shared-memory stages while the CTA computes the current tile from the
// other, so loads no longer wait on compute or compute on loads:
//
//   f   own flow populations                  box 32 x 8 x 9 planes
//   gh  phase and enthalpy populations, ring  box (32 + 2 XG) x 10 x 18
//   lag the 7 lag planes, ring                box 40 x 10 x 7
//   phi0                                      box 40 x 10
//
// (the cold mask, one byte per node and read only where the grid has one,
// comes with plain loads: its box would cost the shared memory that keeps
// the one-stage kernel at four CTAs per SM)
//
// The halo boxes start 16 bytes' worth of columns left of the tile (a TMA
// box must start on a 16-byte boundary); only the one-node ring is used.
// Cells of the ring (or of a ragged tile) outside the grid, which TMA fills
// with zeros, are overwritten with the periodic image or the mirrored wall
// node before use.  Operands are then read from shared memory at offsets
// fixed at compile time, and the post-collision populations are pushed to
// global memory as in step_tile.  Waits on the copies are bounded; a timeout
// sets *status and the CTA drains its copies and leaves.
#pragma once

#include "lbm_step.cuh"
#include "lbm_tma.cuh"

namespace lbmk {

template <typename S>
struct alignas(128) TileStage {
  static constexpr int XG = 16 / (int)sizeof(S);  // ring offset of the population box
  static constexpr int WG = TX + 2 * XG;          // its width
  static constexpr int XL = 4, WL = TX + 2 * XL;  // float lag and phi0 boxes
  alignas(128) S f[9][TY][TX];
  alignas(128) S gh[18][TY + 2][WG];
  alignas(128) float lag[NLAG + 1][TY + 2][WL];
  alignas(128) float phi0[TY + 2][WL];
  static constexpr uint32_t kBytes =
      (uint32_t)(sizeof(S) * (9 * TY * TX + 18 * (TY + 2) * WG) +
                 sizeof(float) * ((NLAG + 2) * (TY + 2) * WL));
};

template <typename S>
struct TileArgs {
  Args<float, S> a;
  CUtensorMap map_f, map_gh, map_lag, map_phi0;
  int tiles_x, ntiles;
  unsigned* status;  // set to 1 when a copy did not arrive in time
  unsigned extra_tx; // test hook: bytes expected beyond the copies (0)
};

// The five tensor maps of one grid and buffer parity, as the batched tile
// kernel reads them from global memory (written by the host before any
// launch that uses them; 64-byte aligned like every CUtensorMap).
struct TileMaps {
  CUtensorMap f, gh, lag, phi0;
};

// Up to BATCH_MAX_GRIDS float grids in one launch of the TMA-staged tile
// kernel, one CTA per 32 x 8 tile of the concatenated tile list: the step
// arguments travel in parameter space as for lbm_batch_kernel, each grid's
// tensor maps (for its current parity) stay in global memory.
template <typename S>
struct TileBatch {
  int ngrids;
  int tile_base[BATCH_MAX_GRIDS + 1];  // first tile of each grid; [ngrids] = total
  int tiles_x[BATCH_MAX_GRIDS];
  const TileMaps* maps[BATCH_MAX_GRIDS];
  unsigned* status[BATCH_MAX_GRIDS];   // per grid: a copy did not arrive in time
  unsigned extra_tx;                   // test hook: bytes expected beyond the copies (0)
  Args<float, S> args[BATCH_MAX_GRIDS];
};

// Shared memory of a CTA with NST stages (plus room to align them).
template <typename S>
constexpr size_t tile_smem_bytes(int nst) {
  return nst * sizeof(TileStage<S>) + 128;
}

// Resident CTAs per SM the kernel is compiled for: two with two stages (a
// CTA overlaps its own loads and compute; 127 registers), three with one
// stage (the CTAs of an SM overlap one another; 80 registers).
template <int NST>
constexpr int tile_min_blocks() {
  return NST == 2 ? 2 : 3;
}

__device__ __forceinline__ float lds(const float* p) { return *p; }
__device__ __forceinline__ float lds(const __half* p) { return __half2float(*p); }

// The inputs of the tile at (x0, y0) into stage st, completing on bar.
template <typename S>
__device__ __forceinline__ void tile_issue_maps(const CUtensorMap* mf, const CUtensorMap* mgh,
                                                const CUtensorMap* mlag, const CUtensorMap* mphi0,
                                                unsigned extra_tx,
                                                TileStage<S>& st, uint64_t* bar, int x0, int y0) {
  using St = TileStage<S>;
  mbar_arrive_expect_tx(bar, St::kBytes + extra_tx);
  tma_load_3d(&st.f[0][0][0], mf, x0, y0, 0, bar);
  tma_load_3d(&st.gh[0][0][0], mgh, x0 - St::XG, y0 - 1, 9, bar);
  tma_load_3d(&st.lag[0][0][0], mlag, x0 - St::XL, y0 - 1, 0, bar);
  tma_load_3d(&st.phi0[0][0], mphi0, x0 - St::XL, y0 - 1, 0, bar);
}

// Tile t of a single grid's launch into stage st, completing on bar.
template <typename S>
__device__ __forceinline__ void tile_issue(const TileArgs<S>& ta, TileStage<S>& st,
                                           uint64_t* bar, int t) {
  tile_issue_maps(&ta.map_f, &ta.map_gh, &ta.map_lag, &ta.map_phi0, ta.extra_tx,
                  st, bar, (t % ta.tiles_x) * TX, (t / ta.tiles_x) * TY);
}

// Ring cells (and cells of a ragged tile) outside the grid: the periodic
// image or the mirrored wall node, as step_tile loads them.  Block-uniform
// test first; every thread takes cells tid, tid + NT.
template <typename S>
__device__ __forceinline__ void tile_fix_edges(const Args<float, S>& a, TileStage<S>& st, int x0,
                                               int y0, int tid) {
  using St = TileStage<S>;
  const Geom& g = a.g;
  if (x0 >= 1 && x0 + TX < g.nx && y0 >= 1 && y0 + TY < g.ny) return;
  const int P = (int)g.plane;
  for (int k = tid; k < HN; k += NT) {
    const int hx = k % HX, hy = k / HX;
    const int X = x0 - 1 + hx, Y = y0 - 1 + hy;
    if (X >= 0 && X < g.nx && Y >= 0 && Y < g.ny) continue;
    const int m = wrap_or_clamp(Y, g.ny, g.bc[2], g.bc[3]) * g.pitch +
                  wrap_or_clamp(X, g.nx, g.bc[0], g.bc[1]);
#pragma unroll
    for (int i = 0; i < 18; i++) st.gh[i][hy][hx - 1 + St::XG] = a.pin[(9 + i) * P + m];
#pragma unroll
    for (int j = 0; j < NLAG + 1; j++) st.lag[j][hy][hx + St::XL - 1] = a.lin[j * P + m];
    st.phi0[hy][hx + St::XL - 1] = a.phi0[m];
  }
}

// The cold-mask bytes of this thread's own cell and (threads below RING) of
// its ring cell for the tile at (x0, y0): 0 where the grid has no mask.
// Cells beyond the grid take their periodic image's or the edge node's byte,
// as tile_fix_edges takes their fields.  Loaded before the wait for the
// tile's copies, so that their latency overlaps the copies'.
struct TileMask {
  uint8_t own, ring;
};
template <typename S>
__device__ __forceinline__ TileMask tile_mask(const Args<float, S>& a, int x0, int y0, int tid) {
  const Geom& g = a.g;
  TileMask m{0, 0};
  if (!g.has_mask) return m;
  const int tx = tid % TX, ty = tid / TX;
  m.own = a.mask[wrap_or_clamp(y0 + ty, g.ny, g.bc[2], g.bc[3]) * g.pitch +
                 wrap_or_clamp(x0 + tx, g.nx, g.bc[0], g.bc[1])];
  if (tid < RING) {
    int hx, hy;
    ring_pos(tid, hx, hy);
    m.ring = a.mask[wrap_or_clamp(y0 + hy - 1, g.ny, g.bc[2], g.bc[3]) * g.pitch +
                    wrap_or_clamp(x0 + hx - 1, g.nx, g.bc[0], g.bc[1])];
  }
  return m;
}

// The step for one staged tile (bx, by), tile index b of nb; mk: the
// thread's mask bytes (tile_mask).  Every thread
// of the CTA calls it; the caller synchronises before and after.
template <typename S, bool DIAG, int LATC>
__device__ __forceinline__ void tile_step(const Args<float, S>& a, const TileStage<S>& st,
                                          int bx, int by, int b, int nb, float* s_phi,
                                          float* s_fs, float* s_rho, float* s_T,
                                          float (*s_red)[NDIAG], TileMask mk) {
  using St = TileStage<S>;
  using R = float;
  const Geom& g = a.g;
  const Coef<R>& c = a.c;
  const int lat = LATC ? LATC : g.lattices;
  const int P = (int)g.plane;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int tid = ty * TX + tx;
  const int x0 = bx * TX, y0 = by * TY;
  const int gx = x0 + tx, gy = y0 + ty;
  const bool valid = gx < g.nx && gy < g.ny;
  const int n = gy * g.pitch + gx;  // used by valid nodes only
  const int hc = (ty + 1) * HX + (tx + 1);
  // the node's cells in the staged boxes
  const int cg = (ty + 1) * St::WG + tx + St::XG;
  const int cl = (ty + 1) * St::WL + tx + St::XL;
  const int PG = (TY + 2) * St::WG, PL = (TY + 2) * St::WL;
  const S* gh = &st.gh[0][0][0];
  const float* lag = &st.lag[0][0][0];

  // ---- phase A1: own node -------------------------------------------------
  const R phi0 = st.phi0[ty + 1][tx + St::XL];
  const R flp = lag[LAG_FL * PL + cl], wp = lag[LAG_W * PL + cl];
  const R pp = lag[LAG_P * PL + cl], Qp = lag[LAG_Q * PL + cl];
  const bool masked = (lat & LAT_HEAT) && mk.own;
  R Tp = R(0), Cp = R(0);
  if (lat & LAT_HEAT) {
    Tp = lag[LAG_T * PL + cl];
    Cp = cap_rn(c, fs_rn(wp, flp, phi0), wp);
  }
  R sg = R(0), sh = R(0);
  if (lat & LAT_PHASE) {
    R v[9];
#pragma unroll
    for (int i = 0; i < 9; i++) v[i] = lds(gh + i * PG + cg);
    sg = sum_g(v);
  }
  if (lat & LAT_HEAT) {
    R v[9];
    if (masked) {
      cold_mask_h(c, wp, phi0, v);
      v[0] -= ref_h0(c, wp, flp, Tp, Cp);
#pragma unroll
      for (int i = 1; i < 9; i++) v[i] -= ref_hi(i <= 4 ? c.wrr1 : c.wrr5, Tp);
    } else {
#pragma unroll
      for (int i = 0; i < 9; i++) v[i] = lds(gh + (9 + i) * PG + cg);
    }
    sh = sum_h(v);
  }
  const Local<R> L = local_state_wb(c, lat, sg, sh, flp, wp, Qp, Tp, Cp, phi0);
  s_phi[hc] = L.phi;
  s_fs[hc] = L.fs;
  s_rho[hc] = L.rho;
  s_T[hc] = L.T;

  // ---- phase A2: the ring ----------------------------------------------------
  if (tid < RING) {
    int hx, hy;
    ring_pos(tid, hx, hy);
    const int hi = hy * HX + hx;
    const int rg = hy * St::WG + hx - 1 + St::XG, rl = hy * St::WL + hx - 1 + St::XL;
    const R q0 = st.phi0[hy][hx - 1 + St::XL];
    const R flq = lag[LAG_FL * PL + rl], wq = lag[LAG_W * PL + rl];
    const R Qq = lag[LAG_Q * PL + rl];
    R Tq = R(0), Cq = R(0);
    if (lat & LAT_HEAT) {
      Tq = lag[LAG_T * PL + rl];
      Cq = cap_rn(c, fs_rn(wq, flq, q0), wq);
    }
    R sgq = R(0), shq = R(0);
    if (lat & LAT_PHASE) {
      R v[9];
#pragma unroll
      for (int i = 0; i < 9; i++) v[i] = lds(gh + i * PG + rg);
      sgq = sum_g(v);
    }
    if (lat & LAT_HEAT) {
      R v[9];
      if (mk.ring) {
        cold_mask_h(c, wq, q0, v);
        v[0] -= ref_h0(c, wq, flq, Tq, Cq);
#pragma unroll
        for (int i = 1; i < 9; i++) v[i] -= ref_hi(i <= 4 ? c.wrr1 : c.wrr5, Tq);
      } else {
#pragma unroll
        for (int i = 0; i < 9; i++) v[i] = lds(gh + (9 + i) * PG + rg);
      }
      shq = sum_h(v);
    }
    const Local<R> Lq = local_state_wb(c, lat, sgq, shq, flq, wq, Qq, Tq, Cq, q0);
    s_phi[hi] = Lq.phi;
    s_fs[hi] = Lq.fs;
    s_rho[hi] = Lq.rho;
    s_T[hi] = Lq.T;
  }
  __syncthreads();

  // ---- phase B: stencils, macros, collisions, streaming -------------------
  // Instantiated twice: for a tile whose nodes and ring are all inside the
  // grid (block-uniform branch) no node needs boundary logic.
  auto phase_b = [&](auto interior) {
  constexpr bool IN = decltype(interior)::value;
  R dvals[NDIAG];
  Macro<R> M;
  const bool inner = IN || (gx > 0 && gx < g.nx - 1 && gy > 0 && gy < g.ny - 1);
  const bool valid_n = IN || valid;
  R f[9];
  if (valid_n) {
    if (lat & LAT_FLOW) {
#pragma unroll
      for (int i = 0; i < 9; i++) f[i] = lds(&st.f[i][ty][tx]);
    }
    node_macros<R, true>(g, c, lat, gx, gy, inner, L, phi0, pp, f, s_phi + hc, s_fs + hc,
                         s_rho + hc, HX, lag + LAG_P * PL + cl, &st.phi0[ty + 1][tx + St::XL],
                         St::WL, M);
    if (DIAG) diag_values(c, lat, L, M, sg, sh, f, dvals);
  } else if (DIAG) {
#pragma unroll
    for (int k = 0; k < NDIAG; k++) dvals[k] = R(0);
  }
  if (DIAG) block_diag_warps(dvals, s_red, tid);

  if (valid_n) {
    S* out = a.pout;
    if (lat & LAT_FLOW) {
      if (inner) collide_flow_wb<true>(g, c, out, P, gx, gy, n, f, L.rho, M);
      else collide_flow_wb<false>(g, c, out, P, gx, gy, n, f, L.rho, M);
    }
    if (lat & LAT_PHASE) {
      R gq[9];
#pragma unroll
      for (int i = 0; i < 9; i++) gq[i] = lds(gh + i * PG + cg);
      const R phuxp = lag[LAG_PHUX * PL + cl], phuyp = lag[LAG_PHUY * PL + cl];
      const R dref = ref_delta(rest_ref_g(L.w, phi0), rest_ref_g(wp, phi0));
      if (inner)
        collide_phase<R, true>(g, c, out + 9 * P, P, gx, gy, n, gq, L.phi, L.phir, L.mdot,
                               phuxp, phuyp, M, dref);
      else
        collide_phase<R, false>(g, c, out + 9 * P, P, gx, gy, n, gq, L.phi, L.phir, L.mdot,
                                phuxp, phuyp, M, dref);
    }
    if (lat & LAT_HEAT) {
      R hq[9];
      if (masked) {
        cold_mask_h(c, wp, phi0, hq);
        hq[0] -= ref_h0(c, wp, flp, Tp, Cp);
#pragma unroll
        for (int i = 1; i < 9; i++) hq[i] -= ref_hi(i <= 4 ? c.wrr1 : c.wrr5, Tp);
      } else {
#pragma unroll
        for (int i = 0; i < 9; i++) hq[i] = lds(gh + (9 + i) * PG + cg);
      }
      const R dref0 = ref_delta(ref_h0(c, L.w, L.fl, L.T, M.cap), ref_h0(c, wp, flp, Tp, Cp));
      const R aold = ref_hi(c.wrr1, Tp), dold = ref_hi(c.wrr5, Tp);
      if (inner)
        collide_heat_wb<true>(g, c, out + 18 * P, P, gx, gy, n, hq, L.fs, L.w, L.T, L.T - Tp,
                              L.rhoHr, L.mdot, M, aold, dold, dref0, s_T, hc);
      else
        collide_heat_wb<false>(g, c, out + 18 * P, P, gx, gy, n, hq, L.fs, L.w, L.T, L.T - Tp,
                               L.rhoHr, L.mdot, M, aold, dold, dref0, s_T, hc);
    }
    a.lout[LAG_FL * P + n] = L.fl;
    a.lout[LAG_W * P + n] = L.w;
    a.lout[LAG_P * P + n] = (lat & LAT_FLOW) ? M.pr : R(0);
    a.lout[LAG_PHUX * P + n] = (lat & LAT_PHASE) ? M.phux : R(0);
    a.lout[LAG_PHUY * P + n] = (lat & LAT_PHASE) ? M.phuy : R(0);
    a.lout[LAG_Q * P + n] = (lat & LAT_HEAT) ? M.cap * L.T * L.mdot : R(0);
    a.lout[LAG_T * P + n] = L.T;
  }
  };
  if (x0 >= 1 && x0 + TX < g.nx && y0 >= 1 && y0 + TY < g.ny) phase_b(std::true_type{});
  else phase_b(std::false_type{});
  if (DIAG) block_diag_finish(s_red, a.diag_partial, tid, b, nb);
}

template <typename S, bool DIAG, int LATC, int NST>
__global__ void __launch_bounds__(NT, tile_min_blocks<NST>())
    lbm_tile_kernel(const __grid_constant__ TileArgs<S> ta) {
  static_assert(NST == 1 || NST == 2, "one or two stages");
  using St = TileStage<S>;
  extern __shared__ unsigned char tile_smem[];
  St* stage = reinterpret_cast<St*>(tile_smem + ((128u - (smem_u32(tile_smem) & 127u)) & 127u));
  __shared__ __align__(8) uint64_t bar[NST];
  __shared__ float s_phi[HN], s_fs[HN], s_rho[HN], s_T[HN];
  __shared__ float s_red[NT / 32][NDIAG];
  const int tid = threadIdx.y * TX + threadIdx.x;
  if (tid == 0) {
    for (int i = 0; i < NST; i++) mbar_init(&bar[i], 1);
    fence_barrier_init();
    tma_prefetch_map(&ta.map_f);
    tma_prefetch_map(&ta.map_gh);
    tma_prefetch_map(&ta.map_lag);
  }
  __syncthreads();
  int t = blockIdx.x, k = 0;
  if (tid == 0 && t < ta.ntiles) tile_issue(ta, stage[0], &bar[0], t);
  bool timed_out = false;
  for (; t < ta.ntiles; t += gridDim.x, k++) {
    const int s = NST == 2 ? (k & 1) : 0;
    const uint32_t parity = NST == 2 ? ((k >> 1) & 1) : (k & 1);
    const int tn = t + gridDim.x;
    // two stages: stage s ^ 1 was released by the barrier that ended the
    // previous tile, so the next tile's copies start now
    if (NST == 2 && tid == 0 && tn < ta.ntiles) {
      fence_proxy_async();
      tile_issue(ta, stage[s ^ 1], &bar[s ^ 1], tn);
    }
    const int bx = t % ta.tiles_x, by = t / ta.tiles_x;
    const TileMask mk = tile_mask(ta.a, bx * TX, by * TY, tid);
    const bool ok = mbar_wait(&bar[s], parity);
    if (__syncthreads_or(!ok)) {
      timed_out = true;
      break;
    }
    tile_fix_edges(ta.a, stage[s], bx * TX, by * TY, tid);
    __syncthreads();
    tile_step<S, DIAG, LATC>(ta.a, stage[s], bx, by, t, ta.ntiles, s_phi, s_fs, s_rho, s_T,
                             s_red, mk);
    // this thread's reads (and edge writes) of stage s come before the TMA
    // writes that will refill it
    fence_proxy_async();
    __syncthreads();
    // one stage: the next tile's copies start once this one is done with
    if (NST == 1 && tid == 0 && tn < ta.ntiles) tile_issue(ta, stage[0], &bar[0], tn);
  }
  if (timed_out && tid == 0) {
    atomicExch(ta.status, 1u);
    // drain: the late copy and (two stages) the prefetch of the next tile,
    // if issued, must land before the CTA's shared memory goes away
    if (NST == 2) {
      mbar_wait(&bar[k & 1], (k >> 1) & 1);
      if (t + (int)gridDim.x < ta.ntiles) mbar_wait(&bar[(k + 1) & 1], ((k + 1) >> 1) & 1);
    } else {
      mbar_wait(&bar[0], k & 1);
    }
  }
}

// One tile per CTA, one stage, no loop over tiles (kept apart from the
// persistent loop above, whose bookkeeping costs the registers this form
// needs): stage the tile at (bx, by) with the given maps, wait (bounded),
// step it.  On a timeout the grid's status word is set and the CTA waits
// (bounded) for the late copy before it leaves.
template <typename S, bool DIAG, int LATC>
__device__ __forceinline__ void tile_once(const Args<float, S>& a, const CUtensorMap* mf,
                                          const CUtensorMap* mgh, const CUtensorMap* mlag,
                                          const CUtensorMap* mphi0,
                                          unsigned extra_tx, unsigned* status, int bx, int by,
                                          int b, int nb) {
  using St = TileStage<S>;
  extern __shared__ unsigned char tile_smem[];
  St* stage = reinterpret_cast<St*>(tile_smem + ((128u - (smem_u32(tile_smem) & 127u)) & 127u));
  __shared__ __align__(8) uint64_t bar;
  __shared__ float s_phi[HN], s_fs[HN], s_rho[HN], s_T[HN];
  __shared__ float s_red[NT / 32][NDIAG];
  const int tid = threadIdx.y * TX + threadIdx.x;
  if (tid == 0) {
    mbar_init(&bar, 1);
    fence_barrier_init();
    tile_issue_maps(mf, mgh, mlag, mphi0, extra_tx, stage[0], &bar, bx * TX, by * TY);
  }
  __syncthreads();
  const TileMask mk = tile_mask(a, bx * TX, by * TY, tid);
  const bool ok = mbar_wait(&bar, 0);
  if (__syncthreads_or(!ok)) {
    if (tid == 0) {
      atomicExch(status, 1u);
      mbar_wait(&bar, 0);  // the late copy must land before the CTA leaves
    }
    return;
  }
  tile_fix_edges(a, stage[0], bx * TX, by * TY, tid);
  __syncthreads();
  tile_step<S, DIAG, LATC>(a, stage[0], bx, by, b, nb, s_phi, s_fs, s_rho, s_T, s_red, mk);
}

// CTAs per SM of the loop-free one-stage kernels: four for one grid (64
// registers, 56 KB of shared memory each); three for the batched kernel,
// whose grid lookup does not fit 64 registers without spills (at four it
// measured 632 us per step of the 64-grid batch against 610 us at three).
constexpr int kTileOnceBlocks = 4;
constexpr int kTileBatchBlocks = 3;

// One grid, one CTA per tile, one stage (kernel form 1).
template <typename S, bool DIAG, int LATC>
__global__ void __launch_bounds__(NT, kTileOnceBlocks)
    lbm_tile1_kernel(const __grid_constant__ TileArgs<S> ta) {
  const int t = blockIdx.x;
  tile_once<S, DIAG, LATC>(ta.a, &ta.map_f, &ta.map_gh, &ta.map_lag, &ta.map_phi0,
                           ta.extra_tx, ta.status, t % ta.tiles_x, t / ta.tiles_x, t, ta.ntiles);
}

// Many float grids in one launch of the one-stage TMA-staged step: CTA t
// takes tile t of the concatenated tile list (its grid by bisection over the
// prefix sums, as lbm_batch_kernel) and stages it with that grid's tensor
// maps from global memory.
template <typename S, bool DIAG, int LATC>
__global__ void __launch_bounds__(NT, kTileBatchBlocks)
    lbm_tile_batch_kernel(const __grid_constant__ TileBatch<S> B) {
  const int t = blockIdx.x;
  int lo = 0, hi = B.ngrids;  // tile_base[lo] <= t < tile_base[hi]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (B.tile_base[mid] <= t) lo = mid;
    else hi = mid;
  }
  const int local = t - B.tile_base[lo];
  const TileMaps* m = B.maps[lo];
  tile_once<S, DIAG, LATC>(B.args[lo], &m->f, &m->gh, &m->lag, &m->phi0, B.extra_tx,
                           B.status[lo], local % B.tiles_x[lo], local / B.tiles_x[lo], local,
                           B.tile_base[lo + 1] - B.tile_base[lo]);
}

}  // namespace lbmk
