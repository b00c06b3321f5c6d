// lbm_split.cuh -- the time step as two barrier-free kernels (sm_103a).
//
//   lbm_macro_kernel    enthalpy inversion, order parameter and properties
//                       (Eqs. (8), (22), (10)) for every node: phi, fs, rho into three
//                       scratch planes (12 B per node in FP32, written once and
//                       read back from L2 by the second kernel).
//   lbm_collide_kernel  the rest of the step: the own node's local state again from its
//                       populations, the isotropic stencils from the scratch
//                       planes and the lagged pressure (neighbours are cache
//                       hits), velocity and pressure, the three pairwise
//                       collisions with push streaming, lag store and fused
//                       diagnostics.
//
// Neither kernel uses shared memory for the stencil nor a CTA barrier on its
// main path, and the halo is not recomputed: each node's macros are computed
// once.  One thread per node; CTA = 32 x 8 nodes.  Plain (FP64) populations
// only: the well-balanced float storage refers the pushed enthalpy
// populations to their destinations' new temperatures, which this form
// would have to write out and read back.
#pragma once

#include "lbm_kernels.cuh"
#include "lbm_step.cuh"

namespace lbmk {

enum { SC_PHI = 0, SC_FS, SC_RHO, NSCRATCH };

template <typename R>
struct SplitArgs {
  Args<R> a;                    // buffers, constants, diagnostics
  R* __restrict__ sc;           // NSCRATCH planes: phi, fs, rho
};

template <typename R, int LATC>
__global__ void __launch_bounds__(NT) lbm_macro_kernel(const SplitArgs<R> s) {
  static_assert(!kShift<R>, "the two-kernel step takes plain populations only");
  const Args<R>& a = s.a;
  const Geom& g = a.g;
  const Coef<R>& c = a.c;
  const int lat = LATC ? LATC : g.lattices;
  const int P = (int)g.plane;
  const int gx = blockIdx.x * TX + threadIdx.x, gy = blockIdx.y * TY + threadIdx.y;
  if (gx >= g.nx || gy >= g.ny) return;
  const int n = gy * g.pitch + gx;
  const R* pn = a.pin + n;
  const R phi0 = a.phi0[n];
  const R wp = a.lin[LAG_W * P + n];
  R sg = R(0), sh = R(0);
  if (lat & LAT_PHASE) {
    R v[9];
#pragma unroll
    for (int i = 0; i < 9; i++) v[i] = pn[(9 + i) * P];
    sg = sum_g(v);
  }
  if (lat & LAT_HEAT) {
    R v[9];
    if (g.has_mask && a.mask[n]) {
      cold_mask_h(c, wp, phi0, v);
    } else {
#pragma unroll
      for (int i = 0; i < 9; i++) v[i] = pn[(18 + i) * P];
    }
    sh = sum_h(v);
  }
  const Local<R> L =
      local_state(c, lat, sg, sh, a.lin[LAG_FL * P + n], wp, a.lin[LAG_Q * P + n], phi0);
  s.sc[SC_PHI * P + n] = L.phi;
  s.sc[SC_FS * P + n] = L.fs;
  s.sc[SC_RHO * P + n] = L.rho;
}

template <typename R, bool DIAG, int LATC>
__global__ void __launch_bounds__(NT, sizeof(R) == 4 ? LBM_MIN_BLOCKS_F32 : 1)
    lbm_collide_kernel(const SplitArgs<R> s) {
  const Args<R>& a = s.a;
  const Geom& g = a.g;
  const Coef<R>& c = a.c;
  const int lat = LATC ? LATC : g.lattices;
  const int P = (int)g.plane;

  __shared__ R s_red[NT / 32][NDIAG];

  const int tx = threadIdx.x, ty = threadIdx.y;
  const int tid = ty * TX + tx;
  const int gx = blockIdx.x * TX + tx, gy = blockIdx.y * TY + ty;
  const bool valid = gx < g.nx && gy < g.ny;
  R dvals[NDIAG];
  if (valid) {
    const int n = gy * g.pitch + gx;
    const R* pn = a.pin + n;
    const R phi0 = a.phi0[n];
    const R flp = a.lin[LAG_FL * P + n];
    const R wp = a.lin[LAG_W * P + n];
    const R Qp = a.lin[LAG_Q * P + n];
    const bool masked = (lat & LAT_HEAT) && g.has_mask && a.mask[n];
    R f[9];
    if (lat & LAT_FLOW) {
#pragma unroll
      for (int i = 0; i < 9; i++) f[i] = pn[i * P];
    }
    R sg = R(0), sh = R(0);
    if (lat & LAT_PHASE) {
      R v[9];
#pragma unroll
      for (int i = 0; i < 9; i++) v[i] = ld_sum(pn + (9 + i) * P);
      sg = sum_g(v);
    }
    if (lat & LAT_HEAT) {
      R v[9];
      if (masked) {
        cold_mask_h(c, wp, phi0, v);
      } else {
#pragma unroll
        for (int i = 0; i < 9; i++) v[i] = ld_sum(pn + (18 + i) * P);
      }
      sh = sum_h(v);
    }
    const Local<R> L = local_state(c, lat, sg, sh, flp, wp, Qp, phi0);

    // stencil neighbours: interior nodes use fixed offsets; edge nodes wrap
    // (periodic) or mirror the wall node (reading R-BC)
    const bool inner = gx > 0 && gx < g.nx - 1 && gy > 0 && gy < g.ny - 1;
    int nb[9];
#pragma unroll
    for (int i = 1; i < 9; i++) {
      if (inner) {
        nb[i] = n + qy(i) * g.pitch + qx(i);
      } else {
        const int xx = wrap_or_clamp(gx + qx(i), g.nx, g.bc[0], g.bc[1]);
        const int yy = wrap_or_clamp(gy + qy(i), g.ny, g.bc[2], g.bc[3]);
        nb[i] = yy * g.pitch + xx;
      }
    }
    // isotropic stencils (reading R-FD): grad = 3 sum w_i c_i chi(x + c_i),
    // lap = 6 sum w_i (chi(x + c_i) - chi(x)); the own node's phi, fs, rho
    // are the values the macro kernel stored
    const R* sphi = s.sc + SC_PHI * P;
    const R* sfs = s.sc + SC_FS * P;
    const R* srho = s.sc + SC_RHO * P;
    const R* spp = a.lin + LAG_P * P;
    const R phic = sphi[n], fsc = sfs[n];
    R gphx = R(0), gphy = R(0), lphi = R(0), lphi0 = R(0), lfs = R(0);
    R grx = R(0), gry = R(0), gpx = R(0), gpy = R(0);
#pragma unroll
    for (int i = 1; i < 9; i++) {
      const int m = nb[i];
      const R wi = qw<R>(i);
      const R cxi = R(qx(i)), cyi = R(qy(i));
      if (lat & LAT_PHASE) {
        const R ph = sphi[m];
        gphx += wi * cxi * ph;
        gphy += wi * cyi * ph;
        lphi += R(2) * wi * (ph - phic);
        lphi0 += R(2) * wi * (a.phi0[m] - phi0);
        lfs += R(2) * wi * (sfs[m] - fsc);
      }
      if (lat & LAT_FLOW) {
        const R rq = srho[m], pq = spp[m];
        grx += wi * cxi * rq;
        gry += wi * cyi * rq;
        gpx += wi * cxi * pq;
        gpy += wi * cyi * pq;
      }
    }
    gphx *= R(3); gphy *= R(3); lphi *= R(3); lphi0 *= R(3); lfs *= R(3);
    grx *= R(3); gry *= R(3); gpx *= R(3); gpy *= R(3);

    const R phi = L.phi, fs = L.fs, rho = L.rho, T = L.T, mdot = L.mdot;
    Macro<R> M;
    M.muphi = R(0);
    R Fx, Fy;
    {
      R Fsx = R(0), Fsy = R(0);
      if (lat & LAT_PHASE) {
        M.muphi = chem_local(c, phi, phi0, fs) -
                  c.klap * (lphi + c.cos_th * lphi0 + c.cos_ps * lfs);
        Fsx = M.muphi * gphx;
        Fsy = M.muphi * gphy;
      }
      Fx = Fsx + rho * c.gx;
      Fy = Fsy + rho * c.gy;
    }
    M.ux = R(0); M.uy = R(0); M.uu = R(0); M.pr = R(0);
    if (lat & LAT_FLOW) {
      const R mu = interp(fs, L.w, c.mu_s, c.mu_l, c.mu_g);
      const R jx = (f[1] - f[3]) + (f[5] - f[6]) + (f[8] - f[7]);
      const R jy = (f[2] - f[4]) + (f[5] + f[6]) - (f[7] + f[8]);
      const R snz = (f[1] + f[2] + f[3] + f[4]) + (f[5] + f[6] + f[7] + f[8]);
      // Eq. (17a,b) with the penalty force f = fs (u_s - u*), u_s = 0
      const R usx = qdiv(jx + R(0.5) * Fx, rho), usy = qdiv(jy + R(0.5) * Fy, rho);
      const R fpx = -fs * usx, fpy = -fs * usy;
      M.ux = usx + R(0.5) * fpx;
      M.uy = usy + R(0.5) * fpy;
      M.uu = M.ux * M.ux + M.uy * M.uy;
      M.S = rho * mdot + M.ux * grx + M.uy * gry;
      // modified force (reading R-FT), lagged pressure (reading R-FP)
      M.Ftx = Fx - (gpx - grx * R(1.0 / 3.0));
      M.Fty = Fy - (gpy - gry * R(1.0 / 3.0));
      M.uFt = M.ux * M.Ftx + M.uy * M.Fty;
      M.tauf = qdiv(mu, rho * R(1.0 / 3.0)) + R(0.5);
      M.Gx = Fx + rho * fpx;
      M.Gy = Fy + rho * fpy;
      R F0 = qw<R>(0) * (M.S + (R(0) - R(2) / R(3) * M.uFt) * R(4.5));
      if (c.readings & 1u) F0 += qw<R>(0) * (M.S * (R(0) - R(2) / R(3)) * R(1.5));
      const R s0 = qw<R>(0) * (-M.uu * R(1.5));
      M.pr = (R(1) / R(3)) / (R(1) - qw<R>(0)) *
             (snz + R(0.5) * M.S + (M.tauf - R(0.5)) * F0 + rho * s0);  // Eq. (17c)
    }
    M.phux = phi * M.ux;
    M.phuy = phi * M.uy;
    M.cap = rho * interp(fs, L.w, c.cp_s, c.cp_l, c.cp_g);

    R* out = a.pout;
    if (lat & LAT_FLOW) {
      if (inner) collide_flow<R, true>(g, c, out, P, gx, gy, n, f, rho, M);
      else collide_flow<R, false>(g, c, out, P, gx, gy, n, f, rho, M);
    }
    if (lat & LAT_PHASE) {
      R gq[9];
#pragma unroll
      for (int i = 0; i < 9; i++) gq[i] = pn[(9 + i) * P];
      const R phuxp = a.lin[LAG_PHUX * P + n];
      const R phuyp = a.lin[LAG_PHUY * P + n];
      if (inner) collide_phase<R, true>(g, c, out + 9 * P, P, gx, gy, n, gq, phi, phi, mdot, phuxp, phuyp, M, R(0));
      else collide_phase<R, false>(g, c, out + 9 * P, P, gx, gy, n, gq, phi, phi, mdot, phuxp, phuyp, M, R(0));
    }
    if (lat & LAT_HEAT) {
      R hq[9];
      if (masked) {
        cold_mask_h(c, wp, phi0, hq);
      } else {
#pragma unroll
        for (int i = 0; i < 9; i++) hq[i] = pn[(18 + i) * P];
      }
      if (inner) collide_heat<R, true>(g, c, out + 18 * P, P, gx, gy, n, hq, fs, L.w, T, L.rhoH, mdot, M, R(0));
      else collide_heat<R, false>(g, c, out + 18 * P, P, gx, gy, n, hq, fs, L.w, T, L.rhoH, mdot, M, R(0));
    }
    a.lout[LAG_FL * P + n] = L.fl;
    a.lout[LAG_W * P + n] = L.w;
    a.lout[LAG_P * P + n] = (lat & LAT_FLOW) ? M.pr : R(0);
    a.lout[LAG_PHUX * P + n] = (lat & LAT_PHASE) ? M.phux : R(0);
    a.lout[LAG_PHUY * P + n] = (lat & LAT_PHASE) ? M.phuy : R(0);
    a.lout[LAG_Q * P + n] = (lat & LAT_HEAT) ? M.cap * T * mdot : R(0);
    if (DIAG) {
      dvals[0] = rho;
      dvals[1] = L.w * (c.rho_s * (R(1) - L.fl) + c.rho_l * L.fl);
      dvals[2] = L.rhoH;
      dvals[3] = L.w * L.fl;
      dvals[4] = L.w;
      dvals[5] = L.w * (R(1) - L.fl);
      dvals[6] = phi;
      dvals[7] = R(0.5) * rho * M.uu;
      R tot = sg + sh;
      if (lat & LAT_FLOW) {
#pragma unroll
        for (int i = 0; i < 9; i++) tot += f[i];
      }
      dvals[8] = isfinite(tot) ? R(0) : R(1);
    }
  } else if (DIAG) {
#pragma unroll
    for (int k = 0; k < NDIAG; k++) dvals[k] = R(0);
  }

  if (DIAG)
    block_diag(dvals, s_red, a.diag_partial, tid, blockIdx.y * gridDim.x + blockIdx.x,
               gridDim.x * gridDim.y);
}

}  // namespace lbmk
