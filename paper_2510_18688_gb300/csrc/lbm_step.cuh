// lbm_step.cuh -- the fused time step (MODE_STEP) and the field read-out
// (MODE_READ) kernel for sm_103a, built on the helpers of lbm_kernels.cuh.
//
// Register budget drives the structure: the populations are never all live
// at once.  Phase A keeps only the sums of the phase and enthalpy
// populations (the loads go through the read-only path with an opaque load so
// that phase B re-reads them from L1 instead of holding them in registers
// across the barriers); the flow populations are prefetched before the
// barriers.  Phase B collides and pushes one lattice at a time.  Links that
// stay inside the grid take a branch-free streaming path; nodes on the grid
// edge take the general path with wrap, bounce-back and anti-bounce-back.
#pragma once

#include "lbm_kernels.cuh"

// resident CTAs per SM the float kernel is compiled for (register budget)
#ifndef LBM_MIN_BLOCKS_F32
#define LBM_MIN_BLOCKS_F32 4
#endif
// 1: the float step also keeps the flow populations in shared memory
#ifndef LBM_STASH_F
#define LBM_STASH_F 0
#endif

namespace lbmk {

// Loads that the compiler may not merge with later loads of the same
// address (read-only, non-coherent path; the input buffer is never written
// during a launch).
__device__ __forceinline__ float ld_sum(const float* p) {
  float v;
  asm volatile("ld.global.nc.f32 %0, [%1];" : "=f"(v) : "l"(p));
  return v;
}
__device__ __forceinline__ double ld_sum(const double* p) {
  double v;
  asm volatile("ld.global.nc.f64 %0, [%1];" : "=d"(v) : "l"(p));
  return v;
}

// Own-node population load: plain (kept in shared memory afterwards) or
// through ld_sum (re-read in phase B).
template <bool PLAIN, typename S>
__device__ __forceinline__ auto ld_pop(const S* p) {
  if constexpr (PLAIN || !(std::is_same<S, float>::value || std::is_same<S, double>::value))
    return ldp(p);
  else return ld_sum(p);
}

// Store of one post-collision population of direction i from node (x, y)
// (index n) into the destination buffer.  INNER: the link stays in the grid.
// For the enthalpy lattice (HEAT) a link leaving through a Dirichlet wall
// returns by anti-bounce-back, through an adiabatic wall by bounce-back.
template <typename R, bool INNER, bool HEAT, typename S>
__device__ __forceinline__ void push(const Geom& g, const Coef<R>& c, S* __restrict__ plane0,
                                     int P, int i, int x, int y, int n, R v) {
  if (INNER) {
    stp(plane0 + i * P + n + qy(i) * g.pitch + qx(i), v);
  } else {
    int wall;
    const long long t = stream_target(g, x, y, qx(i), qy(i), wall);
    if (t >= 0) {
      stp(plane0 + i * P + (int)t, v);
    } else {
      if (HEAT && g.bc[wall] == BC_DIRICHLET) v = -v + R(2) * qw<R>(i) * c.rr * c.T_wall[wall];
      stp(plane0 + qopp(i) * P + n, v);
    }
  }
}

// Macroscopic quantities of one node that the collisions need.
template <typename R>
struct Macro {
  R ux, uy, uu, pr, S, Ftx, Fty, uFt, Gx, Gy, tauf, muphi, phux, phuy, cap;
  R prl;  // well-balanced storage: the pressure's rounding residual (exact p = pr + prl)
};

// The three collisions are evaluated pairwise over (i, opposite of i): in
// every equilibrium and source of Eqs. (14)-(16), (19)-(20) and (25) the
// terms even in c_i are shared by the pair and the odd terms change sign, so
// each pair costs one evaluation of each part.  Pairs: (1,3), (2,4) with
// weight 1/9 and (5,7), (6,8) with weight 1/36.

// Flow collision Eqs. (11), (14)-(16) and push.
template <typename R, bool INNER, typename S>
__device__ __forceinline__ void collide_flow(const Geom& g, const Coef<R>& c, S* __restrict__ out,
                                             int P, int x, int y, int n, const R* f, R rho,
                                             const Macro<R>& M) {
  const R itau = qdiv(R(1), M.tauf);
  const R omi = R(1) - itau;
  const R fcoef = R(1) - R(0.5) * itau;
  const bool iso = (c.readings & 1u) != 0;
  // terms shared by all directions
  const R sym0 = rho * (-R(1.5) * M.uu);           // rho s_i / w_i without c_i terms
  const R fsym0 = M.S - R(3) * M.uFt;              // F_i / w_i without c_i terms
  // rest population
  {
    R F0 = fsym0;
    if (iso) F0 += M.S * (R(0) - R(2) / R(3)) * R(1.5);
    const R feq0 = M.pr * R(3) * (qw<R>(0) - R(1)) + rho * qw<R>(0) * (-R(1.5) * M.uu);
    push<R, INNER, false>(g, c, out, P, 0, x, y, n,
                          f[0] * omi + itau * feq0 + fcoef * qw<R>(0) * F0);
  }
#pragma unroll
  for (int i = 1; i <= 8; i++) {
    if (i == 3 || i == 4 || i == 7 || i == 8) continue;  // handled with its pair
    const int o = qopp(i);
    const R wi = qw<R>(i);
    const R cu = R(qx(i)) * M.ux + R(qy(i)) * M.uy;
    const R cF = R(qx(i)) * M.Gx + R(qy(i)) * M.Gy;
    const R cFt = R(qx(i)) * M.Ftx + R(qy(i)) * M.Fty;
    // even parts (equilibrium and source), odd parts
    const R eqS = M.pr * R(3) + rho * (R(4.5) * cu * cu) + sym0;
    const R eqA = rho * (R(3) * cu);
    R srcS = fsym0 + R(9) * cu * cFt;
    if (iso) srcS += M.S * (R(qx(i) * qx(i) + qy(i) * qy(i)) - R(2) / R(3)) * R(1.5);
    const R srcA = R(3) * cF;
    const R Ps = wi * (itau * eqS + fcoef * srcS);
    const R Pa = wi * (itau * eqA + fcoef * srcA);
    push<R, INNER, false>(g, c, out, P, i, x, y, n, f[i] * omi + Ps + Pa);
    push<R, INNER, false>(g, c, out, P, o, x, y, n, f[o] * omi + Ps - Pa);
  }
}

// Phase-field collision Eqs. (18)-(20) and push.  gq[0] and phir are the
// rest population and phi relative to the reader's reference (kShift), and
// dref = new reference - old reference is taken off the stored rest
// population (all three are the plain values, and dref = 0, otherwise).
template <typename R, bool INNER, typename S>
__device__ __forceinline__ void collide_phase(const Geom& g, const Coef<R>& c,
                                              S* __restrict__ out, int P, int x, int y, int n,
                                              const R* gq, R phi, R phir, R mdot, R phuxp,
                                              R phuyp, const Macro<R>& M, R dref) {
  const R itg = c.inv_tau_g;
  const R omg = R(1) - itg;
  const R gcoef = R(1) - R(0.5) * itg;
  const R emu = c.eta * M.muphi;
  // even part per unit weight: itg * eta mu + gcoef * phi mdot;
  // odd part: 3 c_i . (itg * phi u + gcoef * d(phi u)/dt)
  const R Zs = itg * emu + gcoef * phi * mdot;
  const R Vx = R(3) * (itg * M.phux + gcoef * (M.phux - phuxp));
  const R Vy = R(3) * (itg * M.phuy + gcoef * (M.phuy - phuyp));
  {
    const R geq0 = phir + (qw<R>(0) - R(1)) * emu;
    push<R, INNER, false>(g, c, out, P, 0, x, y, n,
                          gq[0] * omg + itg * geq0 + gcoef * qw<R>(0) * phi * mdot - dref);
  }
#pragma unroll
  for (int i = 1; i <= 8; i++) {
    if (i == 3 || i == 4 || i == 7 || i == 8) continue;
    const int o = qopp(i);
    const R wi = qw<R>(i);
    const R Ps = wi * Zs;
    const R Pa = wi * (R(qx(i)) * Vx + R(qy(i)) * Vy);
    push<R, INNER, false>(g, c, out, P, i, x, y, n, gq[i] * omg + Ps + Pa);
    push<R, INNER, false>(g, c, out, P, o, x, y, n, gq[o] * omg + Ps - Pa);
  }
}

// Enthalpy TRT collision Eqs. (23)-(27) and push.  h[0] and rhoHr are the
// rest population and rho H relative to the reader's reference (kShift);
// dref as in collide_phase.
template <typename R, bool INNER, typename S>
__device__ __forceinline__ void collide_heat(const Geom& g, const Coef<R>& c, S* __restrict__ out,
                                             int P, int x, int y, int n, const R* h, R fs, R w,
                                             R T, R rhoHr, R mdot, const Macro<R>& M, R dref) {
  const R lam = interp(fs, w, c.lam_s, c.lam_l, c.lam_g);
  const R taua = R(0.5) + lam * c.inv_rr3;
  // magic relation of the TRT (Eq. (27)): 1/tau_s + 1/tau_a = 2
  const R ia = qdiv(R(1), taua), is = R(2) - ia;
  const R hcoef = R(1) - R(0.5) * ia;
  const R CT = M.cap * T;
  const R Hsrc = hcoef * CT * mdot;
  const R rrT = c.rr * T;
  {
    // rest population: purely symmetric
    const R heq0 = rhoHr - rrT + qw<R>(0) * (rrT - CT * M.uu * R(1.5));
    push<R, INNER, true>(g, c, out, P, 0, x, y, n,
                         h[0] - (h[0] - heq0) * is + qw<R>(0) * Hsrc - dref);
  }
#pragma unroll
  for (int i = 1; i <= 8; i++) {
    if (i == 3 || i == 4 || i == 7 || i == 8) continue;
    const int o = qopp(i);
    const R wi = qw<R>(i);
    const R cu = R(qx(i)) * M.ux + R(qy(i)) * M.uy;
    const R es = wi * (rrT + CT * (R(4.5) * cu * cu - R(1.5) * M.uu));
    const R ea = wi * (CT * (R(3) * cu));
    const R hs = R(0.5) * (h[i] + h[o]), ha = R(0.5) * (h[i] - h[o]);
    const R Da = (ha - ea) * ia;
    const R Ds = (hs - es) * is - wi * Hsrc;
    push<R, INNER, true>(g, c, out, P, i, x, y, n, h[i] - Da - Ds);
    push<R, INNER, true>(g, c, out, P, o, x, y, n, h[o] + Da - Ds);
  }
}

// ---------------------------------------------------------------------------
// well-balanced float storage (kShift; see lbm_kernels.cuh)
// ---------------------------------------------------------------------------

// True when the node upstream of (x, y) in direction i, (x, y) - c_i, lies
// beyond a wall: population i of (x, y) then came back from (x, y) itself.
__device__ __forceinline__ bool upstream_wall(const Geom& g, int x, int y, int i) {
  const int tx = x - qx(i), ty = y - qy(i);
  return (tx < 0 && g.bc[0] != BC_PERIODIC) || (tx >= g.nx && g.bc[1] != BC_PERIODIC) ||
         (ty < 0 && g.bc[2] != BC_PERIODIC) || (ty >= g.ny && g.bc[3] != BC_PERIODIC);
}

// Flow collision Eqs. (11), (14)-(16) and push for remainders: fb[i] = f_i -
// 3 (w_i - delta_i0) p, the populations referred to p = M.pr, the node's new
// pressure as stored (node_macros forms them; the exact pressure is p +
// M.prl).  The pressure part of the equilibrium and the references then meet
// as f*_i - 3 (w_i - delta_i0) p = (1 - 1/tau) fb_i + (rho s_i + 3 (w_i -
// delta_i0) prl) / tau + (1 - 1/2tau) F_i.
template <bool INNER, typename S>
__device__ __forceinline__ void collide_flow_wb(const Geom& g, const Coef<float>& c,
                                                S* __restrict__ out, int P, int x, int y, int n,
                                                const float* fb, float rho,
                                                const Macro<float>& M) {
  const float itau = qdiv(1.f, M.tauf);
  const float omi = 1.f - itau;
  const float fcoef = 1.f - 0.5f * itau;
  const bool iso = (c.readings & 1u) != 0;
  const float sym0 = rho * (-1.5f * M.uu);
  const float fsym0 = M.S - 3.f * M.uFt;
  {
    float F0 = fsym0;
    if (iso) F0 += M.S * (0.f - 2.f / 3.f) * 1.5f;
    push<float, INNER, false>(g, c, out, P, 0, x, y, n,
                              fb[0] * omi +
                                  itau * (qw<float>(0) * sym0 + 3.f * (qw<float>(0) - 1.f) * M.prl) +
                                  fcoef * qw<float>(0) * F0);
  }
#pragma unroll
  for (int i = 1; i <= 8; i++) {
    if (i == 3 || i == 4 || i == 7 || i == 8) continue;  // handled with its pair
    const int o = qopp(i);
    const float wi = qw<float>(i);
    const float cu = float(qx(i)) * M.ux + float(qy(i)) * M.uy;
    const float cF = float(qx(i)) * M.Gx + float(qy(i)) * M.Gy;
    const float cFt = float(qx(i)) * M.Ftx + float(qy(i)) * M.Fty;
    const float eqS = rho * (4.5f * cu * cu) + sym0 + 3.f * M.prl;
    const float eqA = rho * (3.f * cu);
    float srcS = fsym0 + 9.f * cu * cFt;
    if (iso) srcS += M.S * (float(qx(i) * qx(i) + qy(i) * qy(i)) - 2.f / 3.f) * 1.5f;
    const float srcA = 3.f * cF;
    const float Ps = wi * (itau * eqS + fcoef * srcS);
    const float Pa = wi * (itau * eqA + fcoef * srcA);
    push<float, INNER, false>(g, c, out, P, i, x, y, n, fb[i] * omi + Ps + Pa);
    push<float, INNER, false>(g, c, out, P, o, x, y, n, fb[o] * omi + Ps - Pa);
  }
}

// Store of an enthalpy remainder X (the post-collision population minus the
// writer's old reference ref_old = w_i rho_ref Cp_ref T') referred to the
// destination's new reference w_i rho_ref Cp_ref T_dest (T_self for a
// population a wall returns).  Anti-bounce-back at a Dirichlet wall:
// -h* + 2 w_i rho_ref Cp_ref T_w, as remainder -X + (wTw - ref_old) + (wTw
// - ref_new).
template <bool INNER, typename S>
__device__ __forceinline__ void push_h(const Geom& g, const Coef<float>& c, S* __restrict__ plane0,
                                       int P, int i, int x, int y, int n, float X, float ref_old,
                                       float wrr, float T_self, float T_dest) {
  if (INNER) {
    stp(plane0 + i * P + n + qy(i) * g.pitch + qx(i),
        X - ref_delta(ref_hi(wrr, T_dest), ref_old));
  } else {
    int wall;
    const long long t = stream_target(g, x, y, qx(i), qy(i), wall);
    if (t >= 0) {
      stp(plane0 + i * P + (int)t, X - ref_delta(ref_hi(wrr, T_dest), ref_old));
    } else {
      const float rn = ref_hi(wrr, T_self);
      float v;
      if (g.bc[wall] == BC_DIRICHLET) {
        const float wTw = ref_hi(wrr, c.T_wall[wall]);
        v = -X + (ref_delta(wTw, ref_old) + ref_delta(wTw, rn));
      } else {
        v = X - ref_delta(rn, ref_old);
      }
      stp(plane0 + qopp(i) * P + n, v);
    }
  }
}

// Enthalpy TRT collision Eqs. (23)-(27) and push for remainders: hr[i] = h_i
// minus the node's old references (ref_h0 for i = 0, aold = w_1 rho_ref
// Cp_ref T' on the axes, dold = w_5 rho_ref Cp_ref T' on the diagonals),
// e = rho H minus the sum of those references, dT = T - T'.  With these the
// non-equilibrium parts are h0 - heq0 = hr0 - e + (1 - w_0) rho_ref Cp_ref
// dT + 3/2 w_0 C T u.u and, for a pair, hs - es = hs' - w_i (rho_ref Cp_ref
// dT + C T (9/2 (c.u)^2 - 3/2 u.u)); the rest remainder takes off dref0 =
// new ref_h0 - old ref_h0, the others are referred to their destinations
// (push_h).  sT: new temperatures of the tile and its ring, hc: own index.
template <bool INNER, typename S>
__device__ __forceinline__ void collide_heat_wb(const Geom& g, const Coef<float>& c,
                                                S* __restrict__ out, int P, int x, int y, int n,
                                                const float* hr, float fs, float w, float T,
                                                float dT, float e, float mdot,
                                                const Macro<float>& M, float aold, float dold,
                                                float dref0, const float* sT, int hc) {
  const float lam = interp(fs, w, c.lam_s, c.lam_l, c.lam_g);
  const float taua = 0.5f + lam * c.inv_rr3;
  // magic relation of the TRT (Eq. (27)): 1/tau_s + 1/tau_a = 2
  const float ia = qdiv(1.f, taua), is = 2.f - ia;
  const float hcoef = 1.f - 0.5f * ia;
  const float CT = M.cap * T;
  const float Hsrc = hcoef * CT * mdot;
  const float rrdT = c.rr * dT;
  {
    const float d0 = hr[0] - e + c.rr_rest * dT + 1.5f * qw<float>(0) * CT * M.uu;
    stp(out + n, hr[0] - d0 * is + qw<float>(0) * Hsrc - dref0);
  }
#pragma unroll
  for (int i = 1; i <= 8; i++) {
    if (i == 3 || i == 4 || i == 7 || i == 8) continue;
    const int o = qopp(i);
    const float wi = qw<float>(i);
    const float cu = float(qx(i)) * M.ux + float(qy(i)) * M.uy;
    const float es = wi * (rrdT + CT * (4.5f * cu * cu - 1.5f * M.uu));
    const float ea = wi * (CT * (3.f * cu));
    const float hs = 0.5f * (hr[i] + hr[o]), ha = 0.5f * (hr[i] - hr[o]);
    const float Da = (ha - ea) * ia;
    const float Ds = (hs - es) * is - wi * Hsrc;
    const float ro = i <= 4 ? aold : dold;
    const float wrr = i <= 4 ? c.wrr1 : c.wrr5;
    push_h<INNER>(g, c, out, P, i, x, y, n, hr[i] - Da - Ds, ro, wrr, T,
                  sT[hc + qy(i) * HX + qx(i)]);
    push_h<INNER>(g, c, out, P, o, x, y, n, hr[o] + Da - Ds, ro, wrr, T,
                  sT[hc + qy(o) * HX + qx(o)]);
  }
}

// Phase B of one node up to its collisions: the isotropic stencils (reading
// R-FD: grad chi = 3 sum w_i c_i chi(x + c_i), lap chi = 6 sum w_i (chi(x +
// c_i) - chi(x))) of phi, phi0, f_s, rho and the lagged pressure, the
// chemical potential of Eq. (6), the surface-tension, body and penalty
// forces, velocity and pressure of Eq. (17), the source S and the modified
// force of Eq. (16) (readings R-FT, R-FP).  cphi, cfs, crho point at the node
// in halo arrays of row stride sh; cp, cphi0 at the node in arrays of row
// stride sb.  f: the node's flow populations; with well-balanced storage
// (WB) they are remainders over 3 (w_i - delta_i0) p_src(i), the lagged
// pressure of the node each came from (the node itself for a population a
// wall returned), and on return they are referred to the node's new pressure
// M.pr instead (the form collide_flow_wb takes).
// sum_i w_i c_i v(x + c_i) over opposite neighbours taken in pairs: the
// difference of two close neighbour values is exact in float, so a small
// gradient of a large field (the pressure of a compressed gas, ~1e-9 per node
// against p ~ 6e-4) keeps its relative precision instead of being lost in
// the rounding of the products w_i v.
template <typename R>
__device__ __forceinline__ void grad_pairs(const R* v, int s, R& gx, R& gy) {
  const R d13 = v[1] - v[-1], d24 = v[s] - v[-s];
  const R d57 = v[s + 1] - v[-s - 1], d86 = v[-s + 1] - v[s - 1];
  gx = qw<R>(1) * d13 + qw<R>(5) * (d57 + d86);
  gy = qw<R>(1) * d24 + qw<R>(5) * (d57 - d86);
}

template <typename R, bool WB>
__device__ __forceinline__ void node_macros(const Geom& g, const Coef<R>& c, int lat, int gx,
                                            int gy, bool inner, const Local<R>& L, R phi0, R pp,
                                            R* f, const R* cphi, const R* cfs,
                                            const R* crho, int sh, const R* cp,
                                            const R* cphi0, int sb, Macro<R>& M) {
  R gphx = R(0), gphy = R(0), lphi = R(0), lphi0 = R(0), lfs = R(0);
  R grx = R(0), gry = R(0), gpx = R(0), gpy = R(0);
  if (lat & LAT_PHASE) {
#pragma unroll
    for (int i = 1; i < 9; i++) {
      const int oh = qy(i) * sh + qx(i), ob = qy(i) * sb + qx(i);
      const R wi = qw<R>(i);
      lphi += R(2) * wi * (cphi[oh] - cphi[0]);
      lphi0 += R(2) * wi * (cphi0[ob] - cphi0[0]);
      lfs += R(2) * wi * (cfs[oh] - cfs[0]);
    }
    grad_pairs(cphi, sh, gphx, gphy);
  }
  if (lat & LAT_FLOW) {
    grad_pairs(crho, sh, grx, gry);
    grad_pairs(cp, sb, gpx, gpy);
  }
  gphx *= R(3); gphy *= R(3); lphi *= R(3); lphi0 *= R(3); lfs *= R(3);
  grx *= R(3); gry *= R(3); gpx *= R(3); gpy *= R(3);

  const R phi = L.phi, fs = L.fs, rho = L.rho, mdot = L.mdot;
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
    R jx = (f[1] - f[3]) + (f[5] - f[6]) + (f[8] - f[7]);
    R jy = (f[2] - f[4]) + (f[5] + f[6]) - (f[7] + f[8]);
    // opposite populations summed first: near equilibrium they differ mainly
    // by the +-3 w_i rho c_i.u part, which then cancels exactly instead of
    // after a rounding, and the small remainder keeps its precision
    R snz = ((f[1] + f[3]) + (f[2] + f[4])) + ((f[5] + f[7]) + (f[6] + f[8]));
    R dps[WB ? 9 : 1];  // well-balanced storage: p_src(i) - pp, then p_src(i) - p
    if constexpr (WB) {
      // add the moments of the references 3 w_i p_src(i), as differences
      // from the node's own lagged pressure pp (whose share, 3 (1 - w_0) pp
      // in the sum, returns pp itself in Eq. (17c) below)
      dps[0] = R(0);
#pragma unroll
      for (int i = 1; i < 9; i++)
        dps[i] = (!inner && upstream_wall(g, gx, gy, i)) ? R(0)
                                                         : cp[-(qy(i) * sb + qx(i))] - pp;
      const R w1 = qw<R>(1), w5 = qw<R>(5);
      jx += R(3) * (w1 * (dps[1] - dps[3]) + w5 * ((dps[5] - dps[6]) + (dps[8] - dps[7])));
      jy += R(3) * (w1 * (dps[2] - dps[4]) + w5 * ((dps[5] + dps[6]) - (dps[7] + dps[8])));
      snz += R(3) * (w1 * ((dps[1] + dps[3]) + (dps[2] + dps[4])) +
                     w5 * ((dps[5] + dps[7]) + (dps[6] + dps[8])));
    }
    // Eq. (17a,b) with the penalty force f = fs (u_s - u*), u_s = 0
    const R irho = qdiv(R(1), rho);
    R fpx, fpy;
    if constexpr (WB) {
      // Float states: u = (1 - fs/2) (j + F/2) / rho rounded once.  The
      // weakly damped acoustics of a long run (the closed gas column of the
      // Stefan problem) carry the velocity's per-step rounding forward: with
      // (j + F/2) multiplied by a rounded 1/rho the 50,000-step Stefan
      // velocity is 2.5e-4 off the FP64 oracle, with this 7.4e-5.  j + F/2
      // is kept as s + e (TwoSum), the quotient of s is corrected by its
      // exact residual (FMA) plus e, divided by rho.
      float sx, esx, sy, esy;
      two_sum(jx, 0.5f * Fx, sx, esx);
      two_sum(jy, 0.5f * Fy, sy, esy);
      const float qx = qdiv(sx, rho), qy = qdiv(sy, rho);
      const float qxl = (fmaf(-qx, rho, sx) + esx) * irho;
      const float qyl = (fmaf(-qy, rho, sy) + esy) * irho;
      const float k = 1.f - 0.5f * fs;
      M.ux = fmaf(qx, k, qxl * k);
      M.uy = fmaf(qy, k, qyl * k);
      fpx = -fs * (qx + qxl);
      fpy = -fs * (qy + qyl);
    } else {
      const R usx = (jx + R(0.5) * Fx) * irho, usy = (jy + R(0.5) * Fy) * irho;
      fpx = -fs * usx;
      fpy = -fs * usy;
      M.ux = usx + R(0.5) * fpx;
      M.uy = usy + R(0.5) * fpy;
    }
    M.uu = M.ux * M.ux + M.uy * M.uy;
    M.S = rho * mdot + M.ux * grx + M.uy * gry;
    // modified force (reading R-FT), lagged pressure (reading R-FP)
    M.Ftx = Fx - (gpx - grx * R(1.0 / 3.0));
    M.Fty = Fy - (gpy - gry * R(1.0 / 3.0));
    M.uFt = M.ux * M.Ftx + M.uy * M.Fty;
    if constexpr (WB) {
      // tau_f = 3 mu / rho + 1/2 rounded once (with the velocity above but
      // tau_f from two roundings the Stefan velocity stays at 1.2e-4; the
      // same tau_f alone, velocity as before, leaves it at 2.5e-4):
      // mu / rho = q0 + qe (qe from the
      // exact residual of q0, by FMA), then 3 (q0 + qe) + 1/2 with the
      // errors of 3 q0 (FMA) and of the sum (TwoSum) added back once
      const float q0 = qdiv(mu, rho);
      const float qe = fmaf(-q0, rho, mu) * irho;
      const float t1 = 3.f * q0, t1e = fmaf(3.f, q0, -t1);
      float sm, se;
      two_sum(t1, 0.5f, sm, se);
      M.tauf = sm + (se + (t1e + 3.f * qe));
    } else {
      M.tauf = R(3) * mu * irho + R(0.5);
    }
    M.Gx = Fx + rho * fpx;
    M.Gy = Fy + rho * fpy;
    // F_0 of Eq. (16)
    R F0 = qw<R>(0) * (M.S + (R(0) - R(2) / R(3) * M.uFt) * R(4.5));
    if (c.readings & 1u) F0 += qw<R>(0) * (M.S * (R(0) - R(2) / R(3)) * R(1.5));
    const R s0 = qw<R>(0) * (-M.uu * R(1.5));
    const R dp = (R(1) / R(3)) / (R(1) - qw<R>(0)) *
                 (snz + R(0.5) * M.S + (M.tauf - R(0.5)) * F0 + rho * s0);  // Eq. (17c)
    M.prl = R(0);
    if constexpr (WB) {
      // p = pp + dp, rounded once; the rounding residual (exact, TwoSum)
      // goes into the stored remainders through the equilibrium (see
      // collide_flow_wb), so that a slowly rising pressure is not rounded
      // off step after step
      M.pr = pp + dp;
      const R bb = M.pr - pp;
      M.prl = (pp - (M.pr - bb)) + (dp - bb);
#pragma unroll
      for (int i = 0; i < 9; i++) dps[i] -= bb;  // p_src(i) - p
      // the populations referred to the new pressure
      f[0] += R(3) * (qw<R>(0) - R(1)) * dps[0];
#pragma unroll
      for (int i = 1; i < 9; i++) f[i] += R(3) * qw<R>(i) * dps[i];
    } else {
      M.pr = dp;
    }
  }
  M.phux = phi * M.ux;
  M.phuy = phi * M.uy;
  // heat capacity rho Cp (Eq. (10)); float storage forms it as the next
  // step's reader of this node will (its reference state)
  if constexpr (WB) M.cap = cap_rn(c, fs, L.w);
  else M.cap = rho * interp(fs, L.w, c.cp_s, c.cp_l, c.cp_g);
}

// The node's contributions to the FP64 diagnostics (lbm_diag order) and a
// non-finite flag: a non-finite population anywhere makes one of the sums
// non-finite.
template <typename R>
__device__ __forceinline__ void diag_values(const Coef<R>& c, int lat, const Local<R>& L,
                                            const Macro<R>& M, R sg, R sh, const R* f,
                                            R* dvals) {
  dvals[0] = L.rho;
  dvals[1] = L.w * (c.rho_s * (R(1) - L.fl) + c.rho_l * L.fl);
  dvals[2] = L.rhoH;
  dvals[3] = L.w * L.fl;
  dvals[4] = L.w;
  dvals[5] = L.w * (R(1) - L.fl);
  dvals[6] = L.phi;
  dvals[7] = R(0.5) * L.rho * M.uu;
  R tot = sg + sh;
  if (lat & LAT_FLOW) {
#pragma unroll
    for (int i = 0; i < 9; i++) tot += f[i];
  }
  dvals[8] = finite(tot) ? R(0) : R(1);
}

// One tile (bx, by) of one grid: the whole step (or read-out) for its
// TX x TYS nodes (a Shape).  b / nb: the tile's index and the grid's tile
// count for the diagnostic partials (b < 0: taken from the CTA's position in
// its grid).  LATC: compile-time lattice set (7 = all three) or 0 (read at
// run time).  Every thread of the CTA calls it.
template <typename R, int MODE, bool DIAG, int LATC, typename S = R, int TYS = TY>
__device__ __forceinline__ void step_tile(const Args<R, S>& a, int bx, int by, int b, int nb) {
  // the tile's shape; these hide the namespace's 32 x 8 constants
  constexpr int TY = Shape<TYS>::TY, HN = Shape<TYS>::HN, NT = Shape<TYS>::NT;
  constexpr int RING = Shape<TYS>::RING;
  const Geom& g = a.g;
  const Coef<R>& c = a.c;
  const int lat = LATC ? LATC : g.lattices;
  const int P = (int)g.plane;  // 27 planes fit in 31 bits (checked at create)

  // FP32 steps keep the own node's phase and enthalpy populations in shared
  // memory between phase A and phase B (18 KB per 256-node CTA) instead of
  // reading them again through L1/L2; 32 x 16 tiles have no room for it
  // within the 48 KB of static shared memory and read them again
  constexpr bool STASH = sizeof(R) == 4 && MODE == MODE_STEP && TYS <= 8;
  constexpr bool STASHF = STASH && LBM_STASH_F;
  __shared__ R s_pop[STASH ? 18 : 1][NT];
  __shared__ R s_fpop[STASHF ? 9 : 1][NT];
  __shared__ R s_phu[STASH ? 2 : 1][NT];  // lagged phi u of the own node
  __shared__ R s_phi[HN], s_fs[HN], s_rho[HN], s_p[HN], s_phi0[HN];
  __shared__ R s_rsg[RING][NPART], s_rsh[RING][NPART];
  __shared__ R s_rfl[RING], s_rw[RING], s_rQ[RING];
  // well-balanced float storage: new temperatures of the tile and its ring
  // (references of the pushed enthalpy populations), lagged temperatures of
  // the ring and the own node's old temperature and heat capacity
  constexpr bool WB = kShift<R>;
  __shared__ R s_T[WB ? HN : 1], s_rT[WB ? RING : 1];
  __shared__ R s_Tp[WB ? 2 : 1][NT];
  __shared__ int s_rmask[RING];
  __shared__ R s_red[NT / 32][NDIAG];

  const int tx = threadIdx.x, ty = threadIdx.y;
  const int tid = ty * TX + tx;
  const int x0 = bx * TX, y0 = by * TY;
  const int gx = x0 + tx, gy = y0 + ty;
  const bool valid = gx < g.nx && gy < g.ny;
  const int mx = wrap_or_clamp(gx, g.nx, g.bc[0], g.bc[1]);
  const int my = wrap_or_clamp(gy, g.ny, g.bc[2], g.bc[3]);
  const int n = my * g.pitch + mx;

  // ---- phase A0: a third of one ring node's phase/enthalpy populations ----
  // (job j: ring node j / NPART, part j % NPART; one pass of the CTA unless
  // the tile is short)
  auto ring_load = [&](int job) {
    const int k = job / NPART, part = job - k * NPART;
    int hx, hy;
    ring_pos<TYS>(k, hx, hy);
    const int rx = wrap_or_clamp(x0 + hx - 1, g.nx, g.bc[0], g.bc[1]);
    const int ry = wrap_or_clamp(y0 + hy - 1, g.ny, g.bc[2], g.bc[3]);
    const int m = ry * g.pitch + rx;
    const bool masked = g.has_mask && a.mask[m];
    const S* pm = a.pin + m;
    // part 0: g0..g5; part 1: g6..g8 and h0..h2; part 2: h3..h8
    R sgp = R(0), shp = R(0);
    if (part == 0) {
      if (lat & LAT_PHASE) {
        R v[6];
#pragma unroll
        for (int i = 0; i < 6; i++) v[i] = ldp(pm + (9 + i) * P);
        sgp = v[0] + v[1] + v[2] + v[3] + v[4] + v[5];
      }
      const int hi = hy * HX + hx;
      s_phi0[hi] = a.phi0[m];
      s_p[hi] = a.lin[LAG_P * P + m];
      s_rfl[k] = a.lin[LAG_FL * P + m];
      s_rw[k] = a.lin[LAG_W * P + m];
      s_rQ[k] = a.lin[LAG_Q * P + m];
      if constexpr (WB) s_rT[k] = a.lin[LAG_T * P + m];
      s_rmask[k] = masked ? 1 : 0;
    } else if (part == 1) {
      if (lat & LAT_PHASE) sgp = ldp(pm + 15 * P) + ldp(pm + 16 * P) + ldp(pm + 17 * P);
      if ((lat & LAT_HEAT) && !masked) shp = ldp(pm + 18 * P) + ldp(pm + 19 * P) + ldp(pm + 20 * P);
    } else {
      if ((lat & LAT_HEAT) && !masked) {
        R v[6];
#pragma unroll
        for (int i = 0; i < 6; i++) v[i] = ldp(pm + (21 + i) * P);
        shp = v[0] + v[1] + v[2] + v[3] + v[4] + v[5];
      }
    }
    s_rsg[k][part] = sgp;
    s_rsh[k][part] = shp;
  };
  if constexpr (RING * NPART <= NT) {
    if (tid < RING * NPART) ring_load(tid);
  } else {
    for (int job = tid; job < RING * NPART; job += NT) ring_load(job);
  }

  // ---- phase A1: own node (sums only; f prefetched for phase B) ----------
  const S* pn = a.pin + n;
  const R phi0 = a.phi0[n];
  const R flp = a.lin[LAG_FL * P + n];
  const R wp = a.lin[LAG_W * P + n];
  const R pp = a.lin[LAG_P * P + n];
  const R Qp = a.lin[LAG_Q * P + n];
  // the lagged phi u is needed only by the phase collision in phase B; it is
  // loaded here with everything else so that no load waits in phase B
  R phuxp = R(0), phuyp = R(0);
  if (MODE == MODE_STEP && (lat & LAT_PHASE)) {
    phuxp = a.lin[LAG_PHUX * P + n];
    phuyp = a.lin[LAG_PHUY * P + n];
    if (STASH) {
      s_phu[0][tid] = phuxp;
      s_phu[STASH ? 1 : 0][tid] = phuyp;
    }
  }
  const bool masked = (lat & LAT_HEAT) && g.has_mask && a.mask[n];
  R f[9];
  if (lat & LAT_FLOW) {
#pragma unroll
    for (int i = 0; i < 9; i++) f[i] = ldp(pn + i * P);
    if (STASHF) {
#pragma unroll
      for (int i = 0; i < 9; i++) s_fpop[STASHF ? i : 0][tid] = f[i];
    }
  }
  R sg = R(0), sh = R(0);
  if (lat & LAT_PHASE) {
    R v[9];
#pragma unroll
    for (int i = 0; i < 9; i++) v[i] = ld_pop<STASH>(pn + (9 + i) * P);
    sg = sum_g(v);
    if (STASH) {
#pragma unroll
      for (int i = 0; i < 9; i++) s_pop[i][tid] = v[i];
    }
  }
  // well-balanced float storage: the node's lagged temperature and its heat
  // capacity at the lags (the reference state of its enthalpy populations)
  R Tp = R(0), Cp = R(0);
  if constexpr (WB) {
    if (lat & LAT_HEAT) {
      Tp = a.lin[LAG_T * P + n];
      Cp = cap_rn(c, fs_rn(wp, flp, phi0), wp);
      s_Tp[0][tid] = Tp;
      s_Tp[WB ? 1 : 0][tid] = Cp;
    }
  }
  if (lat & LAT_HEAT) {
    R v[9];
    if (masked) {
      cold_mask_h(c, wp, phi0, v);
      if constexpr (WB) {
        v[0] -= ref_h0(c, wp, flp, Tp, Cp);
#pragma unroll
        for (int i = 1; i < 9; i++) v[i] -= ref_hi(i <= 4 ? c.wrr1 : c.wrr5, Tp);
      }
    } else {
#pragma unroll
      for (int i = 0; i < 9; i++) v[i] = ld_pop<STASH>(pn + (18 + i) * P);
    }
    sh = sum_h(v);
    if (STASH) {
#pragma unroll
      for (int i = 0; i < 9; i++) s_pop[STASH ? 9 + i : 0][tid] = v[i];
    }
  }
  Local<R> L;
  if constexpr (WB) L = local_state_wb(c, lat, sg, sh, flp, wp, Qp, Tp, Cp, phi0);
  else L = local_state(c, lat, sg, sh, flp, wp, Qp, phi0);
  {
    const int hi = (ty + 1) * HX + (tx + 1);
    s_phi[hi] = L.phi;
    s_fs[hi] = L.fs;
    s_rho[hi] = L.rho;
    s_p[hi] = pp;
    s_phi0[hi] = phi0;
    if constexpr (WB) s_T[hi] = L.T;
  }
  __syncthreads();

  // ---- phase A2: inversion, order parameter, properties of the ring ---------
  if (tid < RING) {
    const int k = tid;
    int hx, hy;
    ring_pos<TYS>(k, hx, hy);
    const int hi = hy * HX + hx;
    const R q0 = s_phi0[hi];
    const R wq = s_rw[k];
    const R sgq = s_rsg[k][0] + s_rsg[k][1];
    R Tq = R(0), Cq = R(0);
    if constexpr (WB) {
      if (lat & LAT_HEAT) {
        Tq = s_rT[k];
        Cq = cap_rn(c, fs_rn(wq, s_rfl[k], q0), wq);
      }
    }
    R shq;
    if ((lat & LAT_HEAT) && s_rmask[k]) {
      R hq[9];
      cold_mask_h(c, wq, q0, hq);
      if constexpr (WB) {
        hq[0] -= ref_h0(c, wq, s_rfl[k], Tq, Cq);
#pragma unroll
        for (int i = 1; i < 9; i++) hq[i] -= ref_hi(i <= 4 ? c.wrr1 : c.wrr5, Tq);
      }
      shq = sum_h(hq);
    } else {
      shq = s_rsh[k][1] + s_rsh[k][2];
    }
    Local<R> Lq;
    if constexpr (WB) Lq = local_state_wb(c, lat, sgq, shq, s_rfl[k], wq, s_rQ[k], Tq, Cq, q0);
    else Lq = local_state(c, lat, sgq, shq, s_rfl[k], wq, s_rQ[k], q0);
    s_phi[hi] = Lq.phi;
    s_fs[hi] = Lq.fs;
    s_rho[hi] = Lq.rho;
    if constexpr (WB) s_T[hi] = Lq.T;
  }
  __syncthreads();

  // ---- phase B: stencils, macros, collisions, streaming -------------------
  // Instantiated twice: for a tile whose nodes and ring are all inside the
  // grid (block-uniform branch) every node is valid and every link stays in
  // the grid, so that path carries no boundary logic at all.
  auto phase_b = [&](auto interior) {
  constexpr bool IN = decltype(interior)::value;
  R dvals[NDIAG];
  Macro<R> M;
  // links that stay inside the grid need no boundary logic
  const bool inner = IN || (gx > 0 && gx < g.nx - 1 && gy > 0 && gy < g.ny - 1);
  const bool valid_n = IN || valid;
  if (valid_n) {
    const int hc = (ty + 1) * HX + (tx + 1);
    if (STASHF && (lat & LAT_FLOW)) {
#pragma unroll
      for (int i = 0; i < 9; i++) f[i] = s_fpop[STASHF ? i : 0][tid];
    }
    node_macros<R, WB>(g, c, lat, gx, gy, inner, L, phi0, pp, f, s_phi + hc, s_fs + hc,
                       s_rho + hc, HX, s_p + hc, s_phi0 + hc, HX, M);
    // diagnostics of this state, reduced over the warp before the
    // collisions so that none of their inputs stays live through them
    if (DIAG) diag_values(c, lat, L, M, sg, sh, f, dvals);
  } else if (DIAG) {
#pragma unroll
    for (int k = 0; k < NDIAG; k++) dvals[k] = R(0);
  }
  if (DIAG) block_diag_warps(dvals, s_red, tid);

  if (valid_n) {
    const R phi = L.phi, fs = L.fs, rho = L.rho, T = L.T, mdot = L.mdot;

    if (MODE == MODE_STEP) {
      S* out = a.pout;
      if (lat & LAT_FLOW) {
        if constexpr (WB) {
          if (inner) collide_flow_wb<true>(g, c, out, P, gx, gy, n, f, rho, M);
          else collide_flow_wb<false>(g, c, out, P, gx, gy, n, f, rho, M);
        } else {
          if (inner) collide_flow<R, true>(g, c, out, P, gx, gy, n, f, rho, M);
          else collide_flow<R, false>(g, c, out, P, gx, gy, n, f, rho, M);
        }
      }
      if (lat & LAT_PHASE) {
        R gq[9];
#pragma unroll
        for (int i = 0; i < 9; i++) gq[i] = STASH ? s_pop[i][tid] : ldp(pn + (9 + i) * P);
        if (STASH) {
          phuxp = s_phu[0][tid];
          phuyp = s_phu[STASH ? 1 : 0][tid];
        }
        // change of reference between this step's reader and the next one
        R dref = R(0);
        if constexpr (WB) dref = ref_delta(rest_ref_g(L.w, phi0), rest_ref_g(wp, phi0));
        if (inner) collide_phase<R, true>(g, c, out + 9 * P, P, gx, gy, n, gq, phi, L.phir, mdot, phuxp, phuyp, M, dref);
        else collide_phase<R, false>(g, c, out + 9 * P, P, gx, gy, n, gq, phi, L.phir, mdot, phuxp, phuyp, M, dref);
      }
      if (lat & LAT_HEAT) {
        R hq[9];
        // well-balanced storage: the node's old temperature and heat capacity
        R Tq = R(0), Cq = R(0);
        if constexpr (WB) {
          Tq = s_Tp[0][tid];
          Cq = s_Tp[WB ? 1 : 0][tid];
        }
        if (STASH) {
#pragma unroll
          for (int i = 0; i < 9; i++) hq[i] = s_pop[STASH ? 9 + i : 0][tid];
        } else if (masked) {
          // the populations the cold mask sets, as remainders when stored so
          cold_mask_h(c, wp, phi0, hq);
          if constexpr (WB) {
            hq[0] -= ref_h0(c, wp, flp, Tq, Cq);
#pragma unroll
            for (int i = 1; i < 9; i++) hq[i] -= ref_hi(i <= 4 ? c.wrr1 : c.wrr5, Tq);
          }
        } else {
#pragma unroll
          for (int i = 0; i < 9; i++) hq[i] = ldp(pn + (18 + i) * P);
        }
        if constexpr (WB) {
          // references: this node's old state, and the new one its rest
          // population is stored against
          const R dref0 = ref_delta(ref_h0(c, L.w, L.fl, T, M.cap), ref_h0(c, wp, flp, Tq, Cq));
          const R aold = ref_hi(c.wrr1, Tq), dold = ref_hi(c.wrr5, Tq);
          const int hc = (ty + 1) * HX + (tx + 1);
          if (inner)
            collide_heat_wb<true>(g, c, out + 18 * P, P, gx, gy, n, hq, fs, L.w, T, T - Tq,
                                  L.rhoHr, mdot, M, aold, dold, dref0, s_T, hc);
          else
            collide_heat_wb<false>(g, c, out + 18 * P, P, gx, gy, n, hq, fs, L.w, T, T - Tq,
                                   L.rhoHr, mdot, M, aold, dold, dref0, s_T, hc);
        } else {
          if (inner) collide_heat<R, true>(g, c, out + 18 * P, P, gx, gy, n, hq, fs, L.w, T, L.rhoHr, mdot, M, R(0));
          else collide_heat<R, false>(g, c, out + 18 * P, P, gx, gy, n, hq, fs, L.w, T, L.rhoHr, mdot, M, R(0));
        }
      }
      a.lout[LAG_FL * P + n] = L.fl;
      a.lout[LAG_W * P + n] = L.w;
      a.lout[LAG_P * P + n] = (lat & LAT_FLOW) ? M.pr : R(0);
      a.lout[LAG_PHUX * P + n] = (lat & LAT_PHASE) ? M.phux : R(0);
      a.lout[LAG_PHUY * P + n] = (lat & LAT_PHASE) ? M.phuy : R(0);
      a.lout[LAG_Q * P + n] = (lat & LAT_HEAT) ? M.cap * T * mdot : R(0);
      if constexpr (WB) a.lout[LAG_T * P + n] = T;
    } else {
      const long long d = (long long)gy * g.nx + gx;
      const R vals[NFIELD] = {phi, fs, L.fl, T, L.rhoH, M.pr, M.ux, M.uy, rho, M.muphi, L.w, mdot};
#pragma unroll
      for (int k = 0; k < NFIELD; k++)
        if (a.out[k]) put_out(a.out[k], d, (long long)g.nx * g.ny, vals[k]);
    }
  }
  };
  if (x0 >= 1 && x0 + TX < g.nx && y0 >= 1 && y0 + TY < g.ny) phase_b(std::true_type{});
  else phase_b(std::false_type{});
  if (DIAG) {
    if (b < 0)
      block_diag_finish<R, NT / 32>(s_red, a.diag_partial, tid,
                                    blockIdx.y * gridDim.x + blockIdx.x, gridDim.x * gridDim.y);
    else block_diag_finish<R, NT / 32>(s_red, a.diag_partial, tid, b, nb);
  }
}

// One CTA per 32 x TYS tile; float kernels keep the 64-register budget of
// the 32 x 8 shape (4 CTAs of 256 threads per SM) at every shape.
template <typename R, int MODE, bool DIAG, int LATC, typename S = R, int TYS = TY>
__global__ void __launch_bounds__(Shape<TYS>::NT,
                                  sizeof(R) == 4 ? LBM_MIN_BLOCKS_F32 * TY / TYS : 1)
    lbm_step_kernel(const Args<R, S> a) {
  step_tile<R, MODE, DIAG, LATC, S, TYS>(a, blockIdx.x, blockIdx.y, -1, 0);
}

// Many independent grids (uneven sizes and parameters) advanced in one
// launch.  The whole table -- every grid's arguments and the prefix sums of
// the grids' tile counts -- travels in the kernel's parameter space (up to
// 32 KB on sm_70 and later), so the per-grid constants are read through the
// constant cache, like those of the single-grid kernel, and nothing of the
// table lives in device memory.  CTA t takes tile t of the concatenated tile
// list; its grid is found by bisection over the prefix sums.
constexpr int BATCH_MAX_GRIDS = 64;

template <typename R>
struct BatchTable {
  int ngrids;
  int tile_base[BATCH_MAX_GRIDS + 1];  // first tile of each grid; [ngrids] = total
  Args<R> args[BATCH_MAX_GRIDS];
};

template <typename R, bool DIAG, int LATC>
__global__ void __launch_bounds__(NT, sizeof(R) == 4 ? LBM_MIN_BLOCKS_F32 : 1)
    lbm_batch_kernel(const __grid_constant__ BatchTable<R> B) {
  const int t = blockIdx.x;
  int lo = 0, hi = B.ngrids;  // tile_base[lo] <= t < tile_base[hi]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (B.tile_base[mid] <= t) lo = mid;
    else hi = mid;
  }
  const Args<R>& a = B.args[lo];
  const int local = t - B.tile_base[lo];
  const int tiles_x = (a.g.nx + TX - 1) / TX;
  const int ntiles = B.tile_base[lo + 1] - B.tile_base[lo];
  step_tile<R, MODE_STEP, DIAG, LATC>(a, local % tiles_x, local / tiles_x, local, ntiles);
}

}  // namespace lbmk
