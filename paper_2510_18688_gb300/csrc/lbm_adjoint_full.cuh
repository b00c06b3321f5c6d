// lbm_adjoint_full.cuh -- reverse mode of the whole coupled step (flow,
// phase field and enthalpy lattices; FP64; readings == 0).
//
// On top of the freezing coupling of the phase-field and enthalpy adjoint
// (lbm_adjoint.cuh), the flow lattice moves: the velocity of Eq. (17a,b)
// from the flow populations, the surface-tension and body forces and the
// penalty force; the source S = rho mdot + u . grad rho and the modified
// force F~ = F - grad(p_prev - rho / 3) of Eq. (16); the pressure of
// Eq. (17c); the flow collision Eqs. (11), (14)-(16); phi u in the phase
// equilibrium and source (Eqs. (19)-(20), with its lagged value); u in the
// enthalpy equilibrium (Eq. (25)).  Four stencils are transposed: the
// Laplacians of phi and fs (through mu_phi, Eq. (6)) and the gradients of
// phi (F_s), rho (S and F~) and the lagged pressure (F~).
//
// Per reverse step: a fields kernel (phi, fs, rho of the recomputed state);
// kernel 1 runs the node's whole local reverse and stores what its stencils
// need -- the adjoints of mu_phi and of the three gradients -- with the
// theta and sigma terms; kernel 2 runs the same local reverse again, gathers
// the neighbours' stencil adjoints in a fixed order and finishes the local
// chain to this state's populations and lags (fl, w, p, phi u, Q).
// A cold-mask node reads its enthalpy populations as the equilibrium at
// T_cold (R-BC) built from its lagged w, so their adjoint goes to the lagged
// w, to T_cold and to L instead of to the stored populations.
// Accumulator planes: d/dT_wall[0..3], d/dL, d/dtheta_deg, d/dsigma, d/dgx,
// d/dgy, d/dT_cold.
#pragma once

#include "lbm_adjoint.cuh"

namespace lbmk {

constexpr int FULL_NACC = 10;

struct FullArgs {
  Geom g;
  Coef<double> c;
  const double* __restrict__ pop;     // 27 planes of the forward state: f, g, h
  const double* __restrict__ lag;     // NLAG planes of the forward state
  const double* __restrict__ phi0;
  const unsigned char* __restrict__ mask;  // cold mask (has_mask) or null
  int has_mask;
  double* __restrict__ phi;           // fields of the forward state
  double* __restrict__ fs;
  double* __restrict__ rho;
  const double* __restrict__ lam_in;  // 27 planes: adjoints of the next f, g, h
  const double* __restrict__ llag_in; // NLAG planes: adjoints of the next state's lags
  double* __restrict__ sb;            // 7 planes: adjoints of mu_phi, grad phi, grad rho, grad p
  const double* __restrict__ phib_seed;
  double* __restrict__ lam_out;       // 27 planes
  double* __restrict__ llag_out;      // NLAG planes
  double* __restrict__ acc;           // FULL_NACC planes (+=)
  double dcos_dtheta;
  double inv_sum_w, ff;
  int axis, index;
  double* __restrict__ out;
};

// The phase and enthalpy population sums of node n as the step reads them
// (the enthalpy populations of a cold-mask node: the mask equilibrium); h
// (or null) receives the enthalpy populations.
__device__ __forceinline__ void full_sums(const FullArgs& a, int n, double* sg, double* sh,
                                          double* h) {
  const int P = (int)a.g.plane;
  double v[9];
#pragma unroll
  for (int i = 0; i < 9; i++) v[i] = a.pop[(9 + i) * P + n];
  *sg = sum_g(v);
  if (a.has_mask && a.mask[n]) {
    cold_mask_h(a.c, a.lag[LAG_W * P + n], a.phi0[n], v);
  } else {
#pragma unroll
    for (int i = 0; i < 9; i++) v[i] = a.pop[(18 + i) * P + n];
  }
  *sh = sum_h(v);
  if (h) {
#pragma unroll
    for (int i = 0; i < 9; i++) h[i] = v[i];
  }
}

// Forward values of one node that its reverse needs.
struct FullNode {
  FrzNode q;
  double f[9], h[9];
  double gph[2], gr[2], gp[2], lphi0, mu;
  double muv, irho, F[2], j[2], us[2], fp[2], u[2], uu, S, Ft[2], G[2], uFt, tauf, itau;
  double fsym0, pr, phu[2], phup[2];
};

__device__ __forceinline__ FullNode full_forward(const FullArgs& a, int x, int y, int n) {
  const Geom& g = a.g;
  const Coef<double>& c = a.c;
  const int P = (int)g.plane;
  FullNode r;
  double sg, sh;
  full_sums(a, n, &sg, &sh, r.h);
#pragma unroll
  for (int i = 0; i < 9; i++) r.f[i] = a.pop[i * P + n];
  const double phi0 = a.phi0[n];
  r.q = frz_forward(c, sg, sh, a.lag[LAG_FL * P + n], a.lag[LAG_W * P + n], a.lag[LAG_Q * P + n],
                    phi0);
  // stencils (the forward step's order of summation is not needed here)
  double gx = 0.0, gy = 0.0, rx = 0.0, ry = 0.0, px = 0.0, py = 0.0;
  double lphi = 0.0, lphi0 = 0.0, lfs = 0.0;
#pragma unroll
  for (int i = 1; i < 9; i++) {
    const int m = stencil_index(g, x, y, i);
    const double wi = qw<double>(i);
    gx += wi * qx(i) * a.phi[m];
    gy += wi * qy(i) * a.phi[m];
    rx += wi * qx(i) * a.rho[m];
    ry += wi * qy(i) * a.rho[m];
    px += wi * qx(i) * a.lag[LAG_P * P + m];
    py += wi * qy(i) * a.lag[LAG_P * P + m];
    lphi += 2.0 * wi * (a.phi[m] - a.phi[n]);
    lphi0 += 2.0 * wi * (a.phi0[m] - phi0);
    lfs += 2.0 * wi * (a.fs[m] - a.fs[n]);
  }
  r.gph[0] = 3.0 * gx; r.gph[1] = 3.0 * gy;
  r.gr[0] = 3.0 * rx; r.gr[1] = 3.0 * ry;
  r.gp[0] = 3.0 * px; r.gp[1] = 3.0 * py;
  lphi *= 3.0; lphi0 *= 3.0; lfs *= 3.0;
  r.lphi0 = lphi0;
  const FrzNode& q = r.q;
  r.mu = chem_local(c, q.phi, phi0, q.fs) - c.klap * (lphi + c.cos_th * lphi0 + c.cos_ps * lfs);
  r.F[0] = r.mu * r.gph[0] + q.rho * c.gx;
  r.F[1] = r.mu * r.gph[1] + q.rho * c.gy;
  r.j[0] = (r.f[1] - r.f[3]) + (r.f[5] - r.f[6]) + (r.f[8] - r.f[7]);
  r.j[1] = (r.f[2] - r.f[4]) + (r.f[5] + r.f[6]) - (r.f[7] + r.f[8]);
  const double snz = (r.f[1] + r.f[2] + r.f[3] + r.f[4]) + (r.f[5] + r.f[6] + r.f[7] + r.f[8]);
  r.muv = interp(q.fs, q.w, c.mu_s, c.mu_l, c.mu_g);
  r.irho = 1.0 / q.rho;
  for (int k = 0; k < 2; k++) {
    r.us[k] = (r.j[k] + 0.5 * r.F[k]) * r.irho;
    r.fp[k] = -q.fs * r.us[k];
    r.u[k] = r.us[k] + 0.5 * r.fp[k];
  }
  r.uu = r.u[0] * r.u[0] + r.u[1] * r.u[1];
  r.S = q.rho * q.mdot + r.u[0] * r.gr[0] + r.u[1] * r.gr[1];
  for (int k = 0; k < 2; k++) {
    r.Ft[k] = r.F[k] - (r.gp[k] - r.gr[k] / 3.0);
    r.G[k] = r.F[k] + q.rho * r.fp[k];
  }
  r.uFt = r.u[0] * r.Ft[0] + r.u[1] * r.Ft[1];
  r.tauf = 3.0 * r.muv * r.irho + 0.5;
  r.itau = 1.0 / r.tauf;
  r.fsym0 = r.S - 3.0 * r.uFt;
  const double F0 = qw<double>(0) * r.fsym0;
  const double s0 = qw<double>(0) * (-1.5 * r.uu);
  r.pr = (1.0 / 3.0) / (1.0 - qw<double>(0)) * (snz + 0.5 * r.S + (r.tauf - 0.5) * F0 + q.rho * s0);
  r.phu[0] = q.phi * r.u[0];
  r.phu[1] = q.phi * r.u[1];
  r.phup[0] = a.lag[LAG_PHUX * P + n];
  r.phup[1] = a.lag[LAG_PHUY * P + n];
  return r;
}

// Adjoints of one node's local inputs and stencil outputs.
struct FullAdj {
  double fb[9], gbd[9], hb[9];  // direct adjoints of this node's populations
  double mub, gphb[2], grb[2], gpb[2];
  double phib, fsb, wb, rhob, mdotb, Tb, rhoHb, flb;
  double phupb[2];
  double dTw[4], dg[2];
};

// The local reverse of one node: pulls, the three collisions, the flow
// macros, the lag outputs; stops at (phi, fs, w, rho, mdot, T, rho H, fl)
// and the stencil outputs.
__device__ __forceinline__ void full_local_reverse(const FullArgs& a, const FullNode& r, int x,
                                                   int y, int n, FullAdj& d) {
  const Geom& g = a.g;
  const Coef<double>& c = a.c;
  const FrzNode& q = r.q;
  const int P = (int)g.plane;
  double fbs[9], gbs[9], hbs[9];
  for (int k = 0; k < 4; k++) d.dTw[k] = 0.0;
#pragma unroll
  for (int i = 0; i < 9; i++) {
    int wall;
    const long long t = stream_target(g, x, y, qx(i), qy(i), wall);
    if (t >= 0) {
      fbs[i] = a.lam_in[i * P + (int)t];
      gbs[i] = a.lam_in[(9 + i) * P + (int)t];
      hbs[i] = a.lam_in[(18 + i) * P + (int)t];
    } else {
      fbs[i] = a.lam_in[qopp(i) * P + n];
      gbs[i] = a.lam_in[(9 + qopp(i)) * P + n];
      const double lb = a.lam_in[(18 + qopp(i)) * P + n];
      if (g.bc[wall] == BC_DIRICHLET) {
        hbs[i] = -lb;
        d.dTw[wall] += lb * 2.0 * qw<double>(i) * c.rr;
      } else {
        hbs[i] = lb;
      }
    }
  }
  const double* ll = a.llag_in;
  double ub[2] = {0.0, 0.0}, uub = 0.0, rhob = 0.0, mdotb = 0.0, Sb = 0.0, uFtb = 0.0;
  double Ftb[2] = {0.0, 0.0}, Gb[2] = {0.0, 0.0}, Fb[2] = {0.0, 0.0};
  double prb = ll[LAG_P * P + n], itaub = 0.0, omib = 0.0, fcoefb = 0.0, fsym0b = 0.0;
  double phib = 0.0, mub = 0.0, Tb = 0.0, rhoHb = 0.0, Cb = 0.0, fsb = 0.0, wb = 0.0;
  double phub[2] = {ll[LAG_PHUX * P + n], ll[LAG_PHUY * P + n]};

  // ---- flow collision (Eqs. (11), (14)-(16)) -------------------------------
  {
    const double itau = r.itau, omi = 1.0 - itau, fcoef = 1.0 - 0.5 * itau;
    const double sym0 = q.rho * (-1.5 * r.uu);
    double sym0b = 0.0;
    {
      const double A0 = fbs[0];
      const double feq0 = r.pr * 3.0 * (qw<double>(0) - 1.0) + q.rho * qw<double>(0) * (-1.5 * r.uu);
      d.fb[0] = A0 * omi;
      omib += A0 * r.f[0];
      itaub += A0 * feq0;
      const double feq0b = A0 * itau;
      fcoefb += A0 * qw<double>(0) * r.fsym0;
      fsym0b += A0 * fcoef * qw<double>(0);
      prb += 3.0 * (qw<double>(0) - 1.0) * feq0b;
      rhob += qw<double>(0) * (-1.5 * r.uu) * feq0b;
      uub += -1.5 * q.rho * qw<double>(0) * feq0b;
    }
#pragma unroll
    for (int i = 1; i <= 8; i++) {
      if (i == 3 || i == 4 || i == 7 || i == 8) continue;
      const int o = qopp(i);
      const double wi = qw<double>(i);
      const double cu = qx(i) * r.u[0] + qy(i) * r.u[1];
      const double cG = qx(i) * r.G[0] + qy(i) * r.G[1];
      const double cFt = qx(i) * r.Ft[0] + qy(i) * r.Ft[1];
      const double eqS = r.pr * 3.0 + q.rho * (4.5 * cu * cu) + sym0;
      const double eqA = q.rho * (3.0 * cu);
      const double srcS = r.fsym0 + 9.0 * cu * cFt;
      const double srcA = 3.0 * cG;
      const double A = fbs[i], B = fbs[o];
      d.fb[i] = A * omi;
      d.fb[o] = B * omi;
      omib += A * r.f[i] + B * r.f[o];
      const double Psb = A + B, Pab = A - B;
      itaub += Psb * wi * eqS + Pab * wi * eqA;
      fcoefb += Psb * wi * srcS + Pab * wi * srcA;
      const double eqSb = Psb * wi * itau, srcSb = Psb * wi * fcoef;
      const double eqAb = Pab * wi * itau, srcAb = Pab * wi * fcoef;
      prb += 3.0 * eqSb;
      rhob += eqSb * 4.5 * cu * cu + eqAb * 3.0 * cu;
      const double cub = eqSb * 9.0 * q.rho * cu + eqAb * 3.0 * q.rho + srcSb * 9.0 * cFt;
      sym0b += eqSb;
      fsym0b += srcSb;
      const double cFtb = srcSb * 9.0 * cu, cGb = srcAb * 3.0;
      ub[0] += cub * qx(i); ub[1] += cub * qy(i);
      Ftb[0] += cFtb * qx(i); Ftb[1] += cFtb * qy(i);
      Gb[0] += cGb * qx(i); Gb[1] += cGb * qy(i);
    }
    rhob += -1.5 * r.uu * sym0b;
    uub += -1.5 * q.rho * sym0b;
    itaub -= omib;
    itaub -= 0.5 * fcoefb;
  }
  // ---- phase collision (Eqs. (18)-(20)) ---------------------------------------
  {
    const double itg = c.inv_tau_g, gcoef = 1.0 - 0.5 * itg, omg = 1.0 - itg;
    double S = 0.0, Vb[2] = {0.0, 0.0};
#pragma unroll
    for (int i = 0; i < 9; i++) {
      d.gbd[i] = omg * gbs[i];
      S += qw<double>(i) * gbs[i];
    }
#pragma unroll
    for (int i = 1; i <= 8; i++) {
      if (i == 3 || i == 4 || i == 7 || i == 8) continue;
      const double Pab = gbs[i] - gbs[qopp(i)];
      Vb[0] += qw<double>(i) * qx(i) * Pab;
      Vb[1] += qw<double>(i) * qy(i) * Pab;
    }
    double m = (qw<double>(0) - 1.0) * gbs[0];
#pragma unroll
    for (int i = 1; i < 9; i++) m += qw<double>(i) * gbs[i];
    mub += itg * c.eta * m;
    phib += itg * gbs[0] + gcoef * q.mdot * S;
    mdotb += gcoef * q.phi * S;
    for (int k = 0; k < 2; k++) {
      phub[k] += 3.0 * (itg + gcoef) * Vb[k];
      d.phupb[k] = -3.0 * gcoef * Vb[k];
    }
  }
  // ---- enthalpy TRT collision (Eqs. (23)-(27)) --------------------------------
  double isb = 0.0, iab = 0.0, Hsrcb = 0.0, rrTb = 0.0, CTb = 0.0;
  {
    const double rrT = c.rr * q.T;
    const double A0 = hbs[0];
    const double heq0 = q.rhoH - rrT + qw<double>(0) * (rrT - q.CT * r.uu * 1.5);
    d.hb[0] = A0 * (1.0 - q.is);
    const double heq0b = A0 * q.is;
    isb += -A0 * (r.h[0] - heq0);
    Hsrcb += qw<double>(0) * A0;
    rhoHb += heq0b;
    rrTb += (qw<double>(0) - 1.0) * heq0b;
    CTb += -1.5 * qw<double>(0) * r.uu * heq0b;
    uub += -1.5 * qw<double>(0) * q.CT * heq0b;
#pragma unroll
    for (int i = 1; i <= 8; i++) {
      if (i == 3 || i == 4 || i == 7 || i == 8) continue;
      const int o = qopp(i);
      const double wi = qw<double>(i);
      const double cu = qx(i) * r.u[0] + qy(i) * r.u[1];
      const double es = wi * (rrT + q.CT * (4.5 * cu * cu - 1.5 * r.uu));
      const double ea = wi * (q.CT * (3.0 * cu));
      const double hs = 0.5 * (r.h[i] + r.h[o]), ha = 0.5 * (r.h[i] - r.h[o]);
      const double A = hbs[i], B = hbs[o];
      const double Dab = -A + B, Dsb = -A - B;
      const double hab = Dab * q.ia, eab = -Dab * q.ia;
      iab += Dab * (ha - ea);
      const double hsb = Dsb * q.is, esb = -Dsb * q.is;
      isb += Dsb * (hs - es);
      Hsrcb += -wi * Dsb;
      d.hb[i] = A + 0.5 * hsb + 0.5 * hab;
      d.hb[o] = B + 0.5 * hsb - 0.5 * hab;
      rrTb += wi * esb;
      CTb += wi * (4.5 * cu * cu - 1.5 * r.uu) * esb + 3.0 * wi * cu * eab;
      const double cub = wi * q.CT * 9.0 * cu * esb + 3.0 * wi * q.CT * eab;
      uub += -1.5 * wi * q.CT * esb;
      ub[0] += cub * qx(i); ub[1] += cub * qy(i);
    }
  }
  // ---- the heat source and the lag Q = C T mdot ---------------------------
  {
    const double lqb = ll[LAG_Q * P + n];
    const double hcoefb = Hsrcb * q.CT * q.mdot;
    CTb += Hsrcb * q.hcoef * q.mdot + lqb * q.mdot;
    mdotb += Hsrcb * q.hcoef * q.CT + lqb * q.CT;
    iab += -0.5 * hcoefb;
    iab -= isb;
    Tb += c.rr * rrTb + CTb * q.C;
    Cb += CTb * q.T;
    const double lamb = -iab / (q.taua * q.taua) * c.inv_rr3;
    fsb += lamb * dinterp_dfs(q.w, c.lam_s, c.lam_l, c.lam_g);
    wb += lamb * dinterp_dw(q.fs, c.lam_l, c.lam_g);
    // C = rho cp(fs, w)
    rhob += Cb * q.cp;
    const double cpb = Cb * q.rho;
    fsb += cpb * dinterp_dfs(q.w, c.cp_s, c.cp_l, c.cp_g);
    wb += cpb * dinterp_dw(q.fs, c.cp_l, c.cp_g);
  }
  // ---- pressure Eq. (17c), modified force, source, velocity ---------------
  {
    const double K = (1.0 / 3.0) / (1.0 - qw<double>(0));
    const double F0 = qw<double>(0) * r.fsym0;
    const double s0 = qw<double>(0) * (-1.5 * r.uu);
    const double snzb = K * prb;
    Sb += 0.5 * K * prb;
    double taufb = K * F0 * prb;
    const double F0b = K * (r.tauf - 0.5) * prb;
    rhob += K * s0 * prb;
    uub += -1.5 * qw<double>(0) * K * q.rho * prb;
    fsym0b += qw<double>(0) * F0b;
    Sb += fsym0b;
    uFtb += -3.0 * fsym0b;
    taufb += -itaub / (r.tauf * r.tauf);
    const double muvb = 3.0 * r.irho * taufb;
    double irhob = 3.0 * r.muv * taufb;
    fsb += muvb * dinterp_dfs(q.w, c.mu_s, c.mu_l, c.mu_g);
    wb += muvb * dinterp_dw(q.fs, c.mu_l, c.mu_g);
    // phi u (equilibrium, source, lag)
    phib += phub[0] * r.u[0] + phub[1] * r.u[1];
    for (int k = 0; k < 2; k++) ub[k] += q.phi * phub[k];
    for (int k = 0; k < 2; k++) {
      ub[k] += uFtb * r.Ft[k];
      Ftb[k] += uFtb * r.u[k];
    }
    for (int k = 0; k < 2; k++) {
      Fb[k] += Ftb[k] + Gb[k];
      d.gpb[k] = -Ftb[k];
      d.grb[k] = Ftb[k] / 3.0 + Sb * r.u[k];
      ub[k] += Sb * r.gr[k];
    }
    rhob += Gb[0] * r.fp[0] + Gb[1] * r.fp[1] + Sb * q.mdot;
    mdotb += Sb * q.rho;
    double fpb[2] = {q.rho * Gb[0], q.rho * Gb[1]};
    for (int k = 0; k < 2; k++) ub[k] += 2.0 * uub * r.u[k];
    // u = us + fp / 2, fp = -fs us, us = (j + F / 2) / rho
    double usb[2], jb[2];
    for (int k = 0; k < 2; k++) {
      fpb[k] += 0.5 * ub[k];
      usb[k] = ub[k] - q.fs * fpb[k];
      fsb += -fpb[k] * r.us[k];
      jb[k] = usb[k] * r.irho;
      Fb[k] += 0.5 * usb[k] * r.irho;
      irhob += usb[k] * (r.j[k] + 0.5 * r.F[k]);
    }
    rhob += -irhob * r.irho * r.irho;
#pragma unroll
    for (int i = 0; i < 9; i++) {
      d.fb[i] += qx(i) * jb[0] + qy(i) * jb[1];
      if (i > 0) d.fb[i] += snzb;
    }
    // F = mu grad(phi) + rho g
    mub += Fb[0] * r.gph[0] + Fb[1] * r.gph[1];
    d.gphb[0] = r.mu * Fb[0];
    d.gphb[1] = r.mu * Fb[1];
    rhob += Fb[0] * c.gx + Fb[1] * c.gy;
    d.dg[0] = Fb[0] * q.rho;
    d.dg[1] = Fb[1] * q.rho;
  }
  d.mub = mub;
  d.phib = phib;
  d.fsb = fsb;
  d.wb = wb + ll[LAG_W * P + n];
  d.rhob = rhob;
  d.mdotb = mdotb;
  d.Tb = Tb;
  d.rhoHb = rhoHb;
  d.flb = ll[LAG_FL * P + n];
}

#ifdef LBM_ADJOINT_KERNELS
static __global__ void __launch_bounds__(NT) lbm_full_fields_kernel(const FullArgs a) {
  const Geom& g = a.g;
  const int x = blockIdx.x * TX + threadIdx.x, y = blockIdx.y * TY + threadIdx.y;
  if (x >= g.nx || y >= g.ny) return;
  const int P = (int)g.plane;
  const int n = y * g.pitch + x;
  double sg, sh;
  full_sums(a, n, &sg, &sh, nullptr);
  const FrzNode q = frz_forward(a.c, sg, sh, a.lag[LAG_FL * P + n], a.lag[LAG_W * P + n],
                                a.lag[LAG_Q * P + n], a.phi0[n]);
  a.phi[n] = q.phi;
  a.fs[n] = q.fs;
  a.rho[n] = q.rho;
}
#endif  // LBM_ADJOINT_KERNELS

// Kernel 1: the adjoints the neighbours' stencils need, and the theta and
// sigma terms of mu_phi's adjoint.
#ifdef LBM_ADJOINT_KERNELS
static __global__ void __launch_bounds__(NT) lbm_full_k1_kernel(const FullArgs a) {
  const Geom& g = a.g;
  const Coef<double>& c = a.c;
  const int x = blockIdx.x * TX + threadIdx.x, y = blockIdx.y * TY + threadIdx.y;
  if (x >= g.nx || y >= g.ny) return;
  const int P = (int)g.plane;
  const int n = y * g.pitch + x;
  const FullNode r = full_forward(a, x, y, n);
  FullAdj d;
  full_local_reverse(a, r, x, y, n, d);
  a.sb[n] = d.mub;
  a.sb[1 * P + n] = d.gphb[0];
  a.sb[2 * P + n] = d.gphb[1];
  a.sb[3 * P + n] = d.grb[0];
  a.sb[4 * P + n] = d.grb[1];
  a.sb[5 * P + n] = d.gpb[0];
  a.sb[6 * P + n] = d.gpb[1];
  double dphi, dfs, dcos;
  chem_partials(c, r.q.phi, a.phi0[n], r.q.fs, &dphi, &dfs, &dcos);
  a.acc[5 * P + n] += d.mub * (dcos - c.klap * r.lphi0) * a.dcos_dtheta;
  a.acc[6 * P + n] += d.mub * r.mu / c.sigma;
}
#endif  // LBM_ADJOINT_KERNELS

// Kernel 2: the local reverse again, the gathered stencil transposes and the
// local chain to this state's populations and lags.
#ifdef LBM_ADJOINT_KERNELS
static __global__ void __launch_bounds__(NT) lbm_full_k2_kernel(const FullArgs a) {
  const Geom& g = a.g;
  const Coef<double>& c = a.c;
  const int x = blockIdx.x * TX + threadIdx.x, y = blockIdx.y * TY + threadIdx.y;
  if (x >= g.nx || y >= g.ny) return;
  const int P = (int)g.plane;
  const int n = y * g.pitch + x;
  const FullNode r = full_forward(a, x, y, n);
  const FrzNode& q = r.q;
  FullAdj d;
  full_local_reverse(a, r, x, y, n, d);
  double phib = d.phib, fsb = d.fsb, wb = d.wb, rhob = d.rhob, mdotb = d.mdotb;
  double flb = d.flb, rhoHb = d.rhoHb;
  if (a.phib_seed) phib += a.phib_seed[n];
  const double phi0 = a.phi0[n];
  // mu_phi of this node: local part and the centre of the Laplacians
  {
    double dphi, dfs, dcos;
    chem_partials(c, q.phi, phi0, q.fs, &dphi, &dfs, &dcos);
    const double self = 6.0 * (1.0 - qw<double>(0));
    phib += d.mub * dphi + c.klap * self * d.mub;
    fsb += d.mub * dfs + c.klap * c.cos_ps * self * d.mub;
  }
  // gathered transposes of the neighbours' stencils
  double lsum = 0.0, gphi = 0.0, grho = 0.0, gpr = 0.0;
  for (int dy = -1; dy <= 1; dy++) {
    int py = y + dy;
    if (py < 0 || py >= g.ny) {
      if (g.bc[2] != BC_PERIODIC) continue;
      py = (py + g.ny) % g.ny;
    }
    if (dy == 1 && py == (y - 1 + g.ny) % g.ny && g.bc[2] == BC_PERIODIC) continue;
    for (int dx = -1; dx <= 1; dx++) {
      int px = x + dx;
      if (px < 0 || px >= g.nx) {
        if (g.bc[0] != BC_PERIODIC) continue;
        px = (px + g.nx) % g.nx;
      }
      if (dx == 1 && px == (x - 1 + g.nx) % g.nx && g.bc[0] == BC_PERIODIC) continue;
      const int m = py * g.pitch + px;
      const double mb = a.sb[m];
      const double gpx = a.sb[1 * P + m], gpy = a.sb[2 * P + m];
      const double grx = a.sb[3 * P + m], gry = a.sb[4 * P + m];
      const double ppx = a.sb[5 * P + m], ppy = a.sb[6 * P + m];
#pragma unroll
      for (int i = 1; i < 9; i++) {
        if (stencil_index(g, px, py, i) != n) continue;
        const double wi = qw<double>(i);
        lsum += 6.0 * wi * mb;
        gphi += 3.0 * wi * (qx(i) * gpx + qy(i) * gpy);
        grho += 3.0 * wi * (qx(i) * grx + qy(i) * gry);
        gpr += 3.0 * wi * (qx(i) * ppx + qy(i) * ppy);
      }
    }
  }
  phib += -c.klap * lsum + gphi;
  fsb += -c.klap * c.cos_ps * lsum;
  rhob += grho;
  // rho = interp(fs, w)
  fsb += rhob * dinterp_dfs(q.w, c.rho_s, c.rho_l, c.rho_g);
  wb += rhob * dinterp_dw(q.fs, c.rho_l, c.rho_g);
  // fs = min(phi0 + w (1 - fl), 1)
  if (!(q.fs_raw > 1.0)) {
    wb += fsb * (1.0 - q.fl);
    flb += -q.w * fsb;
  }
  // w = clamp((1 - phi0 + phi) / 2)
  if (!(q.wraw < 0.0) && !(q.wraw > 1.0)) phib += 0.5 * wb;
  // phi = sum g / (1 - mdot / 2)
  const double sgb = phib / q.D;
  mdotb += phib * 0.5 * q.phi / q.D;
  // mdot = (1 - rho_s / rho_l) w_prev (fl_prev - fl)
  const double wp = a.lag[LAG_W * P + n], flp = a.lag[LAG_FL * P + n];
  double wpb = mdotb * c.one_m_ratio * (flp - q.fl);
  const double flpb = mdotb * c.one_m_ratio * wp;
  flb += -mdotb * c.one_m_ratio * wp;
  // the inversion of Eq. (8)
  double ellb = 0.0;
  const double Tb = d.Tb;
  if (q.branch == 0) {
    rhoHb += Tb / q.Cm;
    const double Cmb = -Tb * q.T / q.Cm;
    double cf, cw;
    dcap(c, q.fsf, wp, &cf, &cw);
    wpb += Cmb * ((q.fsf_clamped ? 0.0 : cf) + cw);
  } else if (q.branch == 1) {
    rhoHb += Tb / q.Cp;
    ellb += -Tb / q.Cp;
    const double Cpb = -Tb * q.T / q.Cp;
    double cf, cw;
    dcap(c, phi0, wp, &cf, &cw);
    wpb += Cpb * cw;
  } else if (q.ell > 0.0) {
    rhoHb += flb / q.ell;
    ellb += -flb * q.rhoH / (q.ell * q.ell);
  }
  wpb += ellb * c.rho_l * c.latent;
  double dL = ellb * wp * c.rho_l, dTc = 0.0;
  const bool masked = a.has_mask && a.mask[n];
  if (masked) {
    // the enthalpy populations read here are h_eq(T_cold, u = 0) at w_prev:
    // h_0 = rho H - rr T + w_0 rr T, h_i = w_i rr T with
    // rho H = cap(w_prev) T + w_prev rho_l L fl_c
    const double Tc = c.T_cold;
    const double flc = Tc < 0.0 ? 0.0 : 1.0;
    double fsf = phi0 + wp;
    const bool fsf_cl = fsf > 1.0;
    if (fsf_cl) fsf = 1.0;
    double cf, cw, cap, dcapw;
    if (Tc < 0.0) {
      cap = heat_cap(c, fsf, wp);
      dcap(c, fsf, wp, &cf, &cw);
      dcapw = (fsf_cl ? 0.0 : cf) + cw;
    } else {
      cap = heat_cap(c, phi0, wp);
      dcap(c, phi0, wp, &cf, &cw);
      dcapw = cw;
    }
    double sb = 0.0;  // sum over i>0 of the adjoints times w_i
#pragma unroll
    for (int i = 1; i < 9; i++) sb += (d.hb[i] + rhoHb) * qw<double>(i);
    const double h0b = d.hb[0] + rhoHb;
    wpb += h0b * (dcapw * Tc + c.rho_l * c.latent * flc);
    dTc = h0b * (cap - c.rr + qw<double>(0) * c.rr) + sb * c.rr;
    dL += h0b * wp * c.rho_l * flc;
  }
#pragma unroll
  for (int i = 0; i < 9; i++) {
    a.lam_out[i * P + n] = d.fb[i];
    a.lam_out[(9 + i) * P + n] = d.gbd[i] + sgb;
    a.lam_out[(18 + i) * P + n] = masked ? 0.0 : d.hb[i] + rhoHb;
  }
  a.llag_out[LAG_FL * P + n] = flpb;
  a.llag_out[LAG_W * P + n] = wpb;
  a.llag_out[LAG_P * P + n] = gpr;
  a.llag_out[LAG_PHUX * P + n] = d.phupb[0];
  a.llag_out[LAG_PHUY * P + n] = d.phupb[1];
  a.llag_out[LAG_Q * P + n] = 0.5 * rhoHb;
#pragma unroll
  for (int k = 0; k < 4; k++) a.acc[k * P + n] += d.dTw[k];
  a.acc[4 * P + n] += dL;
  a.acc[7 * P + n] += d.dg[0];
  a.acc[8 * P + n] += d.dg[1];
  a.acc[9 * P + n] += dTc;
}
#endif  // LBM_ADJOINT_KERNELS

// Frozen-fraction seed: the adjoints of the lags fl and w the final state's
// reader writes (other lag and population adjoints zero).
#ifdef LBM_ADJOINT_KERNELS
static __global__ void __launch_bounds__(NT) lbm_full_seed_ff_kernel(const FullArgs a,
                                                                     double* __restrict__ llag) {
  const Geom& g = a.g;
  const int x = blockIdx.x * TX + threadIdx.x, y = blockIdx.y * TY + threadIdx.y;
  if (x >= g.nx || y >= g.ny) return;
  const int P = (int)g.plane;
  const int n = y * g.pitch + x;
  double sg, sh;
  full_sums(a, n, &sg, &sh, nullptr);
  const FrzNode q = frz_forward(a.c, sg, sh, a.lag[LAG_FL * P + n], a.lag[LAG_W * P + n],
                                a.lag[LAG_Q * P + n], a.phi0[n]);
  llag[LAG_FL * P + n] = -q.w * a.inv_sum_w;
  llag[LAG_W * P + n] = ((1.0 - q.fl) - a.ff) * a.inv_sum_w;
}
#endif  // LBM_ADJOINT_KERNELS

// Crossing seed (one thread), as lbm_frz_seed_crossing_kernel.
#ifdef LBM_ADJOINT_KERNELS
static __global__ void lbm_full_seed_crossing_kernel(const FullArgs a, double* __restrict__ phib) {
  const Geom& g = a.g;
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int len = a.axis == 0 ? g.nx : g.ny;
  const int stride = a.axis == 0 ? 1 : g.pitch;
  const int base = a.axis == 0 ? a.index * g.pitch : a.index;
  double J = __longlong_as_double(0x7ff8000000000000ULL);
  for (int k = len - 2; k >= 0; k--) {
    const int n0 = base + k * stride, n1 = n0 + stride;
    const double va = a.phi[n0], vb = a.phi[n1];
    if ((va <= 0.0) != (vb <= 0.0)) {
      const double dd = va - vb;
      J = k + va / dd;
      phib[n0] = -vb / (dd * dd);
      phib[n1] = va / (dd * dd);
      break;
    }
  }
  a.out[0] = J;
}
#endif  // LBM_ADJOINT_KERNELS

// Gradient with respect to the initial temperature field (a run from
// set_geometry): the initial enthalpy populations are h_eq(rho H, T, u = 0)
// with rho H = cap T + w rho_l L fl (cap: the frozen capacity below T_m,
// the liquid one at and above, Eq. (8)), so dh_0/dT = cap - rr + w_0 rr and
// dh_i/dT = w_i rr; T is recovered from the initial populations (pop, lag)
// by the inversion.  lam: the adjoints of the initial h (9 planes); out:
// dense [ny][nx].
#ifdef LBM_ADJOINT_KERNELS
static __global__ void __launch_bounds__(NT) lbm_full_dT0_kernel(const FullArgs a,
                                                                 const double* __restrict__ lam,
                                                                 double* __restrict__ out) {
  const Geom& g = a.g;
  const Coef<double>& c = a.c;
  const int x = blockIdx.x * TX + threadIdx.x, y = blockIdx.y * TY + threadIdx.y;
  if (x >= g.nx || y >= g.ny) return;
  const int P = (int)g.plane;
  const int n = y * g.pitch + x;
  double sg, sh;
  full_sums(a, n, &sg, &sh, nullptr);
  const FrzNode q = frz_forward(c, sg, sh, a.lag[LAG_FL * P + n], a.lag[LAG_W * P + n],
                                a.lag[LAG_Q * P + n], a.phi0[n]);
  const double cap = q.T < 0.0 ? q.Cm : q.Cp;
  double d = lam[n] * (cap - c.rr + qw<double>(0) * c.rr);
#pragma unroll
  for (int i = 1; i < 9; i++) d += lam[i * P + n] * qw<double>(i) * c.rr;
  out[(long long)y * g.nx + x] = d;
}
#endif  // LBM_ADJOINT_KERNELS

cudaError_t launch_full_dT0(const FullArgs& a, const double* lam, double* out, cudaStream_t s);
cudaError_t launch_full_fields(const FullArgs& a, cudaStream_t s);
cudaError_t launch_full_k1(const FullArgs& a, cudaStream_t s);
cudaError_t launch_full_k2(const FullArgs& a, cudaStream_t s);
cudaError_t launch_full_seed_ff(const FullArgs& a, double* llag, cudaStream_t s);
cudaError_t launch_full_seed_crossing(const FullArgs& a, double* phib, cudaStream_t s);

}  // namespace lbmk
