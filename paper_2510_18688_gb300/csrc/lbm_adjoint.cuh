// lbm_adjoint.cuh -- hand-written reverse-mode (adjoint) kernels of the
// enthalpy-lattice step (contexts whose only lattice is LAT_HEAT, or whose
// flow lattice stays at rest; FP64), of the phase-field step and of the two
// coupled.  A cold-mask node reads its enthalpy populations as the
// equilibrium at T_cold, so their adjoint goes to T_cold (and L, and the
// lagged w where it varies) instead of to the stored populations.
//
// With the enthalpy lattice alone the fluid is at rest (u = 0) and the step
// at one node is local: rho H = sum h + Q_prev / 2 (Eq. (28)), the
// inversion to T and fl (Eq. (8)), the mass source mdot (Eq. (1)), the solid
// fraction and the properties (Eq. (10)), the TRT collision (Eqs. (23)-(27))
// and the push with anti-bounce-back (T_wall) or bounce-back walls.  The
// adjoint kernel runs these in reverse for one step: it pulls the adjoint
// of the next state's populations from the nodes the post-collision
// populations were pushed to (through the walls where they bounced), and
// propagates it back through the collision and the inversion to the
// adjoint of this state's populations and lag fields.  Derivatives with
// respect to the wall temperatures (at anti-bounce-back links) and to the
// latent heat L (through the latent capacity w rho_l L of Eq. (8)) are
// accumulated per node, and summed once at the end in a fixed order.
#pragma once

#include "lbm_kernels.cuh"

namespace lbmk {

// accumulator planes: d/dT_wall[0..3], d/dlatent
constexpr int ADJ_NACC = 5;

struct AdjArgs {
  Geom g;
  Coef<double> c;
  const unsigned char* __restrict__ mask;  // cold mask (has_mask) or null
  int has_mask;
  const double* __restrict__ h;      // 9 enthalpy planes of the forward state
  const double* __restrict__ lag;    // NLAG lag planes of the forward state
  const double* __restrict__ phi0;
  const double* __restrict__ lam_in;  // adjoint of the next state's 9 planes
  const double* __restrict__ lfl_in;  // adjoint of the next state's lag fl
  const double* __restrict__ lq_in;   // adjoint of the next state's lag Q
  double* __restrict__ lam_out;       // adjoint of this state's 9 planes
  double* __restrict__ lfl_out;
  double* __restrict__ lq_out;
  double* __restrict__ acc;           // ADJ_NACC accumulator planes (+=)
  double inv_sum_w;                   // seed only: 1 / sum w
};

// Forward quantities of one node that the reverse pass needs.
struct HeatNode {
  double rhoH, T, fl, mdot, fs, fs_raw, C, ia, is, hcoef, CT, ell, Cm, Cp;
  int branch;  // 0: frozen (rhoH < 0), 1: liquid (rhoH > ell), 2: mushy
};

__device__ __forceinline__ HeatNode heat_forward(const Coef<double>& c, double sh, double flp,
                                                 double wp, double Qp, double phi0) {
  HeatNode q;
  q.rhoH = sh + 0.5 * Qp;
  q.ell = wp * c.rho_l * c.latent;
  double fsf = phi0 + wp;
  fsf = fsf > 1.0 ? 1.0 : fsf;
  q.Cm = heat_cap(c, fsf, wp);
  q.Cp = heat_cap(c, phi0, wp);
  if (q.rhoH < 0.0) {
    q.branch = 0;
    q.fl = 0.0;
    q.T = q.rhoH / q.Cm;
  } else if (q.rhoH > q.ell) {
    q.branch = 1;
    q.fl = 1.0;
    q.T = (q.rhoH - q.ell) / q.Cp;
  } else {
    q.branch = 2;
    q.T = 0.0;
    q.fl = q.ell > 0.0 ? q.rhoH / q.ell : 1.0;
  }
  q.mdot = c.one_m_ratio * wp * (flp - q.fl);
  q.fs_raw = phi0 + wp * (1.0 - q.fl);
  q.fs = q.fs_raw > 1.0 ? 1.0 : q.fs_raw;
  q.C = heat_cap(c, q.fs, wp);
  const double lam = interp(q.fs, wp, c.lam_s, c.lam_l, c.lam_g);
  const double taua = 0.5 + lam * c.inv_rr3;
  q.ia = 1.0 / taua;
  q.is = 2.0 - q.ia;
  q.hcoef = 1.0 - 0.5 * q.ia;
  q.CT = q.C * q.T;
  return q;
}

// Reverse of the inversion and of rho H = sum h + Q_prev / 2: from the
// adjoints of T and fl to those of rho H (returned) and of L (added to *dL).
__device__ __forceinline__ double heat_inversion_reverse(const Coef<double>& c, const HeatNode& q,
                                                         double wp, double Tb, double flb,
                                                         double* dL) {
  double rhoHb = 0.0, ellb = 0.0;
  if (q.branch == 0) {
    rhoHb = Tb / q.Cm;
  } else if (q.branch == 1) {
    rhoHb = Tb / q.Cp;
    ellb = -Tb / q.Cp;
  } else if (q.ell > 0.0) {
    rhoHb = flb / q.ell;
    ellb = -flb * q.rhoH / (q.ell * q.ell);
  }
  *dL += ellb * wp * c.rho_l;
  return rhoHb;
}

// Seed: adjoint of the frozen fraction FF = sum w (1 - fl) / sum w of a
// state with respect to its populations, lag Q and L (lag fl: zero).
#ifdef LBM_ADJOINT_KERNELS
static __global__ void __launch_bounds__(NT) lbm_adjoint_seed_kernel(const AdjArgs a) {
  const Geom& g = a.g;
  const int x = blockIdx.x * TX + threadIdx.x, y = blockIdx.y * TY + threadIdx.y;
  if (x >= g.nx || y >= g.ny) return;
  const int P = (int)g.plane;
  const int n = y * g.pitch + x;
  double h[9];
  const double wp = a.lag[LAG_W * P + n], flp = a.lag[LAG_FL * P + n];
  const double Qp = a.lag[LAG_Q * P + n], phi0 = a.phi0[n];
  if (a.has_mask && a.mask[n]) {
    cold_mask_h(a.c, wp, phi0, h);
  } else {
#pragma unroll
    for (int i = 0; i < 9; i++) h[i] = a.h[i * P + n];
  }
  const HeatNode q = heat_forward(a.c, sum_h(h), flp, wp, Qp, phi0);
  double dL = 0.0;
  const double rhoHb = heat_inversion_reverse(a.c, q, wp, 0.0, -wp * a.inv_sum_w, &dL);
#pragma unroll
  for (int i = 0; i < 9; i++) a.lam_out[i * P + n] = rhoHb;
  a.lq_out[n] = 0.5 * rhoHb;
  a.lfl_out[n] = 0.0;
  a.acc[(ADJ_NACC - 1) * P + n] += dL;
}
#endif  // LBM_ADJOINT_KERNELS

// One step in reverse (see the header).
#ifdef LBM_ADJOINT_KERNELS
static __global__ void __launch_bounds__(NT) lbm_adjoint_step_kernel(const AdjArgs a) {
  const Geom& g = a.g;
  const Coef<double>& c = a.c;
  const int x = blockIdx.x * TX + threadIdx.x, y = blockIdx.y * TY + threadIdx.y;
  if (x >= g.nx || y >= g.ny) return;
  const int P = (int)g.plane;
  const int n = y * g.pitch + x;
  // adjoint of the post-collision populations: pull through the push
  double hb_star[9];
  double dTw[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
  for (int i = 0; i < 9; i++) {
    int wall;
    const long long t = stream_target(g, x, y, qx(i), qy(i), wall);
    if (t >= 0) {
      hb_star[i] = a.lam_in[i * P + (int)t];
    } else {
      const double lb = a.lam_in[qopp(i) * P + n];
      if (g.bc[wall] == BC_DIRICHLET) {
        hb_star[i] = -lb;
        dTw[wall] += lb * 2.0 * qw<double>(i) * c.rr;
      } else {
        hb_star[i] = lb;
      }
    }
  }
  // forward recompute of this node (a cold-mask node reads h_eq(T_cold))
  double h[9];
  const double wp = a.lag[LAG_W * P + n], flp = a.lag[LAG_FL * P + n];
  const double Qp = a.lag[LAG_Q * P + n], phi0 = a.phi0[n];
  const bool masked = a.has_mask && a.mask[n];
  if (masked) {
    cold_mask_h(c, wp, phi0, h);
  } else {
#pragma unroll
    for (int i = 0; i < 9; i++) h[i] = a.h[i * P + n];
  }
  const HeatNode q = heat_forward(c, sum_h(h), flp, wp, Qp, phi0);
  const double rrT = c.rr * q.T;

  // reverse of the TRT collision (Eqs. (23)-(27), u = 0)
  double hb[9];
  double isb = 0.0, iab = 0.0, Hsrcb = 0.0, rrTb = 0.0, rhoHb = 0.0;
  {
    const double A0 = hb_star[0];
    const double heq0 = q.rhoH - rrT + qw<double>(0) * rrT;
    hb[0] = A0 * (1.0 - q.is);
    const double heq0b = A0 * q.is;
    isb += -A0 * (h[0] - heq0);
    Hsrcb += qw<double>(0) * A0;
    rhoHb += heq0b;
    rrTb += (qw<double>(0) - 1.0) * heq0b;
  }
#pragma unroll
  for (int i = 1; i <= 8; i++) {
    if (i == 3 || i == 4 || i == 7 || i == 8) continue;
    const int o = qopp(i);
    const double wi = qw<double>(i);
    const double es = wi * rrT;
    const double hs = 0.5 * (h[i] + h[o]), ha = 0.5 * (h[i] - h[o]);
    const double A = hb_star[i], B = hb_star[o];
    const double Dab = -A + B, Dsb = -A - B;
    double hib = A, hob = B;
    const double hab = Dab * q.ia;
    iab += Dab * ha;
    const double hsb = Dsb * q.is;
    rrTb += -Dsb * q.is * wi;
    isb += Dsb * (hs - es);
    Hsrcb += -wi * Dsb;
    hib += 0.5 * hsb + 0.5 * hab;
    hob += 0.5 * hsb - 0.5 * hab;
    hb[i] = hib;
    hb[o] = hob;
  }
  // sources and the lags written by this step
  const double lflb_new = a.lfl_in[n], lqb_new = a.lq_in[n];
  double hcoefb = Hsrcb * q.CT * q.mdot;
  double CTb = Hsrcb * q.hcoef * q.mdot;
  double mdotb = Hsrcb * q.hcoef * q.CT + lqb_new * q.C * q.T;
  double Cb = lqb_new * q.T * q.mdot + CTb * q.T;
  double Tb = c.rr * rrTb + lqb_new * q.C * q.mdot + CTb * q.C;
  double flb = lflb_new;
  // tau_a, tau_s from lambda(fs)
  iab += -0.5 * hcoefb;
  iab -= isb;
  const double taua = 1.0 / q.ia;
  const double tauab = -iab / (taua * taua);
  const double lamb = tauab * c.inv_rr3;
  const double dinterp_lam = c.lam_s - wp * c.lam_l - (1.0 - wp) * c.lam_g;
  double fsb = lamb * dinterp_lam;
  // C = rho(fs) cp(fs)
  {
    const double rho = interp(q.fs, wp, c.rho_s, c.rho_l, c.rho_g);
    const double cp = interp(q.fs, wp, c.cp_s, c.cp_l, c.cp_g);
    const double drho = c.rho_s - wp * c.rho_l - (1.0 - wp) * c.rho_g;
    const double dcp = c.cp_s - wp * c.cp_l - (1.0 - wp) * c.cp_g;
    fsb += Cb * (drho * cp + rho * dcp);
  }
  if (!(q.fs_raw > 1.0)) flb += -wp * fsb;  // the forward clamps only above 1
  // mdot = (1 - rho_s / rho_l) w (fl_prev - fl)
  const double flpb = c.one_m_ratio * wp * mdotb;
  flb += -c.one_m_ratio * wp * mdotb;
  double dL = 0.0;
  rhoHb += heat_inversion_reverse(c, q, wp, Tb, flb, &dL);
  double dTc = 0.0;
  if (masked) {
    // h_eq(T_cold, u = 0) at the (static) weight w: h_0 = rho H - rr T +
    // w_0 rr T, h_i = w_i rr T, rho H = cap T + w rho_l L fl_c
    const double Tc = c.T_cold;
    const double flc = Tc < 0.0 ? 0.0 : 1.0;
    double fsf = phi0 + wp;
    fsf = fsf > 1.0 ? 1.0 : fsf;
    const double cap = Tc < 0.0 ? heat_cap(c, fsf, wp) : heat_cap(c, phi0, wp);
    double sb = 0.0;
#pragma unroll
    for (int i = 1; i < 9; i++) sb += (hb[i] + rhoHb) * qw<double>(i);
    const double h0b = hb[0] + rhoHb;
    dTc = h0b * (cap - c.rr + qw<double>(0) * c.rr) + sb * c.rr;
    dL += h0b * wp * c.rho_l * flc;
  }
#pragma unroll
  for (int i = 0; i < 9; i++) a.lam_out[i * P + n] = masked ? 0.0 : hb[i] + rhoHb;
  a.lq_out[n] = 0.5 * rhoHb;
  a.lfl_out[n] = flpb;
#pragma unroll
  for (int k = 0; k < 4; k++) a.acc[k * P + n] += dTw[k];
  a.acc[(ADJ_NACC - 1) * P + n] += dL;
  a.acc[ADJ_NACC * P + n] += dTc;  // the caller's accumulator has a plane for T_cold
}
#endif  // LBM_ADJOINT_KERNELS

// Initial-state term: set_geometry builds the rest enthalpy population
// from rho H = C T + w rho_l L fl (Eq. (8)), the other populations from T
// alone (Eq. (25), u = 0), so dh0/dL = w rho_l fl; with lam_in the adjoint
// of the initial populations and lag the initial lag planes.
#ifdef LBM_ADJOINT_KERNELS
static __global__ void __launch_bounds__(NT) lbm_adjoint_init_kernel(const AdjArgs a) {
  const Geom& g = a.g;
  const int x = blockIdx.x * TX + threadIdx.x, y = blockIdx.y * TY + threadIdx.y;
  if (x >= g.nx || y >= g.ny) return;
  const int P = (int)g.plane;
  const int n = y * g.pitch + x;
  const double w = a.lag[LAG_W * P + n], fl = a.lag[LAG_FL * P + n];
  a.acc[(ADJ_NACC - 1) * P + n] += a.lam_in[n] * w * a.c.rho_l * fl;
}
#endif  // LBM_ADJOINT_KERNELS

// Fixed-order sum of the accumulator planes over the grid (one CTA).
#ifdef LBM_ADJOINT_KERNELS
static __global__ void __launch_bounds__(NT) lbm_adjoint_reduce_kernel(const double* __restrict__ acc,
                                                                Geom g, double* __restrict__ out) {
  __shared__ double s[ADJ_NACC][NT / 32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int P = (int)g.plane;
  double v[ADJ_NACC];
#pragma unroll
  for (int k = 0; k < ADJ_NACC; k++) v[k] = 0.0;
  for (int y = 0; y < g.ny; y++)
    for (int x = tid; x < g.nx; x += NT) {
#pragma unroll
      for (int k = 0; k < ADJ_NACC; k++) v[k] += acc[k * P + y * g.pitch + x];
    }
#pragma unroll
  for (int k = 0; k < ADJ_NACC; k++) {
    double w = v[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
    if (lane == 0) s[k][warp] = w;
  }
  __syncthreads();
  if (tid < ADJ_NACC) {
    double t = 0.0;
    for (int w = 0; w < NT / 32; w++) t += s[tid][w];
    out[tid] = t;
  }
}
#endif  // LBM_ADJOINT_KERNELS

// ---------------------------------------------------------------------------
// reverse mode of the phase-field step (lattices == LAT_PHASE: the fluid at
// rest, no heat): g* = (1 - 1/tau_g) g + g_eq / tau_g with g_eq of Eq. (19)
// at u = 0 (Eq. (20) vanishes: no phi u, no mass source), mu_phi of Eq. (6)
// from the isotropic Laplacians of phi, phi0 and fs, half-way bounce-back.
// Observable: the last phi = 0 crossing along a grid line (a column: the
// tip height; a row near the substrate: the contact line).
// Parameters: the contact angle theta (through cos theta in Eq. (6)) and
// sigma (mu_phi is proportional to it).
// ---------------------------------------------------------------------------

constexpr int PADJ_NACC = 2;  // d/dtheta_deg, d/dsigma

struct PhaseAdjArgs {
  Geom g;
  Coef<double> c;
  const double* __restrict__ gpop;   // 9 phase planes of the forward state
  const double* __restrict__ lag;    // NLAG lag planes of the forward state
  const double* __restrict__ phi0;
  double* __restrict__ phi;          // forward phi, fs planes (fields kernel output)
  double* __restrict__ fs;
  const double* __restrict__ lam_in;  // adjoint of the next state's 9 planes
  double* __restrict__ gs;            // 9 planes: adjoint of the post-collision populations
  double* __restrict__ phib;          // adjoint of phi: the node's own terms
  double* __restrict__ fsb;           // adjoint of fs: the node's own terms
  double* __restrict__ mub;           // adjoint of mu_phi
  double* __restrict__ lam_out;       // adjoint of this state's 9 planes
  double* __restrict__ acc;           // PADJ_NACC accumulator planes (+=)
  double dcos_dtheta;                 // d cos(theta) / d theta_deg
  int axis, index;                    // seed: the grid line (as lbm_read_crossings)
  double* __restrict__ out;           // seed: the crossing (1 double)
};

// phi = sum g and fs = min(phi0 + w (1 - fl), 1), w = clamp((1 - phi0 + phi) / 2)
#ifdef LBM_ADJOINT_KERNELS
static __global__ void __launch_bounds__(NT) lbm_phase_fields_kernel(const PhaseAdjArgs a) {
  const Geom& g = a.g;
  const int x = blockIdx.x * TX + threadIdx.x, y = blockIdx.y * TY + threadIdx.y;
  if (x >= g.nx || y >= g.ny) return;
  const int P = (int)g.plane;
  const int n = y * g.pitch + x;
  double v[9];
#pragma unroll
  for (int i = 0; i < 9; i++) v[i] = a.gpop[i * P + n];
  const double ph = sum_g(v);
  const double q0 = a.phi0[n];
  const double w = clamp01((1.0 - q0 + ph) * 0.5);
  const double fs = q0 + w * (1.0 - a.lag[LAG_FL * P + n]);
  a.phi[n] = ph;
  a.fs[n] = fs > 1.0 ? 1.0 : fs;
}
#endif  // LBM_ADJOINT_KERNELS

__device__ __forceinline__ int stencil_index(const Geom& g, int x, int y, int i) {
  const int xx = wrap_or_clamp(x + qx(i), g.nx, g.bc[0], g.bc[1]);
  const int yy = wrap_or_clamp(y + qy(i), g.ny, g.bc[2], g.bc[3]);
  return yy * g.pitch + xx;
}

// 6 sum_i w_i (chi(x + c_i) - chi(x)): the isotropic Laplacian (R-FD)
__device__ __forceinline__ double lap6(const Geom& g, const double* chi, int x, int y, int n) {
  double s = 0.0;
#pragma unroll
  for (int i = 1; i < 9; i++) s += 2.0 * qw<double>(i) * (chi[stencil_index(g, x, y, i)] - chi[n]);
  return 3.0 * s;
}

// Seed: the position J = k + a / (a - b) of the last crossing of phi
// through 0 along the line (one thread), dJ/dphi at the two nodes.
#ifdef LBM_ADJOINT_KERNELS
static __global__ void lbm_phase_seed_kernel(const PhaseAdjArgs a) {
  const Geom& g = a.g;
  const int P = (int)g.plane;
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int len = a.axis == 0 ? g.nx : g.ny;
  const int stride = a.axis == 0 ? 1 : g.pitch;
  const int base = a.axis == 0 ? a.index * g.pitch : a.index;
  double J = __longlong_as_double(0x7ff8000000000000ULL);
  for (int k = len - 2; k >= 0; k--) {
    const int n0 = base + k * stride, n1 = n0 + stride;
    const double va = a.phi[n0], vb = a.phi[n1];
    if ((va <= 0.0) != (vb <= 0.0)) {
      const double d = va - vb;
      J = k + va / d;
      const double da = -vb / (d * d), db = va / (d * d);
#pragma unroll
      for (int i = 0; i < 9; i++) {
        a.lam_out[i * P + n0] = da;
        a.lam_out[i * P + n1] = db;
      }
      break;
    }
  }
  a.out[0] = J;
}
#endif  // LBM_ADJOINT_KERNELS

// Shared pieces of Eq. (6): d chem / d phi, d chem / d fs, d chem / d cos(theta).
__device__ __forceinline__ void chem_partials(const Coef<double>& c, double ph, double q0,
                                              double fs, double* dphi, double* dfs,
                                              double* dcos) {
  *dphi = c.s3 * (3.0 * ph * ph - 1.0) + c.s9 * q0 * q0 + c.s3 * c.cos_th * q0 * 6.0 * ph +
          c.s9 * fs * fs + c.s3 * c.cos_ps * fs * 6.0 * ph;
  *dfs = c.s9 * 2.0 * fs * ph + c.s3 * c.cos_ps * (3.0 * ph * ph + 3.0 * fs * fs - 1.0);
  *dcos = c.s3 * q0 * (3.0 * ph * ph + q0 * q0 - 1.0);
}

// Reverse step, part 1: pull the adjoint through the push and back through
// the collision to mu_phi; store mu_phi's adjoint and the terms of phi's and
// fs's adjoints that come from the node itself (the collision's phi, the
// local part of Eq. (6), the centre of the Laplacians).
#ifdef LBM_ADJOINT_KERNELS
static __global__ void __launch_bounds__(NT) lbm_phase_adjoint1_kernel(const PhaseAdjArgs a) {
  const Geom& g = a.g;
  const Coef<double>& c = a.c;
  const int x = blockIdx.x * TX + threadIdx.x, y = blockIdx.y * TY + threadIdx.y;
  if (x >= g.nx || y >= g.ny) return;
  const int P = (int)g.plane;
  const int n = y * g.pitch + x;
  double gb[9];
#pragma unroll
  for (int i = 0; i < 9; i++) {
    int wall;
    const long long t = stream_target(g, x, y, qx(i), qy(i), wall);
    gb[i] = t >= 0 ? a.lam_in[i * P + (int)t] : a.lam_in[qopp(i) * P + n];
    a.gs[i * P + n] = gb[i];
  }
  const double itg = c.inv_tau_g;
  double mub = (qw<double>(0) - 1.0) * gb[0];
#pragma unroll
  for (int i = 1; i < 9; i++) mub += qw<double>(i) * gb[i];
  mub *= itg * c.eta;
  const double ph = a.phi[n], q0 = a.phi0[n], fs = a.fs[n];
  double dphi, dfs, dcos;
  chem_partials(c, ph, q0, fs, &dphi, &dfs, &dcos);
  const double lphi = lap6(g, a.phi, x, y, n), lphi0 = lap6(g, a.phi0, x, y, n);
  const double lfs = lap6(g, a.fs, x, y, n);
  const double mu = chem_local(c, ph, q0, fs) - c.klap * (lphi + c.cos_th * lphi0 + c.cos_ps * lfs);
  const double self = 6.0 * (1.0 - qw<double>(0));  // 6 sum_{i>0} w_i
  a.mub[n] = mub;
  a.phib[n] = itg * gb[0] + mub * dphi + c.klap * self * mub;
  a.fsb[n] = mub * dfs + c.klap * c.cos_ps * self * mub;
  a.acc[n] += mub * (dcos - c.klap * lphi0) * a.dcos_dtheta;
  a.acc[P + n] += mub * mu / c.sigma;
}
#endif  // LBM_ADJOINT_KERNELS

// Reverse step, part 2: the transposed Laplacian stencils as a gather (every
// node p within one node of n, and every direction i whose clamped or
// wrapped stencil neighbour of p is n, adds -klap 6 w_i mub(p); a fixed
// order, so the sweep is deterministic), then fs -> w -> phi (local) and
// phi = sum g.
#ifdef LBM_ADJOINT_KERNELS
static __global__ void __launch_bounds__(NT) lbm_phase_adjoint2_kernel(const PhaseAdjArgs a) {
  const Geom& g = a.g;
  const Coef<double>& c = a.c;
  const int x = blockIdx.x * TX + threadIdx.x, y = blockIdx.y * TY + threadIdx.y;
  if (x >= g.nx || y >= g.ny) return;
  const int P = (int)g.plane;
  const int n = y * g.pitch + x;
  double lsum = 0.0;  // sum of 6 w_i mub(p) over the stencil links that reach n
  for (int dy = -1; dy <= 1; dy++) {
    int py = y + dy;
    if (py < 0 || py >= g.ny) {
      if (g.bc[2] != BC_PERIODIC) continue;
      py = (py + g.ny) % g.ny;
    }
    // on a periodic axis of length 2, y - 1 and y + 1 are the same node
    if (dy == 1 && py == (y - 1 + g.ny) % g.ny && g.ny > 1 && g.bc[2] == BC_PERIODIC) continue;
    for (int dx = -1; dx <= 1; dx++) {
      int px = x + dx;
      if (px < 0 || px >= g.nx) {
        if (g.bc[0] != BC_PERIODIC) continue;
        px = (px + g.nx) % g.nx;
      }
      if (dx == 1 && px == (x - 1 + g.nx) % g.nx && g.nx > 1 && g.bc[0] == BC_PERIODIC) continue;
      const double mp = a.mub[py * g.pitch + px];
#pragma unroll
      for (int i = 1; i < 9; i++)
        if (stencil_index(g, px, py, i) == n) lsum += 6.0 * qw<double>(i) * mp;
    }
  }
  double phib = a.phib[n] - c.klap * lsum;
  const double fsb = a.fsb[n] - c.klap * c.cos_ps * lsum;
  const double q0 = a.phi0[n], ph = a.phi[n], fl = a.lag[LAG_FL * P + n];
  const double wraw = (1.0 - q0 + ph) * 0.5;
  const double w = clamp01(wraw);
  const double fsraw = q0 + w * (1.0 - fl);
  if (!(fsraw > 1.0) && !(wraw < 0.0) && !(wraw > 1.0)) phib += fsb * (1.0 - fl) * 0.5;
  const double omg = 1.0 - c.inv_tau_g;
#pragma unroll
  for (int i = 0; i < 9; i++) a.lam_out[i * P + n] = omg * a.gs[i * P + n] + phib;
}
#endif  // LBM_ADJOINT_KERNELS

// Initial state (a run from set_geometry): g0 = g_eq(phi0_init, mu_phi0)
// depends on theta and sigma through mu_phi0.
#ifdef LBM_ADJOINT_KERNELS
static __global__ void __launch_bounds__(NT) lbm_phase_init_kernel(const PhaseAdjArgs a) {
  const Geom& g = a.g;
  const Coef<double>& c = a.c;
  const int x = blockIdx.x * TX + threadIdx.x, y = blockIdx.y * TY + threadIdx.y;
  if (x >= g.nx || y >= g.ny) return;
  const int P = (int)g.plane;
  const int n = y * g.pitch + x;
  double mub = (qw<double>(0) - 1.0) * a.lam_in[n];
#pragma unroll
  for (int i = 1; i < 9; i++) mub += qw<double>(i) * a.lam_in[i * P + n];
  mub *= c.eta;
  const double ph = a.phi[n], q0 = a.phi0[n], fs = a.fs[n];
  double dphi, dfs, dcos;
  chem_partials(c, ph, q0, fs, &dphi, &dfs, &dcos);
  const double lphi = lap6(g, a.phi, x, y, n), lphi0 = lap6(g, a.phi0, x, y, n);
  const double lfs = lap6(g, a.fs, x, y, n);
  const double mu = chem_local(c, ph, q0, fs) - c.klap * (lphi + c.cos_th * lphi0 + c.cos_ps * lfs);
  a.acc[n] += mub * (dcos - c.klap * lphi0) * a.dcos_dtheta;
  a.acc[P + n] += mub * mu / c.sigma;
}
#endif  // LBM_ADJOINT_KERNELS

// ---------------------------------------------------------------------------
// reverse mode of the coupled phase-field and enthalpy step (lattices ==
// LAT_PHASE | LAT_HEAT: the fluid at rest).  The freezing
// couples the lattices: the mass source mdot of Eq. (1) enters the order
// parameter (Eq. (22)) and the phase source (Eq. (20)); the weight w and
// the solid fraction fs = phi0 + w (1 - fl) set the properties of Eq. (10)
// (rho Cp and lambda of the enthalpy collision) and the wetting terms of
// Eq. (6); the lagged w enters the inversion of Eq. (8) and mdot.  Per step
// in reverse: a fields kernel (phi, fs of the recomputed state), a kernel for
// the adjoint of mu_phi and its theta and sigma terms, and a kernel that
// pulls the adjoints of both lattices through the push (anti-bounce-back at
// Dirichlet walls), reverses the two collisions, gathers the transposed
// stencils and runs the local chain (fs, w, phi, mdot, the inversion) back
// to the adjoints of this state's populations and lags (fl, w, Q).
// Accumulator planes: d/dT_wall[0..3], d/dL, d/dtheta_deg, d/dsigma.
// ---------------------------------------------------------------------------

constexpr int FRZ_NACC = 8;  // ... and d/dT_cold (cold mask)

struct FrzArgs {
  Geom g;
  Coef<double> c;
  const unsigned char* __restrict__ mask;  // cold mask (has_mask) or null
  int has_mask;
  const double* __restrict__ pop;     // 18 planes of the forward state: g (0-8), h (9-17)
  const double* __restrict__ lag;     // NLAG planes of the forward state
  const double* __restrict__ phi0;
  double* __restrict__ phi;           // fields of the forward state
  double* __restrict__ fs;
  const double* __restrict__ lam_in;  // 18 planes: adjoints of the next g (0-8), h (9-17)
  const double* __restrict__ lfl_in;  // adjoints of the next state's lags fl, w, Q
  const double* __restrict__ lw_in;
  const double* __restrict__ lq_in;
  double* __restrict__ mub;           // adjoint of mu_phi
  const double* __restrict__ phib_seed;  // extra adjoint of phi (observable seed) or null
  double* __restrict__ lam_out;       // 18 planes: adjoints of this state's g, h
  double* __restrict__ lfl_out;
  double* __restrict__ lw_out;
  double* __restrict__ lq_out;
  double* __restrict__ acc;           // FRZ_NACC planes (+=)
  double dcos_dtheta;
  double inv_sum_w, ff;               // frozen-fraction seed
  int axis, index;                    // crossing seed
  double* __restrict__ out;           // crossing value (1 double)
};

// Forward quantities of one node of the coupled step.
struct FrzNode {
  double rhoH, T, fl, mdot, ell, Cm, Cp, fsf;
  int branch;  // 0 frozen, 1 liquid, 2 mushy
  bool fsf_clamped;
  double D, phi, wraw, w, fs_raw, fs, rho, cp, C, lam, taua, ia, is, hcoef, CT;
};

__device__ __forceinline__ double dinterp_dfs(double w, double zs, double zl, double zg) {
  return zs - w * zl - (1.0 - w) * zg;
}
__device__ __forceinline__ double dinterp_dw(double fs, double zl, double zg) {
  return (1.0 - fs) * (zl - zg);
}

__device__ __forceinline__ FrzNode frz_forward(const Coef<double>& c, double sg, double sh,
                                               double flp, double wp, double Qp, double phi0) {
  FrzNode q;
  q.rhoH = sh + 0.5 * Qp;
  q.ell = wp * c.rho_l * c.latent;
  q.fsf = phi0 + wp;
  q.fsf_clamped = q.fsf > 1.0;
  if (q.fsf_clamped) q.fsf = 1.0;
  q.Cm = heat_cap(c, q.fsf, wp);
  q.Cp = heat_cap(c, phi0, wp);
  if (q.rhoH < 0.0) {
    q.branch = 0;
    q.fl = 0.0;
    q.T = q.rhoH / q.Cm;
  } else if (q.rhoH > q.ell) {
    q.branch = 1;
    q.fl = 1.0;
    q.T = (q.rhoH - q.ell) / q.Cp;
  } else {
    q.branch = 2;
    q.T = 0.0;
    q.fl = q.ell > 0.0 ? q.rhoH / q.ell : 1.0;
  }
  q.fl = clamp01(q.fl);
  q.mdot = c.one_m_ratio * wp * (flp - q.fl);
  q.D = 1.0 - 0.5 * q.mdot;
  q.phi = q.mdot == 0.0 ? sg : sg / q.D;
  q.wraw = (1.0 - phi0 + q.phi) * 0.5;
  q.w = clamp01(q.wraw);
  q.fs_raw = phi0 + q.w * (1.0 - q.fl);
  q.fs = q.fs_raw > 1.0 ? 1.0 : q.fs_raw;
  q.rho = interp(q.fs, q.w, c.rho_s, c.rho_l, c.rho_g);
  q.cp = interp(q.fs, q.w, c.cp_s, c.cp_l, c.cp_g);
  q.C = q.rho * q.cp;
  q.lam = interp(q.fs, q.w, c.lam_s, c.lam_l, c.lam_g);
  q.taua = 0.5 + q.lam * c.inv_rr3;
  q.ia = 1.0 / q.taua;
  q.is = 2.0 - q.ia;
  q.hcoef = 1.0 - 0.5 * q.ia;
  q.CT = q.C * q.T;
  return q;
}

__device__ __forceinline__ FrzNode frz_node(const FrzArgs& a, int n) {
  const int P = (int)a.g.plane;
  double v[9];
#pragma unroll
  for (int i = 0; i < 9; i++) v[i] = a.pop[i * P + n];
  const double sg = sum_g(v);
  if (a.has_mask && a.mask[n]) {
    // a cold-mask node reads h_eq(T_cold, u = 0) at its lagged w
    cold_mask_h(a.c, a.lag[LAG_W * P + n], a.phi0[n], v);
  } else {
#pragma unroll
    for (int i = 0; i < 9; i++) v[i] = a.pop[(9 + i) * P + n];
  }
  const double sh = sum_h(v);
  return frz_forward(a.c, sg, sh, a.lag[LAG_FL * P + n], a.lag[LAG_W * P + n],
                     a.lag[LAG_Q * P + n], a.phi0[n]);
}

// d(rho Cp)/dfs and d(rho Cp)/dw at (fs, w)
__device__ __forceinline__ void dcap(const Coef<double>& c, double fs, double w, double* dfs,
                                     double* dw) {
  const double rho = interp(fs, w, c.rho_s, c.rho_l, c.rho_g);
  const double cp = interp(fs, w, c.cp_s, c.cp_l, c.cp_g);
  *dfs = dinterp_dfs(w, c.rho_s, c.rho_l, c.rho_g) * cp + rho * dinterp_dfs(w, c.cp_s, c.cp_l, c.cp_g);
  *dw = dinterp_dw(fs, c.rho_l, c.rho_g) * cp + rho * dinterp_dw(fs, c.cp_l, c.cp_g);
}

#ifdef LBM_ADJOINT_KERNELS
static __global__ void __launch_bounds__(NT) lbm_frz_fields_kernel(const FrzArgs a) {
  const Geom& g = a.g;
  const int x = blockIdx.x * TX + threadIdx.x, y = blockIdx.y * TY + threadIdx.y;
  if (x >= g.nx || y >= g.ny) return;
  const int n = y * g.pitch + x;
  const FrzNode q = frz_node(a, n);
  a.phi[n] = q.phi;
  a.fs[n] = q.fs;
}
#endif  // LBM_ADJOINT_KERNELS

// Adjoint of mu_phi from the pulled phase adjoints, with its theta and
// sigma terms (zero for the seed, whose pulled adjoints are zero).
#ifdef LBM_ADJOINT_KERNELS
static __global__ void __launch_bounds__(NT) lbm_frz_mub_kernel(const FrzArgs a) {
  const Geom& g = a.g;
  const Coef<double>& c = a.c;
  const int x = blockIdx.x * TX + threadIdx.x, y = blockIdx.y * TY + threadIdx.y;
  if (x >= g.nx || y >= g.ny) return;
  const int P = (int)g.plane;
  const int n = y * g.pitch + x;
  double mub = 0.0;
#pragma unroll
  for (int i = 0; i < 9; i++) {
    int wall;
    const long long t = stream_target(g, x, y, qx(i), qy(i), wall);
    const double gb = t >= 0 ? a.lam_in[i * P + (int)t] : a.lam_in[qopp(i) * P + n];
    mub += (qw<double>(i) - (i == 0 ? 1.0 : 0.0)) * gb;
  }
  mub *= c.inv_tau_g * c.eta;
  a.mub[n] = mub;
  const double ph = a.phi[n], q0 = a.phi0[n], fs = a.fs[n];
  double dphi, dfs, dcos;
  chem_partials(c, ph, q0, fs, &dphi, &dfs, &dcos);
  const double lphi = lap6(g, a.phi, x, y, n), lphi0 = lap6(g, a.phi0, x, y, n);
  const double lfs = lap6(g, a.fs, x, y, n);
  const double mu = chem_local(c, ph, q0, fs) - c.klap * (lphi + c.cos_th * lphi0 + c.cos_ps * lfs);
  a.acc[5 * P + n] += mub * (dcos - c.klap * lphi0) * a.dcos_dtheta;
  a.acc[6 * P + n] += mub * mu / c.sigma;
}
#endif  // LBM_ADJOINT_KERNELS

// The rest of one reverse step (see the section header).
#ifdef LBM_ADJOINT_KERNELS
static __global__ void __launch_bounds__(NT) lbm_frz_step_kernel(const FrzArgs a) {
  const Geom& g = a.g;
  const Coef<double>& c = a.c;
  const int x = blockIdx.x * TX + threadIdx.x, y = blockIdx.y * TY + threadIdx.y;
  if (x >= g.nx || y >= g.ny) return;
  const int P = (int)g.plane;
  const int n = y * g.pitch + x;
  // pull the adjoints of both lattices' post-collision populations
  double gb[9], hb_star[9];
  double dTw[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
  for (int i = 0; i < 9; i++) {
    int wall;
    const long long t = stream_target(g, x, y, qx(i), qy(i), wall);
    if (t >= 0) {
      gb[i] = a.lam_in[i * P + (int)t];
      hb_star[i] = a.lam_in[(9 + i) * P + (int)t];
    } else {
      gb[i] = a.lam_in[qopp(i) * P + n];
      const double lb = a.lam_in[(9 + qopp(i)) * P + n];
      if (g.bc[wall] == BC_DIRICHLET) {
        hb_star[i] = -lb;
        dTw[wall] += lb * 2.0 * qw<double>(i) * c.rr;
      } else {
        hb_star[i] = lb;
      }
    }
  }
  const FrzNode q = frz_node(a, n);
  const double phi0 = a.phi0[n];
  const double wp = a.lag[LAG_W * P + n], flp = a.lag[LAG_FL * P + n];
  const bool masked = a.has_mask && a.mask[n];
  double h[9];
  if (masked) {
    cold_mask_h(c, wp, phi0, h);
  } else {
#pragma unroll
    for (int i = 0; i < 9; i++) h[i] = a.pop[(9 + i) * P + n];
  }
  const double rrT = c.rr * q.T;

  // enthalpy TRT collision in reverse (u = 0)
  double hb[9];
  double isb = 0.0, iab = 0.0, Hsrcb = 0.0, rrTb = 0.0, rhoHb = 0.0;
  {
    const double A0 = hb_star[0];
    const double heq0 = q.rhoH - rrT + qw<double>(0) * rrT;
    hb[0] = A0 * (1.0 - q.is);
    const double heq0b = A0 * q.is;
    isb += -A0 * (h[0] - heq0);
    Hsrcb += qw<double>(0) * A0;
    rhoHb += heq0b;
    rrTb += (qw<double>(0) - 1.0) * heq0b;
  }
#pragma unroll
  for (int i = 1; i <= 8; i++) {
    if (i == 3 || i == 4 || i == 7 || i == 8) continue;
    const int o = qopp(i);
    const double wi = qw<double>(i);
    const double es = wi * rrT;
    const double hs = 0.5 * (h[i] + h[o]), ha = 0.5 * (h[i] - h[o]);
    const double A = hb_star[i], B = hb_star[o];
    const double Dab = -A + B, Dsb = -A - B;
    const double hab = Dab * q.ia, hsb = Dsb * q.is;
    iab += Dab * ha;
    rrTb += -Dsb * q.is * wi;
    isb += Dsb * (hs - es);
    Hsrcb += -wi * Dsb;
    hb[i] = A + 0.5 * hsb + 0.5 * hab;
    hb[o] = B + 0.5 * hsb - 0.5 * hab;
  }
  // enthalpy source Hsrc = hcoef C T mdot and the lag Q = C T mdot
  const double lqb = a.lq_in[n];
  const double hcoefb = Hsrcb * q.CT * q.mdot;
  const double CTb = Hsrcb * q.hcoef * q.mdot;
  double mdotb = Hsrcb * q.hcoef * q.CT + lqb * q.C * q.T;
  const double Cb = lqb * q.T * q.mdot + CTb * q.T;
  double Tb = c.rr * rrTb + lqb * q.C * q.mdot + CTb * q.C;
  // relaxation rates from lambda(fs, w), capacity rho Cp (fs, w)
  iab += -0.5 * hcoefb;
  iab -= isb;
  const double lamb = -iab / (q.taua * q.taua) * c.inv_rr3;
  double fsb = lamb * dinterp_dfs(q.w, c.lam_s, c.lam_l, c.lam_g);
  double wb = lamb * dinterp_dw(q.fs, c.lam_l, c.lam_g);
  {
    double cf, cw;
    dcap(c, q.fs, q.w, &cf, &cw);
    fsb += Cb * cf;
    wb += Cb * cw;
  }
  // phase collision in reverse: phi and mdot (the mu_phi part is gathered)
  double S = 0.0;
#pragma unroll
  for (int i = 0; i < 9; i++) S += qw<double>(i) * gb[i];
  const double itg = c.inv_tau_g, gcoef = 1.0 - 0.5 * itg;
  double phib = itg * gb[0] + gcoef * q.mdot * S;
  mdotb += gcoef * q.phi * S;
  if (a.phib_seed) phib += a.phib_seed[n];
  // mu_phi of this node (local part, centre of the Laplacians) and the
  // transposed stencils of the neighbours' mu_phi
  {
    const double mub = a.mub[n];
    double dphi, dfs, dcos;
    chem_partials(c, q.phi, phi0, q.fs, &dphi, &dfs, &dcos);
    const double self = 6.0 * (1.0 - qw<double>(0));
    phib += mub * dphi + c.klap * self * mub;
    fsb += mub * dfs + c.klap * c.cos_ps * self * mub;
    double lsum = 0.0;
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
        const double mp = a.mub[py * g.pitch + px];
#pragma unroll
        for (int i = 1; i < 9; i++)
          if (stencil_index(g, px, py, i) == n) lsum += 6.0 * qw<double>(i) * mp;
      }
    }
    phib -= c.klap * lsum;
    fsb -= c.klap * c.cos_ps * lsum;
  }
  // lags written by this step
  wb += a.lw_in[n];
  double flb = a.lfl_in[n];
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
  double wpb = mdotb * c.one_m_ratio * (flp - q.fl);
  const double flpb = mdotb * c.one_m_ratio * wp;
  flb += -mdotb * c.one_m_ratio * wp;
  // the inversion of Eq. (8) with its dependence on w_prev
  double ellb = 0.0;
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
  if (masked) {
    // the populations read here are h_eq(T_cold, u = 0) at w_prev: their
    // adjoint goes to w_prev, T_cold and L instead of the stored ones
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
    double sb = 0.0;
#pragma unroll
    for (int i = 1; i < 9; i++) sb += (hb[i] + rhoHb) * qw<double>(i);
    const double h0b = hb[0] + rhoHb;
    wpb += h0b * (dcapw * Tc + c.rho_l * c.latent * flc);
    dTc = h0b * (cap - c.rr + qw<double>(0) * c.rr) + sb * c.rr;
    dL += h0b * wp * c.rho_l * flc;
  }
  const double omg = 1.0 - itg;
#pragma unroll
  for (int i = 0; i < 9; i++) {
    a.lam_out[i * P + n] = omg * gb[i] + sgb;
    a.lam_out[(9 + i) * P + n] = masked ? 0.0 : hb[i] + rhoHb;
  }
  a.lfl_out[n] = flpb;
  a.lw_out[n] = wpb;
  a.lq_out[n] = 0.5 * rhoHb;
#pragma unroll
  for (int k = 0; k < 4; k++) a.acc[k * P + n] += dTw[k];
  a.acc[4 * P + n] += dL;
  a.acc[7 * P + n] += dTc;
}
#endif  // LBM_ADJOINT_KERNELS

// Seeds on the final state.  Frozen fraction FF = sum w (1 - fl) / sum w
// (w and fl of this state): the adjoints of the lags this state's reader
// would write, with zero population adjoints.
#ifdef LBM_ADJOINT_KERNELS
static __global__ void __launch_bounds__(NT) lbm_frz_seed_ff_kernel(const FrzArgs a) {
  const Geom& g = a.g;
  const int x = blockIdx.x * TX + threadIdx.x, y = blockIdx.y * TY + threadIdx.y;
  if (x >= g.nx || y >= g.ny) return;
  const int n = y * g.pitch + x;
  const FrzNode q = frz_node(a, n);
  a.lfl_out[n] = -q.w * a.inv_sum_w;
  a.lw_out[n] = ((1.0 - q.fl) - a.ff) * a.inv_sum_w;
}
#endif  // LBM_ADJOINT_KERNELS

// Crossing: the last phi = 0 crossing along the line (one thread), as an
// adjoint of phi at its two nodes.
#ifdef LBM_ADJOINT_KERNELS
static __global__ void lbm_frz_seed_crossing_kernel(const FrzArgs a, double* __restrict__ phib) {
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
      const double d = va - vb;
      J = k + va / d;
      phib[n0] = -vb / (d * d);
      phib[n1] = va / (d * d);
      break;
    }
  }
  a.out[0] = J;
}
#endif  // LBM_ADJOINT_KERNELS

cudaError_t launch_frz_fields(const FrzArgs& a, cudaStream_t s);
cudaError_t launch_frz_mub(const FrzArgs& a, cudaStream_t s);
cudaError_t launch_frz_step(const FrzArgs& a, cudaStream_t s);
cudaError_t launch_frz_seed_ff(const FrzArgs& a, cudaStream_t s);
cudaError_t launch_frz_seed_crossing(const FrzArgs& a, double* phib, cudaStream_t s);
// phi and fs of a state as lbm_set_geometry built it (for the initial-state
// terms): phi = sum g (the initial phase equilibrium sums to the input phi)
// and fs = min(phi0 + w (1 - fl), 1) from the initial lags -- not from the
// enthalpy inversion, which at a cold-mask node need not give back the input
// fl.  gpop: the 9 phase planes; out: two planes.
#ifdef LBM_ADJOINT_KERNELS
static __global__ void __launch_bounds__(NT) lbm_adjoint_init_fields_kernel(
    Geom g, const double* __restrict__ gpop, const double* __restrict__ lag,
    const double* __restrict__ phi0, double* __restrict__ phi, double* __restrict__ fs) {
  const int x = blockIdx.x * TX + threadIdx.x, y = blockIdx.y * TY + threadIdx.y;
  if (x >= g.nx || y >= g.ny) return;
  const int P = (int)g.plane;
  const int n = y * g.pitch + x;
  double v[9];
#pragma unroll
  for (int i = 0; i < 9; i++) v[i] = gpop[i * P + n];
  phi[n] = sum_g(v);
  const double f = phi0[n] + lag[LAG_W * P + n] * (1.0 - lag[LAG_FL * P + n]);
  fs[n] = f > 1.0 ? 1.0 : f;
}
#endif  // LBM_ADJOINT_KERNELS

cudaError_t launch_adjoint_init_fields(const Geom& g, const double* gpop, const double* lag,
                                       const double* phi0, double* phi, double* fs,
                                       cudaStream_t s);
cudaError_t launch_phase_adjoint_fields(const PhaseAdjArgs& a, cudaStream_t s);
cudaError_t launch_phase_adjoint_seed(const PhaseAdjArgs& a, cudaStream_t s);
cudaError_t launch_phase_adjoint_step(const PhaseAdjArgs& a, cudaStream_t s);
cudaError_t launch_phase_adjoint_init(const PhaseAdjArgs& a, cudaStream_t s);

}  // namespace lbmk
