// lbm_kernels.cuh -- device code of the fused coupled LB time step for
// sm_103a (GB300), templated on the arithmetic type R (float or double).
//
// One CTA owns a TX x TY tile of nodes and stages, in shared memory, the
// macroscopic fields of the tile plus a one-node halo.  Phase A issues every
// global load of the CTA at once: each thread loads its own node (27
// populations kept in registers, lag fields, phi0) and, in parallel, a
// third of the 18 phase/enthalpy populations of one halo-ring node; the
// ring partial sums meet in shared memory.  The enthalpy inversion (Eq. (8)),
// order parameter (Eq. (22)), material weight, solid fraction and density
// (Eq. (10)) are evaluated for the own node and then for the ring.  Phase B
// evaluates the isotropic stencils of the gradients and the chemical
// potential (Eq. (6)), the velocity and pressure (Eq. (17)), the three
// collisions (Eqs. (11), (18), (23)), pushes the post-collision populations
// to the neighbours in the other buffer with half-way bounce-back /
// anti-bounce-back at walls and stores the lag fields of the next step.
// Global FP64 diagnostics are reduced in the same launch into per-CTA
// partial sums (warp shuffles, then the warps in a fixed order); a one-CTA
// kernel sums the partials in a fixed order when they are read, so the
// result is bitwise reproducible run to run.
//
// Layout in HBM: structure of arrays, one plane per population or field,
// planes of `plane` elements with rows padded to `pitch` (a multiple of 32
// elements).  Populations: planes 0-8 flow f, 9-17 phase g, 18-26 enthalpy h,
// double-buffered (A/B).  Lag fields (double-buffered because neighbours
// read them): fl, w, p, phi ux, phi uy, Q.  Static: phi0 and a byte mask.
#pragma once

#include <cstdint>
#include <type_traits>

#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "lbm_dual.cuh"

namespace lbmk {

constexpr int TX = 32, TY = 8;
constexpr int HX = TX + 2, HY = TY + 2, HN = HX * HY;
constexpr int NT = TX * TY;
constexpr int RING = HN - NT;  // 84 halo nodes
constexpr int NPART = 3;       // threads per ring node in phase A
constexpr int NDIAG = 9;
constexpr int NFIELD = 12;
static_assert(RING * NPART <= NT, "ring loads must fit one pass of the CTA");

// Tile shapes of the one-CTA-per-tile step: 32 x TY_ nodes (a warp per row,
// so every shape keeps 128-byte rows), TY_ = 4, 8 (the default above) or 16.
// The autotuner picks one per grid: short tiles suit grids a few rows high
// (the one-dimensional columns), tall ones shrink the ring's share (84 ring
// nodes per 256 at 32 x 8, 100 per 512 at 32 x 16).
template <int TY_>
struct Shape {
  static_assert(TY_ == 4 || TY_ == 8 || TY_ == 16, "tile shapes 32 x 4, 32 x 8, 32 x 16");
  static constexpr int TY = TY_, HY = TY_ + 2, HN = HX * HY, NT = TX * TY_, RING = HN - NT;
};
__host__ __device__ constexpr int tiles_y(int ny, int ty) { return (ny + ty - 1) / ty; }
enum { BC_PERIODIC = 0, BC_DIRICHLET = 1, BC_ADIABATIC = 2 };
enum { LAT_FLOW = 1, LAT_PHASE = 2, LAT_HEAT = 4 };
enum { LAG_FL = 0, LAG_W, LAG_P, LAG_PHUX, LAG_PHUY, LAG_Q, NLAG };
// Contexts with float arithmetic (FP32, FP16 storage) keep one more lag plane
// after these: the temperature of the previous step, the reference of their
// well-balanced enthalpy storage (see kShift).
constexpr int LAG_T = NLAG;
enum { F_PHI = 0, F_FS, F_FL, F_T, F_RHOH, F_P, F_UX, F_UY, F_RHO, F_MU, F_W, F_MDOT };
enum { MODE_STEP = 0, MODE_READ = 1 };

// D2Q9 of Eq. (12): rest, axes counter-clockwise from +x, diagonals from (1,1)
__host__ __device__ constexpr int qx(int i) {
  return (i == 1 || i == 5 || i == 8) ? 1 : ((i == 3 || i == 6 || i == 7) ? -1 : 0);
}
__host__ __device__ constexpr int qy(int i) {
  return (i == 2 || i == 5 || i == 6) ? 1 : ((i == 4 || i == 7 || i == 8) ? -1 : 0);
}
__host__ __device__ constexpr int qopp(int i) {
  return i == 0 ? 0 : (i <= 4 ? ((i + 1) % 4) + 1 : ((i - 3) % 4) + 5);
}
template <typename R>
__device__ __forceinline__ R qw(int i) {
  return i == 0 ? R(4.0 / 9.0) : (i <= 4 ? R(1.0 / 9.0) : R(1.0 / 36.0));
}

// Division: IEEE in double.  In float, the quotient from the approximate
// reciprocal (PTX rcp.approx.f32) with one Newton correction on the exact
// residual (Markstein's correction step: e = a - q0 b by FMA, q = q0 + e r),
// which leaves an error of about one ulp without the plain approximate
// quotient's one-sided bias: an error that repeats every step at a slowly
// changing node (1 - mdot/2 in the order parameter, the heat capacity in the
// temperature) would otherwise accumulate.  The divisors are positive normal
// numbers (densities, heat capacities, relaxation times, 1 - mdot/2).  Built
// with LBM_F32_FAST_DIV=0, the IEEE quotient instead.
#ifndef LBM_F32_FAST_DIV
#define LBM_F32_FAST_DIV 1
#endif
__device__ __forceinline__ double qdiv(double a, double b) { return a / b; }
__device__ __forceinline__ float qdiv(float a, float b) {
#if LBM_F32_FAST_DIV
  float r;
  asm("rcp.approx.f32 %0, %1;" : "=f"(r) : "f"(b));
  const float q0 = a * r;
  return fmaf(fmaf(-q0, b, a), r, q0);
#else
  return __fdiv_rn(a, b);
#endif
}

// Per-context constants (derived on the host by lbm_create).
template <typename R>
struct Coef {
  R rho_l, rho_s, rho_g, mu_l, mu_s, mu_g, lam_l, lam_s, lam_g, cp_l, cp_s, cp_g;
  R rr;          // rho_ref * Cp_ref
  R latent, sigma, eps, eta, cos_th, cos_ps, gx, gy;
  R tau_g;       // Eq. (21)
  R T_cold;
  R one_m_ratio; // 1 - rho_s / rho_l
  R T_wall[4];
  // per-context products the kernels would otherwise form per node
  R s3, s9;      // 3 sigma / eps, 9 sigma / eps (Eq. (6))
  R klap;        // 3 eps sigma / 8 (Eq. (6))
  R rr3;         // rho_ref Cp_ref cs^2 (Eq. (26))
  R inv_rr3;     // 1 / rr3
  R inv_tau_g;   // 1 / tau_g
  R wrr1, wrr5;  // w_i rho_ref Cp_ref of the axes and of the diagonals
  R rr_rest;     // (1 - w_0) rho_ref Cp_ref
  uint32_t readings;  // must stay the last member
};

struct Geom {
  int nx, ny, pitch;
  long long plane;
  int lattices;
  int bc[4];
  int has_mask;
};

// R: arithmetic type; S: storage type of the populations (R, or __half
// for FP16 storage with FP32 arithmetic).
template <typename R, typename S = R>
struct Args {
  Geom g;
  Coef<R> c;
  const S* __restrict__ pin;   // 27 planes
  S* __restrict__ pout;        // 27 planes
  const R* __restrict__ lin;   // NLAG planes
  R* __restrict__ lout;        // NLAG planes
  const R* __restrict__ phi0;
  const uint8_t* __restrict__ mask;
  double* out[NFIELD];         // MODE_READ: dense [ny][nx] outputs (or null)
  double* diag_partial;        // [NDIAG][nblocks] per-CTA partial sums
};

template <typename R, typename S = R>
struct InitArgs {
  Geom g;
  Coef<R> c;
  S* __restrict__ pout;
  R* __restrict__ lout;
  R* __restrict__ phi0_out;
  uint8_t* __restrict__ mask_out;
  const double* __restrict__ phi0;
  const uint8_t* __restrict__ mask;
  const double* __restrict__ phi;
  const double* __restrict__ T;
  const double* __restrict__ fl;
};

// ---------------------------------------------------------------------------
// local physics
// ---------------------------------------------------------------------------

template <typename R>
__device__ __forceinline__ R clamp01(R v) {
  return v < R(0) ? R(0) : (v > R(1) ? R(1) : v);
}

// Eq. (10)
template <typename R>
__device__ __forceinline__ R interp(R fs, R w, R zs, R zl, R zg) {
  return fs * zs + (R(1) - fs) * w * zl + (R(1) - fs) * (R(1) - w) * zg;
}

template <typename R>
__device__ __forceinline__ R heat_cap(const Coef<R>& c, R fs, R w) {
  return interp(fs, w, c.rho_s, c.rho_l, c.rho_g) * interp(fs, w, c.cp_s, c.cp_l, c.cp_g);
}

// Eq. (8) with T_m = 0, latent capacity w rho_l L, sensible capacities at
// the fully frozen (fs = min(phi0 + w, 1)) and fully liquid (fs = phi0)
// states; ties to the mushy branch.
template <typename R>
__device__ __forceinline__ void invert_enthalpy(const Coef<R>& c, R rhoH, R w, R phi0, R& T,
                                                R& fl) {
  R ell = w * c.rho_l * c.latent;
  R fsf = phi0 + w;
  fsf = fsf > R(1) ? R(1) : fsf;
  if (rhoH < R(0)) {
    fl = R(0);
    T = qdiv(rhoH, heat_cap(c, fsf, w));
  } else if (rhoH > ell) {
    fl = R(1);
    T = qdiv(rhoH - ell, heat_cap(c, phi0, w));
  } else {
    T = R(0);
    fl = ell > R(0) ? qdiv(rhoH, ell) : R(1);
  }
  fl = clamp01(fl);
}

// Enthalpy equilibrium Eq. (25) at temperature T with velocity (ux, uy);
// rrC = rr / C.
template <typename R>
__device__ __forceinline__ R heq_i(int i, R rhoH, R C, R T, R rr, R rrC, R ux, R uy, R uu) {
  if (i == 0) return rhoH - rr * T + qw<R>(0) * C * T * (rrC - uu * R(1.5));
  R cu = R(qx(i)) * ux + R(qy(i)) * uy;
  return qw<R>(i) * C * T * (rrC + R(3) * cu + R(4.5) * cu * cu - R(1.5) * uu);
}

// Enthalpy populations of a cold-mask node: h_eq(T_cold, u = 0) at the
// node's weight w and phi0 (the reset that follows streaming, applied when
// the populations are read).
template <typename R>
__device__ __forceinline__ void cold_mask_h(const Coef<R>& c, R w, R phi0, R* h) {
  R T = c.T_cold;
  R flc = T < R(0) ? R(0) : R(1);
  R fsf = phi0 + w;
  fsf = fsf > R(1) ? R(1) : fsf;
  R cap = T < R(0) ? heat_cap(c, fsf, w) : heat_cap(c, phi0, w);
  R rhoH = cap * T + w * c.rho_l * c.latent * flc;
  R fs = phi0 + w * (R(1) - flc);
  fs = fs > R(1) ? R(1) : fs;
  R C = heat_cap(c, fs, w);
  R rrC = qdiv(c.rr, C);
#pragma unroll
  for (int i = 0; i < 9; i++) h[i] = heq_i<R>(i, rhoH, C, T, c.rr, rrC, R(0), R(0), R(0));
}

// Canonical summation order of the phase and enthalpy populations, shared
// by the own-node and the ring paths so that a node's sums do not depend on
// which CTA evaluates it: g = (g0..g5) + (g6..g8), h = (h0..h2) + (h3..h8).
// ---------------------------------------------------------------------------
// population storage: the arithmetic type itself, or FP16 (round to nearest)
// ---------------------------------------------------------------------------

// Read-out of one field value at dense index d of an N-node field; a
// tangent value writes its derivative N entries further on.
__device__ __forceinline__ void put_out(double* p, long long d, long long, float v) { p[d] = v; }
__device__ __forceinline__ void put_out(double* p, long long d, long long, double v) { p[d] = v; }
__device__ __forceinline__ void put_out(double* p, long long d, long long N, const Dual& v) {
  p[d] = v.v;
  p[d + N] = v.d;
}

__device__ __forceinline__ float ldp(const float* p) { return *p; }
__device__ __forceinline__ double ldp(const double* p) { return *p; }
__device__ __forceinline__ float ldp(const __half* p) { return __half2float(*p); }
__device__ __forceinline__ void stp(float* p, float v) { *p = v; }
__device__ __forceinline__ void stp(double* p, double v) { *p = v; }
__device__ __forceinline__ void stp(__half* p, float v) { *p = __float2half_rn(v); }

// Well-balanced storage of float states (FP32 and FP16 storage).  Every
// population that carries a large, slowly varying part is stored -- and
// handled in the arithmetic of the step -- as its difference from a
// reference that the writer and the next reader compute identically from
// the lag fields:
//
//   g0       2 w - 1 + phi0 (= phi where w is not clamped), the bulk of the
//            rest population phi + (w_0 - 1) eta mu of Eq. (19);
//   h_i      w_i rho_ref Cp_ref T' (i > 0), h0 ell fl' + (C' - (1 - w_0)
//            rho_ref Cp_ref) T': the equilibrium of Eq. (25) at rest at the
//            node's own previous state (T', fl', w', C' = rho Cp of
//            Eq. (10) there, ell = w' rho_l L); the h_i are referred to
//            the node they are streamed TO, whose new temperature the
//            writer holds in shared memory, the reader its own lag T;
//   f_i      3 (w_i - delta_i0) p' of the node they are streamed FROM
//            (the node itself for a population returned by a wall), the
//            pressure part of Eq. (14); the reader has that lagged
//            pressure for its stencil of Eq. (17).
//
// Stored as they are, a step's small change of h0 ~ rho H ~ 10, of h_i ~
// w_i T or of f_i ~ w_i p falls below half an ulp of float and is lost, so a
// slowly freezing or warming region drifts and the small velocity of the
// volume change is buried under the pressure.  Relative to the references
// only the small remainders are rounded; a change of reference enters as a
// difference of two references (exact in float when they are close).  The
// FP64 and tangent steps keep the populations as they are.
template <typename R>
constexpr bool kShift = std::is_same<R, float>::value;

// The references are formed with explicitly rounded operations
// (__fmul_rn, __fadd_rn, which the compiler never contracts into a fused
// multiply-add), so that every evaluation -- by the writer, by the next
// reader, in any kernel variant -- gives the same float.
template <typename R>
__device__ __forceinline__ R rest_ref_g(R w, R phi0) {
  return R(2) * w - R(1) + phi0;
}
__device__ __forceinline__ float rest_ref_g(float w, float phi0) {
  return __fadd_rn(__fadd_rn(__fmul_rn(2.f, w), -1.f), phi0);
}
// latent capacity ell = w rho_l L (Eq. (8) with reading R-T1)
template <typename R>
__device__ __forceinline__ R latent_cap(const Coef<R>& c, R w) {
  return w * c.rho_l * c.latent;
}
__device__ __forceinline__ float latent_cap(const Coef<float>& c, float w) {
  return __fmul_rn(__fmul_rn(w, c.rho_l), c.latent);
}
// Eq. (10), explicitly rounded
__device__ __forceinline__ float interp_rn(float fs, float w, float zs, float zl, float zg) {
  const float a = __fsub_rn(1.f, fs);
  return __fadd_rn(__fadd_rn(__fmul_rn(fs, zs), __fmul_rn(__fmul_rn(a, w), zl)),
                   __fmul_rn(__fmul_rn(a, __fsub_rn(1.f, w)), zg));
}
// solid fraction min(phi0 + w (1 - fl), 1) and heat capacity rho Cp of a
// state given by its weight and liquid fraction: fl = 1 gives the fully
// liquid capacity C+ (fs = phi0), fl = 0 the fully frozen C- (fs = min(phi0
// + w, 1)) of the inversion, bit for bit
__device__ __forceinline__ float fs_rn(float w, float fl, float phi0) {
  return fminf(__fadd_rn(phi0, __fmul_rn(w, __fsub_rn(1.f, fl))), 1.f);
}
__device__ __forceinline__ float cap_rn(const Coef<float>& c, float fs, float w) {
  return __fmul_rn(interp_rn(fs, w, c.rho_s, c.rho_l, c.rho_g),
                   interp_rn(fs, w, c.cp_s, c.cp_l, c.cp_g));
}
// reference of h0: ell fl + (C - (1 - w_0) rho_ref Cp_ref) T
__device__ __forceinline__ float ref_h0(const Coef<float>& c, float w, float fl, float T,
                                        float C) {
  return __fadd_rn(__fmul_rn(latent_cap(c, w), fl), __fmul_rn(__fsub_rn(C, c.rr_rest), T));
}
// reference of h_i, i > 0: w_i rho_ref Cp_ref T (wrr = c.wrr1 or c.wrr5)
__device__ __forceinline__ float ref_hi(float wrr, float T) { return __fmul_rn(wrr, T); }
// new reference - old reference
__device__ __forceinline__ float ref_delta(float r_new, float r_old) {
  return __fsub_rn(r_new, r_old);
}

// Error-free sum (Knuth's TwoSum): s + e == x + y exactly, s = fl(x + y).
__device__ __forceinline__ void two_sum(float x, float y, float& s, float& e) {
  s = __fadd_rn(x, y);
  const float bv = __fsub_rn(s, x);
  e = __fadd_rn(__fsub_rn(x, __fsub_rn(s, bv)), __fsub_rn(y, bv));
}

template <typename R>
__device__ __forceinline__ R sum_g(const R* v) {
  return (v[0] + v[1] + v[2] + v[3] + v[4] + v[5]) + (v[6] + v[7] + v[8]);
}
template <typename R>
__device__ __forceinline__ R sum_h(const R* v) {
  return (v[0] + v[1] + v[2]) + (v[3] + v[4] + v[5] + v[6] + v[7] + v[8]);
}

template <typename R>
struct Local {
  R T, fl, mdot, rhoH, phi, w, fs, rho;
  R rhoHr;  // rho H minus its reference (float storage), else rho H
  R phir;   // phi minus the reference of g0 (float storage), else phi
};

// Rows a1-a2 for one node from its population sums and lag fields (plain
// populations: FP64, tangent and the 3-D step).
template <typename R>
__device__ __forceinline__ Local<R> local_state(const Coef<R>& c, int lat, R sg, R sh, R flp,
                                                R wp, R Qp, R phi0) {
  Local<R> L;
  L.T = R(0);
  L.fl = flp;
  L.rhoH = R(0);
  L.mdot = R(0);
  if (lat & LAT_HEAT) {
    L.rhoH = sh + R(0.5) * Qp;  // Eq. (28), lagged source
    invert_enthalpy(c, L.rhoH, wp, phi0, L.T, L.fl);
    L.mdot = c.one_m_ratio * wp * (flp - L.fl);  // Eq. (1), phase-change part
  }
  L.rhoHr = L.rhoH;
  if (lat & LAT_PHASE) {
    // Eq. (22) solved for phi.  Without phase change the divisor is exactly
    // 1, and the FP64 step (bound by its FP64 pipe, where a division costs
    // about ten operations) skips it; a tangent still divides (the
    // derivative of mdot need not vanish).
    if constexpr (std::is_same<R, double>::value)
      L.phi = L.mdot == R(0) ? sg : qdiv(sg, R(1) - R(0.5) * L.mdot);
    else
      L.phi = qdiv(sg, R(1) - R(0.5) * L.mdot);
    L.w = clamp01((R(1) - phi0 + L.phi) * R(0.5));
  } else {
    L.w = wp;
    L.phi = R(2) * wp - R(1) + phi0;
  }
  L.phir = L.phi;
  R fs = phi0 + L.w * (R(1) - L.fl);
  L.fs = fs > R(1) ? R(1) : fs;
  L.rho = interp(L.fs, L.w, c.rho_s, c.rho_l, c.rho_g);
  return L;
}

// Rows a1-a2 of a well-balanced float state: sg, sh are sums of the stored
// remainders; Tp, flp, wp the node's lags, Cp its heat capacity at the lags
// (cap_rn(fs_rn(wp, flp, phi0), wp)), so that rho H = e + ell flp + Cp Tp
// with e = sh + Q/2 (Eq. (28)).
//
// Eq. (8) for such a state.  A node that was fully liquid (flp = 1) has
// rho H - ell = e + C+ Tp; if the new temperature Tp + e / C+ stays above
// the liquidus it is the answer, exact in float as an increment of Tp.
// Likewise a fully frozen node (flp = 0, rho H = e + C- Tp) below the
// solidus.  Every other node -- the ones near the melting point -- takes the
// branch test, the liquid fraction and its clamp to [0, 1] in FP64 and
// rounds once.
__device__ __forceinline__ Local<float> local_state_wb(const Coef<float>& c, int lat, float sg,
                                                       float sh, float flp, float wp, float Qp,
                                                       float Tp, float Cp, float phi0) {
  Local<float> L;
  L.T = 0.f;
  L.fl = flp;
  L.rhoH = 0.f;
  L.rhoHr = 0.f;
  L.mdot = 0.f;
  if (lat & LAT_HEAT) {
    const float e = sh + 0.5f * Qp;
    const float ell = latent_cap(c, wp);
    L.rhoHr = e;
    bool done = false;
    if (flp == 1.f) {  // Cp is C+ here
      const float T1 = Tp + qdiv(e, Cp);
      if (T1 > 0.f) {
        L.T = T1;
        L.fl = 1.f;
        done = true;
      }
    } else if (flp == 0.f) {  // Cp is C- here
      const float T1 = Tp + qdiv(e, Cp);
      if (T1 < 0.f) {
        L.T = T1;
        L.fl = 0.f;
        done = true;
      }
    }
    if (!done) {
      const double rH = (double)e + (double)ell * (double)flp + (double)Cp * (double)Tp;
      const double ld = (double)ell;
      if (rH < 0.0) {
        L.fl = 0.f;
        L.T = (float)(rH / (double)cap_rn(c, fs_rn(wp, 0.f, phi0), wp));
      } else if (rH > ld) {
        L.fl = 1.f;
        L.T = (float)((rH - ld) / (double)cap_rn(c, phi0, wp));
      } else {
        double f = ld > 0.0 ? rH / ld : 1.0;
        f = f < 0.0 ? 0.0 : (f > 1.0 ? 1.0 : f);
        L.fl = (float)f;
        L.T = 0.f;
      }
    }
    L.rhoH = e + (ell * flp + Cp * Tp);
    L.mdot = c.one_m_ratio * wp * (flp - L.fl);  // Eq. (1), phase-change part
  }
  if (lat & LAT_PHASE) {
    // Eq. (22) solved for phi, relative to r0 = 2 wp - 1 + phi0:
    // phi - r0 = (sum g' + mdot r0 / 2) / (1 - mdot / 2), and the weight
    // (1 - phi0 + phi) / 2 = wp + (phi - r0) / 2
    const float r0 = rest_ref_g(wp, phi0);
    L.phir = qdiv(sg + 0.5f * L.mdot * r0, 1.f - 0.5f * L.mdot);
    L.phi = r0 + L.phir;
    L.w = clamp01(wp + 0.5f * L.phir);
  } else {
    L.w = wp;
    L.phi = 2.f * wp - 1.f + phi0;
    L.phir = 0.f;
  }
  L.fs = fs_rn(L.w, L.fl, phi0);
  L.rho = interp(L.fs, L.w, c.rho_s, c.rho_l, c.rho_g);
  return L;
}

// Eq. (6) without the Laplacian terms.
template <typename R>
__device__ __forceinline__ R chem_local(const Coef<R>& c, R phi, R phi0, R fs) {
  const R s3 = c.s3, s9 = c.s9;
  return s3 * phi * (phi - R(1)) * (phi + R(1)) + s9 * phi0 * phi0 * phi +
         s3 * c.cos_th * phi0 * (R(3) * phi * phi + phi0 * phi0 - R(1)) + s9 * fs * fs * phi +
         s3 * c.cos_ps * fs * (R(3) * phi * phi + fs * fs - R(1));
}

__device__ __forceinline__ int wrap_or_clamp(int v, int n, int bc_lo, int bc_hi) {
  if (v < 0) return bc_lo == BC_PERIODIC ? ((v % n) + n) % n : 0;
  if (v >= n) return bc_hi == BC_PERIODIC ? v % n : n - 1;
  return v;
}

// Streaming target of direction (cx, cy) from (x, y): returns the node index
// in the destination plane, or -1 with `wall` set when the link leaves
// through a wall (the x wall decides at corners).
__device__ __forceinline__ long long stream_target(const Geom& g, int x, int y, int cx, int cy,
                                                   int& wall) {
  int tx = x + cx, ty = y + cy;
  wall = -1;
  if (tx < 0) {
    if (g.bc[0] == BC_PERIODIC) tx += g.nx; else wall = 0;
  } else if (tx >= g.nx) {
    if (g.bc[1] == BC_PERIODIC) tx -= g.nx; else wall = 1;
  }
  if (wall < 0) {
    if (ty < 0) {
      if (g.bc[2] == BC_PERIODIC) ty += g.ny; else wall = 2;
    } else if (ty >= g.ny) {
      if (g.bc[3] == BC_PERIODIC) ty -= g.ny; else wall = 3;
    }
  }
  return wall >= 0 ? -1 : (long long)ty * g.pitch + tx;
}

// Halo-ring position k (0 <= k < RING) in the (HX x HY) tile of height TYS.
template <int TYS = TY>
__device__ __forceinline__ void ring_pos(int k, int& hx, int& hy) {
  if (k < HX) {
    hx = k; hy = 0;
  } else if (k < 2 * HX) {
    hx = k - HX; hy = TYS + 1;
  } else {
    const int r = k - 2 * HX;  // 2 * TY side nodes
    hy = 1 + (r >> 1);
    hx = (r & 1) ? HX - 1 : 0;
  }
}

template <typename R>
__device__ __forceinline__ R warp_sum(R v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ Dual warp_sum(Dual v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += shfl_xor(v, o);
  return v;
}

// Per-tile partial sums of the diagnostics in a fixed order (warp shuffles,
// then the warps in order), written to partial[k * nb + b] for tile b of nb.
// Every thread of the CTA calls it; s_red is shared memory of the arithmetic
// type.  In float the warps' sums are added with Knuth's TwoSum (the
// rounding error of every addition is carried along and added back at the
// end), so one conversion to double per diagnostic keeps the accuracy of a
// double-precision sum without work on the slow FP64 pipe.  The grid-wide
// sum is lbm_diag_finalize_kernel.
// Reduce-scatter of eight per-lane values over a warp: each exchange
// halves the number of values a lane carries, so the eight warp sums take 9
// shuffles instead of 40.  On return lane l holds the warp sum of value
// (l >> 2) & 7.
template <typename R>
__device__ __forceinline__ R warp_sum8(const R* v, int lane) {
  const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4;
  R a[4];
#pragma unroll
  for (int j = 0; j < 4; j++) {
    const R keep = b4 ? v[4 + j] : v[j], send = b4 ? v[j] : v[4 + j];
    a[j] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
  }
  R h[2];
#pragma unroll
  for (int j = 0; j < 2; j++) {
    const R keep = b3 ? a[2 + j] : a[j], send = b3 ? a[j] : a[2 + j];
    h[j] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
  }
  R q;
  {
    const R keep = b2 ? h[1] : h[0], send = b2 ? h[0] : h[1];
    q = keep + __shfl_xor_sync(0xffffffffu, send, 4);
  }
  q += __shfl_xor_sync(0xffffffffu, q, 2);
  q += __shfl_xor_sync(0xffffffffu, q, 1);
  return q;
}

#ifndef LBM_DIAG_BUTTERFLY
#define LBM_DIAG_BUTTERFLY 1
#endif

// Stage 1 (every thread, no barrier): the warp's sums of the nine values
// into s_red[warp][k].
template <typename R>
__device__ __forceinline__ void block_diag_warps(const R* dvals, R (*s_red)[NDIAG], int tid) {
  const int lane = tid & 31, warp = tid >> 5;
  static_assert(NDIAG == 9, "the reduce-scatter covers diagnostics 0-7, the ninth is separate");
  if constexpr (LBM_DIAG_BUTTERFLY && sizeof(R) == 4) {
    const R v = warp_sum8(dvals, lane);
    if ((lane & 3) == 0) s_red[warp][(lane >> 2) & 7] = v;
    const R v8 = warp_sum(dvals[8]);
    if (lane == 0) s_red[warp][8] = v8;
  } else {
#pragma unroll
    for (int k = 0; k < NDIAG; k++) {
      const R v = warp_sum(dvals[k]);
      if (lane == 0) s_red[warp][k] = v;
    }
  }
}

// Stage 2 (every thread; one barrier): the warps' sums in order into
// partial[k * nb + b] for tile b of nb.
template <typename R, int NW = NT / 32>
__device__ __forceinline__ void block_diag_finish(const R (*s_red)[NDIAG],
                                                  double* __restrict__ partial, int tid, int b,
                                                  int nb) {
  __syncthreads();
  if (tid < NDIAG) {
    if constexpr (is_dual<R>::value) {
      // tangent step: values in the first NDIAG * nb partials, derivatives
      // in the next NDIAG * nb
      R acc = R(0);
#pragma unroll
      for (int w = 0; w < NW; w++) acc += s_red[w][tid];
      partial[(long long)tid * nb + b] = acc.v;
      partial[(long long)(NDIAG + tid) * nb + b] = acc.d;
    } else if constexpr (sizeof(R) == 8) {
      double acc = 0.0;
#pragma unroll
      for (int w = 0; w < NW; w++) acc += (double)s_red[w][tid];
      partial[(long long)tid * nb + b] = acc;
    } else {
      R sum = R(0), err = R(0);
#pragma unroll
      for (int w = 0; w < NW; w++) {
        const R y = s_red[w][tid];
        const R t = sum + y;
        const R yv = t - sum;          // the part of y that went into t
        err += (sum - (t - yv)) + (y - yv);
        sum = t;
      }
      partial[(long long)tid * nb + b] = (double)sum + (double)err;
    }
  }
}

// Per-tile partial sums of the diagnostics in a fixed order (warp sums, then
// the warps in order), written to partial[k * nb + b] for tile b of nb.
// Every thread of the CTA calls it; s_red is shared memory of the arithmetic
// type.  In float the warps' sums are added with Knuth's TwoSum (the
// rounding error of every addition is carried along and added back at the
// end), so one conversion to double per diagnostic keeps the accuracy of a
// double-precision sum without work on the slow FP64 pipe.  The grid-wide
// sum is lbm_diag_finalize_kernel.
template <typename R>
__device__ __forceinline__ void block_diag(const R* dvals, R (*s_red)[NDIAG],
                                           double* __restrict__ partial, int tid, int b, int nb) {
  block_diag_warps(dvals, s_red, tid);
  block_diag_finish(s_red, partial, tid, b, nb);
}

// Single-grid launch: the tile is the CTA.
template <typename R>
__device__ __forceinline__ void block_diag(const R* dvals, R (*s_red)[NDIAG],
                                           double* __restrict__ partial, int tid) {
  block_diag(dvals, s_red, partial, tid, blockIdx.y * gridDim.x + blockIdx.x,
             gridDim.x * gridDim.y);
}

// Grid-wide FP64 diagnostics from the per-CTA partials, one CTA, fixed order
// (bitwise reproducible): out[0..NDIAG-1] = sums, out[NDIAG] = step index.
static __global__ void __launch_bounds__(NT) lbm_diag_finalize_kernel(const double* __restrict__ partial,
                                                               int nb, double* __restrict__ out,
                                                               long long step) {
  __shared__ double s_red[NT / 32][NDIAG];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  double acc[NDIAG];
#pragma unroll
  for (int k = 0; k < NDIAG; k++) acc[k] = 0.0;
  for (int j = tid; j < nb; j += NT) {
#pragma unroll
    for (int k = 0; k < NDIAG; k++) acc[k] += partial[(long long)k * nb + j];
  }
#pragma unroll
  for (int k = 0; k < NDIAG; k++) {
    double v = acc[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) s_red[warp][k] = v;
  }
  __syncthreads();
  if (tid < NDIAG) {
    double t = 0.0;
#pragma unroll
    for (int w = 0; w < NT / 32; w++) t += s_red[w][tid];
    out[tid] = t;
  }
  if (tid == 0) out[NDIAG] = (double)step;
}

// ---------------------------------------------------------------------------
// initial state
// ---------------------------------------------------------------------------

template <typename R, typename S = R>
__global__ void __launch_bounds__(NT) lbm_init_kernel(const InitArgs<R, S> a) {
  const Geom& g = a.g;
  const Coef<R>& c = a.c;
  const long long P = g.plane;
  __shared__ R s_phi[HN], s_fs[HN], s_phi0[HN];

  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
  for (int k = tid; k < HN; k += NT) {
    const int hx = k % HX, hy = k / HX;
    const int rx = wrap_or_clamp(x0 + hx - 1, g.nx, g.bc[0], g.bc[1]);
    const int ry = wrap_or_clamp(y0 + hy - 1, g.ny, g.bc[2], g.bc[3]);
    const long long d = (long long)ry * g.nx + rx;
    const R q0 = (R)a.phi0[d];
    const R ph = (R)a.phi[d];
    const R w = clamp01((R(1) - q0 + ph) * R(0.5));
    const R fl = clamp01((R)a.fl[d]);
    R fs = q0 + w * (R(1) - fl);
    s_phi[k] = ph;
    s_fs[k] = fs > R(1) ? R(1) : fs;
    s_phi0[k] = q0;
  }
  __syncthreads();
  const int gx = x0 + tx, gy = y0 + ty;
  if (gx >= g.nx || gy >= g.ny) return;
  const long long d = (long long)gy * g.nx + gx;
  const long long n = (long long)gy * g.pitch + gx;
  const int hc = (ty + 1) * HX + (tx + 1);
  const R phi = s_phi[hc], fs = s_fs[hc], q0 = s_phi0[hc];
  const R w = clamp01((R(1) - q0 + phi) * R(0.5));
  const R fl = clamp01((R)a.fl[d]);
  const R T = (R)a.T[d];
  R lphi = R(0), lphi0 = R(0), lfs = R(0);
#pragma unroll
  for (int i = 1; i < 9; i++) {
    const int hn = hc + qy(i) * HX + qx(i);
    lphi += R(2) * qw<R>(i) * (s_phi[hn] - phi);
    lphi0 += R(2) * qw<R>(i) * (s_phi0[hn] - q0);
    lfs += R(2) * qw<R>(i) * (s_fs[hn] - fs);
  }
  lphi *= R(3); lphi0 *= R(3); lfs *= R(3);
  const R muphi = chem_local(c, phi, q0, fs) -
                  c.klap * (lphi + c.cos_th * lphi0 + c.cos_ps * lfs);
  const R ell = w * c.rho_l * c.latent;
  R fsf = q0 + w;
  fsf = fsf > R(1) ? R(1) : fsf;
  const R capT = T < R(0) ? heat_cap(c, fsf, w) : heat_cap(c, q0, w);
  const R rhoH = capT * T + ell * fl;
  const R C = heat_cap(c, fs, w);
  const R rrC = qdiv(c.rr, C);
  const R emu = c.eta * muphi;
  // float states: the remainders of the well-balanced storage (kShift),
  // referred to this node's own state (streaming has not happened yet)
  R sg0 = R(0), sh0 = R(0), sha = R(0), shd = R(0);
  if constexpr (kShift<R>) {
    sg0 = rest_ref_g(w, q0);
    sh0 = ref_h0(c, w, fl, T, cap_rn(c, fs_rn(w, fl, q0), w));
    sha = ref_hi(c.wrr1, T);
    shd = ref_hi(c.wrr5, T);
  }
#pragma unroll
  for (int i = 0; i < 9; i++) {
    stp(a.pout + i * P + n, R(0));
    stp(a.pout + (9 + i) * P + n,
        (i == 0) ? phi + (qw<R>(0) - R(1)) * emu - sg0 : qw<R>(i) * emu);
    stp(a.pout + (18 + i) * P + n,
        heq_i<R>(i, rhoH, C, T, c.rr, rrC, R(0), R(0), R(0)) -
            (i == 0 ? sh0 : (i <= 4 ? sha : shd)));
  }
  a.lout[LAG_FL * P + n] = fl;
  a.lout[LAG_W * P + n] = w;
  a.lout[LAG_P * P + n] = R(0);
  a.lout[LAG_PHUX * P + n] = R(0);
  a.lout[LAG_PHUY * P + n] = R(0);
  a.lout[LAG_Q * P + n] = R(0);
  if constexpr (kShift<R>) a.lout[LAG_T * P + n] = T;
  a.phi0_out[n] = q0;
  if (a.mask_out) a.mask_out[n] = a.mask ? (a.mask[d] != 0) : 0;
}

}  // namespace lbmk
