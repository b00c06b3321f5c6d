// lbm3d.cu -- the three-dimensional form of the coupled step on the D3Q19
// lattice (Sec. 3.1, Eq. (13)) for sm_103a, and its C ABI (lbm3_* in
// include/lbm.h).
//
// The model is the two-dimensional one with every lattice sum taken over the
// 19 velocities and every vector carrying a z component (flow Eqs. (11),
// (14)-(17); phase field Eqs. (18)-(22); enthalpy Eqs. (23)-(28); the
// isotropic stencils built on the D3Q19 weights).  The lattice-independent
// local physics (the inversion of Eq. (8), the mass source, the order
// parameter, Eq. (10), the local part of Eq. (6)) is shared with the 2-D
// step through lbm_kernels.cuh.
//
// A step is two kernels over the whole grid:
//   lbm3_local_kernel    per node: the sums of the phase and enthalpy
//                        populations, the inversion, mdot, phi, w, fs and
//                        rho, stored as eight planes (phi, fs, rho for the
//                        neighbours' stencils; T, fl, mdot, rho H, w for the
//                        node itself);
//   lbm3_collide_kernel  per node: the 18-neighbour stencils of phi, phi0,
//                        fs, rho and the lagged pressure (neighbour planes
//                        are read through L1/L2; a 32 x 4 x 2 block keeps
//                        its halo in L1), mu_phi, forces, velocity and
//                        pressure, the three collisions one lattice at a
//                        time, push streaming with the wall rules, lag store.
// The 2-D step fuses both halves with a recomputed halo ring; in 3-D the
// ring of a 256-node tile is 2.2 times the tile, so the split form moves
// fewer bytes: the eight local planes (32 B per node in FP32) instead of the
// ring's population sums.
//
// Layout: structure-of-arrays planes of pitch * ny * nz elements (pitch =
// nx rounded up to 32, planes to 64 elements); node (x, y, z) at
// (z * ny + y) * pitch + x.  Populations f (planes 0-18), g (19-37), h
// (38-56) in two buffers (push streaming from one into the other); lag
// fields fl, w, p, phi u (3), Q in two buffers (the collide kernel reads its
// neighbours' lagged pressure while it writes its own).
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>

#include "lbm_host.h"
#include "lbm_kernels.cuh"

namespace lbm3 {

using lbmk::Coef;
using lbmk::LAT_FLOW;
using lbmk::LAT_HEAT;
using lbmk::LAT_PHASE;
using lbmk::BC_DIRICHLET;
using lbmk::BC_PERIODIC;

constexpr int Q = 19;
// thread block (x fastest) and the resident blocks per SM the FP32 collide
// kernel is compiled for
#ifndef LBM3_BY
#define LBM3_BY 4
#endif
#ifndef LBM3_BZ
#define LBM3_BZ 2
#endif
#ifndef LBM3_MINB_F32
#define LBM3_MINB_F32 3
#endif
constexpr int BX = 32, BY = LBM3_BY, BZ = LBM3_BZ, NT = BX * BY * BZ;
enum { L_FL = 0, L_W, L_P, L_PHUX, L_PHUY, L_PHUZ, L_Q, NLAG };
enum { S_PHI = 0, S_FS, S_RHO, S_T, S_FL, S_MDOT, S_RHOH, S_W, NLOC };
constexpr int NFIELD3 = 13;  // phi fs fl T rhoH p ux uy uz rho mu w mdot
constexpr int NDIAG3 = 9;

// D3Q19 of Eq. (13): rest; the six axes; the twelve edge diagonals, in the
// column order of the printed velocity matrix.
__host__ __device__ constexpr int cx(int i) {
  return (i == 1 || i == 7 || i == 9 || i == 11 || i == 13)    ? 1
         : (i == 2 || i == 8 || i == 10 || i == 12 || i == 14) ? -1
                                                               : 0;
}
__host__ __device__ constexpr int cy(int i) {
  return (i == 3 || i == 7 || i == 10 || i == 15 || i == 17)   ? 1
         : (i == 4 || i == 8 || i == 9 || i == 16 || i == 18) ? -1
                                                               : 0;
}
__host__ __device__ constexpr int cz(int i) {
  return (i == 5 || i == 11 || i == 14 || i == 15 || i == 18)   ? 1
         : (i == 6 || i == 12 || i == 13 || i == 16 || i == 17) ? -1
                                                                : 0;
}
// opposite directions come in (odd, even) pairs: (1,2), (3,4), ..., (17,18)
__host__ __device__ constexpr int opp(int i) { return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1); }
template <typename R>
__device__ __forceinline__ R wq(int i) {
  return i == 0 ? R(1.0 / 3.0) : (i <= 6 ? R(1.0 / 18.0) : R(1.0 / 36.0));
}

struct Geom3 {
  int nx, ny, nz, pitch;
  long long plane;  // elements per plane (node offsets within a plane fit 31 bits)
  int bc[6];
  int lattices;
  int has_mask;
};

template <typename R>
struct Args3 {
  Geom3 g;
  Coef<R> c;
  R gz;
  R T_wall[6];  // x-low, x-high, y-low, y-high, z-low, z-high
  const R* __restrict__ pin;
  R* __restrict__ pout;
  const R* __restrict__ lin;
  R* __restrict__ lout;
  const R* __restrict__ phi0;
  const unsigned char* __restrict__ mask;
  R* __restrict__ loc;     // NLOC planes
  double* __restrict__ fld;  // read mode: NFIELD3 dense [nz][ny][nx] planes
};

__device__ __forceinline__ int wrap_or_clamp(int v, int n, int lo, int hi) {
  if (v < 0) return lo == BC_PERIODIC ? v + n : 0;
  if (v >= n) return hi == BC_PERIODIC ? v - n : n - 1;
  return v;
}

__device__ __forceinline__ int node(const Geom3& g, int x, int y, int z) {
  return (z * g.ny + y) * g.pitch + x;
}

// Streaming target of direction i from (x, y, z), or -1 with `wall` set to
// the face it leaves through (the first wall crossed in the order x, y, z).
__device__ __forceinline__ int stream_target(const Geom3& g, int x, int y, int z, int i,
                                             int& wall) {
  const int p[3] = {x + cx(i), y + cy(i), z + cz(i)};
  const int n[3] = {g.nx, g.ny, g.nz};
  int t[3];
  wall = -1;
#pragma unroll
  for (int a = 0; a < 3; a++) {
    t[a] = p[a];
    if (wall >= 0) continue;
    if (p[a] < 0) {
      if (g.bc[2 * a] == BC_PERIODIC) t[a] = p[a] + n[a]; else wall = 2 * a;
    } else if (p[a] >= n[a]) {
      if (g.bc[2 * a + 1] == BC_PERIODIC) t[a] = p[a] - n[a]; else wall = 2 * a + 1;
    }
  }
  return wall >= 0 ? -1 : node(g, t[0], t[1], t[2]);
}

// Store of one post-collision population of direction i from node n; for
// the enthalpy lattice (HEAT) a link leaving through a Dirichlet wall
// returns by anti-bounce-back, through an adiabatic wall by bounce-back.
template <typename R, bool HEAT, typename I>
__device__ __forceinline__ void push(const Args3<R>& a, R* __restrict__ plane0, I P, int i,
                                     int x, int y, int z, int n, bool inner, R v) {
  const Geom3& g = a.g;
  if (inner) {
    plane0[i * P + n + (cz(i) * g.ny + cy(i)) * g.pitch + cx(i)] = v;
  } else {
    int wall;
    const int t = stream_target(g, x, y, z, i, wall);
    if (t >= 0) {
      plane0[i * P + t] = v;
    } else {
      if (HEAT && g.bc[wall] == BC_DIRICHLET) v = -v + R(2) * wq<R>(i) * a.c.rr * a.T_wall[wall];
      plane0[opp(i) * P + n] = v;
    }
  }
}


// Enthalpy populations of a cold-mask node: the equilibrium of Eq. (25) at
// T_cold with u = 0, at the node's weight w and phi0 (applied when the
// populations are read).
template <typename R>
__device__ __forceinline__ void cold_mask_h19(const Coef<R>& c, R w, R phi0, R* h) {
  const R T = c.T_cold;
  const R flc = T < R(0) ? R(0) : R(1);
  R fsf = phi0 + w;
  fsf = fsf > R(1) ? R(1) : fsf;
  const R cap = T < R(0) ? lbmk::heat_cap(c, fsf, w) : lbmk::heat_cap(c, phi0, w);
  const R rhoH = cap * T + w * c.rho_l * c.latent * flc;
  const R rrT = c.rr * T;
  h[0] = rhoH - rrT + wq<R>(0) * rrT;
#pragma unroll
  for (int i = 1; i < Q; i++) h[i] = wq<R>(i) * rrT;
}

template <typename R>
__device__ __forceinline__ R sum19(const R* v) {
  R s = v[0];
#pragma unroll
  for (int i = 1; i < Q; i++) s += v[i];
  return s;
}

// ---------------------------------------------------------------------------
// kernel 1: local state of every node
// ---------------------------------------------------------------------------

// I: the type of plane offsets (int while 57 population planes fit 31
// bits, which keeps the index arithmetic in 32-bit registers; long long for
// larger grids)
template <typename R, typename I>
__global__ void __launch_bounds__(NT) lbm3_local_kernel(const Args3<R> a) {
  const Geom3& g = a.g;
  const Coef<R>& c = a.c;
  const int x = blockIdx.x * BX + threadIdx.x;
  const int y = blockIdx.y * BY + threadIdx.y;
  const int z = blockIdx.z * BZ + threadIdx.z;
  if (x >= g.nx || y >= g.ny || z >= g.nz) return;
  const I P = (I)g.plane;
  const int n = node(g, x, y, z);
  const int lat = g.lattices;
  const R phi0 = a.phi0[n];
  const R flp = a.lin[L_FL * P + n], wp = a.lin[L_W * P + n], Qp = a.lin[L_Q * P + n];
  R sg = R(0), sh = R(0);
  if (lat & LAT_PHASE) {
    R v[Q];
#pragma unroll
    for (int i = 0; i < Q; i++) v[i] = a.pin[(Q + i) * P + n];
    sg = sum19(v);
  }
  if (lat & LAT_HEAT) {
    R v[Q];
    if (g.has_mask && a.mask[n]) {
      cold_mask_h19(c, wp, phi0, v);
    } else {
#pragma unroll
      for (int i = 0; i < Q; i++) v[i] = a.pin[(2 * Q + i) * P + n];
    }
    sh = sum19(v);
  }
  const lbmk::Local<R> L = lbmk::local_state(c, lat, sg, sh, flp, wp, Qp, phi0);
  R* loc = a.loc + n;
  loc[S_PHI * P] = L.phi;
  loc[S_FS * P] = L.fs;
  loc[S_RHO * P] = L.rho;
  loc[S_T * P] = L.T;
  loc[S_FL * P] = L.fl;
  loc[S_MDOT * P] = L.mdot;
  loc[S_RHOH * P] = L.rhoH;
  loc[S_W * P] = L.w;
}

// ---------------------------------------------------------------------------
// kernel 2: stencils, macroscopic fields, collisions, streaming
// ---------------------------------------------------------------------------

template <typename R>
struct Macro3 {
  R u[3], uu, pr, S, Ft[3], uFt, G[3], tauf, muphi, phu[3], cap;
};

// Flow collision Eqs. (11), (14)-(16) over the opposite pairs (i, i + 1):
// the terms even in c_i are shared by the pair, the odd ones change sign.
template <typename R, typename I>
__device__ __forceinline__ void collide_flow(const Args3<R>& a, R* out, I P, int x, int y,
                                             int z, int n, bool inner, const R* f, R rho,
                                             const Macro3<R>& M) {
  const R itau = lbmk::qdiv(R(1), M.tauf);
  const R omi = R(1) - itau;
  const R fcoef = R(1) - R(0.5) * itau;
  const bool iso = (a.c.readings & 1u) != 0;
  const R sym0 = rho * (-R(1.5) * M.uu);
  const R fsym0 = M.S - R(3) * M.uFt;
  {
    R F0 = fsym0;
    if (iso) F0 += M.S * (R(0) - R(1)) * R(1.5);
    const R feq0 = M.pr * R(3) * (wq<R>(0) - R(1)) + rho * wq<R>(0) * (-R(1.5) * M.uu);
    push<R, false, I>(a, out, P, 0, x, y, z, n, inner, f[0] * omi + itau * feq0 + fcoef * wq<R>(0) * F0);
  }
#pragma unroll
  for (int i = 1; i < Q; i += 2) {
    const int o = i + 1;
    const R wi = wq<R>(i);
    const R cu = R(cx(i)) * M.u[0] + R(cy(i)) * M.u[1] + R(cz(i)) * M.u[2];
    const R cG = R(cx(i)) * M.G[0] + R(cy(i)) * M.G[1] + R(cz(i)) * M.G[2];
    const R cFt = R(cx(i)) * M.Ft[0] + R(cy(i)) * M.Ft[1] + R(cz(i)) * M.Ft[2];
    const R eqS = M.pr * R(3) + rho * (R(4.5) * cu * cu) + sym0;
    const R eqA = rho * (R(3) * cu);
    R srcS = fsym0 + R(9) * cu * cFt;
    if (iso) srcS += M.S * (R(cx(i) * cx(i) + cy(i) * cy(i) + cz(i) * cz(i)) - R(1)) * R(1.5);
    const R srcA = R(3) * cG;
    const R Ps = wi * (itau * eqS + fcoef * srcS);
    const R Pa = wi * (itau * eqA + fcoef * srcA);
    push<R, false, I>(a, out, P, i, x, y, z, n, inner, f[i] * omi + Ps + Pa);
    push<R, false, I>(a, out, P, o, x, y, z, n, inner, f[o] * omi + Ps - Pa);
  }
}

// Phase-field collision Eqs. (18)-(20).
template <typename R, typename I>
__device__ __forceinline__ void collide_phase(const Args3<R>& a, R* out, I P, int x, int y,
                                              int z, int n, bool inner, const R* gq, R phi,
                                              R mdot, const R* phup, const Macro3<R>& M) {
  const Coef<R>& c = a.c;
  const R itg = c.inv_tau_g;
  const R omg = R(1) - itg;
  const R gcoef = R(1) - R(0.5) * itg;
  const R emu = c.eta * M.muphi;
  const R Zs = itg * emu + gcoef * phi * mdot;
  R V[3];
#pragma unroll
  for (int k = 0; k < 3; k++) V[k] = R(3) * (itg * M.phu[k] + gcoef * (M.phu[k] - phup[k]));
  {
    const R geq0 = phi + (wq<R>(0) - R(1)) * emu;
    push<R, false, I>(a, out, P, 0, x, y, z, n, inner,
                   gq[0] * omg + itg * geq0 + gcoef * wq<R>(0) * phi * mdot);
  }
#pragma unroll
  for (int i = 1; i < Q; i += 2) {
    const int o = i + 1;
    const R wi = wq<R>(i);
    const R Ps = wi * Zs;
    const R Pa = wi * (R(cx(i)) * V[0] + R(cy(i)) * V[1] + R(cz(i)) * V[2]);
    push<R, false, I>(a, out, P, i, x, y, z, n, inner, gq[i] * omg + Ps + Pa);
    push<R, false, I>(a, out, P, o, x, y, z, n, inner, gq[o] * omg + Ps - Pa);
  }
}

// Enthalpy TRT collision Eqs. (23)-(27) with the magic relation.
template <typename R, typename I>
__device__ __forceinline__ void collide_heat(const Args3<R>& a, R* out, I P, int x, int y,
                                             int z, int n, bool inner, const R* h, R fs, R w,
                                             R T, R rhoH, R mdot, const Macro3<R>& M) {
  const Coef<R>& c = a.c;
  const R lam = lbmk::interp(fs, w, c.lam_s, c.lam_l, c.lam_g);
  const R taua = R(0.5) + lam * c.inv_rr3;
  const R ia = lbmk::qdiv(R(1), taua), is = R(2) - ia;
  const R hcoef = R(1) - R(0.5) * ia;
  const R CT = M.cap * T;
  const R Hsrc = hcoef * CT * mdot;
  const R rrT = c.rr * T;
  {
    const R heq0 = rhoH - rrT + wq<R>(0) * (rrT - CT * M.uu * R(1.5));
    push<R, true, I>(a, out, P, 0, x, y, z, n, inner, h[0] - (h[0] - heq0) * is + wq<R>(0) * Hsrc);
  }
#pragma unroll
  for (int i = 1; i < Q; i += 2) {
    const int o = i + 1;
    const R wi = wq<R>(i);
    const R cu = R(cx(i)) * M.u[0] + R(cy(i)) * M.u[1] + R(cz(i)) * M.u[2];
    const R es = wi * (rrT + CT * (R(4.5) * cu * cu - R(1.5) * M.uu));
    const R ea = wi * (CT * (R(3) * cu));
    const R hs = R(0.5) * (h[i] + h[o]), ha = R(0.5) * (h[i] - h[o]);
    const R Da = (ha - ea) * ia;
    const R Ds = (hs - es) * is - wi * Hsrc;
    push<R, true, I>(a, out, P, i, x, y, z, n, inner, h[i] - Da - Ds);
    push<R, true, I>(a, out, P, o, x, y, z, n, inner, h[o] + Da - Ds);
  }
}

template <typename R, bool READ, typename I>
__global__ void __launch_bounds__(NT, (sizeof(R) == 4 ? LBM3_MINB_F32 : (sizeof(R) == 8 ? 2 : 1)))
    lbm3_collide_kernel(const Args3<R> a) {
  const Geom3& g = a.g;
  const Coef<R>& c = a.c;
  const int x = blockIdx.x * BX + threadIdx.x;
  const int y = blockIdx.y * BY + threadIdx.y;
  const int z = blockIdx.z * BZ + threadIdx.z;
  if (x >= g.nx || y >= g.ny || z >= g.nz) return;
  const I P = (I)g.plane;
  const int n = node(g, x, y, z);
  const int lat = g.lattices;
  const R* loc = a.loc;
  const R phi = loc[S_PHI * P + n], fs = loc[S_FS * P + n], rho = loc[S_RHO * P + n];
  const R T = loc[S_T * P + n], fl = loc[S_FL * P + n], mdot = loc[S_MDOT * P + n];
  const R rhoH = loc[S_RHOH * P + n], w = loc[S_W * P + n];
  const R phi0 = a.phi0[n];

  // isotropic stencils (reading R-FD) over the 18 neighbours; wall axes
  // mirror the boundary node (zero normal gradient)
  R gph[3] = {R(0), R(0), R(0)}, gr[3] = {R(0), R(0), R(0)}, gp[3] = {R(0), R(0), R(0)};
  R lphi = R(0), lphi0 = R(0), lfs = R(0);
#pragma unroll
  for (int i = 1; i < Q; i++) {
    const int xx = wrap_or_clamp(x + cx(i), g.nx, g.bc[0], g.bc[1]);
    const int yy = wrap_or_clamp(y + cy(i), g.ny, g.bc[2], g.bc[3]);
    const int zz = wrap_or_clamp(z + cz(i), g.nz, g.bc[4], g.bc[5]);
    const int m = node(g, xx, yy, zz);
    const R wi = wq<R>(i);
    const R vphi = loc[S_PHI * P + m];
    if (lat & LAT_PHASE) {
      const R vphi0 = a.phi0[m], vfs = loc[S_FS * P + m];
      gph[0] += wi * R(cx(i)) * vphi;
      gph[1] += wi * R(cy(i)) * vphi;
      gph[2] += wi * R(cz(i)) * vphi;
      lphi += R(2) * wi * (vphi - phi);
      lphi0 += R(2) * wi * (vphi0 - phi0);
      lfs += R(2) * wi * (vfs - fs);
    }
    if (lat & LAT_FLOW) {
      const R vrho = loc[S_RHO * P + m], vp = a.lin[L_P * P + m];
      gr[0] += wi * R(cx(i)) * vrho;
      gr[1] += wi * R(cy(i)) * vrho;
      gr[2] += wi * R(cz(i)) * vrho;
      gp[0] += wi * R(cx(i)) * vp;
      gp[1] += wi * R(cy(i)) * vp;
      gp[2] += wi * R(cz(i)) * vp;
    }
  }
#pragma unroll
  for (int k = 0; k < 3; k++) {
    gph[k] *= R(3);
    gr[k] *= R(3);
    gp[k] *= R(3);
  }
  lphi *= R(3); lphi0 *= R(3); lfs *= R(3);

  Macro3<R> M;
  M.muphi = R(0);
  R F[3];
  {
    R Fs[3] = {R(0), R(0), R(0)};
    if (lat & LAT_PHASE) {
      M.muphi = lbmk::chem_local(c, phi, phi0, fs) -
                c.klap * (lphi + c.cos_th * lphi0 + c.cos_ps * lfs);
#pragma unroll
      for (int k = 0; k < 3; k++) Fs[k] = M.muphi * gph[k];
    }
    F[0] = Fs[0] + rho * c.gx;
    F[1] = Fs[1] + rho * c.gy;
    F[2] = Fs[2] + rho * a.gz;
  }
  M.u[0] = M.u[1] = M.u[2] = R(0);
  M.uu = R(0);
  M.pr = R(0);
  R f[Q];
  if (lat & LAT_FLOW) {
#pragma unroll
    for (int i = 0; i < Q; i++) f[i] = a.pin[i * P + n];
    R j[3] = {R(0), R(0), R(0)}, snz = R(0);
#pragma unroll
    for (int i = 0; i < Q; i++) {
      j[0] += R(cx(i)) * f[i];
      j[1] += R(cy(i)) * f[i];
      j[2] += R(cz(i)) * f[i];
      if (i > 0) snz += f[i];
    }
    const R mu = lbmk::interp(fs, w, c.mu_s, c.mu_l, c.mu_g);
    const R irho = lbmk::qdiv(R(1), rho);
    // Eq. (17a,b) with the penalty force f = fs (u_s - u*), u_s = 0
    R fp[3];
#pragma unroll
    for (int k = 0; k < 3; k++) {
      const R us = (j[k] + R(0.5) * F[k]) * irho;
      fp[k] = -fs * us;
      M.u[k] = us + R(0.5) * fp[k];
    }
    M.uu = M.u[0] * M.u[0] + M.u[1] * M.u[1] + M.u[2] * M.u[2];
    M.S = rho * mdot + M.u[0] * gr[0] + M.u[1] * gr[1] + M.u[2] * gr[2];
    // modified force (reading R-FT) with the lagged pressure (reading R-FP)
#pragma unroll
    for (int k = 0; k < 3; k++) {
      M.Ft[k] = F[k] - (gp[k] - gr[k] * R(1.0 / 3.0));
      M.G[k] = F[k] + rho * fp[k];
    }
    M.uFt = M.u[0] * M.Ft[0] + M.u[1] * M.Ft[1] + M.u[2] * M.Ft[2];
    M.tauf = R(3) * mu * irho + R(0.5);
    // F_0 of Eq. (16) and Eq. (17c)
    R F0 = wq<R>(0) * (M.S + (R(0) - R(2) / R(3) * M.uFt) * R(4.5));
    if (c.readings & 1u) F0 += wq<R>(0) * (M.S * (R(0) - R(1)) * R(1.5));
    const R s0 = wq<R>(0) * (-M.uu * R(1.5));
    M.pr = (R(1) / R(3)) / (R(1) - wq<R>(0)) *
           (snz + R(0.5) * M.S + (M.tauf - R(0.5)) * F0 + rho * s0);
  }
#pragma unroll
  for (int k = 0; k < 3; k++) M.phu[k] = phi * M.u[k];
  M.cap = rho * lbmk::interp(fs, w, c.cp_s, c.cp_l, c.cp_g);

  if (READ) {
    const long long N = (long long)g.nx * g.ny * g.nz;
    const long long d = ((long long)z * g.ny + y) * g.nx + x;
    const R vals[NFIELD3] = {phi, fs, fl, T, rhoH, M.pr, M.u[0], M.u[1], M.u[2],
                             rho, M.muphi, w, mdot};
#pragma unroll
    for (int k = 0; k < NFIELD3; k++) lbmk::put_out(a.fld + k * N, d, NFIELD3 * N, vals[k]);
    return;
  }

  const bool inner = x > 0 && x < g.nx - 1 && y > 0 && y < g.ny - 1 && z > 0 && z < g.nz - 1;
  R* out = a.pout;
  if (lat & LAT_FLOW) collide_flow(a, out, P, x, y, z, n, inner, f, rho, M);
  if (lat & LAT_PHASE) {
    R gq[Q];
#pragma unroll
    for (int i = 0; i < Q; i++) gq[i] = a.pin[(Q + i) * P + n];
    const R phup[3] = {a.lin[L_PHUX * P + n], a.lin[L_PHUY * P + n], a.lin[L_PHUZ * P + n]};
    collide_phase(a, out + Q * P, P, x, y, z, n, inner, gq, phi, mdot, phup, M);
  }
  if (lat & LAT_HEAT) {
    R hq[Q];
    if (g.has_mask && a.mask[n]) {
      cold_mask_h19(c, a.lin[L_W * P + n], phi0, hq);
    } else {
#pragma unroll
      for (int i = 0; i < Q; i++) hq[i] = a.pin[(2 * Q + i) * P + n];
    }
    collide_heat(a, out + 2 * Q * P, P, x, y, z, n, inner, hq, fs, w, T, rhoH, mdot, M);
  }
  a.lout[L_FL * P + n] = fl;
  a.lout[L_W * P + n] = w;
  a.lout[L_P * P + n] = (lat & LAT_FLOW) ? M.pr : R(0);
  a.lout[L_PHUX * P + n] = (lat & LAT_PHASE) ? M.phu[0] : R(0);
  a.lout[L_PHUY * P + n] = (lat & LAT_PHASE) ? M.phu[1] : R(0);
  a.lout[L_PHUZ * P + n] = (lat & LAT_PHASE) ? M.phu[2] : R(0);
  a.lout[L_Q * P + n] = (lat & LAT_HEAT) ? M.cap * T * mdot : R(0);
}

// ---------------------------------------------------------------------------
// initial state and diagnostics
// ---------------------------------------------------------------------------

// Per node from the dense inputs: phi, w, fl, fs, rho, T into the local
// planes, phi0 and the mask, and the initial lags (fl, w; p = phi u = Q = 0).
template <typename R>
__global__ void __launch_bounds__(NT) lbm3_init_local_kernel(
    const Args3<R> a, const double* __restrict__ phi0d, const unsigned char* __restrict__ maskd,
    const double* __restrict__ phid, const double* __restrict__ Td,
    const double* __restrict__ fld0, R* __restrict__ phi0_out, unsigned char* __restrict__ mask_out) {
  const Geom3& g = a.g;
  const Coef<R>& c = a.c;
  const int x = blockIdx.x * BX + threadIdx.x;
  const int y = blockIdx.y * BY + threadIdx.y;
  const int z = blockIdx.z * BZ + threadIdx.z;
  if (x >= g.nx || y >= g.ny || z >= g.nz) return;
  const long long P = g.plane;
  const int n = node(g, x, y, z);
  const long long d = ((long long)z * g.ny + y) * g.nx + x;
  const R q0 = (R)phi0d[d], ph = (R)phid[d];
  const R w = lbmk::clamp01((R(1) - q0 + ph) * R(0.5));
  const R fl = lbmk::clamp01((R)fld0[d]);
  R fs = q0 + w * (R(1) - fl);
  fs = fs > R(1) ? R(1) : fs;
  R* loc = a.loc + n;
  loc[S_PHI * P] = ph;
  loc[S_FS * P] = fs;
  loc[S_RHO * P] = lbmk::interp(fs, w, c.rho_s, c.rho_l, c.rho_g);
  loc[S_T * P] = (R)Td[d];
  loc[S_FL * P] = fl;
  loc[S_MDOT * P] = R(0);
  loc[S_RHOH * P] = R(0);
  loc[S_W * P] = w;
  phi0_out[n] = q0;
  mask_out[n] = maskd ? (maskd[d] != 0) : 0;
  R* lag = a.lout + n;
  lag[L_FL * P] = fl;
  lag[L_W * P] = w;
  lag[L_P * P] = R(0);
  lag[L_PHUX * P] = R(0);
  lag[L_PHUY * P] = R(0);
  lag[L_PHUZ * P] = R(0);
  lag[L_Q * P] = R(0);
}

// Initial populations: f at rest (p = 0, u = 0: all zero), g = g_eq(phi,
// mu_phi, u = 0) of Eq. (19) with mu_phi from the stencils of the initial
// fields, h = h_eq(rho H, T, u = 0) of Eq. (25) (cold-mask nodes: the mask
// equilibrium).
template <typename R>
__global__ void __launch_bounds__(NT) lbm3_init_pops_kernel(const Args3<R> a) {
  const Geom3& g = a.g;
  const Coef<R>& c = a.c;
  const int x = blockIdx.x * BX + threadIdx.x;
  const int y = blockIdx.y * BY + threadIdx.y;
  const int z = blockIdx.z * BZ + threadIdx.z;
  if (x >= g.nx || y >= g.ny || z >= g.nz) return;
  const long long P = g.plane;
  const int n = node(g, x, y, z);
  const R* loc = a.loc;
  const R phi = loc[S_PHI * P + n], fs = loc[S_FS * P + n], T = loc[S_T * P + n];
  const R fl = loc[S_FL * P + n], w = loc[S_W * P + n];
  const R q0 = a.phi0[n];
  R lphi = R(0), lphi0 = R(0), lfs = R(0);
#pragma unroll
  for (int i = 1; i < Q; i++) {
    const int xx = wrap_or_clamp(x + cx(i), g.nx, g.bc[0], g.bc[1]);
    const int yy = wrap_or_clamp(y + cy(i), g.ny, g.bc[2], g.bc[3]);
    const int zz = wrap_or_clamp(z + cz(i), g.nz, g.bc[4], g.bc[5]);
    const int m = node(g, xx, yy, zz);
    const R wi = wq<R>(i);
    lphi += R(2) * wi * (loc[S_PHI * P + m] - phi);
    lphi0 += R(2) * wi * (a.phi0[m] - q0);
    lfs += R(2) * wi * (loc[S_FS * P + m] - fs);
  }
  lphi *= R(3); lphi0 *= R(3); lfs *= R(3);
  const R muphi = lbmk::chem_local(c, phi, q0, fs) -
                  c.klap * (lphi + c.cos_th * lphi0 + c.cos_ps * lfs);
  const R emu = c.eta * muphi;
  R fsf = q0 + w;
  fsf = fsf > R(1) ? R(1) : fsf;
  const R capT = T < R(0) ? lbmk::heat_cap(c, fsf, w) : lbmk::heat_cap(c, q0, w);
  const R rhoH = capT * T + w * c.rho_l * c.latent * fl;
  const R rrT = c.rr * T;
  R hq[Q];
  if (g.has_mask && a.mask[n]) {
    cold_mask_h19(c, w, q0, hq);
  } else {
    hq[0] = rhoH - rrT + wq<R>(0) * rrT;
#pragma unroll
    for (int i = 1; i < Q; i++) hq[i] = wq<R>(i) * rrT;
  }
  R* out = a.pout + n;
#pragma unroll
  for (int i = 0; i < Q; i++) {
    out[i * P] = R(0);
    out[(Q + i) * P] = i == 0 ? phi + (wq<R>(0) - R(1)) * emu : wq<R>(i) * emu;
    out[(2 * Q + i) * P] = hq[i];
  }
}

__device__ __forceinline__ double vv(float x) { return x; }
__device__ __forceinline__ double vv(double x) { return x; }
__device__ __forceinline__ double vv(const lbmk::Dual& x) { return x.v; }

// Per-block FP64 partial sums of the diagnostics of the state whose fields
// the read-out pass left in a.fld (dense order; block b covers nodes
// b NT ... (b + 1) NT - 1), summed in a fixed tree order.  For a tangent
// state (R = Dual) the derivative sums follow as rows NDIAG3 ... 2 NDIAG3 - 1,
// from the derivative planes the read-out wrote NFIELD3 planes further on.
template <typename R>
__global__ void __launch_bounds__(NT) lbm3_diag_partial_kernel(const Args3<R> a,
                                                               double* __restrict__ partial) {
  constexpr bool TAN = lbmk::is_dual<R>::value;
  using V = typename std::conditional<TAN, lbmk::Dual, double>::type;
  constexpr int ND = TAN ? 2 * NDIAG3 : NDIAG3;
  __shared__ double s[ND][NT];
  const Geom3& g = a.g;
  const Coef<R>& c = a.c;
  const int tid = threadIdx.x;
  const long long N = (long long)g.nx * g.ny * g.nz;
  const long long d = (long long)blockIdx.x * NT + tid;
  V v[NDIAG3];
#pragma unroll
  for (int k = 0; k < NDIAG3; k++) v[k] = V(0.0);
  if (d < N) {
    const double* F = a.fld;
    auto get = [&](int k) -> V {
      if constexpr (TAN) return V(F[k * N + d], F[(NFIELD3 + k) * N + d]);
      else return V(F[k * N + d]);
    };
    const V phi = get(0), fl = get(2), rhoH = get(4);
    const V ux = get(6), uy = get(7), uz = get(8);
    const V rho = get(9), w = get(11);
    const double rs = vv(c.rho_s), rl = vv(c.rho_l);
    v[0] = rho;
    v[1] = w * (rs * (1.0 - fl) + rl * fl);
    v[2] = rhoH;
    v[3] = w * fl;
    v[4] = w;
    v[5] = w * (1.0 - fl);
    v[6] = phi;
    v[7] = 0.5 * rho * (ux * ux + uy * uy + uz * uz);
    const int x = (int)(d % g.nx), y = (int)((d / g.nx) % g.ny), z = (int)(d / ((long long)g.nx * g.ny));
    const long long P = g.plane;
    const int n = node(g, x, y, z);
    R tot = R(0);
    if (g.lattices & LAT_FLOW)
      for (int i = 0; i < Q; i++) tot += a.pin[i * P + n];
    if (g.lattices & LAT_PHASE)
      for (int i = 0; i < Q; i++) tot += a.pin[(Q + i) * P + n];
    if (g.lattices & LAT_HEAT) {
      if (g.has_mask && a.mask[n]) {
        R hq[Q];
        cold_mask_h19(c, a.lin[L_W * P + n], a.phi0[n], hq);
        for (int i = 0; i < Q; i++) tot += hq[i];
      } else {
        for (int i = 0; i < Q; i++) tot += a.pin[(2 * Q + i) * P + n];
      }
    }
    v[8] = V(lbmk::finite(tot) ? 0.0 : 1.0);
  }
#pragma unroll
  for (int k = 0; k < NDIAG3; k++) {
    if constexpr (TAN) {
      s[k][tid] = v[k].v;
      s[NDIAG3 + k][tid] = v[k].d;
    } else {
      s[k][tid] = v[k];
    }
  }
  __syncthreads();
  for (int h = NT / 2; h > 0; h >>= 1) {
    if (tid < h) {
#pragma unroll
      for (int k = 0; k < ND; k++) s[k][tid] += s[k][tid + h];
    }
    __syncthreads();
  }
  if (tid < ND) partial[(long long)tid * gridDim.x + blockIdx.x] = s[tid][0];
}

__global__ void __launch_bounds__(NT) lbm3_diag_final_kernel(const double* __restrict__ partial,
                                                             int nb, int nrows,
                                                             double* __restrict__ out) {
  __shared__ double s[NT];
  const int tid = threadIdx.x;
  for (int k = 0; k < nrows; k++) {
    double v = 0.0;
    for (int j = tid; j < nb; j += NT) v += partial[(long long)k * nb + j];
    s[tid] = v;
    __syncthreads();
    for (int h = NT / 2; h > 0; h >>= 1) {
      if (tid < h) s[tid] += s[tid + h];
      __syncthreads();
    }
    if (tid == 0) out[k] = s[0];
    __syncthreads();
  }
}

}  // namespace lbm3

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------

struct lbm3_ctx {
  lbm3_params p;
  lbm3::Geom3 g;
  bool f64;
  bool tangent;  // FP64 values with their derivatives (lbmk::Dual)
  lbmk::Coef<float> cf;
  lbmk::Coef<double> cd;
  lbmk::Coef<lbmk::Dual> ct;
  double h_tan[lbm3::NDIAG3];  // derivative sums of the last diagnostics
  int64_t tan_step;
  void* pop[2];
  void* lag[2];
  void* loc;
  void* phi0;
  unsigned char* mask;
  double* fld;
  double* partial;
  double* dout;
  int nb;  // diagnostic blocks
  int cur;
  int64_t step;
  bool have_geometry;
  char err[256];
};

namespace {

int fail3(lbm3_ctx* c, int code, const char* msg) {
  if (c) std::snprintf(c->err, sizeof(c->err), "%s", msg);
  return code;
}

int cuda_fail3(lbm3_ctx* c, cudaError_t e, const char* what) {
  if (c) std::snprintf(c->err, sizeof(c->err), "%s: %s", what, cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA;
}

dim3 grid3(const lbm3::Geom3& g) {
  return dim3((g.nx + lbm3::BX - 1) / lbm3::BX, (g.ny + lbm3::BY - 1) / lbm3::BY,
              (g.nz + lbm3::BZ - 1) / lbm3::BZ);
}
dim3 block3() { return dim3(lbm3::BX, lbm3::BY, lbm3::BZ); }

// a wall temperature with (tangent) or without its derivative
template <typename R>
R wall_value(double v, double d) {
  if constexpr (lbmk::is_dual<R>::value) return R(v, d);
  else { (void)d; return (R)v; }
}

template <typename R>
lbm3::Args3<R> args3(lbm3_ctx* c, const lbmk::Coef<R>& coef) {
  lbm3::Args3<R> a;
  std::memset(&a, 0, sizeof(a));
  a.g = c->g;
  a.c = coef;
  a.gz = (R)c->p.gz;
  for (int k = 0; k < 4; k++) a.T_wall[k] = wall_value<R>(c->p.base.T_wall[k], c->p.base.tan_T_wall[k]);
  a.T_wall[4] = wall_value<R>(c->p.T_wall_z[0], c->p.tan_T_wall_z[0]);
  a.T_wall[5] = wall_value<R>(c->p.T_wall_z[1], c->p.tan_T_wall_z[1]);
  a.phi0 = (const R*)c->phi0;
  a.mask = c->mask;
  a.loc = (R*)c->loc;
  a.fld = c->fld;
  a.pin = (const R*)c->pop[c->cur];
  a.pout = (R*)c->pop[c->cur ^ 1];
  a.lin = (const R*)c->lag[c->cur];
  a.lout = (R*)c->lag[c->cur ^ 1];
  return a;
}

// one step (read == false) or the read-out of the current state's fields
// into c->fld (read == true)
template <typename R>
cudaError_t launch3(lbm3_ctx* c, const lbmk::Coef<R>& coef, bool read, cudaStream_t s) {
  const lbm3::Args3<R> a = args3<R>(c, coef);
  if (c->g.plane * 57 < (1LL << 31)) {
    lbm3::lbm3_local_kernel<R, int><<<grid3(c->g), block3(), 0, s>>>(a);
    if (read) lbm3::lbm3_collide_kernel<R, true, int><<<grid3(c->g), block3(), 0, s>>>(a);
    else lbm3::lbm3_collide_kernel<R, false, int><<<grid3(c->g), block3(), 0, s>>>(a);
  } else {
    lbm3::lbm3_local_kernel<R, long long><<<grid3(c->g), block3(), 0, s>>>(a);
    if (read) lbm3::lbm3_collide_kernel<R, true, long long><<<grid3(c->g), block3(), 0, s>>>(a);
    else lbm3::lbm3_collide_kernel<R, false, long long><<<grid3(c->g), block3(), 0, s>>>(a);
  }
  return cudaGetLastError();
}

cudaError_t launch3(lbm3_ctx* c, bool read, cudaStream_t s) {
  if (c->tangent) return launch3<lbmk::Dual>(c, c->ct, read, s);
  return c->f64 ? launch3<double>(c, c->cd, read, s) : launch3<float>(c, c->cf, read, s);
}

template <typename R>
cudaError_t launch_diag3(lbm3_ctx* c, const lbmk::Coef<R>& coef, cudaStream_t s) {
  const lbm3::Args3<R> a = args3<R>(c, coef);
  lbm3::lbm3_diag_partial_kernel<R><<<c->nb, lbm3::NT, 0, s>>>(a, c->partial);
  const int rows = lbmk::is_dual<R>::value ? 2 * lbm3::NDIAG3 : lbm3::NDIAG3;
  lbm3::lbm3_diag_final_kernel<<<1, lbm3::NT, 0, s>>>(c->partial, c->nb, rows, c->dout);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_init3(lbm3_ctx* c, const lbmk::Coef<R>& coef, const double* phi0,
                         const unsigned char* mask, const double* phi, const double* T,
                         const double* fl, cudaStream_t s) {
  lbm3::Args3<R> a = args3<R>(c, coef);
  a.lout = (R*)c->lag[c->cur];
  a.pout = (R*)c->pop[c->cur];
  lbm3::lbm3_init_local_kernel<R><<<grid3(c->g), block3(), 0, s>>>(a, phi0, mask, phi, T, fl,
                                                                 (R*)c->phi0, c->mask);
  lbm3::lbm3_init_pops_kernel<R><<<grid3(c->g), block3(), 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace

extern "C" {

int lbm3_create(const lbm3_params* p, lbm3_ctx** out) {
  if (!p || !out) return LBM_ERR_ARG;
  *out = nullptr;
  char err[256] = {0};
  lbm_params b = p->base;
  if (b.precision != LBM_FP32 && b.precision != LBM_FP64 && b.precision != LBM_FP64_TANGENT)
    return LBM_ERR_UNSUPPORTED;
  // the 2-D checks on the x and y extents and the physics (sizes are
  // checked here for the 3-D grid)
  b.ny = 2;
  b.nx = 2;
  int st = lbmh::validate(&b, err, sizeof(err));
  if (st != LBM_OK) return st;
  if (p->base.nx < 2 || p->base.ny < 2 || p->nz < 2) return LBM_ERR_ARG;
  for (int k = 0; k < 2; k++)
    if (p->bc_z[k] < LBM_BC_PERIODIC || p->bc_z[k] > LBM_BC_ADIABATIC) return LBM_ERR_ARG;
  if ((p->bc_z[0] == LBM_BC_PERIODIC) != (p->bc_z[1] == LBM_BC_PERIODIC)) return LBM_ERR_ARG;
  if (!std::isfinite(p->gz) || !std::isfinite(p->T_wall_z[0]) || !std::isfinite(p->T_wall_z[1]) ||
      !std::isfinite(p->tan_T_wall_z[0]) || !std::isfinite(p->tan_T_wall_z[1]))
    return LBM_ERR_PARAM;
  const long long pitch = (p->base.nx + 31) / 32 * 32;
  const long long plane = (pitch * p->base.ny * p->nz + 63) / 64 * 64;
  if (plane >= (1LL << 31)) return LBM_ERR_ARG;  // node offsets within a plane are 32-bit
  lbm3_ctx* c = new (std::nothrow) lbm3_ctx();
  if (!c) return LBM_ERR_OOM;
  c->p = *p;
  c->g.nx = p->base.nx;
  c->g.ny = p->base.ny;
  c->g.nz = p->nz;
  c->g.pitch = (int)pitch;
  c->g.plane = plane;
  for (int k = 0; k < 4; k++) c->g.bc[k] = p->base.bc[k];
  c->g.bc[4] = p->bc_z[0];
  c->g.bc[5] = p->bc_z[1];
  c->g.lattices = (int)p->base.lattices;
  c->g.has_mask = 0;
  c->f64 = p->base.precision == LBM_FP64;
  c->tangent = p->base.precision == LBM_FP64_TANGENT;
  c->cf = lbmh::make_coef<float>(p->base);
  c->cd = lbmh::make_coef<double>(p->base);
  if (c->tangent) c->ct = lbmh::make_coef_tangent(p->base);
  const size_t es = c->tangent ? 16 : (c->f64 ? 8 : 4);
  const size_t fmul = c->tangent ? 2 : 1;  // read-out and diagnostics: values, then derivatives
  const long long N = (long long)p->base.nx * p->base.ny * p->nz;
  c->nb = (int)((N + lbm3::NT - 1) / lbm3::NT);
  c->tan_step = -1;
  cudaError_t e = cudaSuccess;
  for (int k = 0; k < 2 && e == cudaSuccess; k++) e = cudaMalloc(&c->pop[k], 57 * plane * es);
  for (int k = 0; k < 2 && e == cudaSuccess; k++) e = cudaMalloc(&c->lag[k], lbm3::NLAG * plane * es);
  if (e == cudaSuccess) e = cudaMalloc(&c->loc, lbm3::NLOC * plane * es);
  if (e == cudaSuccess) e = cudaMalloc(&c->phi0, plane * es);
  if (e == cudaSuccess) e = cudaMalloc((void**)&c->mask, plane);
  if (e == cudaSuccess) e = cudaMalloc((void**)&c->fld, fmul * lbm3::NFIELD3 * N * sizeof(double));
  if (e == cudaSuccess)
    e = cudaMalloc((void**)&c->partial, fmul * lbm3::NDIAG3 * (size_t)c->nb * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc((void**)&c->dout, fmul * lbm3::NDIAG3 * sizeof(double));
  // padding nodes are never read; zero them once so that no buffer holds
  // uninitialised values
  for (int k = 0; k < 2 && e == cudaSuccess; k++) e = cudaMemset(c->pop[k], 0, 57 * plane * es);
  for (int k = 0; k < 2 && e == cudaSuccess; k++) e = cudaMemset(c->lag[k], 0, lbm3::NLAG * plane * es);
  if (e == cudaSuccess) e = cudaMemset(c->loc, 0, lbm3::NLOC * plane * es);
  if (e == cudaSuccess) e = cudaMemset(c->phi0, 0, plane * es);
  if (e == cudaSuccess) e = cudaMemset(c->mask, 0, plane);
  if (e != cudaSuccess) {
    const int code = e == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA;
    lbm3_destroy(c);
    return code;
  }
  *out = c;
  return LBM_OK;
}

int lbm3_set_geometry(lbm3_ctx* c, const double* phi0, const uint8_t* mask, const double* phi,
                      const double* T, const double* fl, int where, void* stream) {
  if (!c) return LBM_ERR_ARG;
  if (!phi0 || !phi || !T || !fl) return fail3(c, LBM_ERR_ARG, "null input array");
  if (where != LBM_HOST && where != LBM_DEVICE) return fail3(c, LBM_ERR_ARG, "bad `where`");
  cudaStream_t s = (cudaStream_t)stream;
  const size_t N = (size_t)c->g.nx * c->g.ny * c->g.nz;
  const double* src[4] = {phi0, phi, T, fl};
  const double* dsrc[4] = {phi0, phi, T, fl};
  const unsigned char* dmask = mask;
  double* stage = nullptr;
  unsigned char* mstage = nullptr;
  cudaError_t e = cudaSuccess;
  if (where == LBM_HOST) {
    e = cudaMalloc(&stage, 4 * N * sizeof(double));
    if (e == cudaSuccess && mask) e = cudaMalloc(&mstage, N);
    for (int k = 0; k < 4 && e == cudaSuccess; k++) {
      e = cudaMemcpyAsync(stage + k * N, src[k], N * sizeof(double), cudaMemcpyHostToDevice, s);
      dsrc[k] = stage + k * N;
    }
    if (e == cudaSuccess && mask) {
      e = cudaMemcpyAsync(mstage, mask, N, cudaMemcpyHostToDevice, s);
      dmask = mstage;
    }
  }
  c->g.has_mask = mask ? 1 : 0;
  c->cur = 0;
  if (e == cudaSuccess)
    e = c->tangent ? launch_init3<lbmk::Dual>(c, c->ct, dsrc[0], dmask, dsrc[1], dsrc[2], dsrc[3], s)
        : c->f64   ? launch_init3<double>(c, c->cd, dsrc[0], dmask, dsrc[1], dsrc[2], dsrc[3], s)
                   : launch_init3<float>(c, c->cf, dsrc[0], dmask, dsrc[1], dsrc[2], dsrc[3], s);
  if (where == LBM_HOST) {
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (stage) cudaFree(stage);
    if (mstage) cudaFree(mstage);
  }
  if (e != cudaSuccess) return cuda_fail3(c, e, "lbm3_set_geometry");
  c->step = 0;
  c->have_geometry = true;
  return LBM_OK;
}

int lbm3_step(lbm3_ctx* c, int64_t nsteps, void* stream) {
  if (!c) return LBM_ERR_ARG;
  if (nsteps < 0) return fail3(c, LBM_ERR_ARG, "nsteps < 0");
  if (!c->have_geometry) return fail3(c, LBM_ERR_STATE, "step before lbm3_set_geometry");
  cudaStream_t s = (cudaStream_t)stream;
  for (int64_t k = 0; k < nsteps; k++) {
    const cudaError_t e = launch3(c, false, s);
    if (e != cudaSuccess) return cuda_fail3(c, e, "lbm3_step");
    c->cur ^= 1;
    c->step++;
  }
  return LBM_OK;
}

int lbm3_read_fields(lbm3_ctx* c, uint32_t field_mask, double* const* out, int where,
                     void* stream) {
  if (!c) return LBM_ERR_ARG;
  if (!out || (field_mask >> lbm3::NFIELD3)) return fail3(c, LBM_ERR_ARG, "bad field mask or output");
  if (where != LBM_HOST && where != LBM_DEVICE) return fail3(c, LBM_ERR_ARG, "bad `where`");
  if (!c->have_geometry) return fail3(c, LBM_ERR_STATE, "read before lbm3_set_geometry");
  for (int k = 0; k < lbm3::NFIELD3; k++)
    if ((field_mask >> k & 1u) && !out[k]) return fail3(c, LBM_ERR_ARG, "null output for a selected field");
  cudaStream_t s = (cudaStream_t)stream;
  const size_t N = (size_t)c->g.nx * c->g.ny * c->g.nz;
  cudaError_t e = launch3(c, true, s);
  for (int k = 0; k < lbm3::NFIELD3 && e == cudaSuccess; k++)
    if (field_mask >> k & 1u)
      e = cudaMemcpyAsync(out[k], c->fld + k * N, N * sizeof(double),
                          where == LBM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess && where == LBM_HOST) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail3(c, e, "lbm3_read_fields");
  return LBM_OK;
}

int lbm3_read_tangent_fields(lbm3_ctx* c, uint32_t field_mask, double* const* out, int where,
                             void* stream) {
  if (!c) return LBM_ERR_ARG;
  if (!c->tangent) return fail3(c, LBM_ERR_UNSUPPORTED, "not a tangent context");
  if (!out || (field_mask >> lbm3::NFIELD3)) return fail3(c, LBM_ERR_ARG, "bad field mask or output");
  if (where != LBM_HOST && where != LBM_DEVICE) return fail3(c, LBM_ERR_ARG, "bad `where`");
  if (!c->have_geometry) return fail3(c, LBM_ERR_STATE, "read before lbm3_set_geometry");
  for (int k = 0; k < lbm3::NFIELD3; k++)
    if ((field_mask >> k & 1u) && !out[k]) return fail3(c, LBM_ERR_ARG, "null output for a selected field");
  cudaStream_t s = (cudaStream_t)stream;
  const size_t N = (size_t)c->g.nx * c->g.ny * c->g.nz;
  cudaError_t e = launch3(c, true, s);
  for (int k = 0; k < lbm3::NFIELD3 && e == cudaSuccess; k++)
    if (field_mask >> k & 1u)
      e = cudaMemcpyAsync(out[k], c->fld + (lbm3::NFIELD3 + k) * N, N * sizeof(double),
                          where == LBM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess && where == LBM_HOST) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail3(c, e, "lbm3_read_tangent_fields");
  return LBM_OK;
}

int lbm3_read_tangent_diagnostics(lbm3_ctx* c, lbm_diag* out) {
  if (!c || !out) return LBM_ERR_ARG;
  if (!c->tangent) return fail3(c, LBM_ERR_UNSUPPORTED, "not a tangent context");
  if (c->tan_step < 0) return fail3(c, LBM_ERR_STATE, "no diagnostics computed yet");
  const double* h = c->h_tan;
  out->mass = h[0];
  out->material_mass = h[1];
  out->rhoH = h[2];
  out->liquid_volume = h[3];
  out->material_volume = h[4];
  out->frozen_volume = h[5];
  out->phi_sum = h[6];
  out->kinetic = h[7];
  out->nonfinite = 0.0;
  out->step = c->tan_step;
  return LBM_OK;
}

int lbm3_diagnostics(lbm3_ctx* c, lbm_diag* out, void* stream) {
  if (!c || !out) return LBM_ERR_ARG;
  if (!c->have_geometry) return fail3(c, LBM_ERR_STATE, "diagnostics before lbm3_set_geometry");
  cudaStream_t s = (cudaStream_t)stream;
  double h[2 * lbm3::NDIAG3];
  const size_t rows = c->tangent ? 2 * lbm3::NDIAG3 : lbm3::NDIAG3;
  cudaError_t e = launch3(c, true, s);
  if (e == cudaSuccess)
    e = c->tangent ? launch_diag3<lbmk::Dual>(c, c->ct, s)
        : c->f64   ? launch_diag3<double>(c, c->cd, s)
                   : launch_diag3<float>(c, c->cf, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h, c->dout, rows * sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail3(c, e, "lbm3_diagnostics");
  out->mass = h[0];
  out->material_mass = h[1];
  out->rhoH = h[2];
  out->liquid_volume = h[3];
  out->material_volume = h[4];
  out->frozen_volume = h[5];
  out->phi_sum = h[6];
  out->kinetic = h[7];
  out->nonfinite = h[8];
  out->step = c->step;
  if (c->tangent) {
    for (int k = 0; k < lbm3::NDIAG3; k++) c->h_tan[k] = k == 8 ? 0.0 : h[lbm3::NDIAG3 + k];
    c->tan_step = c->step;
  }
  return h[8] > 0.0 ? LBM_ERR_NONFINITE : LBM_OK;
}

namespace {
// checkpoint header of a 3-D state (the populations and lags follow)
struct State3Header {
  uint32_t magic, version;
  int32_t nx, ny, nz, precision, lattices, pad;
  int64_t step;
};
constexpr uint32_t kMagic3 = 0x4c424d33u;  // "LBM3"
constexpr uint32_t kVersion3 = 1;
}  // namespace

int lbm3_state_size(const lbm3_ctx* c, size_t* bytes) {
  if (!c || !bytes) return LBM_ERR_ARG;
  const size_t es = c->tangent ? 16 : (c->f64 ? 8 : 4);
  *bytes = sizeof(State3Header) + (57 + lbm3::NLAG) * es * (size_t)c->g.plane;
  return LBM_OK;
}

int lbm3_save_state(lbm3_ctx* c, void* host_buf, size_t capacity, void* stream) {
  if (!c || !host_buf) return LBM_ERR_ARG;
  if (!c->have_geometry) return fail3(c, LBM_ERR_STATE, "save before lbm3_set_geometry");
  size_t need;
  lbm3_state_size(c, &need);
  if (capacity < need) return fail3(c, LBM_ERR_ARG, "state buffer too small");
  cudaStream_t s = (cudaStream_t)stream;
  const State3Header h = {kMagic3, kVersion3, c->g.nx, c->g.ny, c->g.nz,
                          c->p.base.precision, (int32_t)c->p.base.lattices, 0, c->step};
  std::memcpy(host_buf, &h, sizeof(h));
  char* dst = (char*)host_buf + sizeof(h);
  const size_t es = c->tangent ? 16 : (c->f64 ? 8 : 4);
  const size_t pb = 57 * es * (size_t)c->g.plane;
  cudaError_t e = cudaMemcpyAsync(dst, c->pop[c->cur], pb, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(dst + pb, c->lag[c->cur], lbm3::NLAG * es * (size_t)c->g.plane,
                        cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail3(c, e, "state download");
  return LBM_OK;
}

int lbm3_load_state(lbm3_ctx* c, const void* host_buf, size_t size, void* stream) {
  if (!c || !host_buf) return LBM_ERR_ARG;
  if (!c->have_geometry) return fail3(c, LBM_ERR_STATE, "load before lbm3_set_geometry");
  size_t need;
  lbm3_state_size(c, &need);
  if (size < need) return fail3(c, LBM_ERR_ARG, "state buffer too small");
  State3Header h;
  std::memcpy(&h, host_buf, sizeof(h));
  if (h.magic != kMagic3 || h.version != kVersion3 || h.nx != c->g.nx || h.ny != c->g.ny ||
      h.nz != c->g.nz || h.precision != c->p.base.precision ||
      h.lattices != (int32_t)c->p.base.lattices)
    return fail3(c, LBM_ERR_ARG, "state does not match this context");
  cudaStream_t s = (cudaStream_t)stream;
  const char* src = (const char*)host_buf + sizeof(h);
  const size_t es = c->tangent ? 16 : (c->f64 ? 8 : 4);
  const size_t pb = 57 * es * (size_t)c->g.plane;
  cudaError_t e = cudaMemcpyAsync(c->pop[c->cur], src, pb, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(c->lag[c->cur], src + pb, lbm3::NLAG * es * (size_t)c->g.plane,
                        cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail3(c, e, "state upload");
  c->step = h.step;
  return LBM_OK;
}

int64_t lbm3_step_count(const lbm3_ctx* c) { return c ? c->step : -1; }

const char* lbm3_last_error(const lbm3_ctx* c) { return c ? c->err : "null context"; }

void lbm3_destroy(lbm3_ctx* c) {
  if (!c) return;
  void* bufs[] = {c->pop[0], c->pop[1], c->lag[0], c->lag[1], c->loc, c->phi0,
                  c->mask,   c->fld,    c->partial, c->dout};
  for (void* b : bufs)
    if (b) cudaFree(b);
  delete c;
}

void lbm3_lattice(int32_t* c, double* w) {
  for (int i = 0; i < lbm3::Q; i++) {
    if (c) {
      c[3 * i] = lbm3::cx(i);
      c[3 * i + 1] = lbm3::cy(i);
      c[3 * i + 2] = lbm3::cz(i);
    }
    if (w) w[i] = i == 0 ? 1.0 / 3.0 : (i <= 6 ? 1.0 / 18.0 : 1.0 / 36.0);
  }
}

}  // extern "C"
