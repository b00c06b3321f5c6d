// lbm_kernels.cuh -- device code of the fused coupled LB time step for
// sm_103a (GB300), templated on the arithmetic type R (float or double).
//
// One CTA owns a TX x TY tile of nodes and stages, in shared memory, the
// macroscopic fields of the tile plus a one-node halo: each thread recovers
// its own node (rows a1-a2: enthalpy inversion, order parameter, material
// weight, solid fraction, density) while keeping its 27 populations in
// registers; a subset of threads then recovers the ring of halo nodes.  After
// one barrier every thread evaluates the isotropic stencils (row a3), the
// velocity and pressure (row a4), the three collisions (rows a5-a7) and
// pushes its post-collision populations to the neighbours in the other
// buffer, with half-way bounce-back / anti-bounce-back at walls (row a8), and
// stores its lag fields (row a9).  Global FP64 diagnostics are reduced in the
// same launch (warp shuffles, then a fixed-order per-block and last-block
// pass, so results are bitwise reproducible).
//
// Layout in HBM: structure of arrays, one plane per population or field,
// planes of `plane` elements with rows padded to `pitch` (a multiple of 32
// elements).  Populations: planes 0-8 flow f, 9-17 phase g, 18-26 enthalpy h,
// double-buffered (A/B).  Lag fields (double-buffered because neighbours
// read them): fl, w, p, phi ux, phi uy, Q.  Static: phi0 and an optional
// byte mask.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace lbmk {

constexpr int TX = 32, TY = 8;
constexpr int HX = TX + 2, HY = TY + 2, HN = HX * HY;
constexpr int NT = TX * TY;
constexpr int RING = HN - NT;
constexpr int NDIAG = 9;
constexpr int NFIELD = 12;
enum { BC_PERIODIC = 0, BC_DIRICHLET = 1, BC_ADIABATIC = 2 };
enum { LAT_FLOW = 1, LAT_PHASE = 2, LAT_HEAT = 4 };
enum { LAG_FL = 0, LAG_W, LAG_P, LAG_PHUX, LAG_PHUY, LAG_Q, NLAG };
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
  uint32_t readings;
};

struct Geom {
  int nx, ny, pitch;
  long long plane;
  int lattices;
  int bc[4];
  int has_mask;
};

template <typename R>
struct Args {
  Geom g;
  Coef<R> c;
  const R* __restrict__ pin;   // 27 planes
  R* __restrict__ pout;        // 27 planes
  const R* __restrict__ lin;   // NLAG planes
  R* __restrict__ lout;        // NLAG planes
  const R* __restrict__ phi0;
  const uint8_t* __restrict__ mask;
  double* out[NFIELD];         // MODE_READ: dense [ny][nx] outputs (or null)
  double* diag_partial;        // [NDIAG][nblocks]
  double* diag_out;            // NDIAG values + step index (as double)
  unsigned* diag_counter;
  long long step_index;
};

template <typename R>
struct InitArgs {
  Geom g;
  Coef<R> c;
  R* __restrict__ pout;
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
    T = rhoH / heat_cap(c, fsf, w);
  } else if (rhoH > ell) {
    fl = R(1);
    T = (rhoH - ell) / heat_cap(c, phi0, w);
  } else {
    T = R(0);
    fl = ell > R(0) ? rhoH / ell : R(1);
  }
  fl = clamp01(fl);
}

// Enthalpy equilibrium Eq. (25) at temperature T with velocity (ux, uy).
template <typename R>
__device__ __forceinline__ R heq_i(int i, R rhoH, R C, R T, R rr, R ux, R uy, R uu) {
  if (i == 0) return rhoH - rr * T + qw<R>(0) * C * T * (rr / C - uu * R(1.5));
  R cu = R(qx(i)) * ux + R(qy(i)) * uy;
  return qw<R>(i) * C * T * (rr / C + R(3) * cu + R(4.5) * cu * cu - R(1.5) * uu);
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
#pragma unroll
  for (int i = 0; i < 9; i++) h[i] = heq_i<R>(i, rhoH, C, T, c.rr, R(0), R(0), R(0));
}

template <typename R>
struct Local {
  R T, fl, mdot, rhoH, phi, w, fs, rho;
};

// Rows a1-a2 for one node from its population sums and lag fields.
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
  if (lat & LAT_PHASE) {
    L.phi = sg / (R(1) - R(0.5) * L.mdot);  // Eq. (22) solved for phi
    L.w = clamp01((R(1) - phi0 + L.phi) * R(0.5));
  } else {
    L.w = wp;
    L.phi = R(2) * wp - R(1) + phi0;
  }
  R fs = phi0 + L.w * (R(1) - L.fl);
  L.fs = fs > R(1) ? R(1) : fs;
  L.rho = interp(L.fs, L.w, c.rho_s, c.rho_l, c.rho_g);
  return L;
}

// Eq. (6) without the Laplacian terms.
template <typename R>
__device__ __forceinline__ R chem_local(const Coef<R>& c, R phi, R phi0, R fs) {
  R s3 = R(3) * c.sigma / c.eps, s9 = R(9) * c.sigma / c.eps;
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

template <typename R>
__device__ __forceinline__ R warp_sum(R v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ---------------------------------------------------------------------------
// the fused step (MODE_STEP) / field read-out (MODE_READ) kernel
// ---------------------------------------------------------------------------

template <typename R, int MODE, bool DIAG>
__global__ void __launch_bounds__(NT, sizeof(R) == 4 ? 2 : 1) lbm_step_kernel(const Args<R> a) {
  const Geom& g = a.g;
  const Coef<R>& c = a.c;
  const int lat = g.lattices;
  const long long P = g.plane;

  __shared__ R s_phi[HN], s_fs[HN], s_rho[HN], s_p[HN], s_phi0[HN];
  __shared__ double s_red[NT / 32][NDIAG];
  __shared__ int s_last;

  const int tx = threadIdx.x, ty = threadIdx.y;
  const int tid = ty * TX + tx;
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
  const int gx = x0 + tx, gy = y0 + ty;
  const bool valid = gx < g.nx && gy < g.ny;
  const int mx = wrap_or_clamp(gx, g.nx, g.bc[0], g.bc[1]);
  const int my = wrap_or_clamp(gy, g.ny, g.bc[2], g.bc[3]);
  const long long n = (long long)my * g.pitch + mx;

  // ---- phase A1: own node, populations kept in registers -----------------
  R f[9], gp[9], h[9];
  const R phi0 = a.phi0[n];
  const R flp = a.lin[LAG_FL * P + n];
  const R wp = a.lin[LAG_W * P + n];
  const R pp = a.lin[LAG_P * P + n];
  const R phuxp = a.lin[LAG_PHUX * P + n];
  const R phuyp = a.lin[LAG_PHUY * P + n];
  const R Qp = a.lin[LAG_Q * P + n];
  R sg = R(0), sh = R(0);
  if (lat & LAT_FLOW) {
#pragma unroll
    for (int i = 0; i < 9; i++) f[i] = a.pin[i * P + n];
  } else {
#pragma unroll
    for (int i = 0; i < 9; i++) f[i] = R(0);
  }
  if (lat & LAT_PHASE) {
#pragma unroll
    for (int i = 0; i < 9; i++) gp[i] = a.pin[(9 + i) * P + n];
#pragma unroll
    for (int i = 0; i < 9; i++) sg += gp[i];
  } else {
#pragma unroll
    for (int i = 0; i < 9; i++) gp[i] = R(0);
  }
  if (lat & LAT_HEAT) {
    if (g.has_mask && a.mask[n]) {
      cold_mask_h(c, wp, phi0, h);
    } else {
#pragma unroll
      for (int i = 0; i < 9; i++) h[i] = a.pin[(18 + i) * P + n];
    }
#pragma unroll
    for (int i = 0; i < 9; i++) sh += h[i];
  } else {
#pragma unroll
    for (int i = 0; i < 9; i++) h[i] = R(0);
  }
  const Local<R> L = local_state(c, lat, sg, sh, flp, wp, Qp, phi0);
  {
    const int hi = (ty + 1) * HX + (tx + 1);
    s_phi[hi] = L.phi;
    s_fs[hi] = L.fs;
    s_rho[hi] = L.rho;
    s_p[hi] = pp;
    s_phi0[hi] = phi0;
  }

  // ---- phase A2: the ring of halo nodes -----------------------------------
  for (int k = tid; k < RING; k += NT) {
    int hx, hy;
    if (k < HX) {
      hx = k; hy = 0;
    } else if (k < 2 * HX) {
      hx = k - HX; hy = HY - 1;
    } else {
      int r = k - 2 * HX;  // 2 * TY side nodes
      hy = 1 + (r >> 1);
      hx = (r & 1) ? HX - 1 : 0;
    }
    const int rx = wrap_or_clamp(x0 + hx - 1, g.nx, g.bc[0], g.bc[1]);
    const int ry = wrap_or_clamp(y0 + hy - 1, g.ny, g.bc[2], g.bc[3]);
    const long long m = (long long)ry * g.pitch + rx;
    const R q0 = a.phi0[m];
    const R wq = a.lin[LAG_W * P + m];
    R sgq = R(0), shq = R(0);
    if (lat & LAT_PHASE) {
#pragma unroll
      for (int i = 0; i < 9; i++) sgq += a.pin[(9 + i) * P + m];
    }
    if (lat & LAT_HEAT) {
      R hq[9];
      if (g.has_mask && a.mask[m]) {
        cold_mask_h(c, wq, q0, hq);
      } else {
#pragma unroll
        for (int i = 0; i < 9; i++) hq[i] = a.pin[(18 + i) * P + m];
      }
#pragma unroll
      for (int i = 0; i < 9; i++) shq += hq[i];
    }
    const Local<R> Lq = local_state(c, lat, sgq, shq, a.lin[LAG_FL * P + m], wq,
                                    a.lin[LAG_Q * P + m], q0);
    const int hi = hy * HX + hx;
    s_phi[hi] = Lq.phi;
    s_fs[hi] = Lq.fs;
    s_rho[hi] = Lq.rho;
    s_p[hi] = a.lin[LAG_P * P + m];
    s_phi0[hi] = q0;
  }
  __syncthreads();

  // ---- phase B: stencils, macros, collisions, streaming -------------------
  R dvals[NDIAG];
  if (valid) {
    const int hc = (ty + 1) * HX + (tx + 1);
    // isotropic stencils (reading R-FD): grad = 3 sum w_i c_i chi(x + c_i),
    // lap = 6 sum w_i (chi(x + c_i) - chi(x))
    R gphx = R(0), gphy = R(0), lphi = R(0), lphi0 = R(0), lfs = R(0);
    R grx = R(0), gry = R(0), gpx = R(0), gpy = R(0);
#pragma unroll
    for (int i = 1; i < 9; i++) {
      const int hn = hc + qy(i) * HX + qx(i);
      const R wi = qw<R>(i);
      const R cxi = R(qx(i)), cyi = R(qy(i));
      if (lat & LAT_PHASE) {
        const R ph = s_phi[hn];
        gphx += wi * cxi * ph;
        gphy += wi * cyi * ph;
        lphi += R(2) * wi * (ph - s_phi[hc]);
        lphi0 += R(2) * wi * (s_phi0[hn] - s_phi0[hc]);
        lfs += R(2) * wi * (s_fs[hn] - s_fs[hc]);
      }
      if (lat & LAT_FLOW) {
        const R rq = s_rho[hn], pq = s_p[hn];
        grx += wi * cxi * rq;
        gry += wi * cyi * rq;
        gpx += wi * cxi * pq;
        gpy += wi * cyi * pq;
      }
    }
    gphx *= R(3); gphy *= R(3); lphi *= R(3); lphi0 *= R(3); lfs *= R(3);
    grx *= R(3); gry *= R(3); gpx *= R(3); gpy *= R(3);

    const R phi = L.phi, fs = L.fs, rho = L.rho, T = L.T, mdot = L.mdot;
    R muphi = R(0), Fx, Fy;
    {
      R Fsx = R(0), Fsy = R(0);
      if (lat & LAT_PHASE) {
        muphi = chem_local(c, phi, phi0, fs) -
                R(3) * c.eps * c.sigma / R(8) * (lphi + c.cos_th * lphi0 + c.cos_ps * lfs);
        Fsx = muphi * gphx;
        Fsy = muphi * gphy;
      }
      Fx = Fsx + rho * c.gx;
      Fy = Fsy + rho * c.gy;
    }
    const R mu = interp(fs, L.w, c.mu_s, c.mu_l, c.mu_g);
    R ux = R(0), uy = R(0), pr = R(0);
    if (lat & LAT_FLOW) {
      R jx = R(0), jy = R(0), snz = R(0);
#pragma unroll
      for (int i = 1; i < 9; i++) {
        jx += R(qx(i)) * f[i];
        jy += R(qy(i)) * f[i];
        snz += f[i];
      }
      // Eq. (17a,b) with the penalty force f = fs (u_s - u*), u_s = 0
      const R usx = (jx + R(0.5) * Fx) / rho, usy = (jy + R(0.5) * Fy) / rho;
      const R fpx = -fs * usx, fpy = -fs * usy;
      ux = usx + R(0.5) * fpx;
      uy = usy + R(0.5) * fpy;
      const R uu = ux * ux + uy * uy;
      const R S = rho * mdot + ux * grx + uy * gry;
      // modified force (reading R-FT), lagged pressure (reading R-FP)
      const R Ftx = Fx - (gpx - grx / R(3)), Fty = Fy - (gpy - gry / R(3));
      const R uFt = ux * Ftx + uy * Fty;
      const R tauf = mu / (rho / R(3)) + R(0.5);
      const bool iso = (c.readings & 1u) != 0;
      // F_0 of Eq. (16)
      R F0 = qw<R>(0) * (S + (R(0) - R(2) / R(3) * uFt) * R(4.5));
      if (iso) F0 += qw<R>(0) * (S * (R(0) - R(2) / R(3)) * R(1.5));
      const R s0 = qw<R>(0) * (-uu * R(1.5));
      pr = (R(1) / R(3)) / (R(1) - qw<R>(0)) *
           (snz + R(0.5) * S + (tauf - R(0.5)) * F0 + rho * s0);  // Eq. (17c)
      if (MODE == MODE_STEP) {
        const R itau = R(1) / tauf;
        const R fcoef = R(1) - R(0.5) * itau;
        const R Gx = Fx + rho * fpx, Gy = Fy + rho * fpy;
#pragma unroll
        for (int i = 0; i < 9; i++) {
          const R cu = R(qx(i)) * ux + R(qy(i)) * uy;
          const R si = qw<R>(i) * (R(3) * cu + R(4.5) * cu * cu - R(1.5) * uu);
          const R feq = pr * R(3) * (qw<R>(i) - (i == 0 ? R(1) : R(0))) + rho * si;
          const R cF = R(qx(i)) * Gx + R(qy(i)) * Gy;
          const R cFt = R(qx(i)) * Ftx + R(qy(i)) * Fty;
          R tens = R(2) * cu * cFt - R(2) / R(3) * uFt;
          if (iso) tens += S / R(3) * (R(qx(i) * qx(i) + qy(i) * qy(i)) - R(2) / R(3));
          const R Fi = qw<R>(i) * (S + R(3) * cF + R(4.5) * tens);
          const R post = f[i] - (f[i] - feq) * itau + fcoef * Fi;  // Eq. (11)
          int wall;
          const long long t = stream_target(g, gx, gy, qx(i), qy(i), wall);
          if (t >= 0) a.pout[i * P + t] = post;
          else a.pout[qopp(i) * P + n] = post;
        }
      }
    }
    const R phux = phi * ux, phuy = phi * uy;
    if (MODE == MODE_STEP && (lat & LAT_PHASE)) {
      // Eqs. (18)-(20)
      const R itg = R(1) / c.tau_g;
      const R gcoef = R(1) - R(0.5) * itg;
      const R dphx = phux - phuxp, dphy = phuy - phuyp;
      const R emu = c.eta * muphi;
#pragma unroll
      for (int i = 0; i < 9; i++) {
        const R wi = qw<R>(i);
        const R cph = R(qx(i)) * phux + R(qy(i)) * phuy;
        const R geq = (i == 0) ? phi + (wi - R(1)) * emu : wi * emu + wi * R(3) * cph;
        const R Gi = wi * (R(qx(i)) * dphx + R(qy(i)) * dphy) * R(3) + wi * phi * mdot;
        const R post = gp[i] - (gp[i] - geq) * itg + gcoef * Gi;
        int wall;
        const long long t = stream_target(g, gx, gy, qx(i), qy(i), wall);
        if (t >= 0) a.pout[(9 + i) * P + t] = post;
        else a.pout[(9 + qopp(i)) * P + n] = post;
      }
    }
    const R cap = rho * interp(fs, L.w, c.cp_s, c.cp_l, c.cp_g);
    if (MODE == MODE_STEP && (lat & LAT_HEAT)) {
      // Eqs. (23)-(27): TRT with the magic relation 1/tau_s + 1/tau_a = 2
      const R lam = interp(fs, L.w, c.lam_s, c.lam_l, c.lam_g);
      const R taua = R(0.5) + lam / (c.rr / R(3));
      const R taus = taua / (R(2) * taua - R(1));
      const R ia = R(1) / taua, is = R(1) / taus;
      const R hcoef = R(1) - R(0.5) * ia;
      const R uu = ux * ux + uy * uy;
      R he[9];
#pragma unroll
      for (int i = 0; i < 9; i++) he[i] = heq_i<R>(i, L.rhoH, cap, T, c.rr, ux, uy, uu);
      const R Hsrc = cap * T * mdot;
#pragma unroll
      for (int i = 0; i < 9; i++) {
        const int o = qopp(i);
        const R hs = R(0.5) * (h[i] + h[o]), ha = R(0.5) * (h[i] - h[o]);
        const R es = R(0.5) * (he[i] + he[o]), ea = R(0.5) * (he[i] - he[o]);
        const R post = h[i] - (ha - ea) * ia - (hs - es) * is + hcoef * qw<R>(i) * Hsrc;
        int wall;
        const long long t = stream_target(g, gx, gy, qx(i), qy(i), wall);
        if (t >= 0) {
          a.pout[(18 + i) * P + t] = post;
        } else {
          const R v = (g.bc[wall] == BC_DIRICHLET)
                          ? -post + R(2) * qw<R>(i) * c.rr * c.T_wall[wall]
                          : post;
          a.pout[(18 + qopp(i)) * P + n] = v;
        }
      }
    }
    if (MODE == MODE_STEP) {
      a.lout[LAG_FL * P + n] = L.fl;
      a.lout[LAG_W * P + n] = L.w;
      a.lout[LAG_P * P + n] = (lat & LAT_FLOW) ? pr : R(0);
      a.lout[LAG_PHUX * P + n] = (lat & LAT_PHASE) ? phux : R(0);
      a.lout[LAG_PHUY * P + n] = (lat & LAT_PHASE) ? phuy : R(0);
      a.lout[LAG_Q * P + n] = (lat & LAT_HEAT) ? cap * T * mdot : R(0);
    } else {
      const long long d = (long long)gy * g.nx + gx;
      const R vals[NFIELD] = {phi, fs, L.fl, T, L.rhoH, pr, ux, uy, rho, muphi, L.w, mdot};
#pragma unroll
      for (int k = 0; k < NFIELD; k++)
        if (a.out[k]) a.out[k][d] = (double)vals[k];
    }
    if (DIAG) {
      dvals[0] = rho;
      dvals[1] = L.w * (c.rho_s * (R(1) - L.fl) + c.rho_l * L.fl);
      dvals[2] = L.rhoH;
      dvals[3] = L.w * L.fl;
      dvals[4] = L.w;
      dvals[5] = L.w * (R(1) - L.fl);
      dvals[6] = phi;
      dvals[7] = R(0.5) * rho * (ux * ux + uy * uy);
      R tot = R(0);
#pragma unroll
      for (int i = 0; i < 9; i++) tot += f[i] + gp[i] + h[i];
      dvals[8] = isfinite(tot) ? R(0) : R(1);
    }
  } else if (DIAG) {
#pragma unroll
    for (int k = 0; k < NDIAG; k++) dvals[k] = R(0);
  }

  if (DIAG) {
    // warp sums in R, then per-block and a last-block pass in FP64, all in a
    // fixed order
    const int lane = tid & 31, warp = tid >> 5;
#pragma unroll
    for (int k = 0; k < NDIAG; k++) {
      const R v = warp_sum(dvals[k]);
      if (lane == 0) s_red[warp][k] = (double)v;
    }
    __syncthreads();
    const int nb = gridDim.x * gridDim.y;
    const int b = blockIdx.y * gridDim.x + blockIdx.x;
    if (tid < NDIAG) {
      double s = 0.0;
#pragma unroll
      for (int w = 0; w < NT / 32; w++) s += s_red[w][tid];
      a.diag_partial[(long long)tid * nb + b] = s;
    }
    __threadfence();
    __syncthreads();
    if (tid == 0) s_last = (atomicAdd(a.diag_counter, 1u) == (unsigned)(nb - 1));
    __syncthreads();
    if (s_last) {
      __threadfence();
      double acc[NDIAG];
#pragma unroll
      for (int k = 0; k < NDIAG; k++) acc[k] = 0.0;
      for (int j = tid; j < nb; j += NT) {
#pragma unroll
        for (int k = 0; k < NDIAG; k++) acc[k] += __ldcg(&a.diag_partial[(long long)k * nb + j]);
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
        double s = 0.0;
#pragma unroll
        for (int w = 0; w < NT / 32; w++) s += s_red[w][tid];
        a.diag_out[tid] = s;
      }
      if (tid == 0) {
        a.diag_out[NDIAG] = (double)a.step_index;
        *a.diag_counter = 0u;
      }
    }
  }
}

// ---------------------------------------------------------------------------
// initial state
// ---------------------------------------------------------------------------

template <typename R>
__global__ void __launch_bounds__(NT) lbm_init_kernel(const InitArgs<R> a) {
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
                  R(3) * c.eps * c.sigma / R(8) * (lphi + c.cos_th * lphi0 + c.cos_ps * lfs);
  const R ell = w * c.rho_l * c.latent;
  R fsf = q0 + w;
  fsf = fsf > R(1) ? R(1) : fsf;
  const R capT = T < R(0) ? heat_cap(c, fsf, w) : heat_cap(c, q0, w);
  const R rhoH = capT * T + ell * fl;
  const R C = heat_cap(c, fs, w);
  const R emu = c.eta * muphi;
#pragma unroll
  for (int i = 0; i < 9; i++) {
    a.pout[i * P + n] = R(0);
    a.pout[(9 + i) * P + n] = (i == 0) ? phi + (qw<R>(0) - R(1)) * emu : qw<R>(i) * emu;
    a.pout[(18 + i) * P + n] = heq_i<R>(i, rhoH, C, T, c.rr, R(0), R(0), R(0));
  }
  a.lout[LAG_FL * P + n] = fl;
  a.lout[LAG_W * P + n] = w;
  a.lout[LAG_P * P + n] = R(0);
  a.lout[LAG_PHUX * P + n] = R(0);
  a.lout[LAG_PHUY * P + n] = R(0);
  a.lout[LAG_Q * P + n] = R(0);
  a.phi0_out[n] = q0;
  if (a.mask_out) a.mask_out[n] = a.mask ? (a.mask[d] != 0) : 0;
}

}  // namespace lbmk
