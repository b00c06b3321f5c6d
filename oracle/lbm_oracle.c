/*
 * lbm_oracle.c -- plain FP64 CPU oracle of the coupled three-lattice lattice
 * Boltzmann (LB) method for three-phase freezing of Huang, Zhan, Chai & Huang,
 * "A diffuse-interface method for the containerless freezing of three-phase
 * flows in complex geometries" (arXiv 2510.18688).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or
 * call this file: only the test-suite, the smoke check and the CPU-baseline
 * leg of the benchmark use it.  It shares no code, header, table or helper
 * with the CUDA library; the two meet only through seeded input arrays.
 *
 * Everything is a literal, slow restatement of the paper in double
 * precision: plain loops over nodes, one pass per stage, no blocking and no
 * fusion.  The stages of one time step follow the order below, and every
 * silent or garbled point of the paper is resolved by a reading, tagged
 * R-xxx and stated where it is applied:
 *
 *   pass 1  (per node)  enthalpy recovery, Eq. (28) with the lagged source
 *           (reading R-IMP), and the liquid-fraction/temperature inversion
 *           of Eq. (8) generalised to a material weight w (R-T1); the mass
 *           source mdot = (1-rho_s/rho_l) dfs/dt of Eq. (1) from the change of
 *           fl (R-DT); the order parameter of Eq. (22) solved for phi
 *           (R-IMP, R-DIV); the material weight and the solid fraction; the
 *           property interpolation of Eq. (10).
 *   pass 2  (per node, reads neighbours of pass-1 fields)  isotropic finite
 *           differences (R-FD) for grad/Laplacian; chemical potential Eq. (6);
 *           surface tension F_s = mu_phi grad(phi) (Sec. 2); velocity and
 *           pressure Eq. (17a-c) with the penalty force f = f_s(u_s-u*)/dt;
 *           BGK collision of the flow populations Eqs. (11),(14)-(16);
 *           BGK collision of the phase populations Eqs. (18)-(21); TRT
 *           collision of the enthalpy populations Eqs. (23)-(27) (R-TRT,
 *           R-HEQ, R-HS).
 *   pass 3  streaming with periodic wrap or half-way bounce-back walls; the
 *           enthalpy populations use anti-bounce-back at Dirichlet walls and
 *           bounce-back at adiabatic walls (R-BC).
 *   pass 4  cold-mask reset: enthalpy populations of masked nodes are set to
 *           the equilibrium at the mask temperature with u = 0 (R-BC).
 *   pass 5  store the lag fields fl, w, p, phi*u, Q = rho Cp T mdot.
 *
 * Lattice: D2Q9 of Eq. (12) with weights 4/9, 1/9, 1/36 (Sec. 3.1),
 * dx = dt = 1, cs^2 = 1/3, T_m = 0.
 *
 * Pins: every routine here is checked by tests/test_oracle_*.py against
 * closed forms and invariants the paper fixes (Neumann and Stefan solutions,
 * conservation, moment identities of the equilibria and sources, the
 * variational derivative of the free energy Eq. (4), equilibrium contact
 * angle).  Parity unpinned: the lagged pressure inside grad(p) of the
 * modified force (reading R-FP) and the ice-water contact angle psi
 * (reading R-PSI) have no independent check beyond the physical pins.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define NQ 9
#define BC_PERIODIC 0
#define BC_DIRICHLET 1
#define BC_ADIABATIC 2
#define LAT_FLOW 1u
#define LAT_PHASE 2u
#define LAT_HEAT 4u
#define READ_FT_ISOTROPIC_S 1u /* variant of the modified force, reading R-FT */

/* D2Q9 velocities in the order of Eq. (12): rest, the four axes
 * counter-clockwise from +x, then the four diagonals from (1,1). */
static const int CX[NQ] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int CY[NQ] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const double WQ[NQ] = {4.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0,
                              1.0 / 9.0,  1.0 / 9.0,  1.0 / 36.0,
                              1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
static const int OPP[NQ] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
static const double CS2 = 1.0 / 3.0;

typedef struct {
  int32_t nx, ny;
  uint32_t lattices;
  int32_t bc[4]; /* x-low, x-high, y-low, y-high */
  double T_wall[4];
  double rho_l, rho_s, rho_g;
  double mu_l, mu_s, mu_g;
  double lambda_l, lambda_s, lambda_g;
  double cp_l, cp_s, cp_g;
  double rho_ref, latent;
  double sigma, eps, mobility, eta;
  double theta_deg, psi_deg;
  double gx, gy;
  double T_cold;
  uint32_t readings;
} oracle_params;

typedef struct {
  oracle_params p;
  long N;
  double cos_theta, cos_psi;
  double rr; /* rho_ref * Cp_ref, Cp_ref = 2 Cp_s Cp_l / (Cp_s + Cp_l), Eq. (25) */
  double tau_g;
  int64_t step;
  /* state: pre-collision populations [q*N + n] and lag fields */
  double *f, *g, *h;
  double *fl_prev, *w_prev, *p_prev, *phux_prev, *phuy_prev, *Q_prev;
  /* static geometry */
  double* phi0;
  uint8_t* mask;
  /* scratch: post-collision populations */
  double *fp, *gp, *hp;
  /* per-node fields of the current step */
  double *T, *fl, *mdot, *rhoH, *phi, *w, *fs, *rho, *mu, *lam, *cp;
  double *ux, *uy, *pr, *muphi, *phux, *phuy;
} oracle_sim;

/* ------------------------------------------------------------------ */
/* local (per-node) building blocks                                     */
/* ------------------------------------------------------------------ */

static double clamp01(double v) { return v < 0.0 ? 0.0 : (v > 1.0 ? 1.0 : v); }

/* Eq. (10): zeta = fs zeta_s + (1-fs) w zeta_l + (1-fs)(1-w) zeta_g, with
 * w = (1 - phi0 + phi)/2 the liquid weight of the paper. */
static double interp(double fs, double w, double zs, double zl, double zg) {
  return fs * zs + (1.0 - fs) * w * zl + (1.0 - fs) * (1.0 - w) * zg;
}

/* Volumetric heat capacity rho*Cp at solid fraction fs and weight w, with
 * rho and Cp each interpolated by Eq. (10). */
static double heat_capacity(const oracle_params* p, double fs, double w) {
  return interp(fs, w, p->rho_s, p->rho_l, p->rho_g) *
         interp(fs, w, p->cp_s, p->cp_l, p->cp_g);
}

/* Eq. (8) with T_m = T_s = T_l = 0, rho_s H_s = 0 and rho_l H_l = rho_l L,
 * generalised by reading R-T1: the latent capacity of a node is w rho_l L
 * (gas and the pre-existing solid carry no latent heat); below the solidus
 * the sensible capacity is rho Cp at the fully frozen state
 * fs = min(phi0 + w, 1), above the liquidus at the fully liquid state
 * fs = phi0.  Ties go to the mushy branch (R-TIE); a node without latent
 * capacity at exactly rhoH = 0 is counted as liquid. */
static void invert_enthalpy(const oracle_params* p, double rhoH, double w,
                            double phi0, double* T, double* fl) {
  double ell = w * p->rho_l * p->latent;
  double fs_frozen = phi0 + w;
  if (fs_frozen > 1.0) fs_frozen = 1.0;
  double c_minus = heat_capacity(p, fs_frozen, w);
  double c_plus = heat_capacity(p, phi0, w);
  if (rhoH < 0.0) {
    *fl = 0.0;
    *T = rhoH / c_minus;
  } else if (rhoH > ell) {
    *fl = 1.0;
    *T = (rhoH - ell) / c_plus;
  } else {
    *T = 0.0;
    *fl = ell > 0.0 ? rhoH / ell : 1.0;
  }
  *fl = clamp01(*fl);
}

/* Inverse of the inversion at a given temperature and liquid fraction,
 * used only to build initial states and the cold-mask equilibrium. */
static double enthalpy_of(const oracle_params* p, double T, double fl,
                          double w, double phi0) {
  double ell = w * p->rho_l * p->latent;
  double fs_frozen = phi0 + w;
  if (fs_frozen > 1.0) fs_frozen = 1.0;
  double c = T < 0.0 ? heat_capacity(p, fs_frozen, w) : heat_capacity(p, phi0, w);
  return c * T + ell * fl;
}

/* Eq. (15) */
static double s_i(int i, double ux, double uy) {
  double cu = CX[i] * ux + CY[i] * uy;
  double uu = ux * ux + uy * uy;
  return WQ[i] * (cu / CS2 + cu * cu / (2.0 * CS2 * CS2) - uu / (2.0 * CS2));
}

/* Eq. (14): pressure-based flow equilibrium. */
static void flow_equilibrium(double pr, double rho, double ux, double uy,
                             double* out) {
  for (int i = 0; i < NQ; i++)
    out[i] = pr / CS2 * (WQ[i] - (i == 0 ? 1.0 : 0.0)) + rho * s_i(i, ux, uy);
}

/* Eq. (16) with F_tilde = F - grad(p - cs^2 rho) (reading R-FT drops the
 * scalar "+cs^2 S"; the variant bit adds cs^2 S I to the tensor instead). */
static void flow_forcing(double S, double Fx, double Fy, double rho,
                         double fpx, double fpy, double ux, double uy,
                         double Ftx, double Fty, uint32_t readings,
                         double* out) {
  double uFt = ux * Ftx + uy * Fty;
  for (int i = 0; i < NQ; i++) {
    double cF = CX[i] * (Fx + rho * fpx) + CY[i] * (Fy + rho * fpy);
    double cu = CX[i] * ux + CY[i] * uy;
    double cFt = CX[i] * Ftx + CY[i] * Fty;
    /* (u Ft + Ft u) : (c c - cs^2 I) = 2 (c.u)(c.Ft) - 2 cs^2 u.Ft */
    double tens = 2.0 * cu * cFt - 2.0 * CS2 * uFt;
    if (readings & READ_FT_ISOTROPIC_S) {
      double cc = (double)(CX[i] * CX[i] + CY[i] * CY[i]);
      tens += CS2 * S * (cc - 2.0 * CS2);
    }
    out[i] = WQ[i] * (S + cF / CS2 + tens / (2.0 * CS2 * CS2));
  }
}

/* Eq. (19), with the mobility factor eta carried on mu_phi (reading R-ETA). */
static void phase_equilibrium(double phi, double muphi, double eta,
                              double phux, double phuy, double* out) {
  out[0] = phi + (WQ[0] - 1.0) * eta * muphi;
  for (int i = 1; i < NQ; i++)
    out[i] = WQ[i] * eta * muphi + WQ[i] * (CX[i] * phux + CY[i] * phuy) / CS2;
}

/* Eq. (20) with d(phi u)/dt a backward difference (R-DT) and div u = mdot
 * (R-DIV). */
static void phase_source(double dphux, double dphuy, double phi, double mdot,
                         double* out) {
  for (int i = 0; i < NQ; i++)
    out[i] = WQ[i] * (CX[i] * dphux + CY[i] * dphuy) / CS2 + WQ[i] * phi * mdot;
}

/* Eq. (25) with rho_ref Cp_ref T in the rest population (reading R-HEQ). */
static void heat_equilibrium(double rhoH, double C, double T, double rr,
                             double ux, double uy, double* out) {
  double uu = ux * ux + uy * uy;
  out[0] = rhoH - rr * T + WQ[0] * C * T * (rr / C - uu / (2.0 * CS2));
  for (int i = 1; i < NQ; i++) {
    double cu = CX[i] * ux + CY[i] * uy;
    out[i] = WQ[i] * C * T *
             (rr / C + cu / CS2 + (cu * cu - CS2 * uu) / (2.0 * CS2 * CS2));
  }
}

/* Source of Eq. (23): H_i = w_i rho Cp T div u with div u = mdot (R-HS). */
static void heat_source(double C, double T, double mdot, double* out) {
  for (int i = 0; i < NQ; i++) out[i] = WQ[i] * C * T * mdot;
}

/* Eq. (6) without its three Laplacian terms. */
static double chem_pot_local(const oracle_params* p, double cth, double cps,
                             double phi, double phi0, double fs) {
  double s = p->sigma, e = p->eps;
  return 3.0 * s / e * phi * (phi - 1.0) * (phi + 1.0) +
         9.0 * s / e * phi0 * phi0 * phi +
         3.0 * s * cth / e * phi0 * (3.0 * phi * phi + phi0 * phi0 - 1.0) +
         9.0 * s / e * fs * fs * phi +
         3.0 * s * cps / e * fs * (3.0 * phi * phi + fs * fs - 1.0);
}

/* ------------------------------------------------------------------ */
/* grid helpers                                                        */
/* ------------------------------------------------------------------ */

/* Neighbour coordinate for the finite-difference stencils: periodic axes
 * wrap, wall axes mirror the boundary node (zero normal gradient, R-BC). */
static int stencil_coord(int c, int n, int bc_lo, int bc_hi) {
  if (c < 0) return bc_lo == BC_PERIODIC ? c + n : 0;
  if (c >= n) return bc_hi == BC_PERIODIC ? c - n : n - 1;
  return c;
}

static void neighbours(const oracle_sim* s, int x, int y, long* nb) {
  const oracle_params* p = &s->p;
  for (int i = 0; i < NQ; i++) {
    int xx = stencil_coord(x + CX[i], p->nx, p->bc[0], p->bc[1]);
    int yy = stencil_coord(y + CY[i], p->ny, p->bc[2], p->bc[3]);
    nb[i] = (long)yy * p->nx + xx;
  }
}

/* Isotropic stencils (reading R-FD):
 *   grad chi = sum_i w_i c_i chi(x + c_i) / cs^2
 *   lap chi  = sum_i 2 w_i (chi(x + c_i) - chi(x)) / cs^2             */
static void grad(const double* a, const long* nb, double* gx, double* gy) {
  double sx = 0.0, sy = 0.0;
  for (int i = 1; i < NQ; i++) {
    sx += WQ[i] * CX[i] * a[nb[i]];
    sy += WQ[i] * CY[i] * a[nb[i]];
  }
  *gx = sx / CS2;
  *gy = sy / CS2;
}

static double lap(const double* a, const long* nb) {
  double s = 0.0;
  for (int i = 1; i < NQ; i++) s += 2.0 * WQ[i] * (a[nb[i]] - a[nb[0]]);
  return s / CS2;
}

/* ------------------------------------------------------------------ */
/* passes                                                              */
/* ------------------------------------------------------------------ */

/* Pass 1: enthalpy, liquid fraction, mass source, order parameter,
 * material weight, solid fraction and properties of every node. */
static void pass_local(oracle_sim* s) {
  const oracle_params* p = &s->p;
  const long N = s->N;
  const int flow = (p->lattices & LAT_FLOW) != 0;
  const int phase = (p->lattices & LAT_PHASE) != 0;
  const int heat = (p->lattices & LAT_HEAT) != 0;
  (void)flow;
#pragma omp parallel for schedule(static)
  for (long n = 0; n < N; n++) {
    double phi0 = s->phi0[n];
    double wp = s->w_prev[n], flp = s->fl_prev[n];
    double T = 0.0, fl = flp, rhoH = 0.0, mdot = 0.0;
    if (heat) {
      double sh = 0.0;
      for (int i = 0; i < NQ; i++) sh += s->h[i * N + n];
      rhoH = sh + 0.5 * s->Q_prev[n]; /* Eq. (28), lagged source */
      invert_enthalpy(p, rhoH, wp, phi0, &T, &fl);
      /* Eq. (1): mdot = (1 - rho_s/rho_l) dfs/dt, the phase-change part of
       * dfs/dt with fs = phi0 + w (1 - fl) (R-T1, R-DT). */
      mdot = (1.0 - p->rho_s / p->rho_l) * wp * (flp - fl);
    }
    double phi, w;
    if (phase) {
      double sg = 0.0;
      for (int i = 0; i < NQ; i++) sg += s->g[i * N + n];
      phi = sg / (1.0 - 0.5 * mdot); /* Eq. (22) solved for phi */
      w = clamp01((1.0 - phi0 + phi) / 2.0);
    } else {
      w = wp;
      phi = 2.0 * wp - 1.0 + phi0;
    }
    double fs = phi0 + w * (1.0 - fl);
    if (fs > 1.0) fs = 1.0;
    s->T[n] = T;
    s->fl[n] = fl;
    s->mdot[n] = mdot;
    s->rhoH[n] = rhoH;
    s->phi[n] = phi;
    s->w[n] = w;
    s->fs[n] = fs;
    s->rho[n] = interp(fs, w, p->rho_s, p->rho_l, p->rho_g);
    s->mu[n] = interp(fs, w, p->mu_s, p->mu_l, p->mu_g);
    s->lam[n] = interp(fs, w, p->lambda_s, p->lambda_l, p->lambda_g);
    s->cp[n] = interp(fs, w, p->cp_s, p->cp_l, p->cp_g);
  }
}

/* Pass 2: stencils, chemical potential, forces, macroscopic velocity and
 * pressure; with collide != 0 also the three collisions into fp, gp, hp. */
static void pass_collide(oracle_sim* s, int collide) {
  const oracle_params* p = &s->p;
  const long N = s->N;
  const int nx = p->nx, ny = p->ny;
  const int flow = (p->lattices & LAT_FLOW) != 0;
  const int phase = (p->lattices & LAT_PHASE) != 0;
  const int heat = (p->lattices & LAT_HEAT) != 0;
#pragma omp parallel for schedule(static)
  for (int y = 0; y < ny; y++) {
    for (int x = 0; x < nx; x++) {
      long n = (long)y * nx + x;
      long nb[NQ];
      neighbours(s, x, y, nb);
      double phi = s->phi[n], fs = s->fs[n], rho = s->rho[n];
      double T = s->T[n], mdot = s->mdot[n], rhoH = s->rhoH[n];

      /* Eq. (6) and F_s = mu_phi grad(phi) (Sec. 2) */
      double muphi = 0.0, Fsx = 0.0, Fsy = 0.0;
      if (phase) {
        double gphx, gphy;
        grad(s->phi, nb, &gphx, &gphy);
        muphi = chem_pot_local(p, s->cos_theta, s->cos_psi, phi, s->phi0[n], fs) -
                3.0 * p->eps * p->sigma / 8.0 *
                    (lap(s->phi, nb) + s->cos_theta * lap(s->phi0, nb) +
                     s->cos_psi * lap(s->fs, nb));
        Fsx = muphi * gphx;
        Fsy = muphi * gphy;
      }
      /* total force F = F_s + G with G = rho g */
      double Fx = Fsx + rho * p->gx, Fy = Fsy + rho * p->gy;

      double ux = 0.0, uy = 0.0, pr = 0.0;
      if (flow) {
        double jx = 0.0, jy = 0.0, snz = 0.0;
        for (int i = 0; i < NQ; i++) {
          double fi = s->f[i * N + n];
          jx += CX[i] * fi;
          jy += CY[i] * fi;
          if (i > 0) snz += fi;
        }
        /* Eq. (17a,b) with f = fs (u_s - u*)/dt and u_s = 0 */
        double usx = (jx + 0.5 * Fx) / rho, usy = (jy + 0.5 * Fy) / rho;
        double fpx = fs * (0.0 - usx), fpy = fs * (0.0 - usy);
        ux = usx + 0.5 * fpx;
        uy = usy + 0.5 * fpy;
        double grx, gry, gpx, gpy;
        grad(s->rho, nb, &grx, &gry);
        grad(s->p_prev, nb, &gpx, &gpy); /* lagged pressure, R-FP */
        double S = rho * mdot + ux * grx + uy * gry;
        double Ftx = Fx - (gpx - CS2 * grx), Fty = Fy - (gpy - CS2 * gry);
        double tauf = s->mu[n] / (rho * CS2) + 0.5; /* Sec. 3.1 */
        double Fi[NQ];
        flow_forcing(S, Fx, Fy, rho, fpx, fpy, ux, uy, Ftx, Fty, p->readings, Fi);
        /* Eq. (17c) */
        pr = CS2 / (1.0 - WQ[0]) *
             (snz + 0.5 * S + (tauf - 0.5) * Fi[0] + rho * s_i(0, ux, uy));
        if (collide) {
          double feq[NQ];
          flow_equilibrium(pr, rho, ux, uy, feq);
          for (int i = 0; i < NQ; i++) {
            double fi = s->f[i * N + n];
            /* Eq. (11) */
            s->fp[i * N + n] = fi - (fi - feq[i]) / tauf + (1.0 - 1.0 / (2.0 * tauf)) * Fi[i];
          }
        }
      }
      double phux = phi * ux, phuy = phi * uy;
      if (phase && collide) {
        double geq[NQ], Gi[NQ];
        phase_equilibrium(phi, muphi, p->eta, phux, phuy, geq);
        phase_source(phux - s->phux_prev[n], phuy - s->phuy_prev[n], phi, mdot, Gi);
        double tg = s->tau_g;
        for (int i = 0; i < NQ; i++) {
          double gi = s->g[i * N + n];
          /* Eq. (18) */
          s->gp[i * N + n] = gi - (gi - geq[i]) / tg + (1.0 - 1.0 / (2.0 * tg)) * Gi[i];
        }
      }
      if (heat && collide) {
        double C = rho * s->cp[n];
        /* Eq. (26) with rho_ref Cp_ref (R-HEQ) and Eq. (27) */
        double taua = 0.5 + s->lam[n] / (s->rr * CS2);
        double taus = taua / (2.0 * taua - 1.0);
        double heq[NQ], Hi[NQ], hh[NQ];
        heat_equilibrium(rhoH, C, T, s->rr, ux, uy, heq);
        heat_source(C, T, mdot, Hi);
        for (int i = 0; i < NQ; i++) hh[i] = s->h[i * N + n];
        for (int i = 0; i < NQ; i++) {
          int o = OPP[i];
          /* Eq. (24) */
          double hs = 0.5 * (hh[i] + hh[o]), ha = 0.5 * (hh[i] - hh[o]);
          double eqs = 0.5 * (heq[i] + heq[o]), eqa = 0.5 * (heq[i] - heq[o]);
          /* Eq. (23), symmetric part relaxed with tau_s (R-TRT) */
          s->hp[i * N + n] = hh[i] - (ha - eqa) / taua - (hs - eqs) / taus +
                             (1.0 - 1.0 / (2.0 * taua)) * Hi[i];
        }
      }
      s->ux[n] = ux;
      s->uy[n] = uy;
      s->pr[n] = pr;
      s->muphi[n] = muphi;
      s->phux[n] = phux;
      s->phuy[n] = phuy;
    }
  }
}

/* Pass 3: streaming.  A population leaving through a wall returns to its
 * node in the opposite direction (half-way bounce-back); for h at a
 * Dirichlet wall the anti-bounce-back h_opp = -h* + 2 w_i rho_ref Cp_ref T_w.
 * When a diagonal leaves through a corner, the x wall decides. */
static void pass_stream(oracle_sim* s) {
  const oracle_params* p = &s->p;
  const long N = s->N;
  const int nx = p->nx, ny = p->ny;
  const int flow = (p->lattices & LAT_FLOW) != 0;
  const int phase = (p->lattices & LAT_PHASE) != 0;
  const int heat = (p->lattices & LAT_HEAT) != 0;
#pragma omp parallel for schedule(static)
  for (int y = 0; y < ny; y++) {
    for (int x = 0; x < nx; x++) {
      long n = (long)y * nx + x;
      for (int i = 0; i < NQ; i++) {
        int tx = x + CX[i], ty = y + CY[i];
        int wall = -1; /* index into bc[] of the wall that is hit */
        if (tx < 0) {
          if (p->bc[0] == BC_PERIODIC) tx += nx; else wall = 0;
        } else if (tx >= nx) {
          if (p->bc[1] == BC_PERIODIC) tx -= nx; else wall = 1;
        }
        if (wall < 0) {
          if (ty < 0) {
            if (p->bc[2] == BC_PERIODIC) ty += ny; else wall = 2;
          } else if (ty >= ny) {
            if (p->bc[3] == BC_PERIODIC) ty -= ny; else wall = 3;
          }
        }
        if (wall >= 0) {
          long dst = (long)OPP[i] * N + n;
          if (flow) s->f[dst] = s->fp[i * N + n];
          if (phase) s->g[dst] = s->gp[i * N + n];
          if (heat) {
            if (p->bc[wall] == BC_DIRICHLET)
              s->h[dst] = -s->hp[i * N + n] + 2.0 * WQ[i] * s->rr * p->T_wall[wall];
            else
              s->h[dst] = s->hp[i * N + n];
          }
        } else {
          long dst = (long)i * N + (long)ty * nx + tx;
          if (flow) s->f[dst] = s->fp[i * N + n];
          if (phase) s->g[dst] = s->gp[i * N + n];
          if (heat) s->h[dst] = s->hp[i * N + n];
        }
      }
    }
  }
}

/* Pass 4: cold mask, enthalpy populations of masked nodes reset to the
 * equilibrium at T_cold with u = 0, using the node's current weight. */
static void pass_mask(oracle_sim* s, const double* wcur) {
  const oracle_params* p = &s->p;
  const long N = s->N;
  if (!(p->lattices & LAT_HEAT)) return;
  for (long n = 0; n < N; n++) {
    if (!s->mask[n]) continue;
    double T = p->T_cold;
    double fl = T < 0.0 ? 0.0 : 1.0;
    double rhoH = enthalpy_of(p, T, fl, wcur[n], s->phi0[n]);
    double fs = s->phi0[n] + wcur[n] * (1.0 - fl);
    if (fs > 1.0) fs = 1.0;
    double C = heat_capacity(p, fs, wcur[n]);
    double heq[NQ];
    heat_equilibrium(rhoH, C, T, s->rr, 0.0, 0.0, heq);
    for (int i = 0; i < NQ; i++) s->h[i * N + n] = heq[i];
  }
}

/* Pass 5: lag fields for the next step. */
static void pass_lag(oracle_sim* s) {
  const oracle_params* p = &s->p;
  const long N = s->N;
  const int flow = (p->lattices & LAT_FLOW) != 0;
  const int phase = (p->lattices & LAT_PHASE) != 0;
  const int heat = (p->lattices & LAT_HEAT) != 0;
  for (long n = 0; n < N; n++) {
    s->fl_prev[n] = s->fl[n];
    s->w_prev[n] = s->w[n];
    s->p_prev[n] = flow ? s->pr[n] : 0.0;
    s->phux_prev[n] = phase ? s->phux[n] : 0.0;
    s->phuy_prev[n] = phase ? s->phuy[n] : 0.0;
    s->Q_prev[n] = heat ? s->rho[n] * s->cp[n] * s->T[n] * s->mdot[n] : 0.0;
  }
}

/* ------------------------------------------------------------------ */
/* public interface (ctypes)                                           */
/* ------------------------------------------------------------------ */

static int params_valid(const oracle_params* p) {
  if (p->nx < 2 || p->ny < 2) return 0;
  for (int k = 0; k < 4; k++)
    if (p->bc[k] < BC_PERIODIC || p->bc[k] > BC_ADIABATIC) return 0;
  if ((p->bc[0] == BC_PERIODIC) != (p->bc[1] == BC_PERIODIC)) return 0;
  if ((p->bc[2] == BC_PERIODIC) != (p->bc[3] == BC_PERIODIC)) return 0;
  if (!(p->rho_l > 0 && p->rho_s > 0 && p->rho_g > 0)) return 0;
  if (!(p->cp_l > 0 && p->cp_s > 0 && p->cp_g > 0 && p->rho_ref > 0)) return 0;
  if (!(p->mu_l > 0 && p->mu_s > 0 && p->mu_g > 0)) return 0;
  if (!(p->lambda_l > 0 && p->lambda_s > 0 && p->lambda_g > 0)) return 0;
  if (!(p->mobility > 0 && p->eta > 0 && p->eps > 0 && p->latent >= 0)) return 0;
  return 1;
}

oracle_sim* oracle_create(const oracle_params* prm) {
  if (!params_valid(prm)) return NULL;
  oracle_sim* s = (oracle_sim*)calloc(1, sizeof(oracle_sim));
  s->p = *prm;
  s->N = (long)prm->nx * prm->ny;
  const double pi = 3.14159265358979323846;
  s->cos_theta = cos(prm->theta_deg * pi / 180.0);
  s->cos_psi = cos(prm->psi_deg * pi / 180.0);
  double cp_ref = 2.0 * prm->cp_s * prm->cp_l / (prm->cp_s + prm->cp_l);
  s->rr = prm->rho_ref * cp_ref;
  s->tau_g = 0.5 + prm->mobility / (prm->eta * CS2); /* Eq. (21) */
  long N = s->N;
  double** pops[] = {&s->f, &s->g, &s->h, &s->fp, &s->gp, &s->hp};
  for (int k = 0; k < 6; k++) *pops[k] = (double*)calloc((size_t)NQ * N, sizeof(double));
  double** flds[] = {&s->fl_prev, &s->w_prev, &s->p_prev, &s->phux_prev, &s->phuy_prev,
                     &s->Q_prev,  &s->phi0,   &s->T,      &s->fl,        &s->mdot,
                     &s->rhoH,    &s->phi,    &s->w,      &s->fs,        &s->rho,
                     &s->mu,      &s->lam,    &s->cp,     &s->ux,        &s->uy,
                     &s->pr,      &s->muphi,  &s->phux,   &s->phuy};
  for (size_t k = 0; k < sizeof(flds) / sizeof(flds[0]); k++)
    *flds[k] = (double*)calloc((size_t)N, sizeof(double));
  s->mask = (uint8_t*)calloc((size_t)N, 1);
  return s;
}

void oracle_destroy(oracle_sim* s) {
  if (!s) return;
  double* all[] = {s->f,     s->g,       s->h,         s->fp,         s->gp,
                   s->hp,    s->fl_prev, s->w_prev,    s->p_prev,     s->phux_prev,
                   s->phuy_prev, s->Q_prev, s->phi0,   s->T,          s->fl,
                   s->mdot,  s->rhoH,    s->phi,       s->w,          s->fs,
                   s->rho,   s->mu,      s->lam,       s->cp,         s->ux,
                   s->uy,    s->pr,      s->muphi,     s->phux,       s->phuy};
  for (size_t k = 0; k < sizeof(all) / sizeof(all[0]); k++) free(all[k]);
  free(s->mask);
  free(s);
}

/* Initial state (no passage in the paper; the build's choice U4):
 * lag fields fl = fl0, w = w0, p = 0, phi u = 0, Q = 0; f = f_eq(p=0,u=0)
 * = 0; g = g_eq(phi0, mu_phi0, u=0); h = h_eq(rhoH0, T0, u=0) with
 * rhoH0 from the inverse of the inversion; then the cold-mask reset. */
void oracle_init(oracle_sim* s, const double* phi0, const uint8_t* mask,
                 const double* phi_init, const double* T_init,
                 const double* fl_init) {
  const oracle_params* p = &s->p;
  const long N = s->N;
  s->step = 0;
  for (long n = 0; n < N; n++) {
    s->phi0[n] = phi0[n];
    s->mask[n] = mask ? (mask[n] != 0) : 0;
    double w = clamp01((1.0 - phi0[n] + phi_init[n]) / 2.0);
    double fl = clamp01(fl_init[n]);
    double fs = phi0[n] + w * (1.0 - fl);
    if (fs > 1.0) fs = 1.0;
    s->phi[n] = phi_init[n];
    s->w[n] = w;
    s->fs[n] = fs;
    s->fl[n] = fl;
    s->T[n] = T_init[n];
    s->rho[n] = interp(fs, w, p->rho_s, p->rho_l, p->rho_g);
    s->cp[n] = interp(fs, w, p->cp_s, p->cp_l, p->cp_g);
    s->rhoH[n] = enthalpy_of(p, T_init[n], fl, w, phi0[n]);
    s->fl_prev[n] = fl;
    s->w_prev[n] = w;
    s->p_prev[n] = 0.0;
    s->phux_prev[n] = 0.0;
    s->phuy_prev[n] = 0.0;
    s->Q_prev[n] = 0.0;
  }
  for (int y = 0; y < p->ny; y++) {
    for (int x = 0; x < p->nx; x++) {
      long n = (long)y * p->nx + x;
      long nb[NQ];
      neighbours(s, x, y, nb);
      double eq[NQ];
      flow_equilibrium(0.0, s->rho[n], 0.0, 0.0, eq);
      for (int i = 0; i < NQ; i++) s->f[i * N + n] = eq[i];
      double muphi = chem_pot_local(p, s->cos_theta, s->cos_psi, s->phi[n], phi0[n], s->fs[n]) -
                     3.0 * p->eps * p->sigma / 8.0 *
                         (lap(s->phi, nb) + s->cos_theta * lap(s->phi0, nb) +
                          s->cos_psi * lap(s->fs, nb));
      phase_equilibrium(s->phi[n], muphi, p->eta, 0.0, 0.0, eq);
      for (int i = 0; i < NQ; i++) s->g[i * N + n] = eq[i];
      heat_equilibrium(s->rhoH[n], s->rho[n] * s->cp[n], s->T[n], s->rr, 0.0, 0.0, eq);
      for (int i = 0; i < NQ; i++) s->h[i * N + n] = eq[i];
    }
  }
  pass_mask(s, s->w_prev);
}

void oracle_step(oracle_sim* s, long nsteps) {
  for (long k = 0; k < nsteps; k++) {
    pass_local(s);
    pass_collide(s, 1);
    pass_stream(s);
    pass_mask(s, s->w);
    pass_lag(s);
    s->step++;
  }
}

/* Fields of the current state (passes 1-2 without collision). */
enum {
  OF_PHI = 0, OF_FS, OF_FL, OF_T, OF_RHOH, OF_P, OF_UX, OF_UY, OF_RHO, OF_MU, OF_W, OF_MDOT,
  OF_COUNT
};

void oracle_fields(oracle_sim* s, double* out /* [OF_COUNT][N] */) {
  const long N = s->N;
  pass_local(s);
  pass_collide(s, 0);
  const double* src[OF_COUNT] = {s->phi, s->fs, s->fl, s->T,   s->rhoH,  s->pr,
                                 s->ux,  s->uy, s->rho, s->muphi, s->w, s->mdot};
  for (int k = 0; k < OF_COUNT; k++) memcpy(out + (size_t)k * N, src[k], sizeof(double) * N);
}

/* Global FP64 diagnostics of the current state, summed in node order:
 * [0] sum rho, [1] material mass sum w (rho_s (1-fl) + rho_l fl),
 * [2] sum rhoH, [3] liquid volume sum w fl, [4] material volume sum w,
 * [5] frozen volume sum w (1 - fl), [6] sum phi, [7] kinetic energy
 * sum rho |u|^2 / 2, [8] number of nodes whose population sums are not
 * finite. */
void oracle_diagnostics(oracle_sim* s, double* d) {
  const oracle_params* p = &s->p;
  const long N = s->N;
  pass_local(s);
  pass_collide(s, 0);
  for (int k = 0; k < 9; k++) d[k] = 0.0;
  for (long n = 0; n < N; n++) {
    double w = s->w[n], fl = s->fl[n], rho = s->rho[n];
    d[0] += rho;
    d[1] += w * (p->rho_s * (1.0 - fl) + p->rho_l * fl);
    d[2] += s->rhoH[n];
    d[3] += w * fl;
    d[4] += w;
    d[5] += w * (1.0 - fl);
    d[6] += s->phi[n];
    d[7] += 0.5 * rho * (s->ux[n] * s->ux[n] + s->uy[n] * s->uy[n]);
    double tot = 0.0;
    for (int i = 0; i < NQ; i++) {
      if (p->lattices & LAT_FLOW) tot += s->f[i * N + n];
      if (p->lattices & LAT_PHASE) tot += s->g[i * N + n];
      if (p->lattices & LAT_HEAT) tot += s->h[i * N + n];
    }
    if (!isfinite(tot)) d[8] += 1.0;
  }
}

/* State access for tests: populations [3][9][N] (f, g, h) and lag fields
 * [6][N] (fl, w, p, phi ux, phi uy, Q). */
void oracle_get_state(const oracle_sim* s, double* pops, double* lags) {
  const long N = s->N;
  if (pops) {
    memcpy(pops, s->f, sizeof(double) * NQ * N);
    memcpy(pops + (size_t)NQ * N, s->g, sizeof(double) * NQ * N);
    memcpy(pops + (size_t)2 * NQ * N, s->h, sizeof(double) * NQ * N);
  }
  if (lags) {
    const double* src[6] = {s->fl_prev, s->w_prev, s->p_prev, s->phux_prev, s->phuy_prev, s->Q_prev};
    for (int k = 0; k < 6; k++) memcpy(lags + (size_t)k * N, src[k], sizeof(double) * N);
  }
}

void oracle_set_state(oracle_sim* s, const double* pops, const double* lags) {
  const long N = s->N;
  if (pops) {
    memcpy(s->f, pops, sizeof(double) * NQ * N);
    memcpy(s->g, pops + (size_t)NQ * N, sizeof(double) * NQ * N);
    memcpy(s->h, pops + (size_t)2 * NQ * N, sizeof(double) * NQ * N);
  }
  if (lags) {
    double* dst[6] = {s->fl_prev, s->w_prev, s->p_prev, s->phux_prev, s->phuy_prev, s->Q_prev};
    for (int k = 0; k < 6; k++) memcpy(dst[k], lags + (size_t)k * N, sizeof(double) * N);
  }
}

int64_t oracle_step_count(const oracle_sim* s) { return s->step; }

/* Number of OpenMP threads for the row loops (results do not depend on it:
 * every pass writes disjoint nodes and the reductions are serial). */
int oracle_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
  return omp_get_max_threads();
#else
  (void)n;
  return 1;
#endif
}

/* --- single-node entry points for the moment pins --- */

void oracle_lattice(int* cx, int* cy, double* w, int* opp) {
  for (int i = 0; i < NQ; i++) {
    cx[i] = CX[i];
    cy[i] = CY[i];
    w[i] = WQ[i];
    opp[i] = OPP[i];
  }
}

void oracle_node_flow(double pr, double rho, double ux, double uy, double S,
                      double Fx, double Fy, double fpx, double fpy,
                      double Ftx, double Fty, uint32_t readings,
                      double* feq, double* Fi) {
  flow_equilibrium(pr, rho, ux, uy, feq);
  flow_forcing(S, Fx, Fy, rho, fpx, fpy, ux, uy, Ftx, Fty, readings, Fi);
}

void oracle_node_phase(double phi, double muphi, double eta, double phux,
                       double phuy, double dphux, double dphuy, double mdot,
                       double* geq, double* Gi) {
  phase_equilibrium(phi, muphi, eta, phux, phuy, geq);
  phase_source(dphux, dphuy, phi, mdot, Gi);
}

void oracle_node_heat(double rhoH, double C, double T, double rr, double ux,
                      double uy, double mdot, double* heq, double* Hi) {
  heat_equilibrium(rhoH, C, T, rr, ux, uy, heq);
  heat_source(C, T, mdot, Hi);
}

/* TRT collision of one node's enthalpy populations, Eqs. (23)-(24). */
void oracle_node_trt(const double* hh, const double* heq, const double* Hi,
                     double taua, double taus, double* out) {
  for (int i = 0; i < NQ; i++) {
    int o = OPP[i];
    double hs = 0.5 * (hh[i] + hh[o]), ha = 0.5 * (hh[i] - hh[o]);
    double eqs = 0.5 * (heq[i] + heq[o]), eqa = 0.5 * (heq[i] - heq[o]);
    out[i] = hh[i] - (ha - eqa) / taua - (hs - eqs) / taus + (1.0 - 1.0 / (2.0 * taua)) * Hi[i];
  }
}

void oracle_invert(const oracle_params* p, const double* rhoH, const double* w,
                   const double* phi0, long n, double* T, double* fl) {
  for (long k = 0; k < n; k++) invert_enthalpy(p, rhoH[k], w[k], phi0[k], &T[k], &fl[k]);
}

/* Chemical potential Eq. (6) of given phi, phi0, fs fields on the grid of p
 * (with the stencil boundary handling of the step). */
void oracle_chemical_potential(const oracle_params* prm, const double* phi,
                               const double* phi0, const double* fs,
                               double* out) {
  oracle_sim* s = oracle_create(prm);
  if (!s) return;
  const long N = s->N;
  memcpy(s->phi, phi, sizeof(double) * N);
  memcpy(s->phi0, phi0, sizeof(double) * N);
  memcpy(s->fs, fs, sizeof(double) * N);
  for (int y = 0; y < prm->ny; y++)
    for (int x = 0; x < prm->nx; x++) {
      long n = (long)y * prm->nx + x, nb[NQ];
      neighbours(s, x, y, nb);
      out[n] = chem_pot_local(prm, s->cos_theta, s->cos_psi, phi[n], phi0[n], fs[n]) -
               3.0 * prm->eps * prm->sigma / 8.0 *
                   (lap(s->phi, nb) + s->cos_theta * lap(s->phi0, nb) +
                    s->cos_psi * lap(s->fs, nb));
    }
  oracle_destroy(s);
}
