/*
 * lbm_oracle3d.c -- plain FP64 CPU oracle of the three-dimensional form of
 * the coupled three-lattice LB method for three-phase freezing (arXiv
 * 2510.18688): the same model as lbm_oracle.c on the D3Q19 lattice that
 * Sec. 3.1 gives for three-dimensional problems (the rough-fracture case of
 * Sec. 4.5).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or
 * call this file: only the test-suite and the CPU-baseline leg of the
 * benchmark use it.  It shares no code, header, table or helper with the
 * CUDA library; the two meet only through seeded input arrays.
 *
 * The stages of one step are those of the two-dimensional oracle, with every
 * sum over the lattice taken over the 19 velocities of Sec. 3.1 and every
 * vector carrying a z component:
 *
 *   pass 1  enthalpy recovery Eq. (28) with the lagged source (R-IMP), the
 *           inversion of Eq. (8) with material weight w (R-T1), the mass
 *           source of Eq. (1) from the change of fl (R-DT), phi from
 *           Eq. (22) (R-IMP), w, fs and the properties of Eq. (10);
 *   pass 2  isotropic stencils (R-FD) built on the D3Q19 weights, Eq. (6),
 *           F_s = mu_phi grad(phi), Eq. (17a-c) with the penalty force, and
 *           the three collisions Eqs. (11), (14)-(16), (18)-(21), (23)-(27)
 *           with cs^2 = 1/3 and the D3Q19 weights;
 *   pass 3  streaming: periodic wrap or half-way bounce-back walls on each
 *           of the six faces; anti-bounce-back of h at Dirichlet walls,
 *           bounce-back at adiabatic walls (R-BC).  A link that leaves
 *           through an edge or a corner is decided by the first wall it
 *           crosses in the order x, y, z;
 *   pass 4  cold-mask reset of the enthalpy populations (R-BC);
 *   pass 5  lag fields fl, w, p, phi u (three components), Q.
 *
 * The one place where the dimension enters a formula beyond the lattice is
 * the trace of cs^2 I in the variant of the modified force (R-FT variant
 * bit): c.c - 3 cs^2 here, c.c - 2 cs^2 in two dimensions.
 *
 * Pins (tests/test_oracle3d.py): the moments of the D3Q19 lattice against
 * the table printed in Sec. 3.1; for fields uniform along z, the sums of the
 * populations over c_z reproduce the two-dimensional oracle (itself pinned
 * to the Neumann and Stefan solutions) for the phase-field and enthalpy
 * lattices exactly (the D3Q19 weights summed over c_z are the D2Q9 weights);
 * the flow lattice against the Poiseuille profile and Laplace's law for a
 * sphere; conservation of sum(phi) and of the rest state.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define NQ 19
#define BC_PERIODIC 0
#define BC_DIRICHLET 1
#define BC_ADIABATIC 2
#define LAT_FLOW 1u
#define LAT_PHASE 2u
#define LAT_HEAT 4u
#define READ_FT_ISOTROPIC_S 1u

/* D3Q19 of Sec. 3.1, Eq. (13), in the column order of its velocity matrix. */
static const int CX[NQ] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
static const int CY[NQ] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1};
static const int CZ[NQ] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};
static double WQ[NQ];
static int OPP[NQ];
static const double CS2 = 1.0 / 3.0;

static void lattice_setup(void) {
  for (int i = 0; i < NQ; i++) {
    int c2 = CX[i] * CX[i] + CY[i] * CY[i] + CZ[i] * CZ[i];
    WQ[i] = c2 == 0 ? 1.0 / 3.0 : (c2 == 1 ? 1.0 / 18.0 : 1.0 / 36.0);
    for (int j = 0; j < NQ; j++)
      if (CX[j] == -CX[i] && CY[j] == -CY[i] && CZ[j] == -CZ[i]) OPP[i] = j;
  }
}

typedef struct {
  int32_t nx, ny, nz;
  uint32_t lattices;
  int32_t bc[6]; /* x-low, x-high, y-low, y-high, z-low, z-high */
  double T_wall[6];
  double rho_l, rho_s, rho_g;
  double mu_l, mu_s, mu_g;
  double lambda_l, lambda_s, lambda_g;
  double cp_l, cp_s, cp_g;
  double rho_ref, latent;
  double sigma, eps, mobility, eta;
  double theta_deg, psi_deg;
  double gx, gy, gz;
  double T_cold;
  uint32_t readings;
} oracle3_params;

typedef struct {
  oracle3_params p;
  long N;
  double cos_theta, cos_psi, rr, tau_g;
  int64_t step;
  double *f, *g, *h;
  double *fl_prev, *w_prev, *p_prev, *phux_prev, *phuy_prev, *phuz_prev, *Q_prev;
  double* phi0;
  uint8_t* mask;
  double *fp, *gp, *hp;
  double *T, *fl, *mdot, *rhoH, *phi, *w, *fs, *rho, *mu, *lam, *cp;
  double *ux, *uy, *uz, *pr, *muphi, *phux, *phuy, *phuz;
} oracle3_sim;

/* ------------------------------------------------------------------ */
/* local building blocks (the two-dimensional oracle's, in 3-D)        */
/* ------------------------------------------------------------------ */

static double clamp01(double v) { return v < 0.0 ? 0.0 : (v > 1.0 ? 1.0 : v); }

/* Eq. (10) */
static double interp(double fs, double w, double zs, double zl, double zg) {
  return fs * zs + (1.0 - fs) * w * zl + (1.0 - fs) * (1.0 - w) * zg;
}

static double heat_capacity(const oracle3_params* p, double fs, double w) {
  return interp(fs, w, p->rho_s, p->rho_l, p->rho_g) * interp(fs, w, p->cp_s, p->cp_l, p->cp_g);
}

/* Eq. (8) with T_m = 0 and the latent capacity w rho_l L (R-T1). */
static void invert_enthalpy(const oracle3_params* p, double rhoH, double w, double phi0,
                            double* T, double* fl) {
  double ell = w * p->rho_l * p->latent;
  double fs_frozen = phi0 + w;
  if (fs_frozen > 1.0) fs_frozen = 1.0;
  if (rhoH < 0.0) {
    *fl = 0.0;
    *T = rhoH / heat_capacity(p, fs_frozen, w);
  } else if (rhoH > ell) {
    *fl = 1.0;
    *T = (rhoH - ell) / heat_capacity(p, phi0, w);
  } else {
    *T = 0.0;
    *fl = ell > 0.0 ? rhoH / ell : 1.0;
  }
  *fl = clamp01(*fl);
}

static double enthalpy_of(const oracle3_params* p, double T, double fl, double w, double phi0) {
  double fs_frozen = phi0 + w;
  if (fs_frozen > 1.0) fs_frozen = 1.0;
  double c = T < 0.0 ? heat_capacity(p, fs_frozen, w) : heat_capacity(p, phi0, w);
  return c * T + w * p->rho_l * p->latent * fl;
}

static double cdot(int i, double ax, double ay, double az) {
  return CX[i] * ax + CY[i] * ay + CZ[i] * az;
}

/* Eq. (15) */
static double s_i(int i, double ux, double uy, double uz) {
  double cu = cdot(i, ux, uy, uz), uu = ux * ux + uy * uy + uz * uz;
  return WQ[i] * (cu / CS2 + cu * cu / (2.0 * CS2 * CS2) - uu / (2.0 * CS2));
}

/* Eq. (14) */
static void flow_equilibrium(double pr, double rho, const double* u, double* out) {
  for (int i = 0; i < NQ; i++)
    out[i] = pr / CS2 * (WQ[i] - (i == 0 ? 1.0 : 0.0)) + rho * s_i(i, u[0], u[1], u[2]);
}

/* Eq. (16) with F_tilde = F - grad(p - cs^2 rho) (R-FT). */
static void flow_forcing(double S, const double* F, double rho, const double* fp,
                         const double* u, const double* Ft, uint32_t readings, double* out) {
  double uFt = u[0] * Ft[0] + u[1] * Ft[1] + u[2] * Ft[2];
  for (int i = 0; i < NQ; i++) {
    double cF = cdot(i, F[0] + rho * fp[0], F[1] + rho * fp[1], F[2] + rho * fp[2]);
    double cu = cdot(i, u[0], u[1], u[2]);
    double cFt = cdot(i, Ft[0], Ft[1], Ft[2]);
    double tens = 2.0 * cu * cFt - 2.0 * CS2 * uFt;
    if (readings & READ_FT_ISOTROPIC_S) {
      double cc = (double)(CX[i] * CX[i] + CY[i] * CY[i] + CZ[i] * CZ[i]);
      tens += CS2 * S * (cc - 3.0 * CS2);
    }
    out[i] = WQ[i] * (S + cF / CS2 + tens / (2.0 * CS2 * CS2));
  }
}

/* Eq. (19) (R-ETA) */
static void phase_equilibrium(double phi, double muphi, double eta, const double* phu,
                              double* out) {
  out[0] = phi + (WQ[0] - 1.0) * eta * muphi;
  for (int i = 1; i < NQ; i++)
    out[i] = WQ[i] * eta * muphi + WQ[i] * cdot(i, phu[0], phu[1], phu[2]) / CS2;
}

/* Eq. (20) (R-DT, R-DIV) */
static void phase_source(const double* dphu, double phi, double mdot, double* out) {
  for (int i = 0; i < NQ; i++)
    out[i] = WQ[i] * cdot(i, dphu[0], dphu[1], dphu[2]) / CS2 + WQ[i] * phi * mdot;
}

/* Eq. (25) (R-HEQ) */
static void heat_equilibrium(double rhoH, double C, double T, double rr, const double* u,
                             double* out) {
  double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  out[0] = rhoH - rr * T + WQ[0] * C * T * (rr / C - uu / (2.0 * CS2));
  for (int i = 1; i < NQ; i++) {
    double cu = cdot(i, u[0], u[1], u[2]);
    out[i] = WQ[i] * C * T * (rr / C + cu / CS2 + (cu * cu - CS2 * uu) / (2.0 * CS2 * CS2));
  }
}

/* R-HS */
static void heat_source(double C, double T, double mdot, double* out) {
  for (int i = 0; i < NQ; i++) out[i] = WQ[i] * C * T * mdot;
}

/* Eq. (6) without its Laplacian terms. */
static double chem_pot_local(const oracle3_params* p, double cth, double cps, double phi,
                             double phi0, double fs) {
  double s = p->sigma, e = p->eps;
  return 3.0 * s / e * phi * (phi - 1.0) * (phi + 1.0) + 9.0 * s / e * phi0 * phi0 * phi +
         3.0 * s * cth / e * phi0 * (3.0 * phi * phi + phi0 * phi0 - 1.0) +
         9.0 * s / e * fs * fs * phi + 3.0 * s * cps / e * fs * (3.0 * phi * phi + fs * fs - 1.0);
}

/* ------------------------------------------------------------------ */
/* grid helpers                                                        */
/* ------------------------------------------------------------------ */

static int stencil_coord(int c, int n, int bc_lo, int bc_hi) {
  if (c < 0) return bc_lo == BC_PERIODIC ? c + n : 0;
  if (c >= n) return bc_hi == BC_PERIODIC ? c - n : n - 1;
  return c;
}

static long node(const oracle3_params* p, int x, int y, int z) {
  return ((long)z * p->ny + y) * p->nx + x;
}

static void neighbours(const oracle3_sim* s, int x, int y, int z, long* nb) {
  const oracle3_params* p = &s->p;
  for (int i = 0; i < NQ; i++) {
    int xx = stencil_coord(x + CX[i], p->nx, p->bc[0], p->bc[1]);
    int yy = stencil_coord(y + CY[i], p->ny, p->bc[2], p->bc[3]);
    int zz = stencil_coord(z + CZ[i], p->nz, p->bc[4], p->bc[5]);
    nb[i] = node(p, xx, yy, zz);
  }
}

/* R-FD: grad chi = sum_i w_i c_i chi(x + c_i) / cs^2,
 *       lap chi  = sum_i 2 w_i (chi(x + c_i) - chi(x)) / cs^2 */
static void grad(const double* a, const long* nb, double* g) {
  double sx = 0.0, sy = 0.0, sz = 0.0;
  for (int i = 1; i < NQ; i++) {
    sx += WQ[i] * CX[i] * a[nb[i]];
    sy += WQ[i] * CY[i] * a[nb[i]];
    sz += WQ[i] * CZ[i] * a[nb[i]];
  }
  g[0] = sx / CS2;
  g[1] = sy / CS2;
  g[2] = sz / CS2;
}

static double lap(const double* a, const long* nb) {
  double s = 0.0;
  for (int i = 1; i < NQ; i++) s += 2.0 * WQ[i] * (a[nb[i]] - a[nb[0]]);
  return s / CS2;
}

/* ------------------------------------------------------------------ */
/* passes                                                              */
/* ------------------------------------------------------------------ */

static void pass_local(oracle3_sim* s) {
  const oracle3_params* p = &s->p;
  const long N = s->N;
  const int phase = (p->lattices & LAT_PHASE) != 0;
  const int heat = (p->lattices & LAT_HEAT) != 0;
#pragma omp parallel for schedule(static)
  for (long n = 0; n < N; n++) {
    double phi0 = s->phi0[n], wp = s->w_prev[n], flp = s->fl_prev[n];
    double T = 0.0, fl = flp, rhoH = 0.0, mdot = 0.0;
    if (heat) {
      double sh = 0.0;
      for (int i = 0; i < NQ; i++) sh += s->h[i * N + n];
      rhoH = sh + 0.5 * s->Q_prev[n];
      invert_enthalpy(p, rhoH, wp, phi0, &T, &fl);
      mdot = (1.0 - p->rho_s / p->rho_l) * wp * (flp - fl);
    }
    double phi, w;
    if (phase) {
      double sg = 0.0;
      for (int i = 0; i < NQ; i++) sg += s->g[i * N + n];
      phi = sg / (1.0 - 0.5 * mdot);
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

static void pass_collide(oracle3_sim* s, int collide) {
  const oracle3_params* p = &s->p;
  const long N = s->N;
  const int flow = (p->lattices & LAT_FLOW) != 0;
  const int phase = (p->lattices & LAT_PHASE) != 0;
  const int heat = (p->lattices & LAT_HEAT) != 0;
  const long rows = (long)p->nz * p->ny;
#pragma omp parallel for schedule(static)
  for (long r = 0; r < rows; r++) {
    const int z = (int)(r / p->ny), y = (int)(r % p->ny);
    for (int x = 0; x < p->nx; x++) {
      long n = node(p, x, y, z);
      long nb[NQ];
      neighbours(s, x, y, z, nb);
      double phi = s->phi[n], fs = s->fs[n], rho = s->rho[n];
      double T = s->T[n], mdot = s->mdot[n], rhoH = s->rhoH[n];
      double muphi = 0.0, Fs[3] = {0.0, 0.0, 0.0};
      if (phase) {
        double gph[3];
        grad(s->phi, nb, gph);
        muphi = chem_pot_local(p, s->cos_theta, s->cos_psi, phi, s->phi0[n], fs) -
                3.0 * p->eps * p->sigma / 8.0 *
                    (lap(s->phi, nb) + s->cos_theta * lap(s->phi0, nb) +
                     s->cos_psi * lap(s->fs, nb));
        for (int k = 0; k < 3; k++) Fs[k] = muphi * gph[k];
      }
      double F[3] = {Fs[0] + rho * p->gx, Fs[1] + rho * p->gy, Fs[2] + rho * p->gz};
      double u[3] = {0.0, 0.0, 0.0}, pr = 0.0;
      if (flow) {
        double j[3] = {0.0, 0.0, 0.0}, snz = 0.0;
        for (int i = 0; i < NQ; i++) {
          double fi = s->f[i * N + n];
          j[0] += CX[i] * fi;
          j[1] += CY[i] * fi;
          j[2] += CZ[i] * fi;
          if (i > 0) snz += fi;
        }
        /* Eq. (17a,b), penalty force with u_s = 0 */
        double us[3], fp[3];
        for (int k = 0; k < 3; k++) {
          us[k] = (j[k] + 0.5 * F[k]) / rho;
          fp[k] = fs * (0.0 - us[k]);
          u[k] = us[k] + 0.5 * fp[k];
        }
        double gr[3], gp[3];
        grad(s->rho, nb, gr);
        grad(s->p_prev, nb, gp); /* R-FP */
        double S = rho * mdot + u[0] * gr[0] + u[1] * gr[1] + u[2] * gr[2];
        double Ft[3];
        for (int k = 0; k < 3; k++) Ft[k] = F[k] - (gp[k] - CS2 * gr[k]);
        double tauf = s->mu[n] / (rho * CS2) + 0.5;
        double Fi[NQ];
        flow_forcing(S, F, rho, fp, u, Ft, p->readings, Fi);
        /* Eq. (17c) */
        pr = CS2 / (1.0 - WQ[0]) * (snz + 0.5 * S + (tauf - 0.5) * Fi[0] + rho * s_i(0, u[0], u[1], u[2]));
        if (collide) {
          double feq[NQ];
          flow_equilibrium(pr, rho, u, feq);
          for (int i = 0; i < NQ; i++) {
            double fi = s->f[i * N + n];
            s->fp[i * N + n] = fi - (fi - feq[i]) / tauf + (1.0 - 1.0 / (2.0 * tauf)) * Fi[i];
          }
        }
      }
      double phu[3] = {phi * u[0], phi * u[1], phi * u[2]};
      if (phase && collide) {
        double geq[NQ], Gi[NQ];
        double dphu[3] = {phu[0] - s->phux_prev[n], phu[1] - s->phuy_prev[n],
                          phu[2] - s->phuz_prev[n]};
        phase_equilibrium(phi, muphi, p->eta, phu, geq);
        phase_source(dphu, phi, mdot, Gi);
        double tg = s->tau_g;
        for (int i = 0; i < NQ; i++) {
          double gi = s->g[i * N + n];
          s->gp[i * N + n] = gi - (gi - geq[i]) / tg + (1.0 - 1.0 / (2.0 * tg)) * Gi[i];
        }
      }
      if (heat && collide) {
        double C = rho * s->cp[n];
        double taua = 0.5 + s->lam[n] / (s->rr * CS2);
        double taus = taua / (2.0 * taua - 1.0);
        double heq[NQ], Hi[NQ], hh[NQ];
        heat_equilibrium(rhoH, C, T, s->rr, u, heq);
        heat_source(C, T, mdot, Hi);
        for (int i = 0; i < NQ; i++) hh[i] = s->h[i * N + n];
        for (int i = 0; i < NQ; i++) {
          int o = OPP[i];
          double hs = 0.5 * (hh[i] + hh[o]), ha = 0.5 * (hh[i] - hh[o]);
          double eqs = 0.5 * (heq[i] + heq[o]), eqa = 0.5 * (heq[i] - heq[o]);
          s->hp[i * N + n] = hh[i] - (ha - eqa) / taua - (hs - eqs) / taus +
                             (1.0 - 1.0 / (2.0 * taua)) * Hi[i];
        }
      }
      s->ux[n] = u[0];
      s->uy[n] = u[1];
      s->uz[n] = u[2];
      s->pr[n] = pr;
      s->muphi[n] = muphi;
      s->phux[n] = phu[0];
      s->phuy[n] = phu[1];
      s->phuz[n] = phu[2];
    }
  }
}

/* Destination coordinate along one axis: wrapped, or -1 when the link
 * leaves through a wall of that axis. */
static int stream_coord(int t, int n, int bc_lo, int bc_hi, int* hit_lo) {
  *hit_lo = 0;
  if (t < 0) {
    if (bc_lo == BC_PERIODIC) return t + n;
    *hit_lo = 1;
    return -1;
  }
  if (t >= n) return bc_hi == BC_PERIODIC ? t - n : -1;
  return t;
}

static void pass_stream(oracle3_sim* s) {
  const oracle3_params* p = &s->p;
  const long N = s->N;
  const int flow = (p->lattices & LAT_FLOW) != 0;
  const int phase = (p->lattices & LAT_PHASE) != 0;
  const int heat = (p->lattices & LAT_HEAT) != 0;
  const int dims[3] = {p->nx, p->ny, p->nz};
  const long rows = (long)p->nz * p->ny;
#pragma omp parallel for schedule(static)
  for (long r = 0; r < rows; r++) {
    const int z = (int)(r / p->ny), y = (int)(r % p->ny);
    for (int x = 0; x < p->nx; x++) {
      long n = node(p, x, y, z);
      const int pos[3] = {x, y, z};
      for (int i = 0; i < NQ; i++) {
        const int c[3] = {CX[i], CY[i], CZ[i]};
        int t[3], wall = -1;
        for (int a = 0; a < 3 && wall < 0; a++) {
          int lo;
          t[a] = stream_coord(pos[a] + c[a], dims[a], p->bc[2 * a], p->bc[2 * a + 1], &lo);
          if (t[a] < 0) wall = 2 * a + (lo ? 0 : 1);
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
          long dst = (long)i * N + node(p, t[0], t[1], t[2]);
          if (flow) s->f[dst] = s->fp[i * N + n];
          if (phase) s->g[dst] = s->gp[i * N + n];
          if (heat) s->h[dst] = s->hp[i * N + n];
        }
      }
    }
  }
}

static void pass_mask(oracle3_sim* s, const double* wcur) {
  const oracle3_params* p = &s->p;
  const long N = s->N;
  if (!(p->lattices & LAT_HEAT)) return;
  const double zero[3] = {0.0, 0.0, 0.0};
  for (long n = 0; n < N; n++) {
    if (!s->mask[n]) continue;
    double T = p->T_cold;
    double fl = T < 0.0 ? 0.0 : 1.0;
    double rhoH = enthalpy_of(p, T, fl, wcur[n], s->phi0[n]);
    double fs = s->phi0[n] + wcur[n] * (1.0 - fl);
    if (fs > 1.0) fs = 1.0;
    double heq[NQ];
    heat_equilibrium(rhoH, heat_capacity(p, fs, wcur[n]), T, s->rr, zero, heq);
    for (int i = 0; i < NQ; i++) s->h[i * N + n] = heq[i];
  }
}

static void pass_lag(oracle3_sim* s) {
  const oracle3_params* p = &s->p;
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
    s->phuz_prev[n] = phase ? s->phuz[n] : 0.0;
    s->Q_prev[n] = heat ? s->rho[n] * s->cp[n] * s->T[n] * s->mdot[n] : 0.0;
  }
}

/* ------------------------------------------------------------------ */
/* public interface (ctypes)                                           */
/* ------------------------------------------------------------------ */

static int params_valid(const oracle3_params* p) {
  if (p->nx < 2 || p->ny < 2 || p->nz < 2) return 0;
  for (int k = 0; k < 6; k++)
    if (p->bc[k] < BC_PERIODIC || p->bc[k] > BC_ADIABATIC) return 0;
  for (int a = 0; a < 3; a++)
    if ((p->bc[2 * a] == BC_PERIODIC) != (p->bc[2 * a + 1] == BC_PERIODIC)) return 0;
  if (!(p->rho_l > 0 && p->rho_s > 0 && p->rho_g > 0)) return 0;
  if (!(p->cp_l > 0 && p->cp_s > 0 && p->cp_g > 0 && p->rho_ref > 0)) return 0;
  if (!(p->mu_l > 0 && p->mu_s > 0 && p->mu_g > 0)) return 0;
  if (!(p->lambda_l > 0 && p->lambda_s > 0 && p->lambda_g > 0)) return 0;
  if (!(p->mobility > 0 && p->eta > 0 && p->eps > 0 && p->latent >= 0)) return 0;
  return 1;
}

#define NFIELD_BUFS 27

/* The per-node arrays of a simulation (allocated and freed together). */
static void field_slots(oracle3_sim* s, double** slots[NFIELD_BUFS]) {
  double** all[NFIELD_BUFS] = {
      &s->fl_prev, &s->w_prev, &s->p_prev, &s->phux_prev, &s->phuy_prev, &s->phuz_prev,
      &s->Q_prev,  &s->phi0,   &s->T,      &s->fl,        &s->mdot,      &s->rhoH,
      &s->phi,     &s->w,      &s->fs,     &s->rho,       &s->mu,        &s->lam,
      &s->cp,      &s->ux,     &s->uy,     &s->uz,        &s->pr,        &s->muphi,
      &s->phux,    &s->phuy,   &s->phuz};
  for (int k = 0; k < NFIELD_BUFS; k++) slots[k] = all[k];
}

oracle3_sim* oracle3_create(const oracle3_params* prm) {
  lattice_setup();
  if (!params_valid(prm)) return NULL;
  oracle3_sim* s = (oracle3_sim*)calloc(1, sizeof(oracle3_sim));
  s->p = *prm;
  s->N = (long)prm->nx * prm->ny * prm->nz;
  const double pi = 3.14159265358979323846;
  s->cos_theta = cos(prm->theta_deg * pi / 180.0);
  s->cos_psi = cos(prm->psi_deg * pi / 180.0);
  s->rr = prm->rho_ref * (2.0 * prm->cp_s * prm->cp_l / (prm->cp_s + prm->cp_l));
  s->tau_g = 0.5 + prm->mobility / (prm->eta * CS2); /* Eq. (21) */
  const long N = s->N;
  double** pops[] = {&s->f, &s->g, &s->h, &s->fp, &s->gp, &s->hp};
  for (int k = 0; k < 6; k++) *pops[k] = (double*)calloc((size_t)NQ * N, sizeof(double));
  double** slots[NFIELD_BUFS];
  field_slots(s, slots);
  for (int k = 0; k < NFIELD_BUFS; k++) *slots[k] = (double*)calloc((size_t)N, sizeof(double));
  s->mask = (uint8_t*)calloc((size_t)N, 1);
  return s;
}

void oracle3_destroy(oracle3_sim* s) {
  if (!s) return;
  free(s->f); free(s->g); free(s->h); free(s->fp); free(s->gp); free(s->hp);
  double** slots[NFIELD_BUFS];
  field_slots(s, slots);
  for (int k = 0; k < NFIELD_BUFS; k++) free(*slots[k]);
  free(s->mask);
  free(s);
}

/* Initial state as in the two-dimensional oracle: lags fl0, w0, p = 0,
 * phi u = 0, Q = 0; f = f_eq(p = 0, u = 0) = 0; g = g_eq(phi0, mu_phi0);
 * h = h_eq(rhoH0, T0, u = 0); then the cold-mask reset.  Arrays are
 * [nz][ny][nx]. */
void oracle3_init(oracle3_sim* s, const double* phi0, const uint8_t* mask,
                  const double* phi_init, const double* T_init, const double* fl_init) {
  const oracle3_params* p = &s->p;
  const long N = s->N;
  const double zero[3] = {0.0, 0.0, 0.0};
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
    s->phux_prev[n] = s->phuy_prev[n] = s->phuz_prev[n] = 0.0;
    s->Q_prev[n] = 0.0;
  }
  for (int z = 0; z < p->nz; z++)
    for (int y = 0; y < p->ny; y++)
      for (int x = 0; x < p->nx; x++) {
        long n = node(p, x, y, z), nb[NQ];
        neighbours(s, x, y, z, nb);
        double eq[NQ];
        flow_equilibrium(0.0, s->rho[n], zero, eq);
        for (int i = 0; i < NQ; i++) s->f[i * N + n] = eq[i];
        double muphi = chem_pot_local(p, s->cos_theta, s->cos_psi, s->phi[n], phi0[n], s->fs[n]) -
                       3.0 * p->eps * p->sigma / 8.0 *
                           (lap(s->phi, nb) + s->cos_theta * lap(s->phi0, nb) +
                            s->cos_psi * lap(s->fs, nb));
        phase_equilibrium(s->phi[n], muphi, p->eta, zero, eq);
        for (int i = 0; i < NQ; i++) s->g[i * N + n] = eq[i];
        heat_equilibrium(s->rhoH[n], s->rho[n] * s->cp[n], s->T[n], s->rr, zero, eq);
        for (int i = 0; i < NQ; i++) s->h[i * N + n] = eq[i];
      }
  pass_mask(s, s->w_prev);
}

void oracle3_step(oracle3_sim* s, long nsteps) {
  for (long k = 0; k < nsteps; k++) {
    pass_local(s);
    pass_collide(s, 1);
    pass_stream(s);
    pass_mask(s, s->w);
    pass_lag(s);
    s->step++;
  }
}

/* Fields of the current state: phi, fs, fl, T, rhoH, p, ux, uy, uz, rho,
 * mu_phi, w, mdot ([13][N]). */
#define OF3_COUNT 13
void oracle3_fields(oracle3_sim* s, double* out) {
  const long N = s->N;
  pass_local(s);
  pass_collide(s, 0);
  const double* src[OF3_COUNT] = {s->phi, s->fs, s->fl,  s->T,     s->rhoH, s->pr,  s->ux,
                                  s->uy,  s->uz, s->rho, s->muphi, s->w,    s->mdot};
  for (int k = 0; k < OF3_COUNT; k++) memcpy(out + (size_t)k * N, src[k], sizeof(double) * N);
}

/* Global diagnostics in node order, as the two-dimensional oracle's (the
 * kinetic energy with all three velocity components). */
void oracle3_diagnostics(oracle3_sim* s, double* d) {
  const oracle3_params* p = &s->p;
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
    d[7] += 0.5 * rho * (s->ux[n] * s->ux[n] + s->uy[n] * s->uy[n] + s->uz[n] * s->uz[n]);
    double tot = 0.0;
    for (int i = 0; i < NQ; i++) {
      if (p->lattices & LAT_FLOW) tot += s->f[i * N + n];
      if (p->lattices & LAT_PHASE) tot += s->g[i * N + n];
      if (p->lattices & LAT_HEAT) tot += s->h[i * N + n];
    }
    if (!isfinite(tot)) d[8] += 1.0;
  }
}

/* Populations [3][19][N] (f, g, h) and lags [7][N] (fl, w, p, phi u, Q). */
void oracle3_get_state(const oracle3_sim* s, double* pops, double* lags) {
  const long N = s->N;
  if (pops) {
    memcpy(pops, s->f, sizeof(double) * NQ * N);
    memcpy(pops + (size_t)NQ * N, s->g, sizeof(double) * NQ * N);
    memcpy(pops + (size_t)2 * NQ * N, s->h, sizeof(double) * NQ * N);
  }
  if (lags) {
    const double* src[7] = {s->fl_prev,   s->w_prev,    s->p_prev, s->phux_prev,
                            s->phuy_prev, s->phuz_prev, s->Q_prev};
    for (int k = 0; k < 7; k++) memcpy(lags + (size_t)k * N, src[k], sizeof(double) * N);
  }
}

void oracle3_set_state(oracle3_sim* s, const double* pops, const double* lags) {
  const long N = s->N;
  if (pops) {
    memcpy(s->f, pops, sizeof(double) * NQ * N);
    memcpy(s->g, pops + (size_t)NQ * N, sizeof(double) * NQ * N);
    memcpy(s->h, pops + (size_t)2 * NQ * N, sizeof(double) * NQ * N);
  }
  if (lags) {
    double* dst[7] = {s->fl_prev,   s->w_prev,    s->p_prev, s->phux_prev,
                      s->phuy_prev, s->phuz_prev, s->Q_prev};
    for (int k = 0; k < 7; k++) memcpy(dst[k], lags + (size_t)k * N, sizeof(double) * N);
  }
}

int64_t oracle3_step_count(const oracle3_sim* s) { return s->step; }

void oracle3_lattice(int* cx, int* cy, int* cz, double* w, int* opp) {
  lattice_setup();
  for (int i = 0; i < NQ; i++) {
    cx[i] = CX[i];
    cy[i] = CY[i];
    cz[i] = CZ[i];
    w[i] = WQ[i];
    opp[i] = OPP[i];
  }
}

/* --- single-node entry points for the moment pins --- */

void oracle3_node_flow(double pr, double rho, const double* u, double S, const double* F,
                       const double* fp, const double* Ft, uint32_t readings, double* feq,
                       double* Fi) {
  lattice_setup();
  flow_equilibrium(pr, rho, u, feq);
  flow_forcing(S, F, rho, fp, u, Ft, readings, Fi);
}

void oracle3_node_phase(double phi, double muphi, double eta, const double* phu,
                        const double* dphu, double mdot, double* geq, double* Gi) {
  lattice_setup();
  phase_equilibrium(phi, muphi, eta, phu, geq);
  phase_source(dphu, phi, mdot, Gi);
}

void oracle3_node_heat(double rhoH, double C, double T, double rr, const double* u, double mdot,
                       double* heq, double* Hi) {
  lattice_setup();
  heat_equilibrium(rhoH, C, T, rr, u, heq);
  heat_source(C, T, mdot, Hi);
}
