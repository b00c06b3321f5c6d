// lbm_host.h -- host-side helpers shared by the library's translation units
// (parameter validation, derived constants, grid layout).
#pragma once

#include <cmath>
#include <cstddef>
#include <cstdio>

#include "../../include/lbm.h"
#include "lbm_kernels.cuh"

namespace lbmh {

using lbmk::Coef;
using lbmk::Geom;

inline bool positive(double v) { return std::isfinite(v) && v > 0.0; }

template <typename R>
inline Coef<R> make_coef(const lbm_params& p) {
  Coef<R> c;
  const double pi = 3.14159265358979323846;
  c.rho_l = (R)p.rho_l; c.rho_s = (R)p.rho_s; c.rho_g = (R)p.rho_g;
  c.mu_l = (R)p.mu_l; c.mu_s = (R)p.mu_s; c.mu_g = (R)p.mu_g;
  c.lam_l = (R)p.lambda_l; c.lam_s = (R)p.lambda_s; c.lam_g = (R)p.lambda_g;
  c.cp_l = (R)p.cp_l; c.cp_s = (R)p.cp_s; c.cp_g = (R)p.cp_g;
  // Cp_ref = 2 Cp_s Cp_l / (Cp_s + Cp_l) (Sec. 3.3)
  c.rr = (R)(p.rho_ref * (2.0 * p.cp_s * p.cp_l / (p.cp_s + p.cp_l)));
  c.latent = (R)p.latent;
  c.sigma = (R)p.sigma;
  c.eps = (R)p.eps;
  c.eta = (R)p.eta;
  c.cos_th = (R)std::cos(p.theta_deg * pi / 180.0);
  c.cos_ps = (R)std::cos(p.psi_deg * pi / 180.0);
  c.gx = (R)p.gx;
  c.gy = (R)p.gy;
  c.tau_g = (R)(0.5 + p.mobility / (p.eta / 3.0));  // Eq. (21)
  c.T_cold = (R)p.T_cold;
  c.one_m_ratio = (R)(1.0 - p.rho_s / p.rho_l);
  for (int k = 0; k < 4; k++) c.T_wall[k] = (R)p.T_wall[k];
  c.s3 = (R)(3.0 * p.sigma / p.eps);
  c.s9 = (R)(9.0 * p.sigma / p.eps);
  c.klap = (R)(3.0 * p.eps * p.sigma / 8.0);
  c.rr3 = (R)(p.rho_ref * (2.0 * p.cp_s * p.cp_l / (p.cp_s + p.cp_l)) / 3.0);
  c.inv_rr3 = (R)(3.0 / (p.rho_ref * (2.0 * p.cp_s * p.cp_l / (p.cp_s + p.cp_l))));
  c.inv_tau_g = (R)(1.0 / (0.5 + p.mobility / (p.eta / 3.0)));
  {
    const double rr = p.rho_ref * (2.0 * p.cp_s * p.cp_l / (p.cp_s + p.cp_l));
    c.wrr1 = (R)(rr / 9.0);
    c.wrr5 = (R)(rr / 36.0);
    c.rr_rest = (R)(rr * 5.0 / 9.0);
  }
  c.readings = p.readings;
  return c;
}

// Tangent constants: the FP64 constants with the derivatives of the
// parameters that the direction moves (cos of the contact angle in degrees).
inline Coef<lbmk::Dual> make_coef_tangent(const lbm_params& p) {
  const Coef<double> v = make_coef<double>(p);
  Coef<lbmk::Dual> c;
  const double* src = (const double*)&v;
  lbmk::Dual* dst = (lbmk::Dual*)&c;
  const size_t nreal = (sizeof(Coef<double>) - sizeof(double)) / sizeof(double);  // all but readings
  static_assert(offsetof(Coef<double>, readings) == (sizeof(Coef<double>) - sizeof(double)),
                "readings is the last member");
  for (size_t k = 0; k < nreal; k++) dst[k] = lbmk::Dual(src[k]);
  c.readings = v.readings;
  const double pi = 3.14159265358979323846;
  for (int k = 0; k < 4; k++) c.T_wall[k].d = p.tan_T_wall[k];
  c.T_cold.d = p.tan_T_cold;
  c.cos_th.d = -std::sin(p.theta_deg * pi / 180.0) * (pi / 180.0) * p.tan_theta_deg;
  c.latent.d = p.tan_latent;
  return c;
}

inline int validate(const lbm_params* p, char* err, size_t n) {
  if (!p) return LBM_ERR_ARG;
  if (p->nx < 2 || p->ny < 2) {
    std::snprintf(err, n, "grid must be at least 2 x 2 (got %d x %d)", p->nx, p->ny);
    return LBM_ERR_ARG;
  }
  // the kernels index the 27 population planes with 32-bit offsets
  const long long plane = ((long long)((p->nx + 31) / 32 * 32) * p->ny + 63) / 64 * 64;
  if (plane * 27 >= (1LL << 31)) {
    std::snprintf(err, n, "grid of %d x %d nodes is too large", p->nx, p->ny);
    return LBM_ERR_ARG;
  }
  if (p->precision != LBM_FP32 && p->precision != LBM_FP64 && p->precision != LBM_FP16S &&
      p->precision != LBM_FP64_TANGENT) {
    std::snprintf(err, n, "unknown precision %d", p->precision);
    return LBM_ERR_ARG;
  }
  if (p->lattices == 0 || (p->lattices & ~7u)) {
    std::snprintf(err, n, "lattices must be a nonzero subset of flow|phase|heat (got %u)",
                  p->lattices);
    return LBM_ERR_ARG;
  }
  for (int k = 0; k < 4; k++) {
    if (p->bc[k] < LBM_BC_PERIODIC || p->bc[k] > LBM_BC_ADIABATIC) {
      std::snprintf(err, n, "unknown boundary type %d on side %d", p->bc[k], k);
      return LBM_ERR_ARG;
    }
  }
  if ((p->bc[0] == LBM_BC_PERIODIC) != (p->bc[1] == LBM_BC_PERIODIC) ||
      (p->bc[2] == LBM_BC_PERIODIC) != (p->bc[3] == LBM_BC_PERIODIC)) {
    std::snprintf(err, n, "a periodic side needs a periodic opposite side");
    return LBM_ERR_ARG;
  }
  if (p->diag_every < 0) {
    std::snprintf(err, n, "diag_every must be >= 0");
    return LBM_ERR_ARG;
  }
  const double props[] = {p->rho_l, p->rho_s,    p->rho_g,    p->mu_l,     p->mu_s,
                          p->mu_g,  p->lambda_l, p->lambda_s, p->lambda_g, p->cp_l,
                          p->cp_s,  p->cp_g,     p->rho_ref,  p->eps,      p->mobility,
                          p->eta};
  for (double v : props) {
    // every relaxation time of Sec. 3 is 1/2 plus a positive property ratio,
    // so positivity of the properties is what keeps tau > 1/2
    if (!positive(v)) {
      std::snprintf(err, n, "densities, viscosities, conductivities, heat capacities, "
                            "rho_ref, eps, mobility and eta must be positive and finite");
      return LBM_ERR_PARAM;
    }
  }
  if (!(std::isfinite(p->latent) && p->latent >= 0.0) ||
      !(std::isfinite(p->sigma) && p->sigma >= 0.0)) {
    std::snprintf(err, n, "latent heat and surface tension must be finite and >= 0");
    return LBM_ERR_PARAM;
  }
  return LBM_OK;
}


// Layout of one grid: rows padded to a multiple of 32 elements, planes to a
// multiple of 64 elements.
inline Geom make_geom(const lbm_params& p) {
  Geom g;
  g.nx = p.nx;
  g.ny = p.ny;
  g.pitch = (p.nx + 31) / 32 * 32;
  const long long plane = (long long)g.pitch * p.ny;
  g.plane = (plane + 63) / 64 * 64;
  g.lattices = (int)p.lattices;
  for (int k = 0; k < 4; k++) g.bc[k] = p.bc[k];
  g.has_mask = 0;
  return g;
}

}  // namespace lbmh
