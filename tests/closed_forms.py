"""Closed forms the paper fixes, used to pin the oracle (arXiv 2510.18688, Sec. 4).

These are independent of the LB method: error-function similarity solutions
of the Stefan problems and the geometry of an equilibrium droplet on a
cylinder.  Roots of transcendental equations are found by bisection with the
host's ``math.erf``/``math.erfc``.
"""
from __future__ import annotations

import math


def bisect(fun, lo, hi, tol=1e-14, it=200):
    flo = fun(lo)
    for _ in range(it):
        mid = 0.5 * (lo + hi)
        fm = fun(mid)
        if (fm > 0) == (flo > 0):
            lo, flo = mid, fm
        else:
            hi = mid
        if hi - lo < tol:
            break
    return 0.5 * (lo + hi)


def neumann_k(cp_s, cp_l, L, T_m, T_b, T0, alpha_s, alpha_l):
    """Root k of the two-phase Neumann equation, Eq. (33); with T0 = T_m it is
    the one-phase Eq. (31)."""
    r = math.sqrt(alpha_s / alpha_l)

    def fun(k):
        a = cp_s * (T_m - T_b) / (L * math.exp(k * k) * math.erf(k))
        b = cp_l * (T0 - T_m) * math.sqrt(alpha_l / alpha_s) / (
            L * math.exp(k * k * alpha_s / alpha_l) * math.erfc(k * r))
        return a - b - k * math.sqrt(math.pi)

    return bisect(fun, 1e-9, 5.0)


def neumann_front(k, alpha_s, t):
    """X_i(t) = 2 k sqrt(alpha_s t) (Sec. 4.1)."""
    return 2.0 * k * math.sqrt(alpha_s * t)


def neumann_T(x, t, k, T_m, T_b, T0, alpha_s, alpha_l):
    """Temperature of Eq. (32) (Eq. (30) when T0 = T_m), with the argument of
    erf read as x / (2 sqrt(alpha_s t))."""
    X = neumann_front(k, alpha_s, t)
    if x < X:
        return T_b - (T_b - T_m) * math.erf(x / (2.0 * math.sqrt(alpha_s * t))) / math.erf(k)
    return T0 + (T_m - T0) * math.erfc(x / (2.0 * math.sqrt(alpha_l * t))) / math.erfc(
        k * math.sqrt(alpha_s / alpha_l))


def stefan_kappa(ste, lam_l, lam_s, T0, T_m, T_w, alpha_s, alpha_l, rho_r):
    """Root of the three-phase Stefan equation, Eq. (35), read as
    exp((sqrt(alpha_r) kappa rho_r)^2) erfc(sqrt(alpha_r) kappa rho_r)."""
    ar = alpha_s / alpha_l
    sa = math.sqrt(ar)

    def fun(k):
        a = ste / (math.exp(k * k) * math.erf(k))
        z = sa * k * rho_r
        b = lam_l * (T0 - T_m) * sa * ste / (lam_s * (T_m - T_w) * math.exp(z * z) * math.erfc(z))
        return a - b - k * math.sqrt(math.pi)

    return bisect(fun, 1e-9, 5.0)


def stefan_final_height(h0, rho_r):
    """h_f = rho_l h0 / rho_s from mass conservation (Sec. 4.2, Table 1)."""
    return h0 / rho_r


def conduction_T(x, t, T0, T_w, alpha):
    """Pure conduction from a wall held at T_w into a medium at T0."""
    return T0 + (T_w - T0) * math.erfc(x / (2.0 * math.sqrt(alpha * t)))


def poiseuille_u(y, H, g, nu):
    """Body-force driven channel flow between walls at y = 0 and y = H."""
    return g / (2.0 * nu) * y * (H - y)


def _circle_overlap(r1, r2, d):
    """Area of the intersection of two circles at centre distance d."""
    if d >= r1 + r2:
        return 0.0
    if d <= abs(r1 - r2):
        return math.pi * min(r1, r2) ** 2
    a1 = math.acos((d * d + r1 * r1 - r2 * r2) / (2 * d * r1))
    a2 = math.acos((d * d + r2 * r2 - r1 * r1) / (2 * d * r2))
    return (r1 * r1 * (a1 - math.sin(2 * a1) / 2) + r2 * r2 * (a2 - math.sin(2 * a2) / 2))


def cylinder_droplet_equilibrium(R0, Rs, theta_deg):
    """Equilibrium droplet on a cylinder (Sec. 4.4, Eqs. (36)-(37), reading
    R-CYL): the drop is a circle of radius R whose centre sits at distance
    k = sqrt(R^2 + Rs^2 - 2 R Rs cos(theta)) from the cylinder axis, with the
    area outside the cylinder equal to that of the initial drop (radius R0
    centred at distance Rs).  Returns (R, k, H_max = k + R)."""
    th = math.radians(theta_deg)
    area0 = math.pi * R0 * R0 - _circle_overlap(R0, Rs, Rs)

    def area(R):
        k = math.sqrt(R * R + Rs * Rs - 2 * R * Rs * math.cos(th))
        return math.pi * R * R - _circle_overlap(R, Rs, k)

    R = bisect(lambda r: area(r) - area0, 1e-6 * R0, 50.0 * R0)
    k = math.sqrt(R * R + Rs * Rs - 2 * R * Rs * math.cos(th))
    return R, k, k + R
