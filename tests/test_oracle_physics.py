"""Physical pins of the oracle: closed forms and invariants of the paper.

Each test runs the FP64 oracle on a seeded synthetic workload and compares
it with something the paper (arXiv 2510.18688) or the mathematics fixes
without reference to the oracle's formulas:

* Sec. 4.1 (Eqs. (30)-(33)): Neumann similarity solutions of one- and
  two-phase conduction-induced freezing, including a solid/liquid
  conductivity ratio different from one (Fig. 3).
* Sec. 4.2 (Table 1): final solid height of the three-phase Stefan problem
  with volume change, h_f = rho_l h0 / rho_s, expansion and shrinkage.
* Sec. 4.3: equilibrium contact angle of a resting droplet on the solid
  Omega_0 for theta below and above 90 degrees (wetting through Eq. (4)).
* Exact invariants: rest state (Eq. (14) with p = 0, u = 0), conservation of
  sum(phi) and sum(rho H) when nothing enters or leaves, material mass.
* Textbook limits: pure conduction from a Dirichlet wall (erfc), Poiseuille
  flow with halfway bounce-back, Laplace's law for a 2-D drop (the Eq. (4)
  normalisation gives surface tension sigma).
"""
import math

import numpy as np
import pytest

import closed_forms as CF
from paper_2510_18688_gb300 import workloads as W


@pytest.fixture(scope="module")
def O(oracle_mod):
    return oracle_mod


def _run(O, wl):
    return O.from_workload(wl)


# ---------------------------------------------------------------------------
# exact invariants
# ---------------------------------------------------------------------------

def test_rest_state_is_exactly_stationary(O):
    """P14: uniform liquid above T_m with p = 0, u = 0: f stays exactly 0, g
    and h stay exactly at their initial equilibria."""
    cfg = W.base_params(24, 16, bc=("periodic", "periodic", "dirichlet", "adiabatic"),
                        T_wall=(0.0, 0.0, 0.3, 0.0))
    z = np.zeros((16, 24))
    o = O.Oracle(cfg).init(z, z + 1.0, z + 0.3, z + 1.0)
    p0, l0 = o.state()
    o.step(200)
    p1, l1 = o.state()
    assert np.all(p1[0] == 0.0)
    assert np.array_equal(p1[1], p0[1])
    # anti-bounce-back at the wall held at the same temperature reproduces
    # the equilibrium up to the rounding of 2 w_i rho_ref Cp_ref T_w
    assert np.allclose(p1[2], p0[2], rtol=0, atol=1e-14)
    assert np.allclose(l1, l0, rtol=0, atol=1e-14)


@pytest.mark.parametrize("seed", [0, 1])
def test_phi_conserved_without_mass_source(O, seed):
    """P6: with rho_s = rho_l the source of Eq. (3) vanishes; streaming and
    bounce-back conserve sum g, so sum(phi) is constant to round-off."""
    cfg, arr = W.random_state(40, 32, seed=seed)
    cfg["rho_s"] = cfg["rho_l"]
    o = _run(O, (cfg, arr))
    s0 = o.diagnostics()["phi_sum"]
    o.step(300)
    d = o.diagnostics()
    assert d["nonfinite"] == 0
    assert abs(d["phi_sum"] - s0) < 1e-12 * cfg["nx"] * cfg["ny"]


def test_enthalpy_conserved_in_closed_box(O):
    """P5: periodic box without Dirichlet walls or cold mask and rho_s =
    rho_l: the TRT collision conserves sum h (Eq. (23) with H_i = 0), so
    sum(rho H) is constant to round-off while the melt front moves."""
    cfg, arr = W.random_state(40, 32, seed=2)
    cfg["rho_s"] = cfg["rho_l"]
    del arr["mask"]
    o = _run(O, (cfg, arr))
    s0 = o.diagnostics()["rhoH"]
    f0 = o.diagnostics()["frozen_volume"]
    o.step(300)
    d = o.diagnostics()
    assert abs(d["rhoH"] - s0) < 1e-12 * (abs(s0) + cfg["nx"] * cfg["ny"])
    assert abs(d["frozen_volume"] - f0) > 1e-3  # something did melt or freeze


def test_threads_do_not_change_results(O):
    """The OpenMP row loops write disjoint nodes: results are bitwise the
    same for any thread count."""
    cfg, arr = W.random_state(33, 21, seed=3)
    n0 = O.set_threads(0)
    try:
        O.set_threads(1)
        a = _run(O, (cfg, arr)).step(40).state()
        O.set_threads(4)
        b = _run(O, (cfg, arr)).step(40).state()
    finally:
        O.set_threads(n0)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


# ---------------------------------------------------------------------------
# Sec. 4.1: conduction-induced freezing (Eqs. (30)-(33))
# ---------------------------------------------------------------------------

def _neumann_check(O, T0, lam_ratio, times, front_tol=0.02, T_tol=0.02):
    cfg, arr = W.neumann(T0=T0, lambda_ratio=lam_ratio)
    a_l = cfg["lambda_l"] / (cfg["rho_l"] * cfg["cp_l"])
    a_s = cfg["lambda_s"] / (cfg["rho_s"] * cfg["cp_s"])
    k = CF.neumann_k(cfg["cp_s"], cfg["cp_l"], cfg["latent"], 0.0, -1.0, T0, a_s, a_l)
    o = _run(O, (cfg, arr))
    done = 0
    x = np.arange(cfg["nx"]) + 0.5
    for t in times:
        o.step(t - done)
        done = t
        X = o.diagnostics()["frozen_volume"] / cfg["ny"]
        Xa = CF.neumann_front(k, a_s, t)
        assert abs(X - Xa) <= max(1.0, front_tol * Xa), (t, X, Xa)
        T = o.fields()["T"][0]
        Ta = np.array([CF.neumann_T(xx, t, k, 0.0, -1.0, T0, a_s, a_l) for xx in x])
        band = np.abs(x - Xa) > 2.0
        assert np.abs(T - Ta)[band].max() <= T_tol * (T0 + 1.0), t


def test_neumann_two_phase(O):
    """P1, Fig. 3 setting with T0 > T_m (T0 = 0.1, Ste = 0.1)."""
    _neumann_check(O, 0.1, 1.0, (2000, 5000, 10000, 20000))


def test_neumann_two_phase_conductivity_ratio(O):
    """P1 with lambda_s / lambda_l = 2 (Fig. 3 varies this ratio)."""
    _neumann_check(O, 0.1, 2.0, (2000, 6000))


def test_neumann_one_phase(O):
    """P2, Sec. 4.1 first case: liquid initially at T_m (Eqs. (30)-(31))."""
    _neumann_check(O, 0.0, 1.0, (2000, 8000), T_tol=0.03)


def test_pure_conduction_erfc(O):
    """P13: no phase change (T stays above T_m): T = T0 + (T_w - T0)
    erfc(x / 2 sqrt(alpha t)) from an anti-bounce-back Dirichlet wall."""
    cfg, arr = W.neumann(T0=0.5)
    cfg["T_wall"] = (0.2, 0.5, 0.0, 0.0)
    alpha = cfg["lambda_l"] / (cfg["rho_l"] * cfg["cp_l"])
    o = _run(O, (cfg, arr)).step(4000)
    x = np.arange(cfg["nx"]) + 0.5
    Ta = np.array([CF.conduction_T(xx, 4000, 0.5, 0.2, alpha) for xx in x])
    assert np.abs(o.fields()["T"][0] - Ta).max() < 0.01 * 0.3


# ---------------------------------------------------------------------------
# flow and surface tension
# ---------------------------------------------------------------------------

def test_poiseuille(O):
    """P12: body-force driven channel with halfway bounce-back walls."""
    ny, g, nu = 32, 1e-6, 0.1
    cfg = W.base_params(4, ny, lattices=W.FLOW, gx=g, nu=nu,
                        bc=("periodic", "periodic", "dirichlet", "dirichlet"))
    z = np.zeros((ny, 4))
    o = O.Oracle(cfg).init(z, z + 1.0, z + 0.5, z + 1.0).step(12000)
    y = np.arange(ny) + 0.5
    ua = CF.poiseuille_u(y, ny, g, nu)
    assert np.abs(o.fields()["ux"][:, 1] - ua).max() < 0.01 * ua.max()


@pytest.mark.parametrize("R", [10.0, 16.0])
def test_laplace_law(O, R):
    """P11: static drop in a periodic box; the pressure jump equals sigma/R
    (Eq. (4) is normalised so that the interface tension is sigma)."""
    n = 64
    cfg = W.base_params(n, n, lattices=W.FLOW | W.PHASE, sigma=0.001)
    X, Y = np.meshgrid(np.arange(n) + 0.5, np.arange(n) + 0.5)
    phi = np.tanh(2 * (R - np.hypot(X - n / 2, Y - n / 2)) / cfg["eps"])
    z = np.zeros((n, n))
    o = O.Oracle(cfg).init(z, phi, z + 0.5, z + 1.0).step(8000)
    f = o.fields()
    p_in = f["p"][n // 2 - 2:n // 2 + 2, n // 2 - 2:n // 2 + 2].mean()
    p_out = f["p"][:3, :3].mean()
    assert (p_in - p_out) == pytest.approx(cfg["sigma"] / R, rel=0.05)


def _circle_fit(px, py):
    A = np.stack([px, py, np.ones_like(px)], 1)
    b = -(px ** 2 + py ** 2)
    c = np.linalg.lstsq(A, b, rcond=None)[0]
    xc, yc = -c[0] / 2, -c[1] / 2
    return xc, yc, math.sqrt(xc * xc + yc * yc - c[2])


@pytest.mark.parametrize("theta", [60.0, 90.0, 120.0])
def test_contact_angle_on_flat_solid(O, theta):
    """P7: a drop placed as a half disc (90 degrees) on a flat Omega_0 layer
    relaxes towards the prescribed contact angle, wetting acting only
    through phi0 in Eq. (4).  The phi = 0 contour above the wall is fitted
    with a circle; cos(theta) = (h_s - y_c)/R for a cap meeting y = h_s.
    Contact-line motion under Cahn-Hilliard mobility is slow, so within the
    CPU budget the check is: the angle moved at least 60 % of the way from 90
    degrees to theta, in the right direction, without passing theta by more
    than 4 degrees (a sign error in the wetting terms of Eq. (6) moves it
    the other way; a missing factor stops it early)."""
    nx, ny, hs, R0 = 64, 40, 8.0, 12.0
    cfg = W.base_params(nx, ny, lattices=W.FLOW | W.PHASE, theta_deg=theta, sigma=0.01,
                        mobility=0.2, bc=("periodic", "periodic", "adiabatic", "adiabatic"))
    X, Y = np.meshgrid(np.arange(nx) + 0.5, np.arange(ny) + 0.5)
    phi0 = 0.5 + 0.5 * np.tanh(2 * (hs - Y) / cfg["eps"])
    phi = (1 - phi0) * np.tanh(2 * (R0 - np.hypot(X - nx / 2, Y - hs)) / cfg["eps"])
    z = np.zeros((ny, nx))
    o = O.Oracle(cfg).init(phi0, phi, z + 0.5, z + 1.0).step(8000)
    f = o.fields()["phi"]
    px, py = [], []
    for j in range(int(hs) + 3, ny - 1):
        row = f[j]
        for i in range(nx - 1):
            if (row[i] > 0) != (row[i + 1] > 0):
                px.append(i + 0.5 + row[i] / (row[i] - row[i + 1]))
                py.append(j + 0.5)
    xc, yc, Rc = _circle_fit(np.array(px), np.array(py))
    measured = math.degrees(math.acos(max(-1.0, min(1.0, (hs - yc) / Rc))))
    if theta == 90.0:
        assert abs(measured - 90.0) < 4.0, measured
    else:
        moved = (measured - 90.0) / (theta - 90.0)
        assert moved > 0.6 and (measured - theta) * np.sign(theta - 90.0) < 4.0, measured


# ---------------------------------------------------------------------------
# Sec. 4.2: three-phase Stefan problem with volume change (Table 1)
# ---------------------------------------------------------------------------

def _crossing(phi_row, start):
    for i in range(start, len(phi_row) - 1):
        if phi_row[i] > 0 >= phi_row[i + 1]:
            return i + 0.5 + phi_row[i] / (phi_row[i] - phi_row[i + 1])
    return float("nan")


def test_stefan_final_height_table1(O):
    """P3 (Sec. 4.2, Table 1): after complete freezing the solid height is
    h_f = rho_l h0 / rho_s.  The configuration is the paper's: the whole
    system initially at T0 = 1, cold wall T_b = -1, T_m = 0, Ste = 0.1,
    eps = 4, sigma = 0.001, M = 0.1, mu = 0.1, unit Cp and conductivity
    ratios; a liquid column of 64 lattice units on a solid layer (phi0) of
    16, gas above.  At rho_s/rho_l = 0.9 the paper reports 1.1108 against
    1.1111 (0.03 %); the oracle must be within 0.5 %.  h_f is read at the
    first check after complete freezing (the phi = 0 crossing above the
    solid layer)."""
    hs, h0, rho_r = 16.0, 80.0, 0.9
    cfg, arr = W.stefan(nx=256, ny=4, hs=hs, h0=h0, rho_ratio=rho_r, T0=1.0, alpha=0.5)
    o = _run(O, (cfg, arr))
    for _ in range(100):
        o.step(2000)
        d = o.diagnostics()
        if d["frozen_volume"] / d["material_volume"] > 0.999:
            break
    assert d["frozen_volume"] / d["material_volume"] > 0.999
    hf = (_crossing(o.fields()["phi"][0], int(hs)) - hs) / (h0 - hs)
    assert hf == pytest.approx(CF.stefan_final_height(1.0, rho_r), rel=0.005)
    assert d["nonfinite"] == 0


def test_stefan_shrinkage_final_height(O):
    """Shrinkage (rho_s/rho_l = 1.2, Table 1: h_f/h0 = 0.8333): a short
    column of liquid initially at T_m on a solid layer.  The height moves in
    the right direction and within 4 % of rho_l h0 / rho_s (the paper's own
    errors at 1.2 are 0.5-0.7 %; after complete freezing the f_s penalty of
    Eq. (4) keeps pushing phi out of the ice, so the phi = 0 crossing creeps
    and the check is made at the first sample after freezing).  Under
    shrinkage the weight w of Eq. (10) overcounts the material near the
    converging interface (about 10 % of the material mass), a limitation of
    the method as read that this pin records rather than hides."""
    hs, h0, rho_r = 8.0, 32.0, 1.2
    cfg, arr = W.stefan(nx=128, ny=4, hs=hs, h0=h0, rho_ratio=rho_r, T0=0.0, alpha=0.5)
    o = _run(O, (cfg, arr))
    m0 = o.diagnostics()["material_mass"]
    for _ in range(20):
        o.step(1000)
        d = o.diagnostics()
        if d["frozen_volume"] / d["material_volume"] > 0.999:
            break
    assert d["frozen_volume"] / d["material_volume"] > 0.999
    hf = (_crossing(o.fields()["phi"][0], int(hs)) - hs) / (h0 - hs)
    assert hf == pytest.approx(CF.stefan_final_height(1.0, rho_r), rel=0.04)
    assert (hf - 1.0) * (1.0 / rho_r - 1.0) > 0.5 * (1.0 / rho_r - 1.0) ** 2
    assert abs(d["material_mass"] / m0 - 1) < 0.15


def _front(f, row=0):
    """Last crossing of the frozen material fraction w (1 - fl) through 1/2,
    in wall coordinates (node i at i + 1/2; the cold wall at 0)."""
    s = f["w"][row] * (1.0 - f["fl"][row]) - 0.5
    out = float("nan")
    for i in range(len(s) - 1):
        if s[i] > 0 >= s[i + 1]:
            out = i + 0.5 + s[i] / (s[i] - s[i + 1])
    return out


def test_stefan_front_and_interface_displacement(O):
    """P3 (Sec. 4.2, Eq. (35)): the freezing front follows h_s(t) = 2 kappa
    sqrt(alpha_s t), kappa the root of Eq. (35); and the liquid above it is
    pushed up by the convection velocity the paper prints, u = (dh_s/dt)(1 -
    rho_s/rho_l), so that the gas-liquid interface has moved by
    (1 - rho_s/rho_l) (h_s - h_s0) -- the integral of that velocity, which
    the standing sound wave of the closed gas column (period ~600 steps)
    does not blur.  Paper configuration (T0 = 1, Ste = 0.1, rho_s/rho_l =
    0.9) on a thin solid layer (one interface width, so that the front
    starts at the wall).  The paper shows the front as a figure only (good
    agreement); the bounds: front within 3 % (the Neumann pins allow 2 %; the
    diffuse layer and the moving liquid add to it), interface displacement
    within 5 % of the front's advance times (1 - rho_s/rho_l), at 10k, 20k
    and 40k steps.  A mass source with the wrong factor or sign (Eq. (1))
    fails the second; a wrong latent heat or Stefan number the first."""
    hs, h0, rho_r = 4.0, 68.0, 0.9
    cfg, arr = W.stefan(nx=256, ny=4, hs=hs, h0=h0, rho_ratio=rho_r, T0=1.0, alpha=0.5)
    a_s = cfg["lambda_s"] / (cfg["rho_s"] * cfg["cp_s"])
    a_l = cfg["lambda_l"] / (cfg["rho_l"] * cfg["cp_l"])
    kappa = CF.stefan_kappa(0.1, cfg["lambda_l"], cfg["lambda_s"], 1.0, 0.0, -1.0, a_s, a_l,
                            rho_r)
    o = _run(O, (cfg, arr))
    x_gl0 = _crossing(o.fields()["phi"][0], int(hs))
    done = 0
    for t in (10000, 20000, 40000):
        o.step(t - done)
        done = t
        f = o.fields()
        X = _front(f)
        want = 2.0 * kappa * math.sqrt(a_s * t)
        assert abs(X - want) <= 0.03 * want, (t, X, want)
        moved = _crossing(f["phi"][0], int(X) + 2) - x_gl0
        expect = (1.0 - rho_r) * (X - hs)
        assert abs(moved - expect) <= 0.05 * expect, (t, moved, expect)


def test_flat_interface_stays_stationary(O):
    """P9: a flat gas-liquid interface started from the equilibrium profile
    phi = tanh(2 x / eps) of Eq. (4) (two interfaces in a periodic column,
    fluid at rest, no heat) stays where it is.  The continuum profile relaxes
    to the discrete equilibrium of the isotropic stencils (a change of about
    1e-2 near the interface, settling: the change between 5,000 and 10,000
    steps is under 3e-3); the phi = 0 crossings move by less than 1e-3
    lattice units and the bulk stays at phi = -1, +1 to 1e-5.  A wrong sign
    or coefficient in the chemical potential of Eq. (6) widens, narrows or
    moves the interface far beyond these bounds."""
    nx, ny = 96, 4
    cfg = W.base_params(nx, ny, lattices=W.FLOW | W.PHASE, sigma=0.001, mobility=0.1)
    x = np.arange(nx) + 0.5
    eps = cfg["eps"]
    prof = np.tanh(2 * (x - 24) / eps) - np.tanh(2 * (x - 72) / eps) - 1.0
    phi = np.tile(prof, (ny, 1))
    z = np.zeros((ny, nx))
    o = O.Oracle(cfg).init(z, phi, z + 0.5, z + 1.0)

    def crossings(row):
        out = []
        for i in range(nx - 1):
            a, b = row[i], row[i + 1]
            if (a <= 0) != (b <= 0):
                out.append(i + 0.5 + a / (a - b))
        return np.array(out)

    c0 = crossings(o.fields()["phi"][1])
    o.step(5000)
    mid = o.fields()["phi"]
    o.step(5000)
    f = o.fields()["phi"]
    assert np.abs(f - np.tile(prof, (ny, 1))).max() < 2e-2
    assert np.abs(f - mid).max() < 3e-3
    c1 = crossings(f[1])
    assert len(c1) == 2 and np.abs(c1 - c0).max() < 1e-3, (c0, c1)
    assert abs(f[1, 48] - 1.0) < 1e-5 and abs(f[1, 0] + 1.0) < 1e-5


@pytest.mark.xfail(strict=True, reason=(
    "the configured gas/liquid density ratio 0.001 of Sec. 4.2 diverges under the readings "
    "used (about step 19,000 of this column: the compressed light gas heats past T0, then "
    "the state turns non-finite; taking the flow's own div u in the enthalpy source does not "
    "cure it); the workloads run at 0.1"))
def test_stefan_column_at_the_configured_gas_density_ratio(O):
    """Records the known limitation: the three-phase Stefan column of Sec. 4.2
    with rho_g/rho_l = 0.001 (the paper's value) stays finite and bounded
    (T within [T_b, T0] up to 1 %, |phi| <= 1.02) for 22,000 steps.  Strict
    xfail: a change of reading that cures it makes this test pass and
    therefore fail the suite, so the fix cannot go unnoticed."""
    cfg, arr = W.stefan()
    rg = 0.001
    cfg = dict(cfg, rho_g=rg, mu_g=rg * 0.1, cp_g=cfg["cp_l"] * cfg["rho_l"] / rg)
    o = _run(O, (cfg, arr))
    o.step(22000)
    f = o.fields()
    assert o.diagnostics()["nonfinite"] == 0
    assert np.isfinite(f["T"]).all() and np.isfinite(f["phi"]).all()
    assert f["T"].max() <= 1.01 and f["T"].min() >= -1.01
    assert np.abs(f["phi"]).max() <= 1.02
