"""Pins of the oracle's local building blocks against what the paper fixes.

Each check compares the oracle with a property that the paper (arXiv
2510.18688, Secs. 2-3) or the mathematics fixes independently of the
oracle's own formulas: the lattice of Eq. (12) and its isotropy, the
macroscopic moments that Eqs. (14), (16), (19), (20), (25) must reproduce
for the model to recover Eqs. (1)-(7), the reduction of the TRT collision
Eq. (23) to BGK, the enthalpy inversion Eq. (8), and the chemical potential
Eq. (6) as the variational derivative of the free energy Eq. (4).
"""
import itertools
import math

import numpy as np
import pytest

CS2 = 1.0 / 3.0


@pytest.fixture(scope="module")
def O(oracle_mod):
    return oracle_mod


@pytest.fixture(scope="module")
def lat(O):
    return O.lattice()


def test_lattice_is_d2q9_of_eq12(lat):
    cx, cy, w, opp = lat
    # Eq. (12): rest, axes at angles (i-1) pi/2, diagonals at (2i-9) pi/4
    for i in range(1, 5):
        a = (i - 1) * math.pi / 2
        assert (cx[i], cy[i]) == (round(math.cos(a)), round(math.sin(a)))
    for i in range(5, 9):
        a = (2 * i - 9) * math.pi / 4
        assert (cx[i], cy[i]) == (round(math.sqrt(2) * math.cos(a)), round(math.sqrt(2) * math.sin(a)))
    assert np.allclose(w, [4 / 9] + [1 / 9] * 4 + [1 / 36] * 4, rtol=0, atol=1e-16)
    for i in range(9):
        assert cx[opp[i]] == -cx[i] and cy[opp[i]] == -cy[i]


def test_lattice_isotropy(lat):
    cx, cy, w, _ = lat
    c = np.stack([cx, cy], 1).astype(float)
    assert abs(w.sum() - 1) < 1e-15
    assert np.allclose(w @ c, 0, atol=1e-16)
    assert np.allclose(np.einsum("i,ia,ib->ab", w, c, c), CS2 * np.eye(2), atol=1e-16)
    assert np.allclose(np.einsum("i,ia,ib,ic->abc", w, c, c, c), 0, atol=1e-16)
    m4 = np.einsum("i,ia,ib,ic,id->abcd", w, c, c, c, c)
    d = np.eye(2)
    iso = CS2 ** 2 * (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d)
                      + np.einsum("ad,bc->abcd", d, d))
    assert np.allclose(m4, iso, atol=1e-16)


def _moments(lat, v):
    cx, cy, w, _ = lat
    c = np.stack([cx, cy], 1).astype(float)
    return v.sum(), c.T @ v, np.einsum("ia,ib,i->ab", c, c, v)


@pytest.mark.parametrize("seed", range(4))
def test_flow_equilibrium_and_forcing_moments(O, lat, seed):
    """Eq. (14): sum f_eq = 0, sum c f_eq = rho u, sum cc f_eq = p I + rho u u;
    Eq. (16): sum F_i = S, sum c F_i = F + rho f, sum cc F_i = cs^2 S I +
    u Ft + Ft u (the isotropic cs^2 S I coming from the w_i S term)."""
    r = np.random.default_rng(seed)
    p, rho = r.uniform(-1e-3, 1e-3), r.uniform(0.1, 1.0)
    u = r.uniform(-0.05, 0.05, 2)
    S, F, fp, Ft = r.normal() * 1e-3, r.normal(size=2) * 1e-3, r.normal(size=2) * 1e-3, r.normal(size=2) * 1e-3
    feq, Fi = O.node_flow(p, rho, u[0], u[1], S, F[0], F[1], fp[0], fp[1], Ft[0], Ft[1])
    m0, m1, m2 = _moments(lat, feq)
    assert abs(m0) < 1e-15
    assert np.allclose(m1, rho * u, rtol=1e-13, atol=1e-17)
    assert np.allclose(m2, p * np.eye(2) + rho * np.outer(u, u), rtol=1e-12, atol=1e-17)
    m0, m1, m2 = _moments(lat, Fi)
    assert abs(m0 - S) < 1e-15
    assert np.allclose(m1, F + rho * fp, rtol=1e-13, atol=1e-18)
    assert np.allclose(m2, CS2 * S * np.eye(2) + np.outer(u, Ft) + np.outer(Ft, u), rtol=1e-12,
                       atol=1e-18)
    # the R-FT variant adds cs^2 S I once more to the second moment only
    _, Fv = O.node_flow(p, rho, u[0], u[1], S, F[0], F[1], fp[0], fp[1], Ft[0], Ft[1], readings=1)
    v0, v1, v2 = _moments(lat, Fv)
    assert abs(v0 - S) < 1e-15 and np.allclose(v1, m1, atol=1e-18)
    assert np.allclose(v2 - m2, CS2 * S * np.eye(2), atol=1e-17)


@pytest.mark.parametrize("seed", range(4))
def test_phase_equilibrium_and_source_moments(O, lat, seed):
    """Eq. (19): sum g_eq = phi, sum c g_eq = phi u, sum cc g_eq = cs^2 eta mu I
    (this recovers the mobility of Eq. (21)); Eq. (20): sum G = phi div u,
    sum c G = d(phi u)/dt."""
    r = np.random.default_rng(10 + seed)
    phi, mu, eta = r.uniform(-1, 1), r.normal() * 1e-3, r.uniform(0.5, 2)
    phu, dphu, md = r.normal(size=2) * 1e-2, r.normal(size=2) * 1e-4, r.normal() * 1e-4
    geq, G = O.node_phase(phi, mu, eta, phu[0], phu[1], dphu[0], dphu[1], md)
    m0, m1, m2 = _moments(lat, geq)
    assert abs(m0 - phi) < 1e-15
    assert np.allclose(m1, phu, atol=1e-16)
    assert np.allclose(m2, CS2 * eta * mu * np.eye(2), atol=1e-17)
    m0, m1, _ = _moments(lat, G)
    assert abs(m0 - phi * md) < 1e-18
    assert np.allclose(m1, dphu, atol=1e-18)


@pytest.mark.parametrize("seed", range(4))
def test_heat_equilibrium_and_source_moments(O, lat, seed):
    """Eq. (25): sum h_eq = rho H, sum c h_eq = rho Cp T u, sum cc h_eq =
    rho_ref Cp_ref T cs^2 I + rho Cp T u u, so that the diffusive flux is
    lambda grad T with Eq. (26); the source of Eq. (23) sums to rho Cp T mdot."""
    r = np.random.default_rng(20 + seed)
    rhoH, C, T, rr = r.uniform(-2, 12), r.uniform(0.5, 2), r.uniform(-1, 1), r.uniform(0.5, 1.5)
    u = r.uniform(-0.05, 0.05, 2)
    md = r.normal() * 1e-3
    heq, H = O.node_heat(rhoH, C, T, rr, u[0], u[1], md)
    m0, m1, m2 = _moments(lat, heq)
    assert abs(m0 - rhoH) < 1e-13
    assert np.allclose(m1, C * T * u, rtol=1e-12, atol=1e-16)
    assert np.allclose(m2, rr * T * CS2 * np.eye(2) + C * T * np.outer(u, u), rtol=1e-12, atol=1e-15)
    assert abs(H.sum() - C * T * md) < 1e-16


def test_trt_reduces_to_bgk_and_conserves(O, lat):
    """Eqs. (23)-(24): with tau_a = tau_s the TRT collision is BGK; the
    collision conserves sum h when h_eq has the same zeroth moment; the first
    moment relaxes with rate 1/tau_a."""
    cx, cy, w, _ = lat
    r = np.random.default_rng(3)
    h = r.normal(size=9)
    heq = r.normal(size=9)
    heq[0] += h.sum() - heq.sum()
    Hi = np.zeros(9)
    tau = 0.83
    out = O.node_trt(h, heq, Hi, tau, tau)
    assert np.allclose(out, h - (h - heq) / tau, atol=1e-14)
    taua = 1.7
    taus = taua / (2 * taua - 1)  # Eq. (27)
    assert abs(1 / taua + 1 / taus - 2) < 1e-15
    out = O.node_trt(h, heq, Hi, taua, taus)
    assert abs(out.sum() - h.sum()) < 1e-13
    c = np.stack([cx, cy], 1)
    j, jeq = c.T @ h, c.T @ heq
    assert np.allclose(c.T @ out, j - (j - jeq) / taua, atol=1e-13)


def _water_cfg(**kw):
    from paper_2510_18688_gb300 import workloads as W
    return W.base_params(4, 4, rho_s=0.9, cp_s=0.5, latent=7.5, **kw)


def test_enthalpy_inversion_eq8_pure_material(O):
    """Eq. (8) for the pure material (w = 1, phi0 = 0) with T_m = 0:
    rho_s H_s = 0, rho_l H_l = rho_l L, T = rhoH / (rho_s Cp_s) below,
    fl = rhoH / (rho_l L) in the mushy range, T = (rhoH - rho_l L)/(rho_l Cp_l)
    above; continuous at both thresholds (P15)."""
    cfg = _water_cfg()
    L, rl, rs, cpl, cps = cfg["latent"], cfg["rho_l"], cfg["rho_s"], cfg["cp_l"], cfg["cp_s"]
    rhoH = np.array([-3.0, -1e-12, 0.0, 0.3 * rl * L, rl * L, rl * L + 1e-12, rl * L + 2.0])
    T, fl = O.invert(cfg, rhoH, np.ones_like(rhoH), np.zeros_like(rhoH))
    assert T[0] == pytest.approx(-3.0 / (rs * cps), rel=1e-15) and fl[0] == 0.0
    assert abs(T[1]) < 1e-11 and fl[1] == 0.0
    assert T[2] == 0.0 and fl[2] == 0.0
    assert T[3] == 0.0 and fl[3] == pytest.approx(0.3, rel=1e-14)
    assert T[4] == 0.0 and fl[4] == 1.0
    assert abs(T[5]) < 1e-11 and fl[5] == 1.0
    assert T[6] == pytest.approx(2.0 / (rl * cpl), rel=1e-14) and fl[6] == 1.0


def test_enthalpy_inversion_reduces_to_typical_when_densities_equal(O):
    """With rho_s = rho_l and Cp_s = Cp_l the inversion is the standard
    enthalpy method: T = (rhoH - rho L fl) / (rho Cp) with fl in [0, 1]."""
    cfg = _water_cfg()
    cfg.update(rho_s=1.0, cp_s=1.0, latent=10.0)
    rhoH = np.linspace(-2, 14, 161)
    T, fl = O.invert(cfg, rhoH, np.ones_like(rhoH), np.zeros_like(rhoH))
    fl_ref = np.clip(rhoH / 10.0, 0, 1)
    T_ref = rhoH - 10.0 * fl_ref
    assert np.allclose(fl, fl_ref, atol=1e-15) and np.allclose(T, T_ref, atol=1e-14)


def test_enthalpy_inversion_gas_and_solid_carry_no_latent_heat(O):
    """Reading R-T1: a node with no material (gas, w = 0) or inside the
    pre-existing solid changes temperature linearly through T_m."""
    cfg = _water_cfg()
    rhoH = np.array([-0.5, 0.0, 0.5])
    for w, phi0 in ((0.0, 0.0), (0.0, 1.0)):
        T, fl = O.invert(cfg, rhoH, np.full(3, w), np.full(3, phi0))
        slope = T[2] / 0.5
        assert T[0] == pytest.approx(-0.5 * slope, rel=1e-14) and T[1] == 0.0


def _free_energy(phi, phi0, fs, sigma, eps, cth, cps):
    """Discrete free energy of Eq. (4) on a periodic grid: bulk densities
    summed over nodes; grad a . grad b written as the sum over the D2Q9
    links sum_x sum_i (w_i / cs^2) (da)(db), which tends to the integral of
    grad a . grad b for smooth fields (sum_i w_i c_i c_i = cs^2 I)."""
    bulk = (3 * sigma / (4 * eps) * (1 - phi) ** 2 * (1 + phi) ** 2
            + 9 * sigma / (2 * eps) * phi0 ** 2 * phi ** 2
            + 3 * sigma * cth / eps * phi0 * phi * (phi ** 2 + phi0 ** 2 - 1)
            + 9 * sigma / (2 * eps) * fs ** 2 * phi ** 2
            + 3 * sigma * cps / eps * fs * phi * (phi ** 2 + fs ** 2 - 1)).sum()
    link = 0.0
    cx = [1, 0, -1, 0, 1, -1, -1, 1]
    cy = [0, 1, 0, -1, 1, 1, -1, -1]
    w = [1 / 9] * 4 + [1 / 36] * 4
    for k in range(8):
        d = lambda a: np.roll(a, (-cy[k], -cx[k]), axis=(0, 1)) - a  # noqa: E731
        dp = d(phi)
        link += w[k] / CS2 * (3 * eps * sigma / 16 * dp * dp
                                    + 3 * eps * sigma * cth / 8 * d(phi0) * dp
                                    + 3 * eps * sigma * cps / 8 * d(fs) * dp).sum()
    return bulk + link


def test_chemical_potential_is_variational_derivative_of_eq4(O):
    """Eq. (6) must equal delta F / delta phi of Eq. (4); checked node by node
    against a central difference of the discrete functional on random
    smooth fields with every wetting and penalty term active."""
    from paper_2510_18688_gb300 import workloads as W
    ny, nx = 10, 12
    r = np.random.default_rng(7)
    yy, xx = np.mgrid[0:ny, 0:nx]

    def smooth(lo, hi):
        a = sum(r.normal() * np.cos(2 * np.pi * (kx * xx / nx + ky * yy / ny) + r.uniform(0, 6))
                for kx, ky in itertools.product(range(3), range(3)))
        a = (a - a.min()) / (a.max() - a.min())
        return lo + (hi - lo) * a

    phi, phi0, fs = smooth(-0.9, 0.9), smooth(0.0, 0.8), smooth(0.0, 0.7)
    cfg = W.base_params(nx, ny, sigma=0.01, eps=3.0, theta_deg=63.0, psi_deg=124.0)
    mu = O.chemical_potential(cfg, phi, phi0, fs)
    cth, cps = math.cos(math.radians(63.0)), math.cos(math.radians(124.0))
    d = 1e-4
    for (j, i) in [(0, 0), (3, 7), (9, 11), (5, 2), (7, 6)]:
        e = np.zeros_like(phi)
        e[j, i] = d
        num = (_free_energy(phi + e, phi0, fs, 0.01, 3.0, cth, cps)
               - _free_energy(phi - e, phi0, fs, 0.01, 3.0, cth, cps)) / (2 * d)
        assert mu[j, i] == pytest.approx(num, rel=1e-7, abs=1e-13)


def test_bulk_free_energy_wells(O):
    """Sec. 2 and Fig. 2: f_b(phi, phi0) is a double well with minima at +-1
    for phi0 = 0 and a single well at phi = 0 for phi0 = 1 (P10): the local
    chemical potential (uniform fields, no Laplacian) vanishes exactly at the
    stationary points and changes sign once per stationary point."""
    from paper_2510_18688_gb300 import workloads as W
    cfg = W.base_params(3, 3, sigma=0.02, eps=3.0, theta_deg=90.0, psi_deg=90.0)
    for phi0, roots in ((0.0, (-1.0, 0.0, 1.0)), (1.0, (0.0,))):
        for p in roots:
            mu = O.chemical_potential(cfg, np.full((3, 3), p), np.full((3, 3), phi0), np.zeros((3, 3)))
            assert np.all(mu == 0.0)
        grid = np.linspace(-1.5, 1.5, 61)
        vals = np.array([O.chemical_potential(cfg, np.full((3, 3), p), np.full((3, 3), phi0),
                                              np.zeros((3, 3)))[0, 0] for p in grid])
        s = np.sign(vals[vals != 0])
        changes = int(np.sum(s[1:] != s[:-1]))
        # double well: minimum, maximum, minimum; single well: one minimum
        assert changes == (3 if phi0 == 0.0 else 1)
        assert s[0] < 0 and s[-1] > 0


def test_flat_profile_is_equilibrium(O):
    """phi = tanh(2x/eps), the profile of Eqs. (34) and (38), makes the
    standard chemical potential vanish; on the lattice the residual is the
    truncation of the Laplacian, second order in 1/eps."""
    from paper_2510_18688_gb300 import workloads as W
    fracs = []
    for eps in (4.0, 8.0):
        nx, ny = 128, 3
        x = np.arange(nx) + 0.5
        phi = np.tanh(2 * (np.minimum(x - 32, 96 - x)) / eps)
        phi = np.tile(phi, (ny, 1))
        cfg = W.base_params(nx, ny, sigma=0.001, eps=eps)
        mu = O.chemical_potential(cfg, phi, np.zeros_like(phi), np.zeros_like(phi))
        scale = 3 * 0.001 / eps * np.abs(phi * (phi ** 2 - 1)).max()
        fracs.append(np.abs(mu).max() / scale)
    assert fracs[0] < 0.15
    assert fracs[1] < fracs[0] / 3.0
