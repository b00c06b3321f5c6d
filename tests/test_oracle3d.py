"""Pins of the three-dimensional (D3Q19) oracle.

The 3-D oracle restates the method of the 2-D oracle on the D3Q19 lattice of
Sec. 3.1.  It is pinned to things other than itself:

* the lattice against the velocity matrix and weights printed in Sec. 3.1
  (golden fixture) and against the moment identities that make the
  equilibria of Eqs. (14), (19) and (25) recover their macroscopic equations;
* z-projection: for fields uniform along a periodic z axis, the sum of the
  D3Q19 populations over c_z obeys the D2Q9 update exactly for the
  phase-field and enthalpy lattices (the D3Q19 weights summed over c_z are
  the D2Q9 weights, and every equilibrium, source, stencil and wall rule of
  these two lattices is linear in the weights at u = 0), so a 3-D run of an
  extruded 2-D state reproduces the pinned 2-D oracle to round-off;
* the flow lattice against textbook limits in 3-D: the Poiseuille profile
  between halfway bounce-back walls and Laplace's law for a sphere
  (pressure jump 2 sigma / R);
* invariants: the rest state and conservation of sum(phi).
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import closed_forms as CF
from paper_2510_18688_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.fixture(scope="module")
def O3():
    from oracle import oracle3d
    oracle3d.build()
    return oracle3d


def test_lattice_is_the_printed_d3q19(O3):
    rows = [l.split() for l in open(os.path.join(GOLDEN, "d3q19_lattice.txt"))
            if l.strip() and not l.startswith("#")]
    cx, cy, cz, w, opp = O3.lattice()
    for r in rows:
        i = int(r[0])
        assert (cx[i], cy[i], cz[i]) == (int(r[1]), int(r[2]), int(r[3]))
        assert w[i] == float(Fraction(r[4]))
    for i in range(19):
        assert (cx[opp[i]], cy[opp[i]], cz[opp[i]]) == (-cx[i], -cy[i], -cz[i])


def test_lattice_moments(O3):
    """sum w = 1, sum w c = 0, sum w c c = cs^2 I, sum w c c c = 0 and the
    fourth moment cs^4 (d_ab d_cd + d_ac d_bd + d_ad d_bc)."""
    cx, cy, cz, w, _ = O3.lattice()
    c = np.stack([cx, cy, cz], 1).astype(float)
    cs2 = 1.0 / 3.0
    assert math.isclose(w.sum(), 1.0, abs_tol=1e-15)
    assert np.abs(w @ c).max() < 1e-15
    M2 = np.einsum("i,ia,ib->ab", w, c, c)
    assert np.allclose(M2, cs2 * np.eye(3), atol=1e-15)
    M3 = np.einsum("i,ia,ib,ic->abc", w, c, c, c)
    assert np.abs(M3).max() < 1e-15
    M4 = np.einsum("i,ia,ib,ic,id->abcd", w, c, c, c, c)
    d = np.eye(3)
    iso = cs2 ** 2 * (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d)
                      + np.einsum("ad,bc->abcd", d, d))
    assert np.allclose(M4, iso, atol=1e-15)


def _project(O3, O, pops3, nz, shape2):
    """The D3Q19 populations of the first z layer summed over c_z, per D2Q9
    direction (with the populations reshaped to [lattice, i, z, y, x])."""
    cx, cy, cz, _, _ = O3.lattice()
    cx2, cy2, _, _ = O.lattice()
    out = np.zeros((pops3.shape[0], 9) + shape2)
    p = pops3.reshape(pops3.shape[0], 19, nz, *shape2)
    for i in range(19):
        j = [k for k in range(9) if (cx2[k], cy2[k]) == (cx[i], cy[i])][0]
        out[:, j] += p[:, i, 0]
    return out, p


@pytest.mark.parametrize("seed", [0, 1, 3])
def test_z_uniform_run_projects_onto_the_2d_oracle(O3, oracle_mod, seed):
    """Phase-field and enthalpy lattices (no flow, so u = 0) on a 2-D random
    state extruded along z: every z layer stays identical, and the sums of
    the D3Q19 populations over c_z equal the D2Q9 populations of the 2-D
    oracle after 60 steps (walls of every kind, cold mask, mushy nodes,
    wetting, the mass source)."""
    O = oracle_mod
    nx, ny, nz = 21, 13, 3
    wl2 = W.random_state(nx, ny, seed=seed, lattices=W.PHASE | W.HEAT)
    o2 = O.from_workload(wl2).step(60)
    o3 = O3.from_workload(W.extrude_z(wl2, nz)).step(60)
    pops2 = o2.state()[0].reshape(3, 9, ny, nx)
    pops3 = o3.state()[0]
    proj, p = _project(O3, O, pops3, nz, (ny, nx))
    for z in range(1, nz):
        assert np.array_equal(p[:, :, z], p[:, :, 0])
    scale = np.abs(pops2[1:]).max()
    assert np.abs(proj[1:] - pops2[1:]).max() <= 1e-13 * scale
    f2, f3 = o2.fields(), o3.fields()
    for k in ("phi", "fs", "fl", "T", "rhoH", "mu", "mdot"):
        assert np.abs(f3[k][1] - f2[k]).max() <= 1e-12 * max(1.0, np.abs(f2[k]).max()), k
    assert np.all(f3["uz"] == 0.0)


def test_rest_state_is_exactly_stationary(O3):
    cfg = dict(W.base_params(10, 8, bc=("periodic", "periodic", "periodic", "periodic")),
               nz=6, gz=0.0, bc=("periodic",) * 4 + ("dirichlet", "adiabatic"),
               T_wall=(0.0, 0.0, 0.0, 0.0, 0.3, 0.0))
    z = np.zeros((6, 8, 10))
    o = O3.Oracle3(cfg).init(z, z + 1.0, z + 0.3, z + 1.0)
    p0, l0 = o.state()
    o.step(100)
    p1, l1 = o.state()
    assert np.all(p1[0] == 0.0)
    assert np.array_equal(p1[1], p0[1])
    assert np.allclose(p1[2], p0[2], rtol=0, atol=1e-14)
    assert np.allclose(l1, l0, rtol=0, atol=1e-14)


def test_phi_conserved_without_mass_source(O3):
    cfg, arr = W.random_state3(14, 10, 8, seed=2)
    cfg = dict(cfg, rho_s=cfg["rho_l"])
    o = O3.Oracle3(cfg).init(arr["phi0"], arr["phi"], arr["T"], arr["fl"], arr["mask"])
    s0 = o.diagnostics()["phi_sum"]
    o.step(80)
    d = o.diagnostics()
    assert d["nonfinite"] == 0
    assert abs(d["phi_sum"] - s0) <= 1e-10 * abs(s0) + 1e-10


def test_poiseuille_3d(O3):
    """Body force along x between halfway bounce-back walls in y (periodic x
    and z): the parabolic profile of plane Poiseuille flow."""
    ny, g, nu = 32, 1e-6, 0.1
    cfg = dict(W.base_params(4, ny, lattices=W.FLOW, gx=g, nu=nu), nz=4, gz=0.0,
               bc=("periodic", "periodic", "dirichlet", "dirichlet", "periodic", "periodic"),
               T_wall=(0.0,) * 6)
    z = np.zeros((4, ny, 4))
    o = O3.Oracle3(cfg).init(z, z + 1.0, z + 0.5, z + 1.0).step(12000)
    f = o.fields()
    y = np.arange(ny) + 0.5
    ua = CF.poiseuille_u(y, ny, g, nu)
    assert np.abs(f["ux"][2, :, 1] - ua).max() < 0.01 * ua.max()
    assert np.abs(f["uz"]).max() < 1e-6 * ua.max()


def test_laplace_law_sphere(O3):
    """A static drop in a periodic box: the pressure jump is 2 sigma / R in
    three dimensions (the normalisation of Eq. (4) gives tension sigma)."""
    n, R = 36, 10.0
    cfg = dict(W.base_params(n, n, lattices=W.FLOW | W.PHASE, sigma=0.001), nz=n, gz=0.0,
               bc=("periodic",) * 6, T_wall=(0.0,) * 6)
    X, Y, Z = W._grid3(n, n, n)
    phi = np.tanh(2 * (R - np.sqrt((X - n / 2) ** 2 + (Y - n / 2) ** 2 + (Z - n / 2) ** 2)) / cfg["eps"])
    z = np.zeros((n, n, n))
    o = O3.Oracle3(cfg).init(z, phi, z + 0.5, z + 1.0).step(1500)
    p = o.fields()["p"]
    c = n // 2
    p_in = p[c - 2:c + 2, c - 2:c + 2, c - 2:c + 2].mean()
    p_out = p[:3, :3, :3].mean()
    assert (p_in - p_out) == pytest.approx(2 * cfg["sigma"] / R, rel=0.06)


@pytest.mark.parametrize("bc", [("periodic",) * 6,
                                ("periodic", "periodic", "dirichlet", "adiabatic", "adiabatic",
                                 "dirichlet")])
def test_axis_permutation_symmetry(O3, bc):
    """D3Q19 is symmetric under a cyclic permutation of the axes, so a state
    whose axes (and gravity, walls and wall temperatures) are permuted
    cyclically evolves into the permuted state: this catches an axis-specific
    slip (a y component where a z one belongs) that the z-uniform projection
    cannot see.  All three lattices, 25 steps; equality up to the rounding of
    the permuted summation order.  A link leaving through an edge between two
    walls is decided by the first of them in the order x, y, z; the cyclic
    permutation keeps that order for y and z, so x stays periodic when the
    other axes have walls."""
    cfg, arr = W.random_state3(11, 9, 7, seed=1, bc=bc)
    o = O3.from_workload((cfg, arr)).step(25)
    f = o.fields()
    # (x, y, z) -> (y, z, x): the new x axis is the old y axis, and so on
    bc, tw = cfg["bc"], cfg["T_wall"]
    cfgp = dict(cfg, nx=cfg["ny"], ny=cfg["nz"], nz=cfg["nx"],
                gx=cfg["gy"], gy=cfg["gz"], gz=cfg["gx"],
                bc=(bc[2], bc[3], bc[4], bc[5], bc[0], bc[1]),
                T_wall=(tw[2], tw[3], tw[4], tw[5], tw[0], tw[1]))
    # arrays are [z, y, x]; permuted arrays are [x, z, y] of the old ones
    arrp = {k: np.ascontiguousarray(np.transpose(v, (2, 0, 1))) for k, v in arr.items()}
    fp = O3.from_workload((cfgp, arrp)).step(25).fields()
    for k in ("phi", "fs", "fl", "T", "rhoH", "p", "rho", "mu", "w", "mdot"):
        back = np.transpose(fp[k], (1, 2, 0))
        scale = max(1e-30, np.abs(f[k]).max())
        assert np.abs(back - f[k]).max() <= 1e-10 * scale, k
    for new, old in (("ux", "uy"), ("uy", "uz"), ("uz", "ux")):
        back = np.transpose(fp[new], (1, 2, 0))
        scale = max(1e-30, np.abs(f[old]).max())
        assert np.abs(back - f[old]).max() <= 1e-9 * scale, (new, old)


def _m3(O3, v):
    cx, cy, cz, _, _ = O3.lattice()
    c = np.stack([cx, cy, cz], 1).astype(float)
    return v.sum(), c.T @ v, np.einsum("ia,ib,i->ab", c, c, v)


@pytest.mark.parametrize("seed", range(3))
def test_equilibrium_and_source_moments_3d(O3, seed):
    """The moments Eqs. (14), (16), (19), (20), (25) must have on D3Q19 for
    the model to recover its macroscopic equations (the 3-D form of the 2-D
    moment pins), including the R-FT variant: its trace term c.c - 3 cs^2
    adds cs^2 S I to the second moment of F_i and nothing to the zeroth (a
    2-D trace c.c - 2 cs^2 would shift the zeroth moment by cs^2 S)."""
    cs2 = 1.0 / 3.0
    r = np.random.default_rng(40 + seed)
    p, rho = r.uniform(-1e-3, 1e-3), r.uniform(0.1, 1.0)
    u = r.uniform(-0.05, 0.05, 3)
    S, F, fp, Ft = r.normal() * 1e-3, r.normal(size=3) * 1e-3, r.normal(size=3) * 1e-3, r.normal(size=3) * 1e-3
    feq, Fi = O3.node_flow(p, rho, u, S, F, fp, Ft)
    m0, m1, m2 = _m3(O3, feq)
    assert abs(m0) < 1e-15
    assert np.allclose(m1, rho * u, rtol=1e-13, atol=1e-17)
    assert np.allclose(m2, p * np.eye(3) + rho * np.outer(u, u), rtol=1e-12, atol=1e-17)
    m0, m1, m2 = _m3(O3, Fi)
    assert abs(m0 - S) < 1e-15
    assert np.allclose(m1, F + rho * fp, rtol=1e-13, atol=1e-18)
    assert np.allclose(m2, cs2 * S * np.eye(3) + np.outer(u, Ft) + np.outer(Ft, u), rtol=1e-12,
                       atol=1e-18)
    _, Fv = O3.node_flow(p, rho, u, S, F, fp, Ft, readings=1)
    v0, v1, v2 = _m3(O3, Fv)
    assert abs(v0 - S) < 1e-15 and np.allclose(v1, m1, atol=1e-18)
    assert np.allclose(v2 - m2, cs2 * S * np.eye(3), atol=1e-17)
    phi, mu, eta = r.uniform(-1, 1), r.normal() * 1e-3, r.uniform(0.5, 2)
    phu, dphu, md = r.normal(size=3) * 1e-2, r.normal(size=3) * 1e-4, r.normal() * 1e-4
    geq, G = O3.node_phase(phi, mu, eta, phu, dphu, md)
    m0, m1, m2 = _m3(O3, geq)
    assert abs(m0 - phi) < 1e-15
    assert np.allclose(m1, phu, atol=1e-16)
    assert np.allclose(m2, cs2 * eta * mu * np.eye(3), atol=1e-17)
    m0, m1, _ = _m3(O3, G)
    assert abs(m0 - phi * md) < 1e-18
    assert np.allclose(m1, dphu, atol=1e-18)
    rhoH, C, T, rr = r.uniform(-2, 12), r.uniform(0.5, 2), r.uniform(-1, 1), r.uniform(0.5, 1.5)
    heq, H = O3.node_heat(rhoH, C, T, rr, u, md)
    m0, m1, m2 = _m3(O3, heq)
    assert abs(m0 - rhoH) < 1e-13
    assert np.allclose(m1, C * T * u, rtol=1e-12, atol=1e-16)
    assert np.allclose(m2, rr * T * cs2 * np.eye(3) + C * T * np.outer(u, u), rtol=1e-12, atol=1e-15)
    assert abs(H.sum() - C * T * md) < 1e-16
