"""Checks of the closed forms and of the paper's printed numbers.

The closed forms in ``closed_forms.py`` are what the oracle is pinned to, so
they are checked themselves: against the values the paper prints (Table 1,
Table 2 and the dimensionless numbers of Sec. 4.3, stored under
``tests/golden/``), against each other where one reduces to another, and
against the identity the paper prints for the cylinder case (Eq. (37)).
"""
import math
import os

import numpy as np
import pytest

import closed_forms as CF
from paper_2510_18688_gb300 import workloads as W

GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _rows(name):
    with open(os.path.join(GOLD, name)) as fh:
        return [ln.split() for ln in fh if ln.strip() and not ln.startswith("#")]


def test_table1_analytic_column_is_mass_conservation():
    """Table 1: the analytical h_f/h0 is rho_l/rho_s to four decimals, and
    the paper's numerical results lie within its stated 1.5 % of it."""
    for r in _rows("table1_final_height.txt"):
        ratio, ana = float(r[0]), float(r[1])
        assert CF.stefan_final_height(1.0, ratio) == pytest.approx(ana, abs=5e-5)
        for num in map(float, r[2:]):
            assert abs(num / ana - 1) < 0.015


def test_table2_gives_the_dimensionless_numbers_of_sec43():
    """Sec. 4.3: water at a -10 C wall gives Ste = 0.13 and rho_s/rho_l = 0.92
    (Table 2); Ste = Cp_l (T_m - T_w) / L with the workload mapping."""
    rows = {r[0]: r[1:] for r in _rows("table2_properties.txt")}
    rho_l, rho_s, _, _, cp_l, _, L, Tm = map(float, rows["water"])
    ste = cp_l * (Tm - (-10.0)) / L
    assert round(ste, 2) == float(rows["water_ste"][0])
    assert round(rho_s / rho_l, 2) == float(rows["water_density_ratio"][0])
    # the workload mapping inverts Ste = Cp_l (T_m - T_w) / L
    assert W.latent_from_stefan(ste, cp_l, -10.0) == pytest.approx(L, rel=1e-12)


def test_stefan_kappa_reduces_to_two_phase_neumann():
    """Reading R-STE: with rho_s = rho_l and equal heat capacities Eq. (35)
    must coincide with the two-phase Neumann equation Eq. (33)."""
    for ste, T0, ar in ((0.1, 1.0, 1.0), (0.2, 0.5, 0.7), (0.15, 1.0, 1.6)):
        a_l = 0.2
        a_s = ar * a_l
        L = 1.0 / ste  # Cp = 1, T_m - T_w = 1
        k = CF.neumann_k(1.0, 1.0, L, 0.0, -1.0, T0, a_s, a_l)
        kap = CF.stefan_kappa(ste, a_l, a_s, T0, 0.0, -1.0, a_s, a_l, 1.0)
        assert kap == pytest.approx(k, rel=1e-9)


def test_neumann_one_phase_limit():
    """With T0 = T_m the two-phase root equals the one-phase root of Eq. (31),
    k exp(k^2) erf(k) sqrt(pi) = Ste."""
    for ste in (0.05, 0.1, 0.5):
        k = CF.neumann_k(1.0, 1.0, 1.0 / ste, 0.0, -1.0, 0.0, 0.2, 0.2)
        assert k * math.exp(k * k) * math.erf(k) * math.sqrt(math.pi) == pytest.approx(ste, rel=1e-10)


@pytest.mark.parametrize("theta", [30.0, 60.0, 90.0, 120.0, 150.0])
def test_cylinder_droplet_satisfies_eq37(theta):
    """Eq. (37) for R0 = Rs: (pi/3 + sqrt(3)/2) Rs^2 = (alpha + theta) R^2
    - alpha Rs^2 + R Rs sin(theta), with alpha = acos((Rs - R cos theta)/k)
    (reading R-CYL of the garbled alpha)."""
    Rs = 50.0
    R, k, H = CF.cylinder_droplet_equilibrium(Rs, Rs, theta)
    th = math.radians(theta)
    alpha = math.acos((Rs - R * math.cos(th)) / k)
    lhs = (math.pi / 3 + math.sqrt(3) / 2) * Rs * Rs
    rhs = (alpha + th) * R * R - alpha * Rs * Rs + R * Rs * math.sin(th)
    assert rhs == pytest.approx(lhs, rel=1e-9)
    assert H == pytest.approx(k + R)
    # more hydrophobic -> taller drop (Fig. 7(b) trend)
    if theta > 30.0:
        assert H > CF.cylinder_droplet_equilibrium(Rs, Rs, theta - 30.0)[2]


def test_poiseuille_and_conduction_closed_forms():
    y = np.linspace(0, 10, 11)
    u = CF.poiseuille_u(y, 10.0, 1e-6, 0.1)
    assert u[0] == 0.0 and u[-1] == 0.0 and u.argmax() == 5
    assert CF.conduction_T(0.0, 100.0, 1.0, 0.0, 0.2) == 0.0
    assert CF.conduction_T(1e6, 100.0, 1.0, 0.0, 0.2) == pytest.approx(1.0)
