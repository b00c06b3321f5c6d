"""Pin of the oracle's cold-mask pass (reading R-BC): the interior Dirichlet
substrate of the droplet workloads of Secs. 4.3-4.4, whose enthalpy
populations are reset after streaming to the equilibrium of Eq. (25) at the
mask temperature T_cold with u = 0.

Two checks that do not restate the oracle's formulas:

* a masked node holds T_cold: the inversion of Eq. (8) of its reset
  populations gives back T_cold to round-off, with the liquid fraction of
  that temperature (a wrong latent part, heat capacity or weight in the
  reset, or a reset applied before streaming, breaks this);
* the masked block is a Dirichlet boundary at its last node: pure
  conduction (no phase change) from it into a uniform medium follows the
  closed form T = T_c + (T0 - T_c) erf((x - x_b) / (2 sqrt(alpha t))) with
  x_b the last masked node and alpha = lambda / (rho C_p), in a warm column
  (everything liquid, T > T_m) and in a frozen one (T < T_m everywhere).
"""
import math

import numpy as np
import pytest

from paper_2510_18688_gb300 import workloads as W


@pytest.fixture(scope="module")
def O(oracle_mod):
    return oracle_mod


def mask_column(T0, T_c, nx=240, ny=4, k=8, lam=0.2):
    """Enthalpy lattice alone; the first k columns masked at T_c; adiabatic
    x walls (the mask alone drives the heat flow), periodic y; rho = C_p = 1
    in every phase, so alpha = lambda."""
    cfg = W.base_params(nx, ny, lattices=W.HEAT, rho_s=1.0, rho_g=1.0, cp_g=1.0,
                        lambda_l=lam, bc=("adiabatic", "adiabatic", "periodic", "periodic"),
                        T_cold=T_c)
    cfg["lambda_s"] = cfg["lambda_g"] = lam
    z = np.zeros((ny, nx))
    mask = np.zeros((ny, nx), dtype=np.uint8)
    mask[:, :k] = 1
    fl = z + (1.0 if T0 >= 0.0 else 0.0)
    return cfg, W._arrays(z, z + 1.0, z + T0, fl, mask)


def erf_profile(x, t, T0, T_c, xb, alpha):
    return T_c + (T0 - T_c) * np.array([math.erf((xi - xb) / (2.0 * math.sqrt(alpha * t)))
                                        for xi in x])


@pytest.mark.parametrize("T0,T_c", [(0.5, 1.5), (-0.5, -1.5)], ids=["warm", "frozen"])
def test_mask_is_a_dirichlet_boundary_at_its_last_node(O, T0, T_c):
    k, lam, t = 8, 0.2, 3000
    wl = mask_column(T0, T_c, k=k, lam=lam)
    o = O.from_workload(wl).step(t)
    f = o.fields()
    T = f["T"]
    # masked nodes read back T_c, and the liquid fraction of T_c
    assert np.abs(T[:, :k] - T_c).max() < 1e-12
    assert np.all(f["fl"][:, :k] == (1.0 if T_c >= 0.0 else 0.0))
    # no phase change anywhere: the liquid fraction stays that of T0
    assert np.all(f["fl"] == (1.0 if T0 >= 0.0 else 0.0))
    x = np.arange(k, 140, dtype=np.float64)
    want = erf_profile(x, t, T0, T_c, k - 1.0, lam)
    err = np.abs(T[1, k:140] - want).max() / abs(T0 - T_c)
    assert err < 0.01, err
    # the Dirichlet point is the last masked node, not the edge half a node
    # further on: the wrong position is clearly worse
    other = erf_profile(x, t, T0, T_c, k - 0.5, lam)
    assert np.abs(T[1, k:140] - other).max() / abs(T0 - T_c) > 2 * err


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_masked_nodes_hold_T_cold_in_random_states(O, seed):
    """Every masked node of a random state with all lattices (moving fluid,
    phase field, solid blobs, mushy band) reads back T_cold after 60 steps,
    whatever its weight w and phi0."""
    cfg, arr = W.random_state(48, 32, seed=seed)
    assert arr["mask"].any()
    o = O.from_workload((cfg, arr)).step(60)
    f = o.fields()
    m = arr["mask"] != 0
    assert np.abs(f["T"][m] - cfg["T_cold"]).max() < 1e-12
    assert np.all(f["fl"][m] == (1.0 if cfg["T_cold"] >= 0.0 else 0.0))
