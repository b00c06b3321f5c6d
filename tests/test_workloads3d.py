"""The synthetic 3-D inputs follow their stated recipes (CPU only): the rough
fracture has the Sec. 4.5 shape (256 x 128 x 30, a 128-wide self-affine
fracture repeated once along x, rock outside an aperture along z, a liquid
column to 0.75 Lx with three bubbles at the printed centres, a cold wall at
x = 0, periodic y and z), and the generators are seeded."""
import numpy as np

from paper_2510_18688_gb300 import workloads as W


def test_rough_fracture_recipe():
    cfg, arr = W.rough_fracture()
    nx, ny, nz = cfg["nx"], cfg["ny"], cfg["nz"]
    assert (nx, ny, nz) == (256, 128, 30)
    assert cfg["bc"] == ("dirichlet", "adiabatic", "periodic", "periodic", "periodic", "periodic")
    assert cfg["T_wall"][0] < 0.0 and cfg["lattices"] == W.ALL
    phi0, phi = arr["phi0"], arr["phi"]
    assert phi0.shape == (nz, ny, nx)
    # repeated once along x: the two halves of the rock are identical
    assert np.array_equal(phi0[:, :, :128], phi0[:, :, 128:])
    # rock outside the aperture along z: solid at the z ends, open in the middle
    solid = phi0 > 0.5
    assert solid[0].mean() > 0.95 and solid[-1].mean() > 0.95
    assert solid[nz // 2].mean() < 0.05
    aperture = (~solid).sum(axis=0)  # [ny, nx]
    assert 10.0 < aperture.mean() < 14.0 and aperture.min() >= 2
    # liquid column up to 0.75 Lx, gas above it (in the open aperture)
    mid = nz // 2
    assert (phi[mid, :, : int(0.70 * nx)] > 0).mean() > 0.9
    assert (phi[mid, :, int(0.80 * nx):] < 0).all()
    # the largest bubble (radius 0.075 Lx) at (0.25 Lx, 0.25 Ly, 0.5 Lz)
    assert phi[mid, int(0.25 * ny), int(0.25 * nx)] < -0.9
    assert np.all(arr["T"] == arr["T"].flat[0]) and np.all(arr["fl"] == 1.0)


def test_rough_fracture_is_seeded():
    a = W.rough_fracture(seed=3)[1]["phi0"]
    b = W.rough_fracture(seed=3)[1]["phi0"]
    c = W.rough_fracture(seed=4)[1]["phi0"]
    assert np.array_equal(a, b) and not np.array_equal(a, c)


def test_random_state3_covers_every_branch():
    """The states of the 3-D parity tests (37 x 13 x 9, one boundary set per
    seed) hold solid, liquid and gas, liquid below and above T_m, a mushy
    band and masked nodes."""
    for seed in range(4):
        cfg, arr = W.random_state3(37, 13, 9, seed=seed)
        assert arr["phi"].shape == (9, 13, 37)
        T, fl = arr["T"], arr["fl"]
        assert (T < 0).any() and (T > 0).any()
        assert ((fl > 0) & (fl < 1)).any()  # a mushy band
        assert arr["mask"].any() and (arr["phi0"] > 0.5).any()
        assert (arr["phi"] > 0.5).any() and (arr["phi"] < -0.5).any()
        assert len(cfg["bc"]) == 6 and len(cfg["T_wall"]) == 6 and "gz" in cfg


def test_extrude_z_repeats_the_2d_state():
    wl2 = W.random_state(21, 13, seed=2)
    cfg, arr = W.extrude_z(wl2, 4)
    assert cfg["nz"] == 4 and cfg["bc"][4:] == ("periodic", "periodic")
    for k, v in wl2[1].items():
        assert arr[k].shape == (4,) + v.shape
        for z in range(4):
            assert np.array_equal(arr[k][z], v)
