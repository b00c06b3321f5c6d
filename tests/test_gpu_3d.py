"""Parity of the three-dimensional (D3Q19) step with the 3-D FP64 oracle,
through the C ABI (lbm3_*).

Grids are chosen ragged against the 32 x 4 x 2 thread blocks (tails in every
axis) and every boundary set of the seeded random states is covered (walls
of both kinds on each axis, periodic axes, edges and corners where walls
meet), with each lattice subset.  FP64 agrees with the oracle to 1e-10 of
each field's scale (element by element), FP32 to 1e-4 in relative L2.  The
full-size rough fracture (256 x 128 x 30, the Sec. 4.5 shape) is compared
node by node after a few steps.
"""
import numpy as np
import pytest

from paper_2510_18688_gb300 import workloads as W

pytestmark = pytest.mark.gpu

F3 = ("phi", "fs", "fl", "T", "rhoH", "p", "ux", "uy", "uz", "rho", "mu", "w", "mdot")


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from oracle import oracle3d as O3
    from paper_2510_18688_gb300 import build, lbm
    build.build()
    lbm.load()
    O3.build()
    return O3, lbm


def _compare(fo, fg, prec, tag=""):
    for k in F3:
        a, b = fo[k], fg[k]
        assert np.all(np.isfinite(b)), (tag, k)
        scale = max(np.abs(a).max(), 1e-30)
        if prec == "fp64":
            err = np.abs(a - b).max() / scale
            assert err <= 1e-10, (tag, k, err)
        else:
            num = np.linalg.norm((a - b).ravel())
            den = max(np.linalg.norm(a.ravel()), 1e-30 * np.sqrt(a.size))
            assert num / den <= 1e-4 or np.abs(a - b).max() <= 1e-6 * max(scale, 1e-3), (tag, k, num / den)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_random_state_matches_oracle(env, prec, seed):
    O3, lbm = env
    wl = W.random_state3(37, 13, 9, seed=seed)
    steps = 40
    o = O3.from_workload(wl).step(steps)
    s = lbm.Solver3(wl[0], prec).set_geometry(wl[1]).step(steps)
    assert s.steps_done == steps
    _compare(o.fields(), s.fields(), prec, f"seed {seed}")
    do, dg = o.diagnostics(), s.diagnostics()
    for k in ("mass", "material_mass", "rhoH", "liquid_volume", "material_volume",
              "frozen_volume", "phi_sum"):
        tol = 1e-10 if prec == "fp64" else 1e-5
        assert abs(dg[k] - do[k]) <= tol * max(1.0, abs(do[k])), (k, dg[k], do[k])
    assert dg["nonfinite"] == 0
    s.close()


@pytest.mark.parametrize("lattices", [W.FLOW, W.PHASE, W.HEAT, W.FLOW | W.PHASE,
                                      W.PHASE | W.HEAT, W.FLOW | W.HEAT])
def test_lattice_subsets_match_oracle(env, lattices):
    O3, lbm = env
    wl = W.random_state3(33, 9, 10, seed=1, lattices=lattices)
    o = O3.from_workload(wl).step(30)
    s = lbm.Solver3(wl[0], "fp64").set_geometry(wl[1]).step(30)
    _compare(o.fields(), s.fields(), "fp64", f"lattices {lattices}")
    s.close()


def test_initial_state_and_host_inputs(env):
    """Step 0 (set_geometry) equals the oracle's initial state, from host and
    from device inputs alike."""
    O3, lbm = env
    wl = W.random_state3(20, 11, 6, seed=3)
    o = O3.from_workload(wl)
    fo = o.fields()
    a = lbm.Solver3(wl[0], "fp64").set_geometry(wl[1], on_device=True)
    b = lbm.Solver3(wl[0], "fp64").set_geometry(wl[1], on_device=False)
    fa, fb = a.fields(), b.fields()
    _compare(fo, fa, "fp64", "device inputs")
    for k in F3:
        assert np.array_equal(fa[k], fb[k]), k
    a.close()
    b.close()


def test_rough_fracture_full_size(env):
    """The 256 x 128 x 30 rough fracture (Sec. 4.5 shape: cold wall at x = 0,
    a liquid column with three bubbles in a self-affine aperture, periodic
    y and z), node by node against the oracle after 4 steps, in FP64 and
    FP32."""
    O3, lbm = env
    wl = W.rough_fracture()
    o = O3.from_workload(wl).step(4)
    fo = o.fields()
    for prec in ("fp64", "fp32"):
        s = lbm.Solver3(wl[0], prec).set_geometry(wl[1]).step(4)
        _compare(fo, s.fields(), prec, f"fracture {prec}")
        s.close()


def test_extruded_2d_state_stays_z_uniform(env):
    """A 2-D state repeated along a periodic z axis stays exactly uniform in
    z on the GPU too (all three lattices)."""
    O3, lbm = env
    wl = W.extrude_z(W.random_state(24, 12, seed=1), 4)
    s = lbm.Solver3(wl[0], "fp64").set_geometry(wl[1]).step(25)
    f = s.fields()
    for k in F3:
        for z in range(1, 4):
            assert np.array_equal(f[k][z], f[k][0]), (k, z)
    # the z component of the stencils cancels up to the rounding of its
    # summation order
    assert np.abs(f["uz"]).max() <= 1e-10 * max(np.abs(f["ux"]).max(), np.abs(f["uy"]).max())
    s.close()


@pytest.mark.parametrize("shape,bc", [
    ((2, 2, 2), ("periodic",) * 6),
    ((2, 2, 2), ("dirichlet", "adiabatic", "adiabatic", "dirichlet", "dirichlet", "dirichlet")),
    ((33, 2, 3), ("periodic", "periodic", "dirichlet", "dirichlet", "periodic", "periodic")),
    ((3, 5, 2), ("adiabatic", "dirichlet", "periodic", "periodic", "dirichlet", "adiabatic")),
])
def test_degenerate_grids_match_oracle(env, shape, bc):
    """The smallest grids: every node is on a face, edge or corner (links
    leave through several walls at once; a periodic axis of length 2 wraps
    both neighbours onto the same node)."""
    O3, lbm = env
    nx, ny, nz = shape
    wl = W.random_state3(nx, ny, nz, seed=5, bc=bc)
    o = O3.from_workload(wl).step(20)
    s = lbm.Solver3(wl[0], "fp64").set_geometry(wl[1]).step(20)
    _compare(o.fields(), s.fields(), "fp64", f"{shape} {bc}")
    s.close()


def test_nonfinite_state_is_reported(env):
    """A non-finite initial temperature makes the state non-finite; the
    diagnostics count the nodes instead of failing silently."""
    O3, lbm = env
    cfg, arr = W.random_state3(20, 8, 6, seed=2)
    arr = dict(arr)
    T = arr["T"].copy()
    T[3, 4, 5] = np.nan
    arr["T"] = T
    s = lbm.Solver3(cfg, "fp32").set_geometry(arr).step(3)
    d = s.diagnostics()
    assert d["nonfinite"] >= 1
    s.close()


def test_checkpoint_resume_is_bit_exact(env):
    """Run 2N steps, or run N, save, load into a fresh context, run N: the
    same state bit for bit (FP32 and FP64)."""
    O3, lbm = env
    wl = W.random_state3(30, 10, 7, seed=1)
    for prec in ("fp32", "fp64"):
        a = lbm.Solver3(wl[0], prec).set_geometry(wl[1]).step(24)
        b = lbm.Solver3(wl[0], prec).set_geometry(wl[1]).step(12)
        blob = b.save_state()
        b.close()
        c = lbm.Solver3(wl[0], prec).set_geometry(wl[1]).load_state(blob).step(12)
        assert c.steps_done == 24
        fa, fc = a.fields(), c.fields()
        for k in F3:
            assert np.array_equal(fa[k], fc[k]), (prec, k)
        other = lbm.Solver3(dict(wl[0], nz=8), prec).set_geometry(W.random_state3(30, 10, 8, seed=1)[1])
        with pytest.raises(lbm.LbmError):
            other.load_state(blob)
        for s in (a, c, other):
            s.close()


def test_tangent_3d_matches_fp64_and_differences(env):
    """Forward mode on D3Q19: the tangent context's values are the FP64
    step's, and its derivatives of the frozen fraction and of the
    temperature field along a wall temperature, the cold-mask temperature,
    the contact angle and L agree with central differences of the FP64 3-D
    step."""
    O3, lbm = env
    cfg, arr = W.random_state3(20, 12, 8, seed=3)
    steps = 40

    def ff_fields(c):
        u = lbm.Solver3(c, "fp64").set_geometry(arr).step(steps)
        d = u.diagnostics()
        f = u.fields(("T", "phi"))
        u.close()
        return d["frozen_volume"] / d["material_volume"], f

    ff0, f0 = ff_fields(cfg)
    dirs = [("T_wall", {"T_wall": [1.0, 0, 0, 0, 0, 0]}, 1e-6),
            ("T_cold", {"T_cold": 1.0}, 1e-6),
            ("theta_deg", {"theta_deg": 1.0}, 1e-4),
            ("latent", {"latent": 1.0}, 1e-6 * cfg["latent"])]
    for name, t, h in dirs:
        s = lbm.Solver3(cfg, "tangent", tangent=t).set_geometry(arr).step(steps)
        d = s.diagnostics()
        dt = s.tangent_diagnostics()
        f = s.fields(("T", "phi"))
        df = s.tangent_fields(("T",))
        s.close()
        fz, mv = d["frozen_volume"], d["material_volume"]
        assert abs(fz / mv - ff0) <= 1e-12
        assert np.abs(f["T"] - f0["T"]).max() <= 1e-12 * max(1.0, np.abs(f0["T"]).max())
        dff = (dt["frozen_volume"] * mv - fz * dt["material_volume"]) / mv ** 2
        if name == "T_wall":
            cp, cm = dict(cfg, T_wall=(cfg["T_wall"][0] + h,) + tuple(cfg["T_wall"][1:])), \
                dict(cfg, T_wall=(cfg["T_wall"][0] - h,) + tuple(cfg["T_wall"][1:]))
        else:
            cp, cm = dict(cfg, **{name: cfg[name] + h}), dict(cfg, **{name: cfg[name] - h})
        (fp, Fp), (fm, Fm) = ff_fields(cp), ff_fields(cm)
        fd = (fp - fm) / (2 * h)
        fdT = (Fp["T"] - Fm["T"]) / (2 * h)
        print(f"\n{name}: dFF tangent {dff:.10e} FD {fd:.10e}; dT max {np.abs(df['T']).max():.4e} "
              f"err {np.abs(df['T'] - fdT).max():.3e}")
        assert abs(dff - fd) <= 1e-4 * abs(fd) + 1e-9, (name, dff, fd)
        assert np.abs(df["T"] - fdT).max() <= 1e-4 * max(np.abs(fdT).max(), 1e-6), name


@pytest.mark.slow
def test_grid_beyond_31_bit_population_offsets(env):
    """A grid whose 57 population planes span more than 2^31 elements (39.3M
    nodes, 64-bit plane offsets): a small periodic state repeated 200 times
    along x must step into exactly the repeated result of the small grid
    (translation symmetry; the small grid itself is checked against the
    oracle above)."""
    O3, lbm = env
    import torch
    reps = 200
    cfg, arr = W.random_state3(48, 64, 64, seed=2)  # periodic on all six faces
    assert all(b == "periodic" for b in cfg["bc"])
    small = lbm.Solver3(cfg, "fp32").set_geometry(arr).step(4)
    fs = small.fields(("phi", "T"))
    small.close()
    big_cfg = dict(cfg, nx=cfg["nx"] * reps)
    big_arr = {k: np.ascontiguousarray(np.tile(v, (1, 1, reps))) for k, v in arr.items()}
    assert 57 * big_cfg["nx"] * cfg["ny"] * cfg["nz"] > 2 ** 31
    big = lbm.Solver3(big_cfg, "fp32").set_geometry(big_arr).step(4)
    fb = big.fields(("phi", "T"))
    d = big.diagnostics()
    big.close()
    torch.cuda.empty_cache()
    for k in ("phi", "T"):
        assert np.array_equal(fb[k], np.tile(fs[k], (1, 1, reps))), k
    assert d["nonfinite"] == 0
