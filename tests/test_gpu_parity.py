"""Parity of the sm_103a path (through the C ABI) with the FP64 oracle.

Same seeded inputs on both sides; the GPU result is compared element by
element with the oracle:

* FP64 path: max |gpu - oracle| <= 1e-10 * max |oracle| per field (the bar
  for the double-precision kernels);
* FP32 path: relative L2 error <= 1e-4 per field (populations stored and
  collided in float); the mass source mdot, a rate formed by differencing
  two consecutive float liquid fractions, is held to 1e-3.

Grids are chosen to span several 32 x 8 tiles with ragged tails in both
directions; the full-size workloads (512^2 droplet, 2048 x 1024 porous
medium, 256^2 cylinder instance, the 400 x 4 and 512 x 8 column problems)
are compared on every node after a step count the oracle finishes in
seconds.
"""
import numpy as np
import pytest

from paper_2510_18688_gb300 import workloads as W

pytestmark = pytest.mark.gpu

FIELDS = ("phi", "fs", "fl", "T", "rhoH", "p", "ux", "uy", "rho", "mu", "w", "mdot")


@pytest.fixture(scope="module")
def env(oracle_mod):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_18688_gb300 import build, lbm
    build.build()
    lbm.load()
    return oracle_mod, lbm


def _max_rel(a, b):
    scale = np.abs(b).max()
    err = np.abs(a - b).max()
    return err / scale if scale > 0 else err


def _l2_rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / nb if nb > 0 else np.linalg.norm(a)


def _vel_l2_rel(got, ref):
    """Relative L2 error of the velocity as one vector field (a component
    that is zero up to round-off in the oracle, e.g. u_y of a column, has no
    relative error of its own)."""
    d = np.hypot(got["ux"] - ref["ux"], got["uy"] - ref["uy"])
    n = np.linalg.norm(np.hypot(ref["ux"], ref["uy"]))
    return np.linalg.norm(d) / n if n > 0 else np.linalg.norm(d)


def _compare(got, ref, prec, tol=None, fields=FIELDS):
    bad = {}
    for k in fields:
        if prec == "fp64":
            e = _max_rel(got[k], ref[k])
            t = 1e-10 if tol is None else tol
        else:
            e = _vel_l2_rel(got, ref) if k in ("ux", "uy") else _l2_rel(got[k], ref[k])
            t = 1e-4 if tol is None else tol
        if not e <= t:
            bad[k] = e
    assert not bad, f"{prec}: fields off the oracle: {bad}"


def _run_pair(env, wl, steps, prec):
    O, lbm = env
    cfg, arr = wl
    ref = O.from_workload(wl).step(steps).fields()
    s = lbm.Solver(cfg, precision=prec).set_geometry(arr).step(steps)
    got = s.fields()
    s.close()
    return got, ref


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("seed,nx,ny", [(0, 45, 19), (1, 67, 33), (2, 37, 41), (3, 96, 24),
                                        (4, 33, 9), (5, 70, 17)])
def test_random_states(env, prec, seed, nx, ny):
    """Every branch: gas, liquid, ice, mushy nodes, solid blobs, cold mask,
    periodic/Dirichlet/adiabatic sides, gravity, random angles."""
    got, ref = _run_pair(env, W.random_state(nx, ny, seed=seed), 120, prec)
    _compare(got, ref, prec)


@pytest.mark.parametrize("prec", ["fp64"])
@pytest.mark.parametrize("seed", [0, 3])
def test_two_kernel_step(env, prec, seed, monkeypatch):
    """The two-kernel form of the step (macro pass, then collide pass),
    selected with LBM_STEP_KERNEL=split when an FP64 context is created
    (float contexts always take the fused step)."""
    monkeypatch.setenv("LBM_STEP_KERNEL", "split")
    got, ref = _run_pair(env, W.random_state(53, 29, seed=seed), 90, prec)
    _compare(got, ref, prec)
    got, ref = _run_pair(env, W.random_state(47, 31, seed=seed, lattices=5), 40, prec)
    _compare(got, ref, prec)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("lat", [1, 2, 4, 3, 5, 6])
def test_lattice_subsets(env, prec, lat):
    """Flow, phase and enthalpy lattices switched on alone and in pairs."""
    got, ref = _run_pair(env, W.random_state(41, 27, seed=7, lattices=lat), 80, prec)
    _compare(got, ref, prec)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_tiny_and_degenerate_grids(env, prec):
    """2 x 2 and single-tile-column grids, all walls and all periodic."""
    for (nx, ny), bc in (((2, 2), ("periodic",) * 4),
                         ((3, 2), ("dirichlet", "adiabatic", "dirichlet", "adiabatic")),
                         ((2, 40), ("adiabatic", "dirichlet", "periodic", "periodic")),
                         ((33, 1 + 1), ("periodic", "periodic", "dirichlet", "dirichlet"))):
        got, ref = _run_pair(env, W.random_state(nx, ny, seed=11, bc=bc, n_blobs=1), 30, prec)
        # on a handful of nodes the velocity and pressure stay at the
        # float noise level of the forcing, so FP32 gets 1e-3 there
        _compare(got, ref, prec, tol=1e-3 if prec == "fp32" else None)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_readings_variant(env, prec):
    """Variant bit of the modified force (reading R-FT)."""
    cfg, arr = W.random_state(40, 30, seed=5)
    cfg["readings"] = 1
    got, ref = _run_pair(env, (cfg, arr), 60, prec)
    _compare(got, ref, prec)


def test_neumann_column_full_run(env):
    """400 x 4 conduction-induced freezing, FP64, the full 20k steps."""
    got, ref = _run_pair(env, W.neumann(), 20000, "fp64")
    _compare(got, ref, "fp64")


def _front_and_frozen(O, f):
    """Ice front along row 0 (crossing of w (1 - fl) through 1/2) and the
    frozen volume sum w (1 - fl) of a field set."""
    x_ice = O.crossings(f["phi"], f["w"], f["fl"], 0, 0)[1]
    return x_ice, float(np.sum(f["w"] * (1.0 - f["fl"])))


def test_neumann_column_fp32_full_run(env):
    """400 x 4 conduction-induced freezing (Sec. 4.1), FP32 against the FP64
    oracle for the full 20k steps: every field within 1e-4 relative L2 (the
    velocity and pressure are zero in the oracle and must stay zero up to
    round-off), the ice front and the frozen volume within 0.5 %."""
    O, lbm = env
    got, ref = _run_pair(env, W.neumann(), 20000, "fp32")
    _compare(got, ref, "fp32", tol=1e-4)
    (xg, vg), (xr, vr) = _front_and_frozen(O, got), _front_and_frozen(O, ref)
    assert abs(xg - xr) <= 0.005 * xr, (xg, xr)
    assert abs(vg - vr) <= 0.005 * vr, (vg, vr)


def test_stefan_column_fp32(env):
    """512 x 8 three-phase Stefan problem, FP32 against FP64, 5000 steps:
    every field (the velocity as a vector: u_y is zero up to round-off in
    the oracle)."""
    got, ref = _run_pair(env, W.stefan(), 5000, "fp32")
    _compare(got, ref, "fp32", tol=1e-4)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_sessile_droplet_512(env, prec):
    """The 512^2 droplet workload at full size (every node compared)."""
    got, ref = _run_pair(env, W.sessile_droplet(512, seed=0), 12, prec)
    _compare(got, ref, prec)


def test_cylinder_instance(env):
    got, ref = _run_pair(env, W.cylinder_droplet(256, seed=3), 30, "fp64")
    _compare(got, ref, "fp64")


def test_porous_2048x1024_fp32(env):
    """The 2048 x 1024 porous medium at full size, FP32, 4 steps."""
    got, ref = _run_pair(env, W.porous(seed=0), 4, "fp32")
    _compare(got, ref, "fp32")


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_diagnostics_match_oracle(env, prec):
    O, lbm = env
    wl = W.random_state(64, 48, seed=3)
    o = O.from_workload(wl).step(50)
    dref = o.diagnostics()
    s = lbm.Solver(wl[0], precision=prec).set_geometry(wl[1]).step(50)
    d = s.diagnostics()
    tol = 1e-12 if prec == "fp64" else 1e-5
    n = 64 * 48
    for k, v in dref.items():
        # sums of O(1) per-node values: relative tolerance plus n * tol
        assert abs(d[k] - v) <= tol * (abs(v) + n), (k, d[k], v)
    assert d["step"] == 50


def test_fused_diagnostics_equal_readout(env):
    """Diagnostics fused into the step kernel (diag_every) equal those of
    the separate read-out pass on the same state, bit for bit."""
    O, lbm = env
    cfg, arr = W.random_state(50, 30, seed=4)
    s = lbm.Solver(cfg, precision="fp64", diag_every=5).set_geometry(arr).step(10)
    # steps 0 and 5 reduce their input states; the latest describes state 5
    fused = s.diagnostics(compute=False)
    assert fused["step"] == 5
    t = lbm.Solver(cfg, precision="fp64").set_geometry(arr).step(5)
    sep = t.diagnostics()
    for k in sep:
        assert fused[k] == sep[k], k


def test_host_and_device_io_agree(env):
    O, lbm = env
    cfg, arr = W.random_state(48, 20, seed=6)
    a = lbm.Solver(cfg, precision="fp64").set_geometry(arr, on_device=True).step(15)
    b = lbm.Solver(cfg, precision="fp64").set_geometry(arr, on_device=False).step(15)
    fa = a.fields(host=True)
    fb = {k: v.cpu().numpy() for k, v in b.fields(host=False).items()}
    for k in FIELDS:
        assert np.array_equal(fa[k], fb[k]), k


def test_checkpoint_resume_is_bitwise(env):
    O, lbm = env
    cfg, arr = W.random_state(40, 24, seed=8)
    a = lbm.Solver(cfg, precision="fp32").set_geometry(arr).step(40)
    b = lbm.Solver(cfg, precision="fp32").set_geometry(arr).step(20)
    blob = b.save()
    c = lbm.Solver(cfg, precision="fp32").set_geometry(arr)
    c.load(blob)
    assert c.steps_done == 20
    c.step(20)
    fa, fc = a.fields(), c.fields()
    for k in FIELDS:
        assert np.array_equal(fa[k], fc[k]), k


def test_runs_are_deterministic(env):
    O, lbm = env
    cfg, arr = W.sessile_droplet(160, seed=2, radius=40)
    r = [lbm.Solver(cfg, precision="fp32", diag_every=1).set_geometry(arr).step(25)
         for _ in range(2)]
    d0, d1 = r[0].diagnostics(compute=False), r[1].diagnostics(compute=False)
    assert d0 == d1
    f0, f1 = r[0].fields(), r[1].fields()
    for k in FIELDS:
        assert np.array_equal(f0[k], f1[k])


def test_nonfinite_state_is_reported(env):
    """A NaN planted in the host input reaches the diagnostics as
    LBM_ERR_NONFINITE (host-side fault injection, no device fault)."""
    O, lbm = env
    cfg, arr = W.random_state(32, 16, seed=9)
    arr = {k: v.copy() for k, v in arr.items()}
    arr["T"][3, 5] = np.nan
    s = lbm.Solver(cfg, precision="fp64").set_geometry(arr).step(3)
    d = s.diagnostics()
    assert d["nonfinite"] > 0


def test_errors_are_status_codes(env):
    O, lbm = env
    cfg, arr = W.random_state(16, 16, seed=1)
    s = lbm.Solver(cfg, precision="fp32")
    with pytest.raises(lbm.LbmError) as e:
        s.step(1)  # before set_geometry
    assert e.value.status == -8
    s.set_geometry(arr)
    with pytest.raises(lbm.LbmError):
        lbm.lbm_step(s.ctx, -1)


@pytest.mark.parametrize("prec,kernel", [("fp64", "fused"), ("fp32", "tile"), ("fp32", "fused")])
def test_batched_grids_match_single_grids_and_oracle(env, prec, kernel, monkeypatch):
    """Grids of uneven sizes and parameters advanced by one launch per step
    give, grid by grid, the results of lbm_step on each grid alone (bit for
    bit in FP64; within a few FP32 roundings in FP32, where the compiler
    contracts the kernels' copies of the step differently), and the oracle's
    within the parity bar.  FP32 batches run as the batched TMA-staged tile
    kernel by default and as the one-CTA-per-tile kernel from global loads
    with LBM_BATCH_KERNEL=fused; both are covered."""
    O, lbm = env
    if kernel == "fused":
        monkeypatch.setenv("LBM_BATCH_KERNEL", "fused")
    wls = [W.random_state(45, 19, seed=0), W.random_state(96, 24, seed=3),
           W.random_state(37, 41, seed=2), W.random_state(70, 17, seed=5),
           W.cylinder_droplet(64, seed=1)]
    steps = 60
    batch_solvers = [lbm.Solver(c, precision=prec, diag_every=10).set_geometry(a) for c, a in wls]
    b = lbm.Batch(batch_solvers).step(31)  # odd: the second call starts on the other parity
    b.step(steps - 31)
    for (cfg, arr), s in zip(wls, batch_solvers):
        alone = lbm.Solver(cfg, precision=prec, diag_every=10).set_geometry(arr).step(steps)
        fa, fb = alone.fields(), s.fields()
        for k in FIELDS:
            if prec == "fp64":
                assert np.array_equal(fa[k], fb[k]), k
            else:
                scale = np.abs(fa[k]).max() + 1e-6
                bound = 1e-5 * scale
                if k == "mdot":
                    # (1 - rho_s/rho_l) w times a change of f_l: a few float
                    # roundings of f_l (ulp 2^-24 below 1) are its resolution
                    bound += 4 * 2.0 ** -24 * abs(1 - cfg["rho_s"] / cfg["rho_l"])
                assert np.abs(fa[k] - fb[k]).max() <= bound, (k, np.abs(fa[k] - fb[k]).max())
        da, db = alone.diagnostics(compute=False), s.diagnostics(compute=False)
        if prec == "fp64":
            assert da == db
        else:
            for k, v in da.items():
                assert abs(db[k] - v) <= 1e-5 * (abs(v) + cfg["nx"] * cfg["ny"]), k
        assert s.steps_done == steps
        ref = O.from_workload((cfg, arr)).step(steps).fields()
        _compare(fb, ref, prec)
    b.close()


def test_fp32_tile_batch_of_many_grids_parities_and_lattice_sets(env):
    """The batched TMA-staged kernel over 70 small FP32 grids (two launches
    per step), with mixed lattice sets, and with one grid stepped on its own
    between batch steps (its tensor maps then belong to the other buffer
    parity): sampled grids against the oracle at the parity bar."""
    O, lbm = env
    wls = [W.random_state(20 + (k % 7) * 5, 10 + (k % 5) * 4, seed=200 + k,
                          lattices=(7, 5, 2)[k % 3] if k % 4 == 0 else 7) for k in range(70)]
    ss = [lbm.Solver(c, precision="fp32").set_geometry(a) for c, a in wls]
    b = lbm.Batch(ss).step(6)
    ss[3].step(1)
    ss[66].step(1)
    b.step(9)
    for k in (0, 3, 4, 8, 65, 66, 69):
        cfg, arr = wls[k]
        assert ss[k].steps_done == (16 if k in (3, 66) else 15)
        ref = O.from_workload((cfg, arr)).step(ss[k].steps_done).fields()
        _compare(ss[k].fields(), ref, "fp32")
    b.close()
    for s in ss:
        s.close()


def test_batch_with_mixed_lattice_sets(env):
    O, lbm = env
    wls = [W.random_state(40, 30, seed=1), W.random_state(33, 21, seed=2, lattices=5),
           W.random_state(50, 12, seed=4, lattices=2)]
    ss = [lbm.Solver(c, precision="fp64").set_geometry(a) for c, a in wls]
    lbm.Batch(ss).step(25)
    for (cfg, arr), s in zip(wls, ss):
        ref = O.from_workload((cfg, arr)).step(25).fields()
        _compare(s.fields(), ref, "fp64")


def test_batch_after_a_single_grid_step(env):
    """A grid stepped on its own between batch steps moves to the other
    buffer parity than the rest of the batch; the batch must follow it."""
    O, lbm = env
    wls = [W.random_state(40, 30, seed=6), W.random_state(52, 22, seed=7)]
    ss = [lbm.Solver(c, precision="fp64").set_geometry(a) for c, a in wls]
    b = lbm.Batch(ss).step(4)
    ss[1].step(1)
    b.step(5)
    assert [s.steps_done for s in ss] == [9, 10]
    for (cfg, arr), s in zip(wls, ss):
        ref = O.from_workload((cfg, arr)).step(s.steps_done).fields()
        _compare(s.fields(), ref, "fp64")
    b.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_interface_crossings(env, prec):
    """Droplet tip height on the droplet axis, and the liquid height and ice
    front of the Stefan column, against the oracle's definition applied to
    the oracle's fields."""
    O, lbm = env
    tol = 1e-8 if prec == "fp64" else 2e-3  # node coordinates
    cases = [(W.sessile_droplet(160, seed=2, radius=40), 150, [(1, 80), (1, 61), (0, 20)]),
             (W.stefan(), 400, [(0, 0), (0, 4), (0, 7)])]
    for (cfg, arr), steps, lines in cases:
        o = O.from_workload((cfg, arr)).step(steps)
        ref = o.fields()
        s = lbm.Solver(cfg, precision=prec).set_geometry(arr).step(steps)
        for axis, index in lines:
            want = O.crossings(ref["phi"], ref["w"], ref["fl"], axis, index)
            got = s.crossings(axis, index)
            for g, w_ in zip(got, want):
                if np.isnan(w_):
                    assert np.isnan(g), (axis, index, got, want)
                else:
                    assert abs(g - w_) <= tol, (axis, index, got, want)
        # the droplet has a tip and the column an interface and an ice front
        assert not np.isnan(s.crossings(*lines[0])[0])
        s.close()


def test_interface_crossings_errors(env):
    O, lbm = env
    cfg, arr = W.random_state(40, 20, seed=3)
    s = lbm.Solver(cfg, precision="fp32").set_geometry(arr)
    for axis, index in ((2, 0), (0, 20), (1, 40), (0, -1)):
        with pytest.raises(lbm.LbmError):
            s.crossings(axis, index)
    s.close()


@pytest.mark.parametrize("prec,diag_every", [("fp32", 0), ("fp32", 3), ("fp64", 4)])
def test_captured_periods_match_single_launches(env, prec, diag_every):
    """Steps replayed from a captured graph (long calls) give the state,
    step count and diagnostics of the same steps launched one by one, from
    any starting parity and phase."""
    O, lbm = env
    cfg, arr = W.random_state(70, 45, seed=21)
    a = lbm.Solver(cfg, precision=prec, diag_every=diag_every).set_geometry(arr)
    b = lbm.Solver(cfg, precision=prec, diag_every=diag_every).set_geometry(arr)
    a.step(1).step(77).step(40)
    for _ in range(118):
        b.step(1)
    assert a.steps_done == b.steps_done == 118
    fa, fb = a.fields(), b.fields()
    for k in FIELDS:
        assert np.array_equal(fa[k], fb[k]), k
    if diag_every:
        assert a.diagnostics(compute=False) == b.diagnostics(compute=False)
    # a new geometry invalidates what was captured for the old one
    _, arr2 = W.random_state(70, 45, seed=22)
    a.set_geometry(arr2).step(70)
    c = lbm.Solver(cfg, precision=prec, diag_every=diag_every).set_geometry(arr2)
    for _ in range(70):
        c.step(1)
    fa, fc = a.fields(), c.fields()
    for k in FIELDS:
        assert np.array_equal(fa[k], fc[k]), k
    for s in (a, b, c):
        s.close()


def test_batch_captured_periods_match_single_launches(env):
    O, lbm = env
    wls = [W.random_state(45, 19, seed=30), W.random_state(66, 40, seed=31)]
    sa = [lbm.Solver(c, precision="fp32", diag_every=5).set_geometry(a) for c, a in wls]
    sb = [lbm.Solver(c, precision="fp32", diag_every=5).set_geometry(a) for c, a in wls]
    ba, bb = lbm.Batch(sa), lbm.Batch(sb)
    ba.step(3).step(81)
    for _ in range(84):
        bb.step(1)
    for x, y in zip(sa, sb):
        assert x.steps_done == y.steps_done == 84
        fx, fy = x.fields(), y.fields()
        for k in FIELDS:
            assert np.array_equal(fx[k], fy[k]), k
        assert x.diagnostics(compute=False) == y.diagnostics(compute=False)
    ba.close()
    bb.close()


@pytest.mark.parametrize("prec", ["fp32", "fp16s", "fp64"])
def test_autotune_keeps_the_state_and_picks_a_variant(env, prec):
    """lbm_autotune times the step forms on the context's own state, restores
    that state bit for bit, and the context then steps on as before (FP32:
    within the parity bar of the oracle whichever form it kept)."""
    O, lbm = env
    cfg, arr = W.random_state(96, 40, seed=33)
    s = lbm.Solver(cfg, precision=prec, diag_every=4).set_geometry(arr).step(5)
    before = s.fields()
    us, chosen = s.autotune(40)
    # the diagnostics of step 4, pending before the call, read as if it had not happened
    ref = lbm.Solver(cfg, precision=prec, diag_every=4).set_geometry(arr).step(5)
    assert s.diagnostics(compute=False) == ref.diagnostics(compute=False)
    ref.close()
    after = s.fields()
    for k in FIELDS:
        assert np.array_equal(before[k], after[k]), k
    assert s.steps_done == 5
    # kernel forms x two graph periods: every precision one CTA per 32 x 4,
    # 32 x 8 and 32 x 16 tile (forms 0, 4, 5); FP64 the two-kernel split
    # (form 1); float the three TMA-staged configurations (forms 1-3)
    forms = (0, 1, 4, 5) if prec == "fp64" else (0, 1, 2, 3, 4, 5)
    run = [v for v in range(len(us)) if v // 2 in forms]
    assert len(us) == 12
    assert all(us[v] > 0 for v in run)
    assert all(u == -1.0 for v, u in enumerate(us) if v not in run)
    # the fastest variant, or the starting one (form 0, period 32: variant 0)
    # where that is within 2 % of the fastest
    assert chosen in run
    assert us[chosen] == min(us[v] for v in run) or (chosen == 0 and
                                                      us[0] <= 1.02 * min(us[v] for v in run))
    s.step(40)
    if prec != "fp16s":
        _compare(s.fields(), O.from_workload((cfg, arr)).step(45).fields(), prec)
    s.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp16s"])
@pytest.mark.parametrize("form", [4, 0, 5])
def test_tile_shapes_match_the_oracle(env, prec, form, monkeypatch):
    """The one-CTA-per-tile step on 32 x 4, 32 x 8 and 32 x 16 tiles (kernel
    forms 4, 0, 5), forced with LBM_KERNEL_FORM: ragged random states with
    every branch, and a column four nodes high (the Neumann shape) whose
    height one 32 x 4 tile fits exactly.  FP64 within 1e-10 of the oracle,
    FP32 at the parity bar; FP16 storage within twice the 32 x 8 run's
    distance from FP64 of that run (the same arithmetic; only a flipped
    binary16 rounding separates them).  The diagnostics fused into the last
    step (one partial sum per CTA, as many as the shape has tiles) match the
    oracle's of the state that step read."""
    O, lbm = env
    for wl, steps in ((W.random_state(70, 45, seed=41), 80), (W.random_state(37, 19, seed=42), 80),
                      (W.neumann(), 300)):
        cfg, arr = wl
        o = O.from_workload(wl).step(steps - 1)
        rd = o.diagnostics()
        ref = o.step(1).fields()
        monkeypatch.setenv("LBM_KERNEL_FORM", str(form))
        s = lbm.Solver(cfg, precision=prec, diag_every=1).set_geometry(arr).step(steps)
        monkeypatch.delenv("LBM_KERNEL_FORM")
        got, d = s.fields(), s.diagnostics(compute=False)
        s.close()
        assert d["step"] == steps - 1
        if prec == "fp16s":
            b = lbm.Solver(cfg, precision=prec).set_geometry(arr).step(steps)
            c = lbm.Solver(cfg, precision="fp64").set_geometry(arr).step(steps)
            fb, fc = b.fields(), c.fields()
            b.close()
            c.close()
            for k in FIELDS:
                e = _l2_rel(got[k], fb[k])
                assert e <= max(1e-5, 2 * _l2_rel(fb[k], fc[k])), (k, e)
        else:
            _compare(got, ref, prec)
        tol = {"fp64": 1e-10, "fp32": 1e-5, "fp16s": 1e-3}[prec]
        for k in ("mass", "material_mass", "rhoH", "frozen_volume", "phi_sum"):
            assert abs(d[k] - rd[k]) <= tol * (abs(rd[k]) + cfg["nx"] * cfg["ny"]), (k, d[k], rd[k])


@pytest.mark.slow
def test_droplet_on_a_cylinder_reaches_the_closed_form_height(env):
    """P8 (Sec. 4.4, Eq. (37)): a drop of radius R0 = 50 placed on a cylinder
    of radius Rs = 50 (300 x 300, sigma = 0.001, M = 0.1, no heat) spreads
    to the equilibrium whose top lies at H_max = k + R from the cylinder axis,
    with R and k fixed by the contact angle and the drop's area.  At 90
    degrees the FP32 path reaches H_max within 2 % after 200,000 steps (the
    contact line creeps: -9 % at 5,000 steps, -3 % at 100,000).  Larger angles
    on the curved solid are not stable with the model as read (theta >= 105
    degrees diverges after 30,000-50,000 steps, identically in FP32 and FP64),
    so they are not part of this pin."""
    import closed_forms as CF
    O, lbm = env
    L, Rs, R0, eps, theta = 300, 50.0, 50.0, 4.0, 90.0
    cfg = W.base_params(L, L, lattices=W.FLOW | W.PHASE, theta_deg=theta, sigma=0.001,
                        mobility=0.1, bc=("periodic", "periodic", "periodic", "periodic"))
    X, Y = np.meshgrid(np.arange(L) + 0.5, np.arange(L) + 0.5)
    cx, cy = L / 2, 0.35 * L
    phi0 = 0.5 + 0.5 * np.tanh(2 * (Rs - np.hypot(X - cx, Y - cy)) / eps)
    phi = (1 - phi0) * np.tanh(2 * (R0 - np.hypot(X - cx, Y - (cy + Rs))) / eps)
    z = np.zeros((L, L))
    s = lbm.Solver(cfg, precision="fp32").set_geometry(
        {"phi0": phi0, "phi": phi, "T": z + 0.5, "fl": z + 1.0})
    s.step(200000)
    H = s.crossings(1, int(cx))[0] + 0.5 - cy
    _, _, H_eq = CF.cylinder_droplet_equilibrium(R0, Rs, theta)
    print(f"\nH_max {H:.2f}, closed form {H_eq:.2f}")
    assert abs(H - H_eq) <= 0.02 * H_eq
    s.close()


_STEFAN_FULL = {}


def _stefan_full(env):
    """The three-phase Stefan column (512 x 8), 50,000 steps: oracle fields,
    FP32 fields and crossings (computed once per session)."""
    if not _STEFAN_FULL:
        O, lbm = env
        cfg, arr = W.stefan()
        steps = 50000
        ref = O.from_workload((cfg, arr)).step(steps).fields()
        s = lbm.Solver(cfg, precision="fp32").set_geometry(arr).step(steps)
        _STEFAN_FULL.update(ref=ref, got=s.fields(), have=s.crossings(0, 4),
                            want=O.crossings(ref["phi"], ref["w"], ref["fl"], 0, 4))
        s.close()
    return _STEFAN_FULL


@pytest.mark.slow
def test_stefan_column_fp32_full_run(env):
    """The three-phase Stefan column (512 x 8) for the full 50,000 steps, FP32
    against the FP64 oracle: every field (the velocity as one vector field)
    within 1e-4 relative L2, the gas-liquid interface and the ice front
    (crossings along a row) within 0.5 % of the column's liquid height, the
    frozen volume within 0.5 %."""
    O, lbm = env
    r = _stefan_full(env)
    ref, got, have, want = r["ref"], r["got"], r["have"], r["want"]
    errs = {k: _l2_rel(got[k], ref[k]) for k in FIELDS}
    errs["u"] = _vel_l2_rel(got, ref)
    print("\nfield errors", {k: f"{v:.1e}" for k, v in errs.items()}, "crossings", have, want)
    column = 80.0 - 16.0  # liquid height h0 - hs of the workload
    for g, w in zip(have, want):
        assert abs(g - w) <= 0.005 * column, (have, want)
    vg, vr = _front_and_frozen(O, got)[1], _front_and_frozen(O, ref)[1]
    assert abs(vg - vr) <= 0.005 * vr, (vg, vr)
    _compare(got, ref, "fp32", tol=1e-4)


@pytest.mark.slow
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_sessile_droplet_512_long_run(env, prec):
    """The benchmark workload itself (512^2 droplet, three lattices, cold
    substrate) for 2,000 steps, every node against the oracle."""
    got, ref = _run_pair(env, W.sessile_droplet(512, seed=0), 2000, prec)
    _compare(got, ref, prec)


def test_batch64_full_size_sampled_grids(env):
    """The benchmark's 64-grid batch (sides from {128, 256, 384, 512}, one
    launch per step, captured periods) at full size: the smallest, a middle
    and the largest grid compared with the oracle on every node after 40
    steps (FP32 parity bar)."""
    O, lbm = env
    r = W.rng(1000)
    sides = r.choice([128, 256, 384, 512], size=64)
    wls = [W.cylinder_droplet(int(sd), seed=i) for i, sd in enumerate(sides)]
    ss = [lbm.Solver(c, precision="fp32").set_geometry(a) for c, a in wls]
    b = lbm.Batch(ss)
    b.step(40)
    order = np.argsort(sides, kind="stable")
    for k in (order[0], order[31], order[-1]):
        cfg, arr = wls[k]
        ref = O.from_workload((cfg, arr)).step(40).fields()
        _compare(ss[k].fields(), ref, "fp32")
    b.close()
    for s in ss:
        s.close()


def test_batch_of_more_than_64_grids(env):
    """More than 64 grids take several launches per step (64 grids per
    argument table); every grid still matches its own lbm_step run bit for
    bit (FP64), through captured periods and single steps."""
    O, lbm = env
    wls = [W.random_state(20 + (k % 7) * 3, 10 + (k % 5) * 4, seed=100 + k) for k in range(70)]
    ss = [lbm.Solver(c, precision="fp64", diag_every=3).set_geometry(a) for c, a in wls]
    b = lbm.Batch(ss)
    b.step(5).step(40)
    for (cfg, arr), s in zip(wls[::9] + [wls[-1]], ss[::9] + [ss[-1]]):
        alone = lbm.Solver(cfg, precision="fp64", diag_every=3).set_geometry(arr).step(45)
        fa, fb = alone.fields(), s.fields()
        for k in FIELDS:
            assert np.array_equal(fa[k], fb[k]), k
        assert alone.diagnostics(compute=False) == s.diagnostics(compute=False)
        alone.close()
    b.close()
    for s in ss:
        s.close()


@pytest.mark.parametrize("prec", ["fp32", "fp16s"])
@pytest.mark.parametrize("wl", ["random", "droplet", "subset", "tiles2"])
def test_tile_kernel_matches_one_cta_per_tile_kernel(env, prec, wl, monkeypatch):
    """The float step runs as the persistent TMA-staged tile kernel; the
    one-CTA-per-tile kernel (LBM_STEP_KERNEL=fused) computes the same
    arithmetic from global loads.  FP32: the same fields up to the last bits
    of float (the compiler may contract multiply-adds differently in the
    two kernels).  FP16 storage: such a last-bit difference now and then
    flips the binary16 rounding of a stored population, and the two runs
    then drift apart by up to the format's own error, so each field of the
    two is held within twice its distance from the FP64 state (the triangle
    bound for two runs each that far from it)."""
    O, lbm = env
    cfg, arr = {"random": lambda: W.random_state(101, 37, seed=21),
                "droplet": lambda: W.sessile_droplet(160, seed=2, radius=40),
                "subset": lambda: W.random_state(67, 29, seed=22, lattices=5),
                "tiles2": lambda: W.sessile_droplet(256, seed=4, radius=60)}[wl]()
    # the two-stage persistent form on a grid with several tiles per CTA
    monkeypatch.setenv("LBM_TILE", "2:2" if wl == "tiles2" else "1:0")
    a = lbm.Solver(cfg, precision=prec).set_geometry(arr).step(60)
    monkeypatch.delenv("LBM_TILE")
    monkeypatch.setenv("LBM_STEP_KERNEL", "fused")
    b = lbm.Solver(cfg, precision=prec).set_geometry(arr).step(60)
    fa, fb = a.fields(), b.fields()
    if prec == "fp16s":
        c = lbm.Solver(cfg, precision="fp64").set_geometry(arr).step(60)
        fc = c.fields()
        c.close()
    for k in FIELDS:
        e = _l2_rel(fa[k], fb[k])
        bound = 1e-5 if prec == "fp32" else max(1e-5, 2 * _l2_rel(fb[k], fc[k]))
        assert e <= bound, (k, e, bound)
    da, db = a.diagnostics(compute=True), b.diagnostics(compute=True)
    assert abs(da["material_mass"] - db["material_mass"]) <= 1e-6 * abs(db["material_mass"])
    a.close()
    b.close()
