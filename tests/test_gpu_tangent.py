"""Forward-mode (tangent) derivatives of the fused step, through the C ABI.

The tangent context carries, beside every FP64 value, its derivative along
one parameter direction.  Checked here: its values are those of the FP64
step; its derivatives of the frozen fraction and of the droplet's tip height
with respect to the wall temperature, the contact angle and the Stefan
number agree with central differences of the FP64 GPU step and of the FP64
oracle; the torch.autograd.Function returns J^T grad.
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
    from paper_2510_18688_gb300 import build, lbm, sensitivity
    build.build()
    lbm.load()
    return oracle_mod, lbm, sensitivity, torch


# central-difference steps per parameter (T_w, theta in degrees, Ste)
H = (1e-4, 1e-3, 1e-5)


def _droplet(n=64):
    cfg, arr = W.sessile_droplet(n, seed=3, radius=n / 4, hs=n / 10, theta_deg=80.0, ste=0.3)
    return cfg, arr, (-1.0, 80.0, 0.3), ("cold", 2), (1, n // 2)


def _fd(observe, p0, h=H):
    out = np.empty((2, 3))
    for j in range(3):
        pp, pm = list(p0), list(p0)
        pp[j] += h[j]
        pm[j] -= h[j]
        out[:, j] = (observe(pp) - observe(pm)) / (2 * h[j])
    return out


def _close(J, ref, rtol, atol):
    return np.all(np.abs(J - ref) <= rtol * np.abs(ref) + atol)


def test_tangent_values_are_the_fp64_step(env):
    O, lbm, S, torch = env
    cfg, arr = W.random_state(70, 45, seed=12)
    a = lbm.Solver(cfg, precision="fp64").set_geometry(arr).step(60)
    t = lbm.Solver(cfg, precision="tangent", tangent={"theta_deg": 1.0, "latent": 2.0}
                   ).set_geometry(arr).step(60)
    fa, ft = a.fields(), t.fields()
    for k in FIELDS:
        scale = np.abs(fa[k]).max() + 1e-300
        assert np.abs(fa[k] - ft[k]).max() <= 1e-12 * scale, k
    dt = t.tangent_fields()
    assert all(np.all(np.isfinite(dt[k])) for k in FIELDS)
    assert np.abs(dt["phi"]).max() > 0.0  # the angle moves the interface
    a.close()
    t.close()


def test_tangent_matches_central_differences_of_the_gpu_step(env):
    O, lbm, S, torch = env
    cfg, arr, p0, wall, line = _droplet()
    steps = 300
    val, J = S.value_and_jacobian(cfg, arr, steps, p0, wall, line)

    def observe(p):
        s = S.run(S.apply_params(cfg, *p, wall), arr, steps)
        v = S.observables(s, line)
        s.close()
        return v

    fd = _fd(observe, p0)
    print("\nJ =\n", J, "\nFD =\n", fd)
    assert val[0] > 0.0 and np.isfinite(val[1])  # ice has formed; the drop has a tip
    assert np.abs(J[0]).max() > 0.0
    assert _close(J, fd, 1e-3, np.array([[1e-9], [1e-7]])), (J, fd)


def test_tangent_of_the_neumann_front(env):
    O, lbm, S, torch = env
    cfg, arr = W.neumann()
    steps, wall, p0 = 3000, (0,), (-1.0, 90.0, 0.1)
    val, J = S.value_and_jacobian(cfg, arr, steps, p0, wall, None)

    def observe(p):
        s = S.run(S.apply_params(cfg, *p, wall), arr, steps)
        v = S.observables(s, None)
        s.close()
        return v

    # The column freezes node by node, so the frozen fraction has a kink
    # (a branch change of Eq. (8)) wherever the front node crosses a
    # threshold; a difference step must be small enough not to straddle one
    # (with 1e-5 in Ste it does: left and right differences then disagree).
    h = (1e-6, 1e-3, 1e-7)
    fd = _fd(observe, p0, h)
    p_right = list(p0)
    p_right[2] += h[2]
    right = (observe(p_right)[0] - val[0]) / h[2]
    print("\nJ =", J[0], "FD =", fd[0], "right difference in Ste", right)
    assert J[0, 1] == 0.0  # no phase field: the angle does not enter
    assert abs(right - fd[0, 2]) <= 1e-4 * abs(fd[0, 2])  # no kink inside the step
    assert _close(J[0], fd[0], 1e-4, 1e-9), (J[0], fd[0])


def test_tangent_matches_central_differences_of_the_oracle(env):
    O, lbm, S, torch = env
    cfg, arr, p0, wall, line = _droplet(40)
    steps = 120
    val, J = S.value_and_jacobian(cfg, arr, steps, p0, wall, line)

    def observe(p):
        o = O.from_workload((S.apply_params(cfg, *p, wall), arr)).step(steps)
        d = o.diagnostics()
        f = o.fields()
        tip = O.crossings(f["phi"], f["w"], f["fl"], *line)[0]
        return np.array([d["frozen_volume"] / d["material_volume"], tip])

    fd = _fd(observe, p0)
    print("\nJ =\n", J, "\noracle FD =\n", fd)
    assert _close(J, fd, 1e-3, np.array([[1e-9], [1e-7]])), (J, fd)


def test_autograd_function_returns_the_jacobian_product(env):
    O, lbm, S, torch = env
    cfg, arr, p0, wall, line = _droplet(48)
    steps = 150
    p = torch.tensor(p0, dtype=torch.float64, requires_grad=True)
    y = S.FreezingObservables.apply(p, cfg, arr, steps, wall, line)
    (y[0] + 0.01 * y[1]).backward()
    val, J = S.value_and_jacobian(cfg, arr, steps, p0, wall, line)
    assert np.allclose(y.detach().numpy(), val, rtol=0, atol=0)
    assert np.allclose(p.grad.numpy(), J[0] + 0.01 * J[1], rtol=1e-12, atol=0)


def test_tangent_rejected_where_unsupported(env):
    O, lbm, S, torch = env
    cfg, arr = W.random_state(40, 20, seed=3)
    s = lbm.Solver(cfg, precision="tangent").set_geometry(arr)
    with pytest.raises(lbm.LbmError):
        lbm.Batch([s])
    f = lbm.Solver(cfg, precision="fp64").set_geometry(arr)
    with pytest.raises(lbm.LbmError) as e:
        f.tangent_fields()
    assert e.value.status == -6
    s.close()
    f.close()


def test_freezing_time_derivative(env):
    """d t*/d T_w and d t*/d Ste of the time at which the frozen fraction of
    a small droplet first reaches 0.9, against central differences of the
    same interpolated time from FP64 runs."""
    O, lbm, S, torch = env
    cfg, arr, p0, wall, line = _droplet(32)
    level = 0.9

    def tstar(p):
        c = S.apply_params(cfg, *p, wall)
        s = lbm.Solver(c, precision="fp64").set_geometry(arr)
        prev = None
        for n in range(200000):
            d = s.diagnostics(compute=True)
            ff = d["frozen_volume"] / d["material_volume"]
            if prev is not None and ff >= level:
                s.close()
                return (n - 1) + (level - prev) / (ff - prev)
            prev = ff
            s.step(1)
        raise AssertionError("the droplet did not freeze")

    for j, name in ((0, "T_w"), (2, "ste")):
        t0, dt = S.freezing_time(cfg, arr, p0, wall, name, level=level)
        h = (1e-6, None, 1e-7)[j]
        pp, pm = list(p0), list(p0)
        pp[j] += h
        pm[j] -= h
        fd = (tstar(pp) - tstar(pm)) / (2 * h)
        print(f"\nt* = {t0:.3f}, dt*/d{name}: tangent {dt:.6f}, FD {fd:.6f}")
        assert np.isfinite(t0) and t0 > 0
        assert abs(dt - fd) <= 1e-3 * abs(fd), (name, dt, fd)


@pytest.mark.slow
def test_porous_medium_gradient_over_4000_steps(env):
    """Freezing of gas-liquid flow in a porous medium (cold wall at x = 0,
    Sec. 4.6 shape, here 1024 x 512): the frozen fraction after 4000 steps
    and its derivatives with respect to the cold-wall temperature and the
    contact angle, against central differences of the FP64 GPU step."""
    O, lbm, S, torch = env
    cfg, arr = W.porous(1024, 512, seed=0)
    steps, wall, p0 = 4000, (0,), (-1.0, 60.0, 0.1)
    val, J = S.value_and_jacobian(cfg, arr, steps, p0, wall, None)

    def observe(p):
        s = S.run(S.apply_params(cfg, *p, wall), arr, steps)
        v = S.observables(s, None)
        s.close()
        return v

    h = (1e-6, 1e-4, 1e-7)
    fd = np.empty(3)
    for j in (0, 1):
        pp, pm = list(p0), list(p0)
        pp[j] += h[j]
        pm[j] -= h[j]
        fd[j] = (observe(pp)[0] - observe(pm)[0]) / (2 * h[j])
    print(f"\nFF = {val[0]:.6f}; dFF/dT_w tangent {J[0, 0]:.8f} FD {fd[0]:.8f}; "
          f"dFF/dtheta tangent {J[0, 1]:.3e} FD {fd[1]:.3e}; dFF/dSte {J[0, 2]:.6f}")
    assert val[0] > 0.0
    assert abs(J[0, 0] - fd[0]) <= 1e-3 * abs(fd[0])
    assert abs(J[0, 1] - fd[1]) <= 1e-3 * abs(fd[1]) + 1e-10


# ---------------------------------------------------------------------------
# reverse mode (hand-written adjoint) of the enthalpy-lattice step
# ---------------------------------------------------------------------------

def _heat_column():
    cfg, arr = W.neumann()
    cfg = dict(cfg, lattices=4)  # the enthalpy lattice alone (the fluid is at rest)
    return cfg, arr


def test_adjoint_gradient_equals_the_tangent_and_differences(env):
    """The reverse sweep gives the gradient of the frozen fraction of the
    conduction-freezing column with respect to the cold-wall temperature and
    the latent heat: equal to the forward-mode tangent (the same discrete
    derivative, another summation order) and to central differences."""
    O, lbm, S, torch = env
    cfg, arr = _heat_column()
    steps = 2000
    s = lbm.Solver(cfg, precision="fp64").set_geometry(arr)
    ff, grad = s.adjoint_frozen_fraction(steps, every=100)
    s.close()
    tan = {}
    for name, direction in (("T_wall0", {"T_wall": [1.0, 0.0, 0.0, 0.0]}), ("latent", {"latent": 1.0})):
        t = lbm.Solver(cfg, precision="tangent", tangent=direction).set_geometry(arr).step(steps)
        d, dt = t.diagnostics(), t.tangent_diagnostics(compute=False)
        fz, mv = d["frozen_volume"], d["material_volume"]
        tan[name] = (dt["frozen_volume"] * mv - fz * dt["material_volume"]) / mv ** 2
        assert abs(fz / mv - ff) <= 1e-12 * ff
        t.close()

    def ff_at(c):
        u = lbm.Solver(c, precision="fp64").set_geometry(arr).step(steps)
        d = u.diagnostics()
        u.close()
        return d["frozen_volume"] / d["material_volume"]

    h = 1e-7
    tw = list(cfg["T_wall"])
    fd_tw = (ff_at(dict(cfg, T_wall=tuple([tw[0] + h] + tw[1:])))
             - ff_at(dict(cfg, T_wall=tuple([tw[0] - h] + tw[1:])))) / (2 * h)
    hl = 1e-7 * cfg["latent"]
    fd_l = (ff_at(dict(cfg, latent=cfg["latent"] + hl)) - ff_at(dict(cfg, latent=cfg["latent"] - hl))) / (2 * hl)
    print(f"\nFF {ff:.8f}; dFF/dT_w adjoint {grad[0]:.10e} tangent {tan['T_wall0']:.10e} FD {fd_tw:.10e}; "
          f"dFF/dL adjoint {grad[4]:.10e} tangent {tan['latent']:.10e} FD {fd_l:.10e}")
    assert abs(grad[0] - tan["T_wall0"]) <= 1e-9 * abs(tan["T_wall0"])
    assert abs(grad[4] - tan["latent"]) <= 1e-9 * abs(tan["latent"])
    assert abs(grad[0] - fd_tw) <= 1e-4 * abs(fd_tw)
    assert abs(grad[4] - fd_l) <= 1e-4 * abs(fd_l)
    assert grad[2] == grad[3] == 0.0  # periodic in y: no wall there
    assert abs(grad[1]) < 1e-6 * abs(grad[0])  # the warm wall is 400 nodes from the front


def test_adjoint_checkpoint_interval_and_final_state(env):
    """The checkpoint interval changes the memory, not the result (the
    recomputed segments repeat the forward steps bit for bit), and the
    context ends in the state nsteps plain steps give."""
    O, lbm, S, torch = env
    cfg, arr = _heat_column()
    steps = 300
    out = []
    for every in (1, 37, 300):
        s = lbm.Solver(cfg, precision="fp64").set_geometry(arr)
        out.append(s.adjoint_frozen_fraction(steps, every=every))
        if every == 37:
            f_adj = s.fields()
            assert s.steps_done == steps
        s.close()
    assert all(o == out[0] for o in out[1:]), out
    plain = lbm.Solver(cfg, precision="fp64").set_geometry(arr).step(steps)
    f_plain = plain.fields()
    for k in FIELDS:
        assert np.array_equal(f_adj[k], f_plain[k]), k
    plain.close()


def test_adjoint_of_the_conduction_column_with_its_resting_flow(env):
    """The conduction-freezing column as configured (flow and enthalpy
    lattices, rho_s = rho_l, no body force): the flow stays at rest, and the
    adjoint gradient equals the tangent of the full step."""
    O, lbm, S, torch = env
    cfg, arr = W.neumann()
    assert cfg["lattices"] == 5 and cfg["rho_s"] == cfg["rho_l"]
    steps = 1500
    s = lbm.Solver(cfg, precision="fp64").set_geometry(arr)
    ff, grad = s.adjoint_frozen_fraction(steps, every=64)
    assert np.abs(s.fields(("ux",))["ux"]).max() == 0.0
    s.close()
    t = lbm.Solver(cfg, precision="tangent", tangent={"T_wall": [1.0, 0.0, 0.0, 0.0]}
                   ).set_geometry(arr).step(steps)
    d, dt = t.diagnostics(), t.tangent_diagnostics(compute=False)
    fz, mv = d["frozen_volume"], d["material_volume"]
    tan = (dt["frozen_volume"] * mv - fz * dt["material_volume"]) / mv ** 2
    t.close()
    assert abs(grad[0] - tan) <= 1e-9 * abs(tan), (grad[0], tan)


def test_adjoint_rejects_other_contexts(env):
    O, lbm, S, torch = env
    cfg, arr = _heat_column()
    for c, prec in ((cfg, "fp32"), (dict(cfg, lattices=7), "fp64"),
                    (dict(cfg, lattices=5, rho_s=0.9), "fp64")):
        s = lbm.Solver(c, precision=prec).set_geometry(arr)
        with pytest.raises(lbm.LbmError) as e:
            s.adjoint_frozen_fraction(10, 5)
        assert e.value.status == -6
        s.close()


def _phase_droplet(n=64):
    """The droplet of _droplet with the phase-field lattice alone (fluid at
    rest, no heat): its cap relaxes towards the contact angle by the
    Cahn-Hilliard flux of Eqs. (18)-(21)."""
    cfg, arr = W.sessile_droplet(n, seed=3, radius=n / 4, hs=n / 10, theta_deg=80.0, ste=0.3)
    return dict(cfg, lattices=2), arr


def test_phase_adjoint_gradient_equals_the_tangent_and_differences(env):
    """The reverse sweep of the phase-field step gives the derivatives of an
    interface crossing with respect to the contact angle and the surface
    tension, from the initial fields: equal to the forward-mode tangent
    (theta) and to central differences of the FP64 step.  Two lines: the
    droplet's axis (the tip height, set by sigma; theta acts there only
    through the slow Cahn-Hilliard relaxation of the cap) and a row just
    above the substrate (the contact line, where the wetting terms of
    Eq. (6) act)."""
    O, lbm, S, torch = env
    cfg, arr = _phase_droplet()
    steps = 600
    lines = ((1, cfg["nx"] // 2), (0, 9))

    def pos_at(c, axis, index):
        u = lbm.Solver(c, precision="fp64").set_geometry(arr).step(steps)
        v = u.crossings(axis, index)[0]
        u.close()
        return v

    for axis, index in lines:
        s = lbm.Solver(cfg, precision="fp64").set_geometry(arr)
        pos, grad = s.adjoint_crossing(steps, axis, index, every=50)
        assert s.crossings(axis, index)[0] == pos
        s.close()
        t = lbm.Solver(cfg, precision="tangent", tangent={"theta_deg": 1.0}).set_geometry(arr)
        t.step(steps)
        pos_t, _, dpos_t, _ = t.crossings_tangent(axis, index)
        t.close()
        assert abs(pos_t - pos) <= 1e-12 * pos
        ht, hs = 1e-3, 1e-5 * cfg["sigma"]
        fd_t = (pos_at(dict(cfg, theta_deg=cfg["theta_deg"] + ht), axis, index)
                - pos_at(dict(cfg, theta_deg=cfg["theta_deg"] - ht), axis, index)) / (2 * ht)
        fd_s = (pos_at(dict(cfg, sigma=cfg["sigma"] + hs), axis, index)
                - pos_at(dict(cfg, sigma=cfg["sigma"] - hs), axis, index)) / (2 * hs)
        print(f"\nline {axis},{index}: crossing {pos:.8f}; d/dtheta adjoint {grad[0]:.10e} "
              f"tangent {dpos_t:.10e} FD {fd_t:.10e}; d/dsigma adjoint {grad[1]:.10e} FD {fd_s:.10e}")
        assert abs(grad[0] - dpos_t) <= 1e-9 * abs(dpos_t)
        assert abs(grad[1] - fd_s) <= 1e-4 * abs(fd_s)
        if axis == 0:
            # the contact line moves with theta (slowly: the fluid is at
            # rest), four orders of magnitude more than the tip
            assert abs(grad[0]) > 1e-6
            assert abs(grad[0] - fd_t) <= 1e-4 * abs(fd_t)


def test_phase_adjoint_checkpoints_final_state_and_rejections(env):
    """The checkpoint interval does not change the result; the context ends
    in the state of plain steps; other contexts are refused."""
    O, lbm, S, torch = env
    cfg, arr = _phase_droplet()
    steps, col = 120, cfg["nx"] // 2
    out = []
    for every in (1, 17, 120):
        s = lbm.Solver(cfg, precision="fp64").set_geometry(arr)
        out.append(s.adjoint_crossing(steps, 1, col, every=every))
        if every == 17:
            f_adj = s.fields()
            assert s.steps_done == steps
        s.close()
    assert all(o == out[0] for o in out[1:]), out
    plain = lbm.Solver(cfg, precision="fp64").set_geometry(arr).step(steps)
    f_plain = plain.fields()
    for k in FIELDS:
        assert np.array_equal(f_adj[k], f_plain[k]), k
    plain.close()
    for c, prec in ((cfg, "fp32"), (dict(cfg, lattices=7), "fp64"), (dict(cfg, sigma=0.0), "fp64")):
        s = lbm.Solver(c, precision=prec).set_geometry(arr)
        with pytest.raises(lbm.LbmError) as e:
            s.adjoint_crossing(10, 1, col, 5)
        assert e.value.status == -6
        s.close()
    s = lbm.Solver(cfg, precision="fp64").set_geometry(arr)
    for axis, index in ((1, cfg["nx"]), (0, cfg["ny"]), (2, 0), (0, -1)):
        with pytest.raises(lbm.LbmError) as e:
            s.adjoint_crossing(10, axis, index, 5)
        assert e.value.status == -1
    s.close()


def test_adjoints_behind_autograd(env):
    """The reverse-mode calls behind torch.autograd: backward returns
    grad_output times the sweep's gradient, and the values are those of plain
    runs with the same parameters."""
    O, lbm, S, torch = env
    cfg, arr = _phase_droplet()
    q = torch.tensor([cfg["theta_deg"], cfg["sigma"]], dtype=torch.float64, requires_grad=True)
    y = S.AdjointCrossing.apply(q, cfg, arr, 200, 0, 9, 50)
    (3.0 * y).backward()
    s = lbm.Solver(cfg, precision="fp64").set_geometry(arr)
    pos, grad = s.adjoint_crossing(200, 0, 9, every=50)
    s.close()
    assert float(y.detach()) == pos
    assert q.grad.tolist() == [3.0 * grad[0], 3.0 * grad[1]]

    hc, ha = _heat_column()
    qh = torch.tensor(list(hc["T_wall"]) + [hc["latent"], hc["T_cold"]], dtype=torch.float64,
                      requires_grad=True)
    ff = S.AdjointFrozenFraction.apply(qh, hc, ha, 300, 100)
    ff.backward()
    t = lbm.Solver(hc, precision="tangent", tangent={"T_wall": [1.0, 0.0, 0.0, 0.0]}).set_geometry(ha).step(300)
    d, dt = t.diagnostics(), t.tangent_diagnostics(compute=False)
    fz, mv = d["frozen_volume"], d["material_volume"]
    tan = (dt["frozen_volume"] * mv - fz * dt["material_volume"]) / mv ** 2
    t.close()
    assert abs(float(ff.detach()) - fz / mv) <= 1e-12 * float(ff.detach())
    assert abs(float(qh.grad[0]) - tan) <= 1e-9 * abs(tan)


def _frz_state(seed, n=(40, 24), mask=False):
    """A random three-phase state with the phase field and the enthalpy
    lattice only (fluid at rest), with or without its cold mask: ice, drops,
    a mushy band and walls of every kind, so freezing couples the two
    lattices."""
    cfg, arr = W.random_state(*n, seed=seed, lattices=W.PHASE | W.HEAT)
    return cfg, {k: v for k, v in arr.items() if mask or k != "mask"}


@pytest.mark.parametrize("seed,mask", [(1, False), (3, False), (4, False), (3, True)])
def test_coupled_adjoint_equals_the_tangent(env, seed, mask):
    """The reverse sweep of the coupled phase-field + enthalpy step gives the
    derivatives of the frozen fraction and of an interface crossing with
    respect to the wall temperatures, L, theta (equal to the forward-mode
    tangent of the same steps) and sigma (central differences)."""
    O, lbm, S, torch = env
    cfg, arr = _frz_state(seed, mask=mask)
    steps = 200
    plain = lbm.Solver(cfg, precision="fp64").set_geometry(arr).step(steps)
    col = next(i for i in range(cfg["nx"]) if np.isfinite(plain.crossings(1, i)[0]))
    plain.close()
    res = {}
    for obs in (0, 1):
        s = lbm.Solver(cfg, precision="fp64").set_geometry(arr)
        res[obs] = s.adjoint_freezing(steps, obs, 1, col, every=37)
        s.close()
    dirs = [("T_wall", k) for k in range(4) if cfg["bc"][k] == "dirichlet"] + [("latent", 4), ("theta_deg", 5)]
    if mask:
        dirs.append(("T_cold", 7))
    rows = []
    for name, k in dirs:
        t = ({"T_wall": [1.0 if j == k else 0.0 for j in range(4)]} if name == "T_wall" else {name: 1.0})
        ts = lbm.Solver(cfg, precision="tangent", tangent=t).set_geometry(arr).step(steps)
        d, dt = ts.diagnostics(), ts.tangent_diagnostics(compute=False)
        fz, mv = d["frozen_volume"], d["material_volume"]
        dff = (dt["frozen_volume"] * mv - fz * dt["material_volume"]) / mv ** 2
        cr = ts.crossings_tangent(1, col)
        ts.close()
        assert abs(fz / mv - res[0][0]) <= 1e-12
        assert abs(cr[0] - res[1][0]) <= 1e-12 * abs(cr[0])
        rows.append((name, k, res[0][1][k], dff, res[1][1][k], cr[2]))

    def val(c, obs):
        u = lbm.Solver(c, precision="fp64").set_geometry(arr).step(steps)
        d = u.diagnostics()
        v = d["frozen_volume"] / d["material_volume"] if obs == 0 else u.crossings(1, col)[0]
        u.close()
        return v

    hs = 1e-5 * cfg["sigma"]
    for obs in (0, 1):
        fd = (val(dict(cfg, sigma=cfg["sigma"] + hs), obs) - val(dict(cfg, sigma=cfg["sigma"] - hs), obs)) / (2 * hs)
        rows.append(("sigma FD", 6, res[obs][1][6], fd, None, None) if obs == 0 else ("sigma FD", 6, None, None, res[obs][1][6], fd))
    print(f"\nseed {seed}, column {col}: FF {res[0][0]:.10f}, crossing {res[1][0]:.8f}")
    for r in rows:
        print("  ", r)
    scale_ff = max(abs(r[3]) for r in rows if r[3] is not None and r[0] != "sigma FD")
    scale_cr = max(abs(r[5]) for r in rows if r[5] is not None and r[0] != "sigma FD")
    for name, k, aff, tff, acr, tcr in rows:
        if name == "sigma FD":
            if aff is not None:
                assert abs(aff - tff) <= 1e-4 * abs(tff) + 1e-9, (name, aff, tff)
            else:
                assert abs(acr - tcr) <= 1e-4 * abs(tcr) + 1e-7, (name, acr, tcr)
            continue
        assert abs(aff - tff) <= 1e-8 * max(abs(tff), 1e-4 * scale_ff), (name, k, aff, tff)
        assert abs(acr - tcr) <= 1e-8 * max(abs(tcr), 1e-4 * scale_cr), (name, k, acr, tcr)
    for k in range(4):
        if cfg["bc"][k] != "dirichlet":
            assert res[0][1][k] == 0.0 and res[1][1][k] == 0.0


def test_coupled_adjoint_checkpoints_and_rejections(env):
    """The checkpoint interval does not change the coupled gradient (bit for
    bit: every reduction and gather runs in a fixed order); the context ends
    in the state of plain steps; other contexts are refused."""
    O, lbm, S, torch = env
    cfg, arr = _frz_state(3)
    steps = 60
    out = []
    for every in (1, 13, 60):
        s = lbm.Solver(cfg, precision="fp64").set_geometry(arr)
        out.append(s.adjoint_freezing(steps, 0, every=every))
        if every == 13:
            f_adj = s.fields()
        s.close()
    assert all(o == out[0] for o in out[1:]), out
    plain = lbm.Solver(cfg, precision="fp64").set_geometry(arr).step(steps)
    f_plain = plain.fields()
    plain.close()
    for k in FIELDS:
        assert np.array_equal(f_adj[k], f_plain[k]), k
    for c, a, prec in ((cfg, arr, "fp32"), (dict(cfg, lattices=7), arr, "fp64"),
                       (dict(cfg, sigma=0.0), arr, "fp64")):
        s = lbm.Solver(c, precision=prec).set_geometry(a)
        with pytest.raises(lbm.LbmError) as e:
            s.adjoint_freezing(5, 0, every=5)
        assert e.value.status == -6
        s.close()
    s = lbm.Solver(cfg, precision="fp64").set_geometry(arr)
    for obs, axis, index in ((2, 0, 0), (1, 0, cfg["ny"]), (1, 3, 0)):
        with pytest.raises(lbm.LbmError) as e:
            s.adjoint_freezing(5, obs, axis, index, every=5)
        assert e.value.status == -1
    s.close()


def test_coupled_adjoint_behind_autograd(env):
    O, lbm, S, torch = env
    cfg, arr = _frz_state(3)
    q = torch.tensor(list(cfg["T_wall"]) + [cfg["latent"], cfg["theta_deg"], cfg["sigma"],
                                            cfg["T_cold"]], dtype=torch.float64, requires_grad=True)
    y = S.AdjointFreezing.apply(q, cfg, arr, 80, 0, 0, 0, 40)
    (2.0 * y).backward()
    s = lbm.Solver(cfg, precision="fp64").set_geometry(arr)
    ff, grad = s.adjoint_freezing(80, 0, every=40)
    s.close()
    assert float(y.detach()) == ff
    assert q.grad.tolist() == [2.0 * v for v in grad]


def _full_state(seed, n=(40, 24), g=(2e-5, -3e-5), mask=False):
    """A random three-phase state with all three lattices (with or without
    its cold mask); a body force strong enough that the flow carries the
    interfaces."""
    cfg, arr = W.random_state(*n, seed=seed, lattices=W.FLOW | W.PHASE | W.HEAT)
    return dict(cfg, gx=g[0], gy=g[1]), {k: v for k, v in arr.items() if mask or k != "mask"}


@pytest.mark.parametrize("seed,mask", [(1, False), (3, False), (3, True), (0, True)])
def test_full_adjoint_equals_the_tangent(env, seed, mask):
    """The reverse sweep of the whole coupled step (moving fluid; with and
    without a cold mask) against the forward-mode tangent (wall
    temperatures, L, theta, the cold-mask temperature) and central
    differences (sigma, the body force)."""
    O, lbm, S, torch = env
    cfg, arr = _full_state(seed, mask=mask)
    steps = 150
    plain = lbm.Solver(cfg, precision="fp64").set_geometry(arr).step(steps)
    assert np.abs(plain.fields(("ux",))["ux"]).max() > 1e-5
    col = next(i for i in range(cfg["nx"]) if np.isfinite(plain.crossings(1, i)[0]))
    plain.close()
    res = {}
    for obs in (0, 1):
        s = lbm.Solver(cfg, precision="fp64").set_geometry(arr)
        res[obs] = s.adjoint_coupled(steps, obs, 1, col, every=37)
        s.close()
    rows = []
    dirs = [("T_wall", k) for k in range(4) if cfg["bc"][k] == "dirichlet"] + [("latent", 4), ("theta_deg", 5)]
    if mask:
        dirs.append(("T_cold", 9))
    for name, k in dirs:
        t = ({"T_wall": [1.0 if j == k else 0.0 for j in range(4)]} if name == "T_wall" else {name: 1.0})
        ts = lbm.Solver(cfg, precision="tangent", tangent=t).set_geometry(arr).step(steps)
        d, dt = ts.diagnostics(), ts.tangent_diagnostics(compute=False)
        fz, mv = d["frozen_volume"], d["material_volume"]
        dff = (dt["frozen_volume"] * mv - fz * dt["material_volume"]) / mv ** 2
        cr = ts.crossings_tangent(1, col)
        ts.close()
        rows.append((name, k, res[0][1][k], dff, res[1][1][k], cr[2]))

    def val(c, obs):
        u = lbm.Solver(c, precision="fp64").set_geometry(arr).step(steps)
        d = u.diagnostics()
        v = d["frozen_volume"] / d["material_volume"] if obs == 0 else u.crossings(1, col)[0]
        u.close()
        return v

    fds = []
    for name, k, h in (("sigma", 6, 1e-5 * cfg["sigma"]), ("gx", 7, 1e-4 * abs(cfg["gx"])),
                       ("gy", 8, 1e-4 * abs(cfg["gy"]))):
        for obs in (0, 1):
            fd = (val(dict(cfg, **{name: cfg[name] + h}), obs)
                  - val(dict(cfg, **{name: cfg[name] - h}), obs)) / (2 * h)
            fds.append((name, obs, res[obs][1][k], fd))
    print(f"\nseed {seed}, column {col}: FF {res[0][0]:.10f}, crossing {res[1][0]:.8f}")
    for r in rows + fds:
        print("  ", r)
    for name, k, aff, tff, acr, tcr in rows:
        assert abs(aff - tff) <= 1e-8 * abs(tff) + 1e-13, (name, k, aff, tff)
        assert abs(acr - tcr) <= 1e-8 * abs(tcr) + 1e-11, (name, k, acr, tcr)
    for name, obs, adj, fd in fds:
        assert abs(adj - fd) <= 1e-5 * abs(fd) + (1e-10 if obs == 0 else 1e-8), (name, obs, adj, fd)


def test_full_adjoint_checkpoints_and_rejections(env):
    O, lbm, S, torch = env
    cfg, arr = _full_state(3)
    steps = 50
    out = []
    for every in (1, 17, 50):
        s = lbm.Solver(cfg, precision="fp64").set_geometry(arr)
        out.append(s.adjoint_coupled(steps, 1, 1, 0, every=every))
        if every == 17:
            f_adj = s.fields()
        s.close()
    assert all(o == out[0] for o in out[1:]), out
    plain = lbm.Solver(cfg, precision="fp64").set_geometry(arr).step(steps)
    f_plain = plain.fields()
    plain.close()
    for k in FIELDS:
        assert np.array_equal(f_adj[k], f_plain[k]), k
    for c, a, prec in ((cfg, arr, "fp32"), (dict(cfg, lattices=6), arr, "fp64"),
                       (dict(cfg, readings=1), arr, "fp64")):
        s = lbm.Solver(c, precision=prec).set_geometry(a)
        with pytest.raises(lbm.LbmError) as e:
            s.adjoint_coupled(5, 0, every=5)
        assert e.value.status == -6
        s.close()


def test_full_adjoint_initial_temperature_gradient(env):
    """The per-node gradient with respect to the initial temperature field
    (one reverse sweep) against central differences of single-node
    perturbations, at nodes away from the T = T_m kink of Eq. (8)."""
    O, lbm, S, torch = env
    cfg, arr = _full_state(3)
    steps = 100
    s = lbm.Solver(cfg, precision="fp64").set_geometry(arr)
    ff, grad, dT0 = s.adjoint_coupled(steps, 0, every=25, initial_T=True)
    s.close()
    T0 = arr["T"]
    cand = [(j, i) for j in range(3, cfg["ny"] - 3) for i in range(3, cfg["nx"] - 3)
            if abs(T0[j, i]) > 0.1]
    nodes = [cand[0], cand[len(cand) // 2], cand[-1]]

    def ff_of(node, delta):
        a2 = dict(arr)
        T = T0.copy()
        T[node] += delta
        a2["T"] = T
        u = lbm.Solver(cfg, precision="fp64").set_geometry(a2).step(steps)
        d = u.diagnostics()
        u.close()
        return d["frozen_volume"] / d["material_volume"]

    h = 1e-6
    for node in nodes:
        fd = (ff_of(node, h) - ff_of(node, -h)) / (2 * h)
        print(f"\nnode {node}: T0 {T0[node]:+.3f} adjoint {dT0[node]:.10e} FD {fd:.10e}")
        assert abs(dT0[node] - fd) <= 1e-5 * abs(fd) + 1e-10, (node, dT0[node], fd)
    assert np.abs(dT0).max() > 0.0
    s = lbm.Solver(cfg, precision="fp64").set_geometry(arr).step(3)
    with pytest.raises(lbm.LbmError) as e:
        s.adjoint_coupled(5, 0, every=5, initial_T=True)
    assert e.value.status == -8
    s.close()


def test_heat_adjoint_with_cold_mask_equals_the_tangent(env):
    """The enthalpy-lattice sweep on a random state with a cold mask: the
    gradient w.r.t. the wall temperatures, L and the mask temperature T_cold
    equals the forward-mode tangent."""
    O, lbm, S, torch = env
    cfg, arr = W.random_state(40, 24, seed=3, lattices=W.HEAT)
    assert "mask" in arr and arr["mask"].any()
    steps = 150
    s = lbm.Solver(cfg, precision="fp64").set_geometry(arr)
    ff, grad = s.adjoint_frozen_fraction(steps, every=40)
    s.close()
    dirs = [("T_wall", k) for k in range(4) if cfg["bc"][k] == "dirichlet"] + [("latent", 4), ("T_cold", 5)]
    for name, k in dirs:
        t = ({"T_wall": [1.0 if j == k else 0.0 for j in range(4)]} if name == "T_wall" else {name: 1.0})
        ts = lbm.Solver(cfg, precision="tangent", tangent=t).set_geometry(arr).step(steps)
        d, dt = ts.diagnostics(), ts.tangent_diagnostics(compute=False)
        ts.close()
        fz, mv = d["frozen_volume"], d["material_volume"]
        tan = (dt["frozen_volume"] * mv - fz * dt["material_volume"]) / mv ** 2
        print(f"\n{name}: adjoint {grad[k]:.12e} tangent {tan:.12e}")
        assert abs(fz / mv - ff) <= 1e-12
        assert abs(grad[k] - tan) <= 1e-9 * abs(tan) + 1e-14, (name, grad[k], tan)
