"""Gradients of freezing observables with respect to the problem's
parameters, from forward-mode (tangent) steps of the fused kernel.

The parameters are those of the paper's problem statement: the wall
temperature T_w (Dirichlet walls and the cold substrate), the contact angle
theta (Eq. (4)) and the Stefan number Ste = Cp_l (T_m - T_w) / L (Eq. (29),
T_m = 0), so the latent heat follows both T_w and Ste.  The initial state is
held fixed.  One tangent context (``precision="tangent"``) per parameter
carries the derivative of every value through the same steps as the FP64
forward run; the observables and their derivatives are read from the FP64
diagnostic sums and the interface crossings:

* frozen fraction FF = sum w (1 - fl) / sum w (Sec. 4.3's freezing measure);
* tip height = the last phi = 0 crossing along a grid line (the droplet
  axis), Secs. 4.3-4.4;
* freezing time = the first time FF reaches a level (0.99), interpolated
  linearly between the two steps that bracket it.

``FreezingObservables`` wraps this as a ``torch.autograd.Function`` of the
parameter vector (T_w, theta_deg, Ste).
"""
from __future__ import annotations

import numpy as np

from . import lbm

PARAMS = ("T_w", "theta_deg", "ste")


def latent(cfg: dict, T_w: float, ste: float) -> float:
    """L of Eq. (29) with T_m = 0."""
    return float(cfg["cp_l"]) * (0.0 - T_w) / ste


def apply_params(cfg: dict, T_w: float, theta_deg: float, ste: float, wall) -> dict:
    """The workload dict with the parameters set.  wall: where T_w applies,
    a collection of wall indices 0-3 (x-low, x-high, y-low, y-high) and/or
    "cold" for the cold-mask temperature."""
    c = dict(cfg)
    tw = list(c["T_wall"])
    for k in wall:
        if k == "cold":
            c["T_cold"] = T_w
        else:
            tw[int(k)] = T_w
    c["T_wall"] = tuple(tw)
    c["theta_deg"] = theta_deg
    c["latent"] = latent(cfg, T_w, ste)
    return c


def direction(cfg: dict, name: str, T_w: float, ste: float, wall) -> dict:
    """Rates of the context parameters per unit of parameter `name`."""
    L = latent(cfg, T_w, ste)
    if name == "T_w":
        rates = [0.0, 0.0, 0.0, 0.0]
        for k in wall:
            if k != "cold":
                rates[int(k)] = 1.0
        return {"T_wall": rates, "T_cold": 1.0 if "cold" in wall else 0.0,
                "latent": -float(cfg["cp_l"]) / ste}
    if name == "theta_deg":
        return {"theta_deg": 1.0}
    if name == "ste":
        return {"latent": -L / ste}
    raise ValueError(name)


def observables(s: "lbm.Solver", line) -> np.ndarray:
    """(FF, tip height) of a solver's current state; tip NaN without line."""
    d = s.diagnostics(compute=True)
    ff = d["frozen_volume"] / d["material_volume"]
    tip = s.crossings(*line)[0] if line is not None else float("nan")
    return np.array([ff, tip])


def tangent_observables(s: "lbm.Solver", line) -> np.ndarray:
    """Derivatives of (FF, tip height) from a tangent solver's state."""
    d = s.diagnostics(compute=True)
    t = s.tangent_diagnostics(compute=False)
    fz, mv = d["frozen_volume"], d["material_volume"]
    dff = (t["frozen_volume"] * mv - fz * t["material_volume"]) / (mv * mv)
    dtip = s.crossings_tangent(*line)[2] if line is not None else float("nan")
    return np.array([dff, dtip])


def run(cfg: dict, arrays: dict, steps: int, precision="fp64", tangent=None) -> "lbm.Solver":
    """A solver advanced `steps` steps from the arrays."""
    return lbm.Solver(cfg, precision=precision, tangent=tangent).set_geometry(arrays).step(steps)


def value_and_jacobian(cfg: dict, arrays: dict, steps: int, p, wall, line):
    """(FF, tip) and their 2 x 3 Jacobian with respect to (T_w, theta, Ste)."""
    T_w, th, ste = (float(v) for v in p)
    c = apply_params(cfg, T_w, th, ste, wall)
    s = run(c, arrays, steps)
    val = observables(s, line)
    s.close()
    J = np.empty((2, 3))
    for j, name in enumerate(PARAMS):
        t = run(c, arrays, steps, precision="tangent",
                tangent=direction(cfg, name, T_w, ste, wall))
        J[:, j] = tangent_observables(t, line)
        t.close()
    return val, J


def _ff(d: dict) -> float:
    return d["frozen_volume"] / d["material_volume"]


def _dff(d: dict, t: dict) -> float:
    fz, mv = d["frozen_volume"], d["material_volume"]
    return (t["frozen_volume"] * mv - fz * t["material_volume"]) / (mv * mv)


def freezing_time(cfg: dict, arrays: dict, p, wall, name: str, level: float = 0.99,
                  max_steps: int = 200000):
    """(t*, dt*/d name): t* = n0 + (level - FF(n0)) / (FF(n0 + 1) - FF(n0)) for
    the step n0 after which FF first reaches `level`; its derivative is the
    exact derivative of that expression, from the tangent diagnostics of the
    two steps.  (nan, nan) if FF stays below `level` for max_steps steps."""
    T_w, th, ste = (float(v) for v in p)
    c = apply_params(cfg, T_w, th, ste, wall)
    t = run(c, arrays, 0, precision="tangent", tangent=direction(cfg, name, T_w, ste, wall))
    prev = None
    try:
        for n in range(max_steps + 1):
            d = t.diagnostics(compute=True)
            ff, dff = _ff(d), _dff(d, t.tangent_diagnostics(compute=False))
            if prev is not None and ff >= level:
                ff0, dff0 = prev
                span = ff - ff0
                frac = (level - ff0) / span
                dfrac = (-dff0 * span - (level - ff0) * (dff - dff0)) / (span * span)
                return (n - 1) + frac, dfrac
            prev = (ff, dff)
            t.step(1)
    finally:
        t.close()
    return float("nan"), float("nan")


class FreezingObservables:
    """``FreezingObservables.apply(p, cfg, arrays, steps, wall, line)``:
    (FF, tip height) after `steps` steps as a differentiable function of
    p = (T_w, theta_deg, Ste) (a float64 tensor); the backward pass returns
    J^T grad from three tangent runs."""

    _fn = None

    @classmethod
    def apply(cls, p, cfg, arrays, steps, wall, line):
        if cls._fn is None:
            import torch

            class _Fn(torch.autograd.Function):
                @staticmethod
                def forward(ctx, p, cfg, arrays, steps, wall, line):
                    val, J = value_and_jacobian(cfg, arrays, steps, p.detach().cpu().numpy(),
                                                wall, line)
                    ctx.save_for_backward(torch.as_tensor(J, dtype=torch.float64))
                    return torch.as_tensor(val, dtype=torch.float64)

                @staticmethod
                def backward(ctx, g):
                    (J,) = ctx.saved_tensors
                    return (J.T @ g.to(J.dtype)).to(g.device), None, None, None, None, None

            cls._fn = _Fn
        return cls._fn.apply(p, cfg, arrays, steps, wall, line)


# --- reverse mode: the hand-written adjoints behind torch.autograd ------------

def _adjoint_fn(name, run):
    """A torch.autograd.Function whose forward runs a reverse-mode library
    call from the initial fields (value and gradient in one sweep) and whose
    backward returns grad_output times the stored gradient."""
    import torch

    class _Fn(torch.autograd.Function):
        @staticmethod
        def forward(ctx, q, *args):
            val, grad = run(q.detach().cpu().numpy().astype(np.float64), *args)
            ctx.save_for_backward(torch.as_tensor(np.asarray(grad), dtype=torch.float64))
            ctx.nargs = len(args)
            return torch.as_tensor(val, dtype=torch.float64)

        @staticmethod
        def backward(ctx, g):
            (grad,) = ctx.saved_tensors
            return ((g.to(grad.dtype) * grad).to(g.device),) + (None,) * ctx.nargs

    _Fn.__name__ = name
    return _Fn


def _run_adjoint_ff(q, cfg, arrays, steps, every):
    c = dict(cfg, T_wall=tuple(float(v) for v in q[:4]), latent=float(q[4]), T_cold=float(q[5]))
    s = lbm.Solver(c, precision="fp64").set_geometry(arrays)
    try:
        return s.adjoint_frozen_fraction(steps, every)
    finally:
        s.close()


def _run_adjoint_crossing(q, cfg, arrays, steps, axis, index, every):
    c = dict(cfg, theta_deg=float(q[0]), sigma=float(q[1]))
    s = lbm.Solver(c, precision="fp64").set_geometry(arrays)
    try:
        return s.adjoint_crossing(steps, axis, index, every)
    finally:
        s.close()


class AdjointFrozenFraction:
    """``AdjointFrozenFraction.apply(q, cfg, arrays, steps, every)``: the
    frozen fraction after `steps` steps of an enthalpy-lattice context (see
    lbm_adjoint_frozen_fraction) as a differentiable function of
    q = (T_wall[0..3], latent, T_cold) (a float64 tensor of 6), from the
    initial fields; one forward-and-reverse sweep gives the value and the
    gradient."""

    _fn = None

    @classmethod
    def apply(cls, q, cfg, arrays, steps, every=64):
        if cls._fn is None:
            cls._fn = _adjoint_fn("AdjointFrozenFraction", _run_adjoint_ff)
        return cls._fn.apply(q, cfg, arrays, steps, every)


class AdjointCrossing:
    """``AdjointCrossing.apply(q, cfg, arrays, steps, axis, index, every)``:
    the last phi = 0 crossing along a grid line after `steps` steps of a
    phase-field context (see lbm_adjoint_crossing) as a differentiable
    function of q = (theta_deg, sigma), from the initial fields."""

    _fn = None

    @classmethod
    def apply(cls, q, cfg, arrays, steps, axis, index, every=64):
        if cls._fn is None:
            cls._fn = _adjoint_fn("AdjointCrossing", _run_adjoint_crossing)
        return cls._fn.apply(q, cfg, arrays, steps, axis, index, every)


def _run_adjoint_freezing(q, cfg, arrays, steps, observable, axis, index, every):
    c = dict(cfg, T_wall=tuple(float(v) for v in q[:4]), latent=float(q[4]),
             theta_deg=float(q[5]), sigma=float(q[6]), T_cold=float(q[7]))
    s = lbm.Solver(c, precision="fp64").set_geometry(arrays)
    try:
        return s.adjoint_freezing(steps, observable, axis, index, every)
    finally:
        s.close()


class AdjointFreezing:
    """``AdjointFreezing.apply(q, cfg, arrays, steps, observable, axis, index,
    every)``: the frozen fraction (observable 0) or an interface crossing
    (observable 1, along grid line (axis, index)) after `steps` steps of the
    coupled phase-field and enthalpy step (see lbm_adjoint_freezing), as a
    differentiable function of q = (T_wall[0..3], latent, theta_deg, sigma,
    T_cold), from the initial fields."""

    _fn = None

    @classmethod
    def apply(cls, q, cfg, arrays, steps, observable=0, axis=0, index=0, every=64):
        if cls._fn is None:
            cls._fn = _adjoint_fn("AdjointFreezing", _run_adjoint_freezing)
        return cls._fn.apply(q, cfg, arrays, steps, observable, axis, index, every)


def _run_adjoint_coupled(q, cfg, arrays, steps, observable, axis, index, every):
    c = dict(cfg, T_wall=tuple(float(v) for v in q[:4]), latent=float(q[4]),
             theta_deg=float(q[5]), sigma=float(q[6]), gx=float(q[7]), gy=float(q[8]),
             T_cold=float(q[9]))
    s = lbm.Solver(c, precision="fp64").set_geometry(arrays)
    try:
        return s.adjoint_coupled(steps, observable, axis, index, every)
    finally:
        s.close()


class AdjointCoupled:
    """``AdjointCoupled.apply(q, cfg, arrays, steps, observable, axis, index,
    every)``: the frozen fraction (observable 0) or an interface crossing
    (observable 1) after `steps` steps of the whole coupled step (see
    lbm_adjoint_coupled) as a differentiable function of
    q = (T_wall[0..3], latent, theta_deg, sigma, gx, gy, T_cold), from the
    initial fields."""

    _fn = None

    @classmethod
    def apply(cls, q, cfg, arrays, steps, observable=0, axis=0, index=0, every=64):
        if cls._fn is None:
            cls._fn = _adjoint_fn("AdjointCoupled", _run_adjoint_coupled)
        return cls._fn.apply(q, cfg, arrays, steps, observable, axis, index, every)
