"""Python binding of the C ABI in ``include/lbm.h`` (argument marshalling only).

Every computation happens in ``_lib/liblbm_gb300.so`` (sm_103a kernels).  The
functions below keep the C names; ``Solver`` wraps one context with PyTorch
tensors for device memory and PyTorch's current CUDA stream.  There is no CPU
path: loading fails loudly when the library is missing.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "liblbm_gb300.so")

LBM_OK, LBM_ERR_NONFINITE = 0, -5
LBM_FP64, LBM_FP32, LBM_FP16S, LBM_FP64_TANGENT = 0, 1, 2, 3
PRECISION = {"fp64": LBM_FP64, "fp32": LBM_FP32, "fp16s": LBM_FP16S, "tangent": LBM_FP64_TANGENT}
LBM_HOST, LBM_DEVICE = 0, 1
BC = {"periodic": 0, "dirichlet": 1, "adiabatic": 2}
FIELDS = ("phi", "fs", "fl", "T", "rhoH", "p", "ux", "uy", "rho", "mu", "w", "mdot")
FIELD_BIT = {k: 1 << i for i, k in enumerate(FIELDS)}


class LbmParams(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
        ("precision", ctypes.c_int32), ("lattices", ctypes.c_uint32),
        ("bc", ctypes.c_int32 * 4), ("T_wall", ctypes.c_double * 4),
        ("rho_l", ctypes.c_double), ("rho_s", ctypes.c_double), ("rho_g", ctypes.c_double),
        ("mu_l", ctypes.c_double), ("mu_s", ctypes.c_double), ("mu_g", ctypes.c_double),
        ("lambda_l", ctypes.c_double), ("lambda_s", ctypes.c_double),
        ("lambda_g", ctypes.c_double),
        ("cp_l", ctypes.c_double), ("cp_s", ctypes.c_double), ("cp_g", ctypes.c_double),
        ("rho_ref", ctypes.c_double), ("latent", ctypes.c_double),
        ("sigma", ctypes.c_double), ("eps", ctypes.c_double),
        ("mobility", ctypes.c_double), ("eta", ctypes.c_double),
        ("theta_deg", ctypes.c_double), ("psi_deg", ctypes.c_double),
        ("gx", ctypes.c_double), ("gy", ctypes.c_double),
        ("T_cold", ctypes.c_double),
        ("readings", ctypes.c_uint32),
        ("diag_every", ctypes.c_int32),
        ("tan_T_wall", ctypes.c_double * 4),
        ("tan_T_cold", ctypes.c_double), ("tan_theta_deg", ctypes.c_double),
        ("tan_latent", ctypes.c_double),
    ]


class LbmDiag(ctypes.Structure):
    _fields_ = [(k, ctypes.c_double) for k in (
        "mass", "material_mass", "rhoH", "liquid_volume", "material_volume",
        "frozen_volume", "phi_sum", "kinetic", "nonfinite")] + [("step", ctypes.c_int64)]


EXPORTS = ("lbm_create", "lbm_set_geometry", "lbm_step", "lbm_read_fields",
           "lbm_compute_diagnostics", "lbm_read_diagnostics", "lbm_state_size",
           "lbm_save_state", "lbm_load_state", "lbm_step_count", "lbm_last_error",
           "lbm_status_string", "lbm_source_hash", "lbm_destroy", "lbm_diagnostics_noalloc",
           "lbm_batch_create", "lbm_batch_step", "lbm_batch_destroy", "lbm_probe_fma_rate",
           "lbm_read_crossings", "lbm_read_tangent_fields", "lbm_read_tangent_diagnostics",
           "lbm_read_crossings_tangent", "lbm_autotune", "lbm_adjoint_frozen_fraction",
           "lbm_adjoint_crossing", "lbm_adjoint_freezing", "lbm_adjoint_coupled",
           "lbm_debug_fail_allocation", "lbm_debug_tile_timeout", "lbm3_create", "lbm3_set_geometry", "lbm3_step",
           "lbm3_read_fields", "lbm3_diagnostics", "lbm3_step_count", "lbm3_last_error",
           "lbm3_destroy", "lbm3_lattice", "lbm3_state_size", "lbm3_save_state",
           "lbm3_load_state", "lbm3_read_tangent_fields", "lbm3_read_tangent_diagnostics")
FIELDS3 = ("phi", "fs", "fl", "T", "rhoH", "p", "ux", "uy", "uz", "rho", "mu", "w", "mdot")

_lib = None


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_2510_18688_gb300/build.py "
                           "(there is no CPU fallback)")
    L = ctypes.CDLL(path)
    vp, dp = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)
    L.lbm_create.argtypes = [ctypes.POINTER(LbmParams), ctypes.POINTER(vp)]
    L.lbm_set_geometry.argtypes = [vp, vp, vp, vp, vp, vp, ctypes.c_int, vp]
    L.lbm_step.argtypes = [vp, ctypes.c_int64, vp]
    L.lbm_read_fields.argtypes = [vp, ctypes.c_uint32, ctypes.POINTER(vp), ctypes.c_int, vp]
    L.lbm_compute_diagnostics.argtypes = [vp, vp]
    L.lbm_read_diagnostics.argtypes = [vp, ctypes.POINTER(LbmDiag)]
    L.lbm_state_size.argtypes = [vp, ctypes.POINTER(ctypes.c_size_t)]
    L.lbm_save_state.argtypes = [vp, vp, ctypes.c_size_t, vp]
    L.lbm_load_state.argtypes = [vp, vp, ctypes.c_size_t, vp]
    L.lbm_step_count.argtypes = [vp]
    L.lbm_step_count.restype = ctypes.c_int64
    L.lbm_last_error.argtypes = [vp]
    L.lbm_last_error.restype = ctypes.c_char_p
    L.lbm_status_string.argtypes = [ctypes.c_int]
    L.lbm_status_string.restype = ctypes.c_char_p
    L.lbm_source_hash.argtypes = []
    L.lbm_source_hash.restype = ctypes.c_char_p
    L.lbm_destroy.argtypes = [vp]
    L.lbm_destroy.restype = None
    L.lbm_diagnostics_noalloc.argtypes = [ctypes.POINTER(LbmParams), vp, vp, vp, vp, vp, vp]
    L.lbm_batch_create.argtypes = [ctypes.POINTER(vp), ctypes.c_int, ctypes.POINTER(vp)]
    L.lbm_batch_step.argtypes = [vp, ctypes.c_int64, vp]
    L.lbm_batch_destroy.argtypes = [vp]
    L.lbm_batch_destroy.restype = None
    L.lbm_probe_fma_rate.argtypes = [ctypes.c_int, dp, vp]
    L.lbm_read_crossings.argtypes = [vp, ctypes.c_int, ctypes.c_int, dp, vp]
    L.lbm_read_crossings_tangent.argtypes = [vp, ctypes.c_int, ctypes.c_int, dp, vp]
    L.lbm_read_tangent_fields.argtypes = [vp, ctypes.c_uint32, ctypes.POINTER(vp), ctypes.c_int, vp]
    L.lbm_read_tangent_diagnostics.argtypes = [vp, ctypes.POINTER(LbmDiag)]
    L.lbm_autotune.argtypes = [vp, ctypes.c_int, vp, dp, ctypes.POINTER(ctypes.c_int)]
    L.lbm_adjoint_frozen_fraction.argtypes = [vp, ctypes.c_int64, ctypes.c_int, dp, dp, vp]
    L.lbm_adjoint_crossing.argtypes = [vp, ctypes.c_int64, ctypes.c_int, ctypes.c_int,
                                       ctypes.c_int, dp, dp, vp]
    L.lbm_adjoint_freezing.argtypes = [vp, ctypes.c_int64, ctypes.c_int, ctypes.c_int,
                                       ctypes.c_int, ctypes.c_int, dp, dp, vp]
    L.lbm_adjoint_coupled.argtypes = [vp, ctypes.c_int64, ctypes.c_int, ctypes.c_int,
                                      ctypes.c_int, ctypes.c_int, dp, dp, dp, vp]
    L.lbm_debug_fail_allocation.argtypes = [ctypes.c_int]
    L.lbm_debug_fail_allocation.restype = None
    L.lbm_debug_tile_timeout.argtypes = [ctypes.c_int]
    L.lbm_debug_tile_timeout.restype = None
    L.lbm3_create.argtypes = [ctypes.POINTER(Lbm3Params), ctypes.POINTER(vp)]
    L.lbm3_set_geometry.argtypes = [vp, vp, vp, vp, vp, vp, ctypes.c_int, vp]
    L.lbm3_step.argtypes = [vp, ctypes.c_int64, vp]
    L.lbm3_read_fields.argtypes = [vp, ctypes.c_uint32, ctypes.POINTER(vp), ctypes.c_int, vp]
    L.lbm3_diagnostics.argtypes = [vp, ctypes.POINTER(LbmDiag), vp]
    L.lbm3_step_count.argtypes = [vp]
    L.lbm3_step_count.restype = ctypes.c_int64
    L.lbm3_last_error.argtypes = [vp]
    L.lbm3_last_error.restype = ctypes.c_char_p
    L.lbm3_destroy.argtypes = [vp]
    L.lbm3_destroy.restype = None
    L.lbm3_lattice.argtypes = [ctypes.POINTER(ctypes.c_int32), dp]
    L.lbm3_state_size.argtypes = [vp, ctypes.POINTER(ctypes.c_size_t)]
    L.lbm3_read_tangent_fields.argtypes = [vp, ctypes.c_uint32, ctypes.POINTER(vp), ctypes.c_int, vp]
    L.lbm3_read_tangent_diagnostics.argtypes = [vp, ctypes.POINTER(LbmDiag)]
    L.lbm3_save_state.argtypes = [vp, vp, ctypes.c_size_t, vp]
    L.lbm3_load_state.argtypes = [vp, vp, ctypes.c_size_t, vp]
    L.lbm3_lattice.restype = None
    for fn in ("lbm3_create", "lbm3_set_geometry", "lbm3_step", "lbm3_read_fields",
               "lbm3_diagnostics", "lbm3_state_size", "lbm3_save_state", "lbm3_load_state",
               "lbm3_read_tangent_fields", "lbm3_read_tangent_diagnostics"):
        getattr(L, fn).restype = ctypes.c_int
    for fn in ("lbm_create", "lbm_set_geometry", "lbm_step", "lbm_read_fields",
               "lbm_compute_diagnostics", "lbm_read_diagnostics", "lbm_state_size",
               "lbm_save_state", "lbm_load_state", "lbm_diagnostics_noalloc",
               "lbm_batch_create", "lbm_batch_step", "lbm_probe_fma_rate",
               "lbm_read_crossings", "lbm_read_crossings_tangent", "lbm_read_tangent_fields",
               "lbm_read_tangent_diagnostics", "lbm_autotune", "lbm_adjoint_frozen_fraction",
               "lbm_adjoint_crossing", "lbm_adjoint_freezing", "lbm_adjoint_coupled"):
        getattr(L, fn).restype = ctypes.c_int
    _lib = L
    return L


class Lbm3Params(ctypes.Structure):
    _fields_ = [("base", LbmParams), ("nz", ctypes.c_int32), ("bc_z", ctypes.c_int32 * 2),
                ("T_wall_z", ctypes.c_double * 2), ("gz", ctypes.c_double),
                ("tan_T_wall_z", ctypes.c_double * 2)]


class LbmError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{msg} (status {status})")
        self.status = status


def make_params(cfg: dict, precision: str = "fp32", diag_every: int = 0,
                tangent: dict = None) -> LbmParams:
    """lbm_params of a workload dict.  tangent (precision "tangent"): the
    parameter direction as rates {"T_wall": [4 values], "T_cold",
    "theta_deg", "latent"} (missing entries: 0)."""
    p = LbmParams()
    p.nx, p.ny = int(cfg["nx"]), int(cfg["ny"])
    p.precision = PRECISION[precision]
    p.lattices = int(cfg["lattices"])
    for k in range(4):
        p.bc[k] = BC[cfg["bc"][k]]
        p.T_wall[k] = float(cfg["T_wall"][k])
    for name in ("rho_l", "rho_s", "rho_g", "mu_l", "mu_s", "mu_g", "lambda_l", "lambda_s",
                 "lambda_g", "cp_l", "cp_s", "cp_g", "rho_ref", "latent", "sigma", "eps",
                 "mobility", "eta", "theta_deg", "psi_deg", "gx", "gy", "T_cold"):
        setattr(p, name, float(cfg[name]))
    p.readings = int(cfg.get("readings", 0))
    p.diag_every = int(diag_every)
    t = tangent or {}
    for k, v in enumerate(t.get("T_wall", (0.0, 0.0, 0.0, 0.0))):
        p.tan_T_wall[k] = float(v)
    p.tan_T_cold = float(t.get("T_cold", 0.0))
    p.tan_theta_deg = float(t.get("theta_deg", 0.0))
    p.tan_latent = float(t.get("latent", 0.0))
    return p


# --- the C entry points, same names ------------------------------------------

def _check(ctx, st, what):
    if st != LBM_OK:
        msg = load().lbm_last_error(ctx).decode() if ctx else ""
        raise LbmError(st, f"{what}: {load().lbm_status_string(st).decode()} {msg}")


def lbm_create(params: LbmParams) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    _check(None, load().lbm_create(ctypes.byref(params), ctypes.byref(h)), "lbm_create")
    return h


def lbm_set_geometry(ctx, phi0, cold_mask, phi, T, fl, where, stream=None):
    _check(ctx, load().lbm_set_geometry(ctx, phi0, cold_mask, phi, T, fl, where, stream),
           "lbm_set_geometry")


def lbm_step(ctx, nsteps: int, stream=None):
    _check(ctx, load().lbm_step(ctx, int(nsteps), stream), "lbm_step")


def lbm_read_fields(ctx, field_mask: int, out_ptrs, where, stream=None):
    arr = (ctypes.c_void_p * len(FIELDS))(*[p or None for p in out_ptrs])
    _check(ctx, load().lbm_read_fields(ctx, field_mask, arr, where, stream), "lbm_read_fields")


def lbm_read_tangent_fields(ctx, field_mask: int, out_ptrs, where, stream=None):
    arr = (ctypes.c_void_p * len(FIELDS))(*[p or None for p in out_ptrs])
    _check(ctx, load().lbm_read_tangent_fields(ctx, field_mask, arr, where, stream),
           "lbm_read_tangent_fields")


def lbm_read_tangent_diagnostics(ctx) -> dict:
    d = LbmDiag()
    _check(ctx, load().lbm_read_tangent_diagnostics(ctx, ctypes.byref(d)),
           "lbm_read_tangent_diagnostics")
    return {k: getattr(d, k) for k, _ in LbmDiag._fields_}


def lbm_read_crossings_tangent(ctx, axis: int, index: int, stream=None):
    """(phi = 0 crossing, ice front, their derivatives) along one line."""
    out = (ctypes.c_double * 4)()
    _check(ctx, load().lbm_read_crossings_tangent(ctx, int(axis), int(index), out, stream),
           "lbm_read_crossings_tangent")
    return tuple(out)


def lbm_adjoint_frozen_fraction(ctx, nsteps: int, every: int, stream=None):
    """(FF after nsteps steps, [dFF/dT_wall[0..3], dFF/dlatent, dFF/dT_cold]);
    see include/lbm.h."""
    ff = ctypes.c_double()
    grad = (ctypes.c_double * 6)()
    _check(ctx, load().lbm_adjoint_frozen_fraction(ctx, int(nsteps), int(every), ctypes.byref(ff),
                                                   grad, stream), "lbm_adjoint_frozen_fraction")
    return ff.value, list(grad)


def lbm_adjoint_crossing(ctx, nsteps: int, every: int, axis: int, index: int, stream=None):
    """(phi = 0 crossing along the line after nsteps steps, [d/dtheta_deg,
    d/dsigma]); see include/lbm.h."""
    pos = ctypes.c_double()
    grad = (ctypes.c_double * 2)()
    _check(ctx, load().lbm_adjoint_crossing(ctx, int(nsteps), int(every), int(axis), int(index),
                                            ctypes.byref(pos), grad, stream),
           "lbm_adjoint_crossing")
    return pos.value, list(grad)


def lbm_adjoint_freezing(ctx, nsteps: int, every: int, observable: int, axis: int = 0,
                         index: int = 0, stream=None):
    """(observable after nsteps steps -- 0: frozen fraction, 1: the phi = 0
    crossing along (axis, index) -- and its gradient w.r.t. (T_wall[0..3],
    latent, theta_deg, sigma, T_cold)); see include/lbm.h."""
    val = ctypes.c_double()
    grad = (ctypes.c_double * 8)()
    _check(ctx, load().lbm_adjoint_freezing(ctx, int(nsteps), int(every), int(observable),
                                            int(axis), int(index), ctypes.byref(val), grad,
                                            stream), "lbm_adjoint_freezing")
    return val.value, list(grad)


def lbm_adjoint_coupled(ctx, nsteps: int, every: int, observable: int, axis: int = 0,
                        index: int = 0, dT0=None, stream=None):
    """(observable after nsteps steps of the whole coupled step and its
    gradient w.r.t. (T_wall[0..3], latent, theta_deg, sigma, gx, gy,
    T_cold)); with dT0 (a float64 [ny, nx] numpy array) also the gradient
    w.r.t. the initial temperature field; see include/lbm.h."""
    val = ctypes.c_double()
    grad = (ctypes.c_double * 10)()
    dptr = None if dT0 is None else dT0.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    _check(ctx, load().lbm_adjoint_coupled(ctx, int(nsteps), int(every), int(observable),
                                           int(axis), int(index), ctypes.byref(val), grad,
                                           dptr, stream), "lbm_adjoint_coupled")
    return val.value, list(grad)


# kernel form ids of lbm_autotune (variant v = form v // 2, period v % 2)
FORMS = ("one CTA per 32x8 tile", "float: TMA-staged, one stage / fp64: two-kernel split",
         "float: TMA-staged, two stages, 2 persistent CTAs per SM",
         "float: TMA-staged, one stage, 3 persistent CTAs per SM", "one CTA per 32x4 tile",
         "one CTA per 32x16 tile")
N_VARIANTS = 2 * len(FORMS)
VARIANTS = tuple(f"{f}, periods >= {p}" for f in FORMS for p in (32, 256))


def lbm_autotune(ctx, steps_per_trial: int = 64, stream=None):
    """(microseconds per step of each variant, index kept); see include/lbm.h."""
    us = (ctypes.c_double * N_VARIANTS)()
    chosen = ctypes.c_int()
    _check(ctx, load().lbm_autotune(ctx, int(steps_per_trial), stream, us, ctypes.byref(chosen)),
           "lbm_autotune")
    return list(us), chosen.value


def lbm_compute_diagnostics(ctx, stream=None):
    _check(ctx, load().lbm_compute_diagnostics(ctx, stream), "lbm_compute_diagnostics")


def lbm_read_diagnostics(ctx) -> dict:
    d = LbmDiag()
    st = load().lbm_read_diagnostics(ctx, ctypes.byref(d))
    if st not in (LBM_OK, LBM_ERR_NONFINITE):
        _check(ctx, st, "lbm_read_diagnostics")
    return {k: getattr(d, k) for k, _ in LbmDiag._fields_}


def lbm_state_size(ctx) -> int:
    n = ctypes.c_size_t()
    _check(ctx, load().lbm_state_size(ctx, ctypes.byref(n)), "lbm_state_size")
    return n.value


def lbm_save_state(ctx, stream=None) -> bytes:
    n = lbm_state_size(ctx)
    buf = ctypes.create_string_buffer(n)
    _check(ctx, load().lbm_save_state(ctx, buf, n, stream), "lbm_save_state")
    return buf.raw


def lbm_load_state(ctx, blob: bytes, stream=None):
    buf = ctypes.create_string_buffer(blob, len(blob))
    _check(ctx, load().lbm_load_state(ctx, buf, len(blob), stream), "lbm_load_state")


def lbm_step_count(ctx) -> int:
    return int(load().lbm_step_count(ctx))


def lbm_diagnostics_noalloc(params: LbmParams, pops, lags, phi0, cold_mask, out,
                            stream=None) -> int:
    """Diagnostics of a caller-held device state without device allocation
    (see include/lbm.h); returns the status code."""
    return int(load().lbm_diagnostics_noalloc(ctypes.byref(params), pops, lags, phi0,
                                              cold_mask, out, stream))


def lbm_read_crossings(ctx, axis: int, index: int, stream=None):
    """(phi = 0 crossing, ice-front crossing) along one grid line; NaN if none."""
    out = (ctypes.c_double * 2)()
    _check(ctx, load().lbm_read_crossings(ctx, int(axis), int(index), out, stream),
           "lbm_read_crossings")
    return out[0], out[1]


def lbm_probe_fma_rate(precision: str = "fp64", stream=None) -> float:
    """Measured FMA throughput of the current device in FLOP/s (2 per FMA)."""
    v = ctypes.c_double()
    st = load().lbm_probe_fma_rate(LBM_FP64 if precision == "fp64" else LBM_FP32,
                                   ctypes.byref(v), stream)
    _check(None, st, "lbm_probe_fma_rate")
    return v.value


def lbm_batch_create(ctxs) -> ctypes.c_void_p:
    arr = (ctypes.c_void_p * len(ctxs))(*[c.value if isinstance(c, ctypes.c_void_p) else c
                                           for c in ctxs])
    h = ctypes.c_void_p()
    _check(None, load().lbm_batch_create(arr, len(ctxs), ctypes.byref(h)), "lbm_batch_create")
    return h


def lbm_batch_step(batch, nsteps: int, stream=None):
    _check(None, load().lbm_batch_step(batch, int(nsteps), stream), "lbm_batch_step")


def lbm_batch_destroy(batch):
    if batch:
        load().lbm_batch_destroy(batch)


def lbm_last_error(ctx) -> str:
    return load().lbm_last_error(ctx).decode()


def lbm_status_string(status: int) -> str:
    return load().lbm_status_string(int(status)).decode()


def lbm_source_hash() -> str:
    return load().lbm_source_hash().decode()


def lbm_destroy(ctx):
    if ctx:
        load().lbm_destroy(ctx)


# --- convenience wrapper with torch tensors ----------------------------------

def _stream():
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


class Solver:
    """One GPU context.  Inputs: the workload dict and arrays of
    ``paper_2510_18688_gb300.workloads``; fields come back as torch tensors
    on the device (or numpy arrays with ``host=True``)."""

    def __init__(self, cfg: dict, precision: str = "fp32", diag_every: int = 0,
                 tangent: dict = None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("Solver needs a CUDA device (no CPU path)")
        load()
        self.cfg = dict(cfg)
        self.nx, self.ny = int(cfg["nx"]), int(cfg["ny"])
        self.precision = precision
        self.params = make_params(cfg, precision, diag_every, tangent)
        self.ctx = lbm_create(self.params)

    def close(self):
        if getattr(self, "ctx", None):
            lbm_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_geometry(self, arrays: dict, on_device: bool = True):
        import torch
        keys = ("phi0", "phi", "T", "fl")
        if on_device:
            t = {k: torch.as_tensor(np.ascontiguousarray(arrays[k], dtype=np.float64),
                                    device="cuda") for k in keys}
            m = arrays.get("mask")
            tm = None if m is None else torch.as_tensor(
                np.ascontiguousarray(m, dtype=np.uint8), device="cuda")
            lbm_set_geometry(self.ctx, t["phi0"].data_ptr(), None if tm is None else tm.data_ptr(),
                             t["phi"].data_ptr(), t["T"].data_ptr(), t["fl"].data_ptr(),
                             LBM_DEVICE, _stream())
            torch.cuda.current_stream().synchronize()
        else:
            h = {k: np.ascontiguousarray(arrays[k], dtype=np.float64) for k in keys}
            m = arrays.get("mask")
            hm = None if m is None else np.ascontiguousarray(m, dtype=np.uint8)
            lbm_set_geometry(self.ctx, h["phi0"].ctypes.data, None if hm is None else hm.ctypes.data,
                             h["phi"].ctypes.data, h["T"].ctypes.data, h["fl"].ctypes.data,
                             LBM_HOST, _stream())
        return self

    def step(self, n: int = 1):
        lbm_step(self.ctx, n, _stream())
        return self

    @property
    def steps_done(self) -> int:
        return lbm_step_count(self.ctx)

    def crossings(self, axis: int, index: int):
        """Interface positions along one line (see lbm_read_crossings)."""
        return lbm_read_crossings(self.ctx, axis, index, _stream())

    def adjoint_frozen_fraction(self, nsteps: int, every: int = 64):
        """Advance nsteps and return (FF, its gradient) by reverse mode
        (enthalpy-lattice FP64 contexts; see lbm_adjoint_frozen_fraction)."""
        return lbm_adjoint_frozen_fraction(self.ctx, nsteps, every, _stream())

    def adjoint_crossing(self, nsteps: int, axis: int, index: int, every: int = 64):
        """Advance nsteps and return (the phi = 0 crossing along the line, its
        gradient with respect to (theta_deg, sigma)) by reverse mode
        (phase-field-only FP64 contexts; see lbm_adjoint_crossing)."""
        return lbm_adjoint_crossing(self.ctx, nsteps, every, axis, index, _stream())

    def adjoint_freezing(self, nsteps: int, observable: int = 0, axis: int = 0, index: int = 0,
                         every: int = 64):
        """Advance nsteps and return (observable, gradient w.r.t. (T_wall[0..3],
        latent, theta_deg, sigma, T_cold)) by reverse mode of the coupled phase-field
        and enthalpy step (see lbm_adjoint_freezing)."""
        return lbm_adjoint_freezing(self.ctx, nsteps, every, observable, axis, index, _stream())

    def adjoint_coupled(self, nsteps: int, observable: int = 0, axis: int = 0, index: int = 0,
                        every: int = 64, initial_T: bool = False):
        """Advance nsteps and return (observable, gradient w.r.t. (T_wall[0..3],
        latent, theta_deg, sigma, gx, gy, T_cold)) by reverse mode of the whole coupled
        step (see lbm_adjoint_coupled); with initial_T also the [ny, nx]
        gradient w.r.t. the initial temperature field, as a third item."""
        if not initial_T:
            return lbm_adjoint_coupled(self.ctx, nsteps, every, observable, axis, index,
                                       None, _stream())
        dT0 = np.empty((self.ny, self.nx), dtype=np.float64)
        v, g = lbm_adjoint_coupled(self.ctx, nsteps, every, observable, axis, index, dT0,
                                   _stream())
        return v, g, dT0

    def autotune(self, steps_per_trial: int = 64):
        """Pick the fastest step form for this grid (state unchanged)."""
        return lbm_autotune(self.ctx, steps_per_trial, _stream())

    def crossings_tangent(self, axis: int, index: int):
        """Crossings and their derivatives (tangent contexts)."""
        return lbm_read_crossings_tangent(self.ctx, axis, index, _stream())

    def tangent_fields(self, names=FIELDS) -> dict:
        """Derivatives of the fields along the parameter direction (host)."""
        return self.fields(names, host=True, deriv=True)

    def tangent_diagnostics(self, compute: bool = True) -> dict:
        if compute:
            lbm_compute_diagnostics(self.ctx, _stream())
        return lbm_read_tangent_diagnostics(self.ctx)

    def fields(self, names=FIELDS, host: bool = True, deriv: bool = False) -> dict:
        import torch
        mask = 0
        ptrs = [None] * len(FIELDS)
        out = {}
        for k in names:
            mask |= FIELD_BIT[k]
            if host:
                out[k] = np.empty((self.ny, self.nx), dtype=np.float64)
                ptrs[FIELDS.index(k)] = out[k].ctypes.data
            else:
                out[k] = torch.empty((self.ny, self.nx), dtype=torch.float64, device="cuda")
                ptrs[FIELDS.index(k)] = out[k].data_ptr()
        read = lbm_read_tangent_fields if deriv else lbm_read_fields
        read(self.ctx, mask, ptrs, LBM_HOST if host else LBM_DEVICE, _stream())
        return out

    def diagnostics(self, compute: bool = True) -> dict:
        if compute:
            lbm_compute_diagnostics(self.ctx, _stream())
        return lbm_read_diagnostics(self.ctx)

    def save(self) -> bytes:
        return lbm_save_state(self.ctx, _stream())

    def load(self, blob: bytes):
        lbm_load_state(self.ctx, blob, _stream())


class Batch:
    """Several Solvers advanced together, one persistent launch per step."""

    def __init__(self, solvers):
        self.solvers = list(solvers)
        self.handle = lbm_batch_create([s.ctx for s in self.solvers])

    def step(self, n: int = 1):
        lbm_batch_step(self.handle, n, _stream())
        return self

    def close(self):
        if getattr(self, "handle", None):
            lbm_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# --- three-dimensional (D3Q19) contexts ---------------------------------------

def make_params3(cfg: dict, precision: str = "fp32", tangent: dict = None) -> Lbm3Params:
    """lbm3_params of a 3-D workload dict (six boundary types and wall
    temperatures: x_lo, x_hi, y_lo, y_hi, z_lo, z_hi; nz; gz).  tangent
    (precision "tangent"): {"T_wall": [6 rates], "T_cold", "theta_deg",
    "latent"} (missing entries: 0)."""
    t = dict(tangent or {})
    tw = list(t.get("T_wall", [0.0] * 6)) + [0.0] * 6
    t2 = dict(t, T_wall=tw[:4])
    base = make_params(dict(cfg, bc=tuple(cfg["bc"][:4]), T_wall=tuple(cfg["T_wall"][:4])),
                       precision, 0, t2)
    p = Lbm3Params()
    p.base = base
    p.nz = int(cfg["nz"])
    for k in range(2):
        p.bc_z[k] = BC[cfg["bc"][4 + k]]
        p.T_wall_z[k] = float(cfg["T_wall"][4 + k])
    p.gz = float(cfg.get("gz", 0.0))
    p.tan_T_wall_z[0], p.tan_T_wall_z[1] = float(tw[4]), float(tw[5])
    return p


def _check3(ctx, st, what):
    if st != LBM_OK:
        msg = load().lbm3_last_error(ctx).decode() if ctx else ""
        raise LbmError(st, f"{what}: {load().lbm_status_string(st).decode()} {msg}")


def lbm_debug_fail_allocation(after: int):
    """Testing hook: the (after + 1)-th allocation of the next lbm_create
    calls fails as out of memory (after < 0 disarms); see include/lbm.h."""
    load().lbm_debug_fail_allocation(int(after))


def lbm_debug_tile_timeout(on: bool):
    """Test hook: the float step's tile kernels expect more bytes than their
    copies deliver, so their bounded waits run out (see include/lbm.h)."""
    load().lbm_debug_tile_timeout(1 if on else 0)


def lbm3_create(params: Lbm3Params) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    _check3(None, load().lbm3_create(ctypes.byref(params), ctypes.byref(h)), "lbm3_create")
    return h


def lbm3_set_geometry(ctx, phi0, cold_mask, phi, T, fl, where, stream=None):
    _check3(ctx, load().lbm3_set_geometry(ctx, phi0, cold_mask, phi, T, fl, where, stream),
            "lbm3_set_geometry")


def lbm3_step(ctx, nsteps: int, stream=None):
    _check3(ctx, load().lbm3_step(ctx, int(nsteps), stream), "lbm3_step")


def lbm3_read_fields(ctx, field_mask: int, out_ptrs, where, stream=None):
    arr = (ctypes.c_void_p * len(FIELDS3))(*[p or None for p in out_ptrs])
    _check3(ctx, load().lbm3_read_fields(ctx, field_mask, arr, where, stream), "lbm3_read_fields")


def lbm3_diagnostics(ctx, stream=None) -> dict:
    """The diagnostic sums (a non-finite state is reported in 'nonfinite',
    not raised)."""
    d = LbmDiag()
    st = load().lbm3_diagnostics(ctx, ctypes.byref(d), stream)
    if st not in (LBM_OK, LBM_ERR_NONFINITE):
        _check3(ctx, st, "lbm3_diagnostics")
    return {k: getattr(d, k) for k, _ in LbmDiag._fields_}


def lbm3_step_count(ctx) -> int:
    return int(load().lbm3_step_count(ctx))


def lbm3_last_error(ctx) -> str:
    return load().lbm3_last_error(ctx).decode()


def lbm3_destroy(ctx):
    load().lbm3_destroy(ctx)


def lbm3_state_size(ctx) -> int:
    n = ctypes.c_size_t()
    _check3(ctx, load().lbm3_state_size(ctx, ctypes.byref(n)), "lbm3_state_size")
    return int(n.value)


def lbm3_save_state(ctx, stream=None) -> bytes:
    buf = ctypes.create_string_buffer(lbm3_state_size(ctx))
    _check3(ctx, load().lbm3_save_state(ctx, buf, len(buf), stream), "lbm3_save_state")
    return buf.raw


def lbm3_load_state(ctx, data: bytes, stream=None):
    buf = ctypes.create_string_buffer(data, len(data))
    _check3(ctx, load().lbm3_load_state(ctx, buf, len(data), stream), "lbm3_load_state")


def lbm3_read_tangent_fields(ctx, field_mask: int, out_ptrs, where, stream=None):
    arr = (ctypes.c_void_p * len(FIELDS3))(*[p or None for p in out_ptrs])
    _check3(ctx, load().lbm3_read_tangent_fields(ctx, field_mask, arr, where, stream),
            "lbm3_read_tangent_fields")


def lbm3_read_tangent_diagnostics(ctx) -> dict:
    d = LbmDiag()
    _check3(ctx, load().lbm3_read_tangent_diagnostics(ctx, ctypes.byref(d)),
            "lbm3_read_tangent_diagnostics")
    return {k: getattr(d, k) for k, _ in LbmDiag._fields_}


def lbm3_lattice():
    """(c [19, 3], w [19]) of the library's D3Q19 lattice (host only)."""
    c = (ctypes.c_int32 * 57)()
    w = (ctypes.c_double * 19)()
    load().lbm3_lattice(c, w)
    return np.array(c[:]).reshape(19, 3), np.array(w[:])


class Solver3:
    """One three-dimensional (D3Q19) GPU context; arrays are [nz, ny, nx]."""

    def __init__(self, cfg: dict, precision: str = "fp32", tangent: dict = None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("Solver3 needs a CUDA device (no CPU path)")
        if precision not in ("fp32", "fp64", "tangent"):
            raise ValueError("3-D contexts take fp32, fp64 or tangent")
        load()
        self.cfg = dict(cfg)
        self.shape = (int(cfg["nz"]), int(cfg["ny"]), int(cfg["nx"]))
        self.precision = precision
        self.params = make_params3(cfg, precision, tangent)
        self.ctx = lbm3_create(self.params)

    def close(self):
        if getattr(self, "ctx", None):
            lbm3_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_geometry(self, arrays: dict, on_device: bool = True):
        import torch
        keys = ("phi0", "phi", "T", "fl")
        m = arrays.get("mask")
        if on_device:
            t = {k: torch.as_tensor(np.ascontiguousarray(arrays[k], dtype=np.float64),
                                    device="cuda") for k in keys}
            tm = None if m is None else torch.as_tensor(np.ascontiguousarray(m, dtype=np.uint8),
                                                        device="cuda")
            ptrs = [t[k].data_ptr() for k in keys]
            mp, where = (None if tm is None else tm.data_ptr()), LBM_DEVICE
        else:
            h = {k: np.ascontiguousarray(arrays[k], dtype=np.float64) for k in keys}
            hm = None if m is None else np.ascontiguousarray(m, dtype=np.uint8)
            ptrs = [h[k].ctypes.data for k in keys]
            mp, where = (None if hm is None else hm.ctypes.data), LBM_HOST
        lbm3_set_geometry(self.ctx, ptrs[0], mp, ptrs[1], ptrs[2], ptrs[3], where, _stream())
        if on_device:
            torch.cuda.current_stream().synchronize()
        return self

    def step(self, n: int = 1):
        lbm3_step(self.ctx, n, _stream())
        return self

    @property
    def steps_done(self) -> int:
        return lbm3_step_count(self.ctx)

    def fields(self, names=FIELDS3) -> dict:
        out = {k: np.empty(self.shape, dtype=np.float64) for k in names}
        mask = 0
        ptrs = [None] * len(FIELDS3)
        for k in names:
            i = FIELDS3.index(k)
            mask |= 1 << i
            ptrs[i] = out[k].ctypes.data
        lbm3_read_fields(self.ctx, mask, ptrs, LBM_HOST, _stream())
        return out

    def diagnostics(self) -> dict:
        return lbm3_diagnostics(self.ctx, _stream())

    def tangent_fields(self, names=FIELDS3) -> dict:
        """Derivatives of the fields along the parameter direction (host)."""
        out = {k: np.empty(self.shape, dtype=np.float64) for k in names}
        mask = 0
        ptrs = [None] * len(FIELDS3)
        for k in names:
            i = FIELDS3.index(k)
            mask |= 1 << i
            ptrs[i] = out[k].ctypes.data
        lbm3_read_tangent_fields(self.ctx, mask, ptrs, LBM_HOST, _stream())
        return out

    def tangent_diagnostics(self) -> dict:
        """Derivatives of the sums of the most recent diagnostics() call."""
        return lbm3_read_tangent_diagnostics(self.ctx)

    def save_state(self) -> bytes:
        return lbm3_save_state(self.ctx, _stream())

    def load_state(self, data: bytes):
        lbm3_load_state(self.ctx, data, _stream())
        return self
