"""ctypes front end of the FP64 CPU oracle (``lbm_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by ``__graft_entry__.smoke``
and by the CPU-baseline leg of ``bench.py``.  The product path (the CUDA
library and its Python binding) never imports this module.

The oracle is a literal restatement of the paper's LB method (arXiv
2510.18688, Secs. 2-3) in double precision; see the header of
``lbm_oracle.c`` for the stage order and the readings it follows.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liblbm_oracle.so")
_lock = threading.Lock()
_lib = None

LAT_FLOW, LAT_PHASE, LAT_HEAT = 1, 2, 4
BC_CODES = {"periodic": 0, "dirichlet": 1, "adiabatic": 2}
FIELDS = ("phi", "fs", "fl", "T", "rhoH", "p", "ux", "uy", "rho", "mu", "w", "mdot")
DIAGS = ("mass", "material_mass", "rhoH", "liquid_volume", "material_volume",
         "frozen_volume", "phi_sum", "kinetic", "nonfinite")


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (FP contraction off, OpenMP over rows)."""
    with _lock:
        os.makedirs(_BUILD, exist_ok=True)
        if (not force and os.path.exists(_LIB)
                and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
            return _LIB
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-ffp-contract=off",
               "-fno-fast-math", "-fopenmp", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
        return _LIB


class OracleParams(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
        ("lattices", ctypes.c_uint32),
        ("bc", ctypes.c_int32 * 4),
        ("T_wall", ctypes.c_double * 4),
        ("rho_l", ctypes.c_double), ("rho_s", ctypes.c_double), ("rho_g", ctypes.c_double),
        ("mu_l", ctypes.c_double), ("mu_s", ctypes.c_double), ("mu_g", ctypes.c_double),
        ("lambda_l", ctypes.c_double), ("lambda_s", ctypes.c_double), ("lambda_g", ctypes.c_double),
        ("cp_l", ctypes.c_double), ("cp_s", ctypes.c_double), ("cp_g", ctypes.c_double),
        ("rho_ref", ctypes.c_double), ("latent", ctypes.c_double),
        ("sigma", ctypes.c_double), ("eps", ctypes.c_double),
        ("mobility", ctypes.c_double), ("eta", ctypes.c_double),
        ("theta_deg", ctypes.c_double), ("psi_deg", ctypes.c_double),
        ("gx", ctypes.c_double), ("gy", ctypes.c_double),
        ("T_cold", ctypes.c_double),
        ("readings", ctypes.c_uint32),
    ]


_SCALARS = ("rho_l", "rho_s", "rho_g", "mu_l", "mu_s", "mu_g", "lambda_l", "lambda_s",
            "lambda_g", "cp_l", "cp_s", "cp_g", "rho_ref", "latent", "sigma", "eps",
            "mobility", "eta", "theta_deg", "psi_deg", "gx", "gy", "T_cold")


def make_params(cfg: dict) -> OracleParams:
    p = OracleParams()
    p.nx, p.ny = int(cfg["nx"]), int(cfg["ny"])
    p.lattices = int(cfg["lattices"])
    for k in range(4):
        p.bc[k] = BC_CODES[cfg["bc"][k]]
        p.T_wall[k] = float(cfg["T_wall"][k])
    for name in _SCALARS:
        setattr(p, name, float(cfg[name]))
    p.readings = int(cfg.get("readings", 0))
    return p


_dp = ctypes.POINTER(ctypes.c_double)
_u8p = ctypes.POINTER(ctypes.c_uint8)


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        L.oracle_create.restype = ctypes.c_void_p
        L.oracle_create.argtypes = [ctypes.POINTER(OracleParams)]
        L.oracle_destroy.argtypes = [ctypes.c_void_p]
        L.oracle_init.argtypes = [ctypes.c_void_p, _dp, _u8p, _dp, _dp, _dp]
        L.oracle_step.argtypes = [ctypes.c_void_p, ctypes.c_long]
        L.oracle_fields.argtypes = [ctypes.c_void_p, _dp]
        L.oracle_diagnostics.argtypes = [ctypes.c_void_p, _dp]
        L.oracle_get_state.argtypes = [ctypes.c_void_p, _dp, _dp]
        L.oracle_set_state.argtypes = [ctypes.c_void_p, _dp, _dp]
        L.oracle_step_count.restype = ctypes.c_int64
        L.oracle_step_count.argtypes = [ctypes.c_void_p]
        L.oracle_set_threads.restype = ctypes.c_int
        L.oracle_set_threads.argtypes = [ctypes.c_int]
        L.oracle_lattice.argtypes = [ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                     _dp, ctypes.POINTER(ctypes.c_int)]
        L.oracle_node_flow.argtypes = [ctypes.c_double] * 11 + [ctypes.c_uint32, _dp, _dp]
        L.oracle_node_phase.argtypes = [ctypes.c_double] * 8 + [_dp, _dp]
        L.oracle_node_heat.argtypes = [ctypes.c_double] * 7 + [_dp, _dp]
        L.oracle_node_trt.argtypes = [_dp, _dp, _dp, ctypes.c_double, ctypes.c_double, _dp]
        L.oracle_invert.argtypes = [ctypes.POINTER(OracleParams), _dp, _dp, _dp, ctypes.c_long,
                                    _dp, _dp]
        L.oracle_chemical_potential.argtypes = [ctypes.POINTER(OracleParams), _dp, _dp, _dp, _dp]
        _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(_dp)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


class Oracle:
    """One oracle simulation on an ``nx`` x ``ny`` grid (arrays are [ny, nx])."""

    def __init__(self, cfg: dict):
        self.cfg = dict(cfg)
        self.params = make_params(cfg)
        self.nx, self.ny = self.params.nx, self.params.ny
        self.N = self.nx * self.ny
        self._h = lib().oracle_create(ctypes.byref(self.params))
        if not self._h:
            raise ValueError("oracle rejected the parameters")

    def close(self):
        if self._h:
            lib().oracle_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def init(self, phi0, phi, T, fl, mask=None):
        phi0, phi, T, fl = (_f64(a).reshape(-1) for a in (phi0, phi, T, fl))
        for a in (phi0, phi, T, fl):
            assert a.size == self.N
        m = None
        if mask is not None:
            m = np.ascontiguousarray(mask, dtype=np.uint8).reshape(-1)
            assert m.size == self.N
        lib().oracle_init(self._h, _ptr(phi0),
                          m.ctypes.data_as(_u8p) if m is not None else None,
                          _ptr(phi), _ptr(T), _ptr(fl))
        self._keep = (phi0, phi, T, fl, m)
        return self

    def step(self, n: int = 1):
        lib().oracle_step(self._h, int(n))
        return self

    @property
    def steps_done(self) -> int:
        return int(lib().oracle_step_count(self._h))

    def fields(self) -> dict:
        out = np.empty((len(FIELDS), self.N), dtype=np.float64)
        lib().oracle_fields(self._h, _ptr(out))
        return {k: out[i].reshape(self.ny, self.nx).copy() for i, k in enumerate(FIELDS)}

    def diagnostics(self) -> dict:
        d = np.empty(len(DIAGS), dtype=np.float64)
        lib().oracle_diagnostics(self._h, _ptr(d))
        return {k: float(d[i]) for i, k in enumerate(DIAGS)}

    def state(self):
        pops = np.empty((3, 9, self.N), dtype=np.float64)
        lags = np.empty((6, self.N), dtype=np.float64)
        lib().oracle_get_state(self._h, _ptr(pops), _ptr(lags))
        return pops, lags

    def set_state(self, pops, lags):
        pops, lags = _f64(pops), _f64(lags)
        assert pops.size == 27 * self.N and lags.size == 6 * self.N
        lib().oracle_set_state(self._h, _ptr(pops), _ptr(lags))


def from_workload(wl) -> Oracle:
    """Build and initialise an oracle from a workload (cfg, arrays)."""
    cfg, arr = wl
    return Oracle(cfg).init(arr["phi0"], arr["phi"], arr["T"], arr["fl"], arr.get("mask"))


def set_threads(n: int) -> int:
    """Set the oracle's OpenMP thread count (0 queries); returns the count."""
    return int(lib().oracle_set_threads(int(n)))


# --- single-node entry points, used by the moment pins -----------------------

def lattice():
    cx = (ctypes.c_int * 9)()
    cy = (ctypes.c_int * 9)()
    w = (ctypes.c_double * 9)()
    opp = (ctypes.c_int * 9)()
    lib().oracle_lattice(cx, cy, w, opp)
    return (np.array(cx[:]), np.array(cy[:]), np.array(w[:]), np.array(opp[:]))


def node_flow(pr, rho, ux, uy, S, Fx, Fy, fpx, fpy, Ftx, Fty, readings=0):
    feq = np.empty(9)
    Fi = np.empty(9)
    lib().oracle_node_flow(pr, rho, ux, uy, S, Fx, Fy, fpx, fpy, Ftx, Fty, readings,
                           _ptr(feq), _ptr(Fi))
    return feq, Fi


def node_phase(phi, muphi, eta, phux, phuy, dphux, dphuy, mdot):
    geq = np.empty(9)
    Gi = np.empty(9)
    lib().oracle_node_phase(phi, muphi, eta, phux, phuy, dphux, dphuy, mdot, _ptr(geq), _ptr(Gi))
    return geq, Gi


def node_heat(rhoH, C, T, rr, ux, uy, mdot):
    heq = np.empty(9)
    Hi = np.empty(9)
    lib().oracle_node_heat(rhoH, C, T, rr, ux, uy, mdot, _ptr(heq), _ptr(Hi))
    return heq, Hi


def node_trt(h, heq, Hi, taua, taus):
    out = np.empty(9)
    h, heq, Hi = _f64(h), _f64(heq), _f64(Hi)
    lib().oracle_node_trt(_ptr(h), _ptr(heq), _ptr(Hi), taua, taus, _ptr(out))
    return out


def invert(cfg: dict, rhoH, w, phi0):
    p = make_params(cfg)
    rhoH, w, phi0 = _f64(rhoH).ravel(), _f64(w).ravel(), _f64(phi0).ravel()
    T = np.empty_like(rhoH)
    fl = np.empty_like(rhoH)
    lib().oracle_invert(ctypes.byref(p), _ptr(rhoH), _ptr(w), _ptr(phi0), rhoH.size,
                        _ptr(T), _ptr(fl))
    return T, fl


def chemical_potential(cfg: dict, phi, phi0, fs):
    p = make_params(cfg)
    phi, phi0, fs = _f64(phi), _f64(phi0), _f64(fs)
    out = np.empty_like(phi)
    lib().oracle_chemical_potential(ctypes.byref(p), _ptr(phi), _ptr(phi0), _ptr(fs), _ptr(out))
    return out


# --- interface observables -----------------------------------------------------

def crossings(phi, w, fl, axis: int, index: int):
    """Interface positions along one grid line, as node coordinates.

    Returns (x_phi, x_ice): the largest coordinate at which phi crosses 0
    (the gas-liquid interface: the liquid height of the Stefan problem of
    Sec. 4.2, the droplet tip height of Secs. 4.3-4.4 on the droplet axis),
    and the largest at which the frozen material fraction s = w (1 - fl)
    crosses 1/2 (the ice front).  Between neighbouring nodes k and k+1 with
    values a and b, a crossing happens when exactly one of a, b is <= 0, at
    k + a / (a - b) (linear interpolation).  NaN where there is none.
    axis 0: along x on row y = index; axis 1: along y on column x = index.
    The line does not wrap across a periodic edge.
    """
    phi, w, fl = np.asarray(phi), np.asarray(w), np.asarray(fl)
    if axis == 0:
        p, s = phi[index, :], w[index, :] * (1.0 - fl[index, :]) - 0.5
    else:
        p, s = phi[:, index], w[:, index] * (1.0 - fl[:, index]) - 0.5
    out = []
    for v in (p, s):
        best = float("nan")
        for k in range(len(v) - 1):
            a, b = float(v[k]), float(v[k + 1])
            if (a <= 0.0) != (b <= 0.0):
                best = k + a / (a - b)
        out.append(best)
    return tuple(out)
