"""ctypes front end of the FP64 CPU oracle of the three-dimensional (D3Q19)
form of the method (``lbm_oracle3d.c``).

TEST INFRASTRUCTURE ONLY: imported by ``tests/`` and by the CPU-baseline leg
of ``bench.py``.  The product path never imports this module.

Arrays are [nz, ny, nx] (x fastest).  The configuration dictionary is the
two-dimensional one with ``nz``, six boundary types and six wall
temperatures (x-low, x-high, y-low, y-high, z-low, z-high) and ``gz``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm_oracle3d.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liblbm_oracle3d.so")
_lock = threading.Lock()
_lib = None

BC_CODES = {"periodic": 0, "dirichlet": 1, "adiabatic": 2}
FIELDS = ("phi", "fs", "fl", "T", "rhoH", "p", "ux", "uy", "uz", "rho", "mu", "w", "mdot")
DIAGS = ("mass", "material_mass", "rhoH", "liquid_volume", "material_volume",
         "frozen_volume", "phi_sum", "kinetic", "nonfinite")
NQ = 19


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


class Oracle3Params(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
        ("lattices", ctypes.c_uint32),
        ("bc", ctypes.c_int32 * 6),
        ("T_wall", ctypes.c_double * 6),
        ("rho_l", ctypes.c_double), ("rho_s", ctypes.c_double), ("rho_g", ctypes.c_double),
        ("mu_l", ctypes.c_double), ("mu_s", ctypes.c_double), ("mu_g", ctypes.c_double),
        ("lambda_l", ctypes.c_double), ("lambda_s", ctypes.c_double), ("lambda_g", ctypes.c_double),
        ("cp_l", ctypes.c_double), ("cp_s", ctypes.c_double), ("cp_g", ctypes.c_double),
        ("rho_ref", ctypes.c_double), ("latent", ctypes.c_double),
        ("sigma", ctypes.c_double), ("eps", ctypes.c_double),
        ("mobility", ctypes.c_double), ("eta", ctypes.c_double),
        ("theta_deg", ctypes.c_double), ("psi_deg", ctypes.c_double),
        ("gx", ctypes.c_double), ("gy", ctypes.c_double), ("gz", ctypes.c_double),
        ("T_cold", ctypes.c_double),
        ("readings", ctypes.c_uint32),
    ]


_SCALARS = ("rho_l", "rho_s", "rho_g", "mu_l", "mu_s", "mu_g", "lambda_l", "lambda_s",
            "lambda_g", "cp_l", "cp_s", "cp_g", "rho_ref", "latent", "sigma", "eps",
            "mobility", "eta", "theta_deg", "psi_deg", "gx", "gy", "gz", "T_cold")


def make_params(cfg: dict) -> Oracle3Params:
    p = Oracle3Params()
    p.nx, p.ny, p.nz = int(cfg["nx"]), int(cfg["ny"]), int(cfg["nz"])
    p.lattices = int(cfg["lattices"])
    for k in range(6):
        p.bc[k] = BC_CODES[cfg["bc"][k]]
        p.T_wall[k] = float(cfg["T_wall"][k])
    for name in _SCALARS:
        setattr(p, name, float(cfg.get(name, 0.0)) if name == "gz" else float(cfg[name]))
    p.readings = int(cfg.get("readings", 0))
    return p


_dp = ctypes.POINTER(ctypes.c_double)
_u8p = ctypes.POINTER(ctypes.c_uint8)
_ip = ctypes.POINTER(ctypes.c_int)


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        L.oracle3_create.restype = ctypes.c_void_p
        L.oracle3_create.argtypes = [ctypes.POINTER(Oracle3Params)]
        L.oracle3_destroy.argtypes = [ctypes.c_void_p]
        L.oracle3_init.argtypes = [ctypes.c_void_p, _dp, _u8p, _dp, _dp, _dp]
        L.oracle3_step.argtypes = [ctypes.c_void_p, ctypes.c_long]
        L.oracle3_fields.argtypes = [ctypes.c_void_p, _dp]
        L.oracle3_diagnostics.argtypes = [ctypes.c_void_p, _dp]
        L.oracle3_get_state.argtypes = [ctypes.c_void_p, _dp, _dp]
        L.oracle3_set_state.argtypes = [ctypes.c_void_p, _dp, _dp]
        L.oracle3_step_count.restype = ctypes.c_int64
        L.oracle3_step_count.argtypes = [ctypes.c_void_p]
        L.oracle3_lattice.argtypes = [_ip, _ip, _ip, _dp, _ip]
        L.oracle3_node_flow.argtypes = [ctypes.c_double, ctypes.c_double, _dp, ctypes.c_double,
                                        _dp, _dp, _dp, ctypes.c_uint32, _dp, _dp]
        L.oracle3_node_phase.argtypes = [ctypes.c_double] * 3 + [_dp, _dp, ctypes.c_double,
                                                                 _dp, _dp]
        L.oracle3_node_heat.argtypes = [ctypes.c_double] * 4 + [_dp, ctypes.c_double, _dp, _dp]
        _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(_dp)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


class Oracle3:
    """One three-dimensional oracle simulation (arrays are [nz, ny, nx])."""

    def __init__(self, cfg: dict):
        self.cfg = dict(cfg)
        self.params = make_params(cfg)
        self.shape = (self.params.nz, self.params.ny, self.params.nx)
        self.N = int(np.prod(self.shape))
        self._h = lib().oracle3_create(ctypes.byref(self.params))
        if not self._h:
            raise ValueError("oracle rejected the parameters")

    def close(self):
        if self._h:
            lib().oracle3_destroy(self._h)
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
        lib().oracle3_init(self._h, _ptr(phi0), m.ctypes.data_as(_u8p) if m is not None else None,
                           _ptr(phi), _ptr(T), _ptr(fl))
        self._keep = (phi0, phi, T, fl, m)
        return self

    def step(self, n: int = 1):
        lib().oracle3_step(self._h, int(n))
        return self

    @property
    def steps_done(self) -> int:
        return int(lib().oracle3_step_count(self._h))

    def fields(self) -> dict:
        out = np.empty((len(FIELDS), self.N), dtype=np.float64)
        lib().oracle3_fields(self._h, _ptr(out))
        return {k: out[i].reshape(self.shape).copy() for i, k in enumerate(FIELDS)}

    def diagnostics(self) -> dict:
        d = np.empty(len(DIAGS), dtype=np.float64)
        lib().oracle3_diagnostics(self._h, _ptr(d))
        return {k: float(d[i]) for i, k in enumerate(DIAGS)}

    def state(self):
        pops = np.empty((3, NQ, self.N), dtype=np.float64)
        lags = np.empty((7, self.N), dtype=np.float64)
        lib().oracle3_get_state(self._h, _ptr(pops), _ptr(lags))
        return pops, lags

    def set_state(self, pops, lags):
        pops, lags = _f64(pops), _f64(lags)
        assert pops.size == 3 * NQ * self.N and lags.size == 7 * self.N
        lib().oracle3_set_state(self._h, _ptr(pops), _ptr(lags))


def from_workload(wl) -> Oracle3:
    cfg, arr = wl
    return Oracle3(cfg).init(arr["phi0"], arr["phi"], arr["T"], arr["fl"], arr.get("mask"))


def lattice():
    cx, cy, cz, opp = ((ctypes.c_int * NQ)() for _ in range(4))
    w = (ctypes.c_double * NQ)()
    lib().oracle3_lattice(cx, cy, cz, w, opp)
    return (np.array(cx[:]), np.array(cy[:]), np.array(cz[:]), np.array(w[:]), np.array(opp[:]))


# --- single-node entry points, used by the moment pins -----------------------

def node_flow(pr, rho, u, S, F, fp, Ft, readings=0):
    feq, Fi = np.empty(NQ), np.empty(NQ)
    u, F, fp, Ft = (_f64(v) for v in (u, F, fp, Ft))
    lib().oracle3_node_flow(pr, rho, _ptr(u), S, _ptr(F), _ptr(fp), _ptr(Ft), readings,
                            _ptr(feq), _ptr(Fi))
    return feq, Fi


def node_phase(phi, muphi, eta, phu, dphu, mdot):
    geq, Gi = np.empty(NQ), np.empty(NQ)
    phu, dphu = _f64(phu), _f64(dphu)
    lib().oracle3_node_phase(phi, muphi, eta, _ptr(phu), _ptr(dphu), mdot, _ptr(geq), _ptr(Gi))
    return geq, Gi


def node_heat(rhoH, C, T, rr, u, mdot):
    heq, Hi = np.empty(NQ), np.empty(NQ)
    u = _f64(u)
    lib().oracle3_node_heat(rhoH, C, T, rr, _ptr(u), mdot, _ptr(heq), _ptr(Hi))
    return heq, Hi
