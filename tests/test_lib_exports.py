"""CPU checks of the C-ABI library: it builds for sm_103a, loads, and exports
every entry point that include/lbm.h declares (no compute without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2510_18688_gb300 import build, lbm
    build.build()
    return lbm.load()


def _declared():
    src = open(os.path.join(ROOT, "include", "lbm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lbm3?_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("lbm_create", "lbm_set_geometry", "lbm_step", "lbm_read_fields",
              "lbm_read_diagnostics", "lbm_destroy"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    for n in _declared():
        assert hasattr(lib, n), n


def test_binding_exports_match_header():
    from paper_2510_18688_gb300 import lbm
    assert sorted(lbm.EXPORTS) == _declared()
    for n in lbm.EXPORTS:
        assert callable(getattr(lbm, n))


def test_create_rejects_invalid_parameters_without_gpu(lib):
    """Validation runs before any device call, so it is testable on CPU."""
    from paper_2510_18688_gb300 import lbm, workloads as W
    cfg = W.base_params(16, 16)
    bad = [dict(nx=1), dict(mu_l=0.0), dict(rho_g=-1.0), dict(lattices=0), dict(lattices=9),
           dict(bc=("periodic", "dirichlet", "periodic", "periodic")), dict(mobility=0.0)]
    for b in bad:
        c = dict(cfg, **b)
        p = lbm.make_params(c)
        h = ctypes.c_void_p()
        st = lib.lbm_create(ctypes.byref(p), ctypes.byref(h))
        assert st in (-1, -2), (b, st)
        assert not h.value
    assert lib.lbm_status_string(-5).decode() == "non-finite state"


def test_null_context_is_an_error_not_a_crash(lib):
    from paper_2510_18688_gb300 import lbm
    assert lib.lbm_step(None, 1, None) == -1
    assert lib.lbm_read_diagnostics(None, None) == -1
    assert lib.lbm_step_count(None) == -1
    lib.lbm_destroy(None)
    assert lbm.LBM_OK == 0


def test_3d_lattice_is_the_printed_d3q19(lib):
    """The kernels' D3Q19 table (a host copy of the same constexpr
    functions) against the velocity matrix and weights printed in Sec. 3.1."""
    from fractions import Fraction
    from paper_2510_18688_gb300 import lbm
    c, w = lbm.lbm3_lattice()
    rows = [l.split() for l in open(os.path.join(ROOT, "tests", "golden", "d3q19_lattice.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 19
    for r in rows:
        i = int(r[0])
        assert tuple(c[i]) == (int(r[1]), int(r[2]), int(r[3]))
        assert w[i] == float(Fraction(r[4]))


def test_3d_create_rejects_invalid_parameters_without_gpu(lib):
    from paper_2510_18688_gb300 import lbm, workloads as W
    cfg, _ = W.random_state3(8, 6, 4, seed=2)
    bad = [dict(nz=1), dict(nx=1), dict(mu_l=0.0),
           dict(bc=("periodic",) * 4 + ("periodic", "dirichlet")),
           dict(bc=("periodic",) * 4 + ("periodic", "sticky"))]
    for b in bad:
        c = dict(cfg, **b)
        try:
            p = lbm.make_params3(c)
        except KeyError:
            continue  # an unknown boundary name never reaches the library
        h = ctypes.c_void_p()
        st = lib.lbm3_create(ctypes.byref(p), ctypes.byref(h))
        assert st in (-1, -2), (b, st)
        assert not h.value
    p = lbm.make_params3(cfg, "fp32")
    p.base.precision = 2  # FP16 storage is not offered in 3-D
    h = ctypes.c_void_p()
    assert lib.lbm3_create(ctypes.byref(p), ctypes.byref(h)) == -6
    assert lib.lbm3_step(None, 1, None) == -1
    assert lib.lbm3_step_count(None) == -1
    lib.lbm3_destroy(None)


def test_3d_create_rejects_grids_beyond_31_bit_offsets(lib):
    """Node offsets within one plane are 32-bit (planes of up to 2^31
    elements; the population planes themselves are addressed with 64-bit
    offsets once they pass 2^31 together); the check runs before any device
    allocation."""
    from paper_2510_18688_gb300 import lbm, workloads as W
    cfg, _ = W.random_state3(8, 6, 4, seed=2)
    p = lbm.make_params3(dict(cfg, nx=2048, ny=1024, nz=1025))  # 2.15 G nodes per plane
    h = ctypes.c_void_p()
    assert lib.lbm3_create(ctypes.byref(p), ctypes.byref(h)) == -1
    assert not h.value


def test_3d_params_marshalling():
    """make_params3 maps a 3-D workload dict onto lbm3_params: the x and y
    faces into the base parameters, the z faces, g_z and the tangent rates of
    all six walls into the 3-D fields."""
    from paper_2510_18688_gb300 import lbm, workloads as W
    cfg, _ = W.random_state3(12, 8, 6, seed=3)
    tw = [0.1, 0.2, 0.3, 0.4, 0.5, 0.6]
    p = lbm.make_params3(cfg, "tangent", {"T_wall": tw, "theta_deg": 1.0})
    assert (p.base.nx, p.base.ny, p.nz) == (12, 8, 6)
    assert p.base.precision == lbm.PRECISION["tangent"]
    assert [p.base.bc[k] for k in range(4)] == [lbm.BC[b] for b in cfg["bc"][:4]]
    assert [p.bc_z[k] for k in range(2)] == [lbm.BC[b] for b in cfg["bc"][4:]]
    assert list(p.base.T_wall) == list(cfg["T_wall"][:4])
    assert list(p.T_wall_z) == list(cfg["T_wall"][4:])
    assert p.gz == cfg["gz"]
    assert list(p.base.tan_T_wall) == tw[:4] and list(p.tan_T_wall_z) == tw[4:]
    assert p.base.tan_theta_deg == 1.0 and p.base.tan_latent == 0.0
