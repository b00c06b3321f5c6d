"""The allocation-free diagnostics entry point, called through the C ABI.

lbm_diagnostics_noalloc serves callers that may not allocate device memory
themselves (their framework's allocator or memory pool owns it, or an
allocation's implicit synchronisation is not acceptable in their loop).  It
reduces a state the caller already holds, using a static device array as
scratch.  Here the state of a context is copied into caller-owned device
buffers and the entry point must reproduce the context's own diagnostics,
on two calls in a row.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

from paper_2510_18688_gb300 import workloads as W

pytestmark = pytest.mark.gpu

HEADER_BYTES = 32  # magic, version, nx, ny, precision, lattices, step
NAMES = ("mass", "material_mass", "rhoH", "liquid_volume", "material_volume",
         "frozen_volume", "phi_sum", "kinetic", "nonfinite")


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_18688_gb300 import build, lbm
    build.build()
    lbm.load()
    return torch, lbm


def _planes(a, nx, ny, pitch, plane, dtype):
    """One [ny][nx] array laid out as a padded plane of the library."""
    buf = np.zeros(plane, dtype=dtype)
    buf[:pitch * ny].reshape(ny, pitch)[:, :nx] = a
    return buf


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_noalloc_matches_context_diagnostics(env, prec):
    torch, lbm = env
    cfg, arr = W.random_state(70, 45, seed=12)
    nx, ny = cfg["nx"], cfg["ny"]
    s = lbm.Solver(cfg, precision=prec).set_geometry(arr).step(25)
    expected = s.diagnostics()
    blob = s.save()
    esize = 4 if prec == "fp32" else 8
    dtype = np.float32 if prec == "fp32" else np.float64
    pitch = (nx + 31) // 32 * 32
    plane = (pitch * ny + 63) // 64 * 64
    body = np.frombuffer(blob, dtype=np.uint8, offset=HEADER_BYTES)
    pops = np.frombuffer(body[:27 * plane * esize].tobytes(), dtype=dtype)
    nlag = 7 if prec == "fp32" else 6  # FP32 states carry the lagged temperature too
    lags = np.frombuffer(body[27 * plane * esize:(27 + nlag) * plane * esize].tobytes(),
                         dtype=dtype)
    phi0 = _planes(arr["phi0"], nx, ny, pitch, plane, dtype)
    mask = _planes(arr["mask"], nx, ny, pitch, plane, np.uint8)
    d_pops = torch.from_numpy(pops.copy()).cuda()
    d_lags = torch.from_numpy(lags.copy()).cuda()
    d_phi0 = torch.from_numpy(phi0).cuda()
    d_mask = torch.from_numpy(mask).cuda()
    params = lbm.make_params(cfg, prec)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    n = nx * ny
    tol = 1e-12 if prec == "fp64" else 1e-5
    for call in range(2):
        out = torch.full((10,), -1.0, dtype=torch.float64, device="cuda")
        st = lbm.lbm_diagnostics_noalloc(params, d_pops.data_ptr(), d_lags.data_ptr(),
                                         d_phi0.data_ptr(), d_mask.data_ptr(), out.data_ptr(),
                                         stream)
        assert st == 0, (call, lbm.lbm_status_string(st))
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        for k, name in enumerate(NAMES):
            v = expected[name]
            assert abs(got[k] - v) <= tol * (abs(v) + n), (call, name, got[k], v)
        assert got[9] == 0.0
    s.close()


def test_noalloc_rejects_grids_beyond_its_scratch(env):
    torch, lbm = env
    cfg = W.base_params(2048, 2048)  # 64 x 256 tiles, above the 4096-tile limit
    params = lbm.make_params(cfg, "fp32")
    dummy = torch.zeros(16, dtype=torch.float64, device="cuda")
    p = dummy.data_ptr()
    st = lbm.lbm_diagnostics_noalloc(params, p, p, p, None, p, None)
    assert st == -6  # LBM_ERR_UNSUPPORTED
    assert lbm.lbm_diagnostics_noalloc(params, None, p, p, None, p, None) == -1
