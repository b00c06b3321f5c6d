"""Failure paths without a GPU fault (host-side fault injection): every
device or pinned allocation of lbm_create is made to fail in turn; each
attempt must return LBM_ERR_OOM, hand back no context, free what it had
allocated, and leave the library usable."""
import ctypes

import numpy as np
import pytest

from paper_2510_18688_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def test_every_allocation_failure_of_lbm_create_is_clean():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_18688_gb300 import build, lbm
    build.build()
    L = lbm.load()
    cfg, arr = W.random_state(64, 48, seed=2)
    p = lbm.make_params(cfg, "fp32")
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    failures = 0
    for k in range(32):
        lbm.lbm_debug_fail_allocation(k)
        h = ctypes.c_void_p()
        st = L.lbm_create(ctypes.byref(p), ctypes.byref(h))
        if st == 0:
            # k is past the last allocation: the create succeeded
            lbm.lbm_debug_fail_allocation(-1)
            L.lbm_destroy(h)
            break
        assert st == -4, (k, st)
        assert not h.value
        failures += 1
    lbm.lbm_debug_fail_allocation(-1)
    assert failures >= 8  # populations, lags, phi0, scratch, mask, diagnostics
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    assert abs(free1 - free0) < 64 << 20, (free0, free1)
    s = lbm.Solver(cfg, precision="fp32").set_geometry(arr).step(10)
    assert s.diagnostics()["nonfinite"] == 0
    s.close()


@pytest.mark.parametrize("prec", ["fp32", "fp16s"])
@pytest.mark.parametrize("tile", ["1:0", "2:2"])
def test_tile_wait_timeout_is_reported(prec, tile, monkeypatch):
    """The float step's tile kernel waits for its TMA copies with a bound of
    about a second.  The test hook makes every such wait run out (the
    kernel expects 16 bytes more than its copies deliver; nothing is left in
    flight, no device fault): the next read reports LBM_ERR_TIMEOUT, and the
    context steps correctly again once the geometry is set anew."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_18688_gb300 import build, lbm
    build.build()
    lbm.load()
    cfg, arr = W.random_state(70, 45, seed=4)
    monkeypatch.setenv("LBM_TILE", tile)  # the tile kernel in this configuration
    s = lbm.Solver(cfg, precision=prec).set_geometry(arr)
    lbm.lbm_debug_tile_timeout(True)
    try:
        s.step(1)
        with pytest.raises(lbm.LbmError) as e:
            s.fields()
        assert e.value.status == -7  # LBM_ERR_TIMEOUT
    finally:
        lbm.lbm_debug_tile_timeout(False)
    s.set_geometry(arr).step(5)
    ref = lbm.Solver(cfg, precision=prec).set_geometry(arr).step(5)
    a, b = s.fields(), ref.fields()
    for k in a:
        assert np.array_equal(a[k], b[k]), k
    s.close()
    ref.close()


def test_batched_tile_wait_timeout_is_reported():
    """The batched TMA-staged kernel (FP32 batches) waits for each tile's
    copies with the same bound; with the test hook every wait runs out (no
    fault, nothing left in flight), each context of the batch reports
    LBM_ERR_TIMEOUT on its next read, and the batch steps correctly again
    once the geometry is set anew."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_18688_gb300 import build, lbm
    build.build()
    lbm.load()
    wls = [W.random_state(70, 45, seed=5), W.random_state(41, 23, seed=6)]
    ss = [lbm.Solver(c, precision="fp32").set_geometry(a) for c, a in wls]
    b = lbm.Batch(ss)
    lbm.lbm_debug_tile_timeout(True)
    try:
        b.step(1)
        for s in ss:
            with pytest.raises(lbm.LbmError) as e:
                s.fields()
            assert e.value.status == -7  # LBM_ERR_TIMEOUT
    finally:
        lbm.lbm_debug_tile_timeout(False)
    for s, (c, a) in zip(ss, wls):
        s.set_geometry(a)
    b.step(5)
    for s, (c, a) in zip(ss, wls):
        ref = lbm.Solver(c, precision="fp32").set_geometry(a)
        lbm.Batch([ref]).step(5)
        x, y = s.fields(), ref.fields()
        for k in x:
            assert np.array_equal(x[k], y[k]), k
        ref.close()
    b.close()
    for s in ss:
        s.close()
