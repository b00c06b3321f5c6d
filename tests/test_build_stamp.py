"""The build is tied to its sources by a hash, not by file times (CPU)."""
import os

from paper_2510_18688_gb300 import build as B


def test_stale_library_with_newer_mtime_is_rebuilt(tmp_path, monkeypatch):
    """A library whose stamp names other sources is out of date even when
    its file time is newer than every source (e.g. a binary copied in)."""
    lib = tmp_path / "liblbm_gb300.so"
    stamp = tmp_path / "liblbm_gb300.so.srchash"
    lib.write_bytes(b"not a library")
    future = max(os.path.getmtime(p) for p in B._sources()) + 3600
    os.utime(lib, (future, future))
    monkeypatch.setattr(B, "LIB", str(lib))
    monkeypatch.setattr(B, "STAMP", str(stamp))
    assert not B.up_to_date()                 # no stamp
    stamp.write_text("0123456789abcdef\n")
    assert not B.up_to_date()                 # stamp of other sources
    stamp.write_text(B.source_hash() + "\n")
    assert B.up_to_date()


def test_hash_covers_every_source_and_the_flags(monkeypatch):
    h0 = B.source_hash()
    monkeypatch.setenv("LBM_NVCC_EXTRA", "-DLBM_MIN_BLOCKS_F32=3")
    assert B.source_hash() != h0
    names = {os.path.basename(p) for p in B._sources()}
    assert {"lbm_step.cuh", "lbm_kernels.cuh", "lbm_api.cu", "lbm.h"} <= names


def test_loaded_library_reports_its_source_hash():
    from paper_2510_18688_gb300 import lbm
    B.build()
    lib = lbm.load()
    assert lib.lbm_source_hash().decode() == B.source_hash()
