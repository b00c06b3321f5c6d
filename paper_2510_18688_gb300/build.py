"""Build the sm_103a shared library ``_lib/liblbm_gb300.so`` with nvcc.

The library is rebuilt whenever the SHA-256 of its sources (every file of
``csrc/``, ``include/lbm.h``) and of the compile command differs from the
stamp written beside it at the last build -- file times are not trusted, so
a library copied in with a newer time than its sources is still rebuilt.
The hash is compiled into the library (``lbm_source_hash``), which ties a
loaded binary to the sources it was built from.

The translation units (host API, FP32, FP64, FP16-storage, tangent and adjoint kernels, the
allocation-free diagnostics, the FMA-rate probe) compile
in parallel and link into one C-ABI library.  Both precisions keep fused
multiply-add contraction: the FP64 step is bound by the FP64 pipe on this
part, and contraction cuts its pipe operations by about a quarter while the
results stay within 1e-10 of the uncontracted oracle.
"""
from __future__ import annotations

import argparse
import concurrent.futures as cf
import hashlib
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_lib")
LIB = os.path.join(OUT_DIR, "liblbm_gb300.so")
STAMP = LIB + ".srchash"
ARCH = "-gencode=arch=compute_103a,code=sm_103a"
UNITS = {
    "lbm_api.cu": [],
    "lbm_f32.cu": [],
    "lbm_f64.cu": [],
    "lbm_f16.cu": [],
    "lbm_tan.cu": [],
    "lbm_adjoint.cu": [],
    "lbm_static.cu": [],
    "lbm_probe.cu": [],
    "lbm3d.cu": [],
}


def nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build liblbm_gb300")


def _sources():
    return sorted(os.path.join(SRC, f) for f in os.listdir(SRC)) + [
        os.path.join(os.path.dirname(HERE), "include", "lbm.h")]


def _flags(verbose: bool = False):
    base = [ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC"]
    base += os.environ.get("LBM_NVCC_EXTRA", "").split()
    if verbose:
        base += ["-Xptxas", "-v"]
    return base


def source_hash() -> str:
    """SHA-256 (first 16 hex digits) of the library's sources and compile
    flags; the file names are hashed with their contents."""
    h = hashlib.sha256()
    for path in _sources():
        h.update(os.path.basename(path).encode() + b"\0")
        with open(path, "rb") as fh:
            h.update(fh.read())
        h.update(b"\0")
    h.update(" ".join(_flags()).encode())
    return h.hexdigest()[:16]


def up_to_date() -> bool:
    """True when the library exists and its stamp holds the current source
    hash (not a comparison of file times)."""
    if not (os.path.exists(LIB) and os.path.exists(STAMP)):
        return False
    with open(STAMP) as fh:
        return fh.read().strip() == source_hash()


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and up_to_date():
        return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    tool = nvcc()
    digest = source_hash()
    base = [tool] + _flags(verbose)

    def compile_one(unit):
        obj = os.path.join(OUT_DIR, unit.replace(".cu", ".o"))
        extra = [f'-DLBM_SOURCE_HASH="{digest}"'] if unit == "lbm_api.cu" else []
        cmd = base + UNITS[unit] + extra + ["-c", os.path.join(SRC, unit), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {unit}:\n{r.stdout}\n{r.stderr}")
        return obj, r.stderr

    with cf.ThreadPoolExecutor(len(UNITS)) as ex:
        results = list(ex.map(compile_one, UNITS))
    if verbose:
        for _, log in results:
            sys.stderr.write(log)
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [tool, ARCH, "-shared", "-o", tmp] + [o for o, _ in results]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    with open(STAMP + f".tmp{os.getpid()}", "w") as fh:
        fh.write(digest + "\n")
    os.replace(STAMP + f".tmp{os.getpid()}", STAMP)
    return LIB


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("--force", action="store_true")
    ap.add_argument("-v", "--verbose", action="store_true")
    args = ap.parse_args()
    print(build(force=args.force, verbose=args.verbose))
