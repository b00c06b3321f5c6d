"""Build the sm_103a shared library ``_lib/liblbm_gb300.so`` with nvcc.

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
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_lib")
LIB = os.path.join(OUT_DIR, "liblbm_gb300.so")
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
    return [os.path.join(SRC, f) for f in os.listdir(SRC)] + [
        os.path.join(os.path.dirname(HERE), "include", "lbm.h")]


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(s) <= t for s in _sources())


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and up_to_date():
        return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    tool = nvcc()
    base = [tool, ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC"]
    base += os.environ.get("LBM_NVCC_EXTRA", "").split()
    if verbose:
        base += ["-Xptxas", "-v"]

    def compile_one(unit):
        obj = os.path.join(OUT_DIR, unit.replace(".cu", ".o"))
        cmd = base + UNITS[unit] + ["-c", os.path.join(SRC, unit), "-o", obj]
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
    return LIB


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("--force", action="store_true")
    ap.add_argument("-v", "--verbose", action="store_true")
    args = ap.parse_args()
    print(build(force=args.force, verbose=args.verbose))
