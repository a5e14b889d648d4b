"""Compile the CUDA library ``libeb.so`` in-tree for sm_103a (GB300).

Each translation unit is compiled by its own nvcc process, in parallel, then
linked into one shared object next to this file.  The set-up units (geometry
and redistribution tables) are compiled without FMA contraction.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OBJ = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libeb.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
UNITS = ["eb_api.cu", "eb_geom.cu", "eb_wsrd_setup.cu", "eb_step.cu", "eb_fast.cu", "eb_scan.cu", "eb_ensemble.cu", "eb_project.cu", "eb_unet.cu", "eb_peak.cu", "eb_sources.cu", "eb_amr.cu"]
# Units compiled without contraction of a * b + c: the set-up (bit-exact
# geometry), and the step units, whose device functions run both in their
# own kernels and inlined into the persistent ensemble kernel and must round
# the same in both (their heavy arithmetic uses explicit FMA intrinsics).
NO_FMA = {"eb_geom.cu", "eb_wsrd_setup.cu", "eb_step.cu", "eb_fast.cu"}


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _sources_mtime() -> float:
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(HERE, "..", "include", "eb.h")]
    return max(os.path.getmtime(f) for f in files)


def build(force: bool = False, verbose: bool = False, extra=()) -> str:
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= _sources_mtime():
        return LIB
    os.makedirs(OBJ, exist_ok=True)
    cc = nvcc()
    base = [cc, "-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xptxas", "-v" if verbose else "-O3",
            *ARCH, *extra]

    def one(u):
        obj = os.path.join(OBJ, u.replace(".cu", ".o"))
        cmd = base + (["-fmad=false"] if u in NO_FMA else []) + ["-c", os.path.join(CSRC, u), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {u}:\n{r.stderr}")
        return obj, r.stderr

    with ThreadPoolExecutor(max_workers=len(UNITS)) as ex:
        results = list(ex.map(one, UNITS))
    if verbose:
        for _, err in results:
            sys.stderr.write(err)
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [cc, "-shared", *ARCH, "-o", tmp] + [o for o, _ in results] + ["-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
