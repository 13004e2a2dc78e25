"""Build libtc.so in-tree with nvcc for sm_103a (GB300).

Each .cu file compiles in parallel to an object file under ``_build/``; the
objects link into ``paper_1908_00587_gb300/libtc.so``.  No cmake, one
-gencode, a minute or less on either host architecture.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(ROOT, "_build")
LIB = os.path.join(PKG, "libtc.so")
# the same sources with -DTC_DEBUG: index checks that record, never trap
LIB_DEBUG = os.path.join(PKG, "libtc_debug.so")

SOURCES = ["tc_host.cu", "nonlinear.cu", "linear.cu", "diag.cu", "ensemble.cu", "restart.cu",
           "theta_tc.cu", "zinv_tc.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2",
         "--expt-relaxed-constexpr", "-I", INCLUDE, "-I", CSRC]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _newer(target: str, deps) -> bool:
    if not os.path.exists(target):
        return False
    t = os.path.getmtime(target)
    return all(os.path.getmtime(d) <= t for d in deps)


def build(verbose: bool = False, force: bool = False, extra: tuple = (),
          debug: bool = True) -> str:
    """Compile libtc.so and (debug=True) libtc_debug.so; returns libtc.so's path."""
    os.makedirs(BUILD, exist_ok=True)
    headers = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    headers.append(os.path.join(INCLUDE, "tc.h"))
    cc = nvcc()
    variants = [("", LIB, ())] + ([("_debug", LIB_DEBUG, ("-DTC_DEBUG",))] if debug else [])

    def compile_one(job):
        src, suffix, defs = job
        s = os.path.join(CSRC, src)
        o = os.path.join(BUILD, src.replace(".cu", suffix + ".o"))
        if not force and _newer(o, [s] + headers):
            return o
        cmd = [cc, "-c", s, "-o", o] + ARCH + FLAGS + list(defs) + list(extra)
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{res.stdout}\n{res.stderr}")
        if verbose and res.stderr:
            print(res.stderr, file=sys.stderr)
        return o

    jobs = [(src, suffix, defs) for suffix, _, defs in variants for src in SOURCES]
    with ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
        objs = list(ex.map(compile_one, jobs))
    for k, (suffix, lib, _) in enumerate(variants):
        vobjs = objs[k * len(SOURCES):(k + 1) * len(SOURCES)]
        if force or not _newer(lib, vobjs):
            cmd = [cc, "-shared", "-o", lib] + vobjs + ARCH
            res = subprocess.run(cmd, capture_output=True, text=True)
            if res.returncode != 0:
                raise RuntimeError(f"link failed:\n{res.stdout}\n{res.stderr}")
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv, force="-f" in sys.argv))
