"""Build libpic.so (the C-ABI CUDA library) for sm_103a with nvcc.

Each translation unit is compiled in parallel into ``_build/`` and linked
in-tree as ``paper_2206_14662_gb300/libpic.so`` (static CUDA runtime, so the
library loads without extra search paths).
"""
from __future__ import annotations

import os
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libpic.so")
SOURCES = ["particle_step.cu", "field_solve.cu", "sort.cu", "capi.cu", "field_static.cu",
           "unet.cu", "moments.cu", "spline.cu", "webspline.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I" + INCLUDE, "-I" + CSRC]
# the particle step writes its multiply-adds out explicitly; no automatic
# contraction keeps every particle's rounding sequence the same
PER_FILE = {"particle_step.cu": ["-fmad=false"]}


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.isabs(cand) and os.path.exists(cand) or not os.path.isabs(cand)):
            return cand
    return "nvcc"


def _stale(target: str, deps: list[str]) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile and link libpic.so if any source or header changed."""
    os.makedirs(BUILD, exist_ok=True)
    headers = [os.path.join(INCLUDE, "pic.h"), os.path.join(CSRC, "pic_internal.cuh"),
               os.path.join(CSRC, "unet_kernels.cuh"), os.path.join(CSRC, "unet_tc.cuh"),
               os.path.join(CSRC, "field_common.cuh"),
               os.path.join(CSRC, "fluid.cuh"), os.path.join(CSRC, "dfloat.cuh")]
    nvcc = _nvcc()
    procs, objs = [], []
    for src in SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(BUILD, src.replace(".cu", ".o"))
        objs.append(o)
        if force or _stale(o, [s] + headers):
            cmd = [nvcc, *ARCH, *FLAGS, *PER_FILE.get(src, []), "-c", s, "-o", o + ".tmp"]
            if verbose:
                print(" ".join(cmd), file=sys.stderr)
            procs.append((o, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    failed = []
    for o, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0:
            failed.append(out.decode(errors="replace"))
        else:
            os.replace(o + ".tmp", o)
    if failed:
        raise RuntimeError("nvcc failed:\n" + "\n".join(failed))
    if force or _stale(LIB, objs):
        tmp = LIB + f".tmp{os.getpid()}"
        subprocess.check_call([nvcc, *ARCH, "-shared", "-o", tmp, *objs])
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
