"""Build the CUDA library libcal.so in-tree for sm_103a (nvcc + g++, no cmake).

Translation units are compiled in parallel and linked with the static CUDA
runtime, so the library has no dependency beyond the driver. Run as
``python -m paper_2008_04772_gb300.build`` or through ``__graft_entry__.build()``.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = os.path.join(HERE, "csrc")
INC = os.path.join(ROOT, "include")
OUT_DIR = os.path.join(HERE, "_lib")
LIB = os.path.join(OUT_DIR, "libcal.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CU_SOURCES = ["assemble.cu", "solve.cu", "gemm_tc.cu", "api.cu", "static_scratch.cu", "field.cu", "hmat.cu"]
CXX_SOURCES = ["host.cpp", "serve.cpp"]


def _nvcc():
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(SRC, f) for f in os.listdir(SRC)] + [os.path.join(INC, "cal.h"), __file__]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and not _stale():
        return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    nvcc = _nvcc()
    common = ["-O3", "-std=c++17", "-I", INC, "-I", SRC]
    jobs = []
    objs = []
    for f in CU_SOURCES:
        o = os.path.join(OUT_DIR, f + ".o")
        objs.append(o)
        # -ftz=true: no denormal fix-ups around the float32 rsqrt/sin/cos/exp
        # hardware approximations (the operands here are never denormal)
        jobs.append([nvcc, *ARCH, "-lineinfo", "-ftz=true", "-Xcompiler", "-fPIC", *common, "-c",
                     os.path.join(SRC, f), "-o", o])
    for f in CXX_SOURCES:
        o = os.path.join(OUT_DIR, f + ".o")
        objs.append(o)
        jobs.append([nvcc, "-x", "cu", *ARCH, "-Xcompiler", "-fPIC", *common, "-c",
                     os.path.join(SRC, f), "-o", o])

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0 or verbose:
            sys.stderr.write(" ".join(cmd) + "\n" + r.stdout + r.stderr)
        if r.returncode != 0:
            raise RuntimeError(f"compile failed: {cmd[-3]}")

    with ThreadPoolExecutor(max_workers=len(jobs)) as ex:
        list(ex.map(run, jobs))
    tmp = LIB + f".tmp{os.getpid()}"
    run([nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-cudart", "static"])
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
