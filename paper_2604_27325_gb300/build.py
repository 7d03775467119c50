"""Builds the CUDA library ``libbed.so`` in-tree (``paper_2604_27325_gb300/_build/``) with nvcc for sm_103a.

Each translation unit is compiled in parallel, then linked into one shared library that exports the C
ABI declared in ``include/bed.h``.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libbed.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")

SOURCES = ["bed_api.cu", "bed_kernel_16.cu", "bed_kernel_32.cu", "bed_kernel_48.cu", "bed_kernel_64.cu", "bed_ragged.cu",
           "bed_backward.cu", "bed_serve.cu", "bed_peak.cu"]
HEADERS = ["bed_internal.h", "bed_kernel.cuh"]
# exports only the C ABI (bed_*): every other symbol, the per-kernel attribute flags included, stays
# local, so that two copies of the library in one process keep separate state
VERSION_SCRIPT = os.path.join(CSRC, "bed.map")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I" + INCLUDE]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libbed.so")


def _stale(target: str, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, extra_flags=()) -> str:
    """Compile (if stale) and return the path of ``libbed.so``."""
    os.makedirs(OUT, exist_ok=True)
    hdrs = [os.path.join(CSRC, h) for h in HEADERS] + [os.path.join(INCLUDE, "bed.h")]
    objs = []
    jobs = []
    cc = nvcc()
    for src in SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(OUT, src.replace(".cu", ".o"))
        objs.append(o)
        if force or _stale(o, [s] + hdrs):
            jobs.append([cc, *FLAGS, *extra_flags, "-c", s, "-o", o])

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed:\n{' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
        if verbose and (r.stdout or r.stderr):
            print(r.stdout + r.stderr)

    with cf.ThreadPoolExecutor(max_workers=len(jobs) or 1) as ex:
        list(ex.map(run, jobs))
    if force or jobs or _stale(LIB, objs + [VERSION_SCRIPT]):
        tmp = LIB + f".{os.getpid()}.tmp"
        run([cc, *ARCH, "-shared", "-Xlinker", "--version-script=" + VERSION_SCRIPT, "-o", tmp, *objs])
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    import sys

    print(build(force="--force" in sys.argv, verbose=True, extra_flags=["-Xptxas", "-v"] if "-v" in sys.argv else []))
