"""Build libqcx.so in-tree (paper_2603_12326_gb300/_build/) for sm_103a.

Each .cu file is compiled to an object in parallel, then linked into one
shared library with the CUDA runtime linked statically.  Used by
``__graft_entry__.build()`` and by the tests when the library is missing.
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
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libqcx.so")
PEAKS_SRC = os.path.join(HERE, "peaks", "fma_peak.cu")
PEAKS_LIB = os.path.join(OUT, "libqcx_peaks.so")   # measurement utility (CUDA-core FMA peaks), not the path
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I" + os.path.join(ROOT, "include"),
         "-I" + SRC]


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def sources():
    return sorted(os.path.join(SRC, f) for f in os.listdir(SRC) if f.endswith(".cu"))


def up_to_date() -> bool:
    if not os.path.exists(LIB) or not os.path.exists(PEAKS_LIB):
        return False
    if os.path.getmtime(PEAKS_SRC) > os.path.getmtime(PEAKS_LIB):
        return False
    t = os.path.getmtime(LIB)
    deps = sources() + [os.path.join(SRC, f) for f in os.listdir(SRC) if f.endswith((".h", ".cuh"))]
    deps.append(os.path.join(ROOT, "include", "qcx.h"))
    return all(os.path.getmtime(d) <= t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and up_to_date():
        return LIB
    os.makedirs(OUT, exist_ok=True)
    nvcc = _nvcc()

    def one(src):
        obj = os.path.join(OUT, os.path.basename(src)[:-3] + ".o")
        cmd = [nvcc, *ARCH, *FLAGS, "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        if verbose and r.stderr:
            sys.stderr.write(r.stderr)
        return obj

    def peaks():
        r = subprocess.run([nvcc, *ARCH, *FLAGS, "-shared", PEAKS_SRC, "-o", PEAKS_LIB + ".tmp"], capture_output=True,
                           text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {PEAKS_SRC}:\n{r.stdout}\n{r.stderr}")
        os.replace(PEAKS_LIB + ".tmp", PEAKS_LIB)

    with ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 2)) as ex:
        fut = ex.submit(peaks)
        objs = list(ex.map(one, sources()))
        fut.result()
    tmp = LIB + ".tmp"
    r = subprocess.run([nvcc, *ARCH, "-shared", "-o", tmp, *objs], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
