"""Build libpgs.so (the CUDA library behind include/pgs.h) in-tree for sm_103a.

    python -m paper_2503_23044_b300.build [--verbose] [--ptxas] [--checked]

Each translation unit is compiled by nvcc in parallel into _build/, then
linked into paper_2503_23044_b300/libpgs.so.  Rebuilds only what changed.
--checked builds the bounds-checked variant instead (-DPGS_CHECKED, objects in
_build/checked/, library libpgs_checked.so; the binding loads it when the
environment sets PGS_LIB=checked).
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(ROOT, "_build")
LIB = os.path.join(PKG, "libpgs.so")
LIB_CHECKED = os.path.join(PKG, "libpgs_checked.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
         "-I" + os.path.join(ROOT, "include")]


def _nvcc() -> str:
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def _headers_mtime() -> float:
    hs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    hs.append(os.path.join(ROOT, "include", "pgs.h"))
    return max(os.path.getmtime(h) for h in hs)


def build(verbose: bool = False, ptxas_verbose: bool = False, checked: bool = False) -> str:
    bdir = os.path.join(BUILD, "checked") if checked else BUILD
    lib = LIB_CHECKED if checked else LIB
    defs = ["-DPGS_CHECKED"] if checked else []
    os.makedirs(bdir, exist_ok=True)
    nvcc = _nvcc()
    hm = _headers_mtime()
    jobs = []
    for src in sources():
        obj = os.path.join(bdir, os.path.basename(src)[:-3] + ".o")
        if os.path.exists(obj) and os.path.getmtime(obj) >= max(os.path.getmtime(src), hm) and not ptxas_verbose:
            continue
        cmd = [nvcc, *ARCH, *FLAGS, *defs, "-c", src, "-o", obj]
        if ptxas_verbose:
            cmd.insert(1, "-Xptxas=-v")
        jobs.append((src, cmd))

    def run(job):
        src, cmd = job
        return src, cmd, subprocess.run(cmd, capture_output=True, text=True)

    with cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
        for src, cmd, r in ex.map(run, jobs):
            if verbose or ptxas_verbose or r.returncode:
                sys.stderr.write(f"[nvcc] {os.path.basename(src)}\n{r.stdout}{r.stderr}")
            if r.returncode:
                raise RuntimeError(f"nvcc failed on {src}:\n{' '.join(cmd)}\n{r.stderr}")
    objs = [os.path.join(bdir, os.path.basename(s)[:-3] + ".o") for s in sources()]
    if jobs or not os.path.exists(lib):
        cmd = [nvcc, *ARCH, "-shared", "-o", lib, *objs, "-lcudart"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode:
            raise RuntimeError(f"link failed:\n{' '.join(cmd)}\n{r.stderr}")
    return lib


if __name__ == "__main__":
    print(build(verbose="--verbose" in sys.argv, ptxas_verbose="--ptxas" in sys.argv, checked="--checked" in sys.argv))
