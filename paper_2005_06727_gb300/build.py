"""Build the CUDA library ``libwmd_gb300.so`` in-tree for sm_103a.

Each translation unit of ``csrc/`` is compiled by its own nvcc process (in
parallel), then the objects are linked into one shared library next to this
file.  Only the ``sm_103a`` target is generated.  Run ``python -m
paper_2005_06727_gb300.build`` or call :func:`build`.
"""
from __future__ import annotations

import concurrent.futures
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OBJ = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libwmd_gb300.so")
ROOT = os.path.dirname(HERE)

SOURCES = ["api.cu", "cdist.cu", "cdist_tc.cu", "sinkhorn.cu", "sinkhorn_conv.cu", "serve.cu",
           "topk.cu", "dense.cu", "noalloc.cu", "peak.cu"]
# cuBLAS serves the dense comparator's two plain GEMMs (dense.cu)
LIBS = ["-lcublas", "-Xlinker", "-rpath,/usr/local/cuda/lib64"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
         "--expt-relaxed-constexpr", "-I", os.path.join(ROOT, "include")]


def nvcc() -> str:
    exe = shutil.which("nvcc")
    if exe is None:
        cand = "/usr/local/cuda/bin/nvcc"
        if os.path.exists(cand):
            return cand
        raise RuntimeError("nvcc not found; the CUDA toolkit is required to build the library")
    return exe


def _sources():
    return [s for s in SOURCES if os.path.exists(os.path.join(CSRC, s))]


def _stale(target: str, deps: list[str]) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(verbose: bool = False, ptxas_verbose: bool = False) -> str:
    """Compile (if needed) and return the path of the shared library."""
    os.makedirs(OBJ, exist_ok=True)
    headers = [os.path.join(CSRC, h) for h in os.listdir(CSRC) if h.endswith((".h", ".cuh"))]
    headers.append(os.path.join(ROOT, "include", "wmd.h"))
    exe = nvcc()
    jobs = []
    for src in _sources():
        s = os.path.join(CSRC, src)
        o = os.path.join(OBJ, src.replace(".cu", ".o"))
        extra = ["-Xptxas", "-v"] if ptxas_verbose else []
        if ptxas_verbose or _stale(o, [s] + headers):
            jobs.append([exe, *ARCH, *FLAGS, *extra, "-c", s, "-o", o])
    if jobs:
        with concurrent.futures.ThreadPoolExecutor(max_workers=len(jobs)) as ex:
            results = list(ex.map(lambda cmd: subprocess.run(cmd, capture_output=True, text=True), jobs))
        for cmd, res in zip(jobs, results):
            if verbose or ptxas_verbose or res.returncode != 0:
                sys.stderr.write(" ".join(cmd) + "\n" + res.stdout + res.stderr)
            if res.returncode != 0:
                raise RuntimeError(f"nvcc failed for {cmd[-3]}")
    objs = [os.path.join(OBJ, s.replace(".cu", ".o")) for s in _sources()]
    if jobs or _stale(LIB, objs):
        tmp = LIB + ".tmp"
        cmd = [exe, *ARCH, "-shared", "-o", tmp, *objs, *LIBS]
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            sys.stderr.write(" ".join(cmd) + "\n" + res.stdout + res.stderr)
            raise RuntimeError("link of libwmd_gb300.so failed")
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build(verbose=True, ptxas_verbose="-v" in sys.argv)
    print(LIB)
