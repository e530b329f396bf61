"""Build libtns.so (the engine) for sm_103a with nvcc, in-tree.

Each translation unit is compiled in parallel, then linked; the result is
``paper_2305_05581_gb300/libtns.so``.  Run ``python -m paper_2305_05581_gb300.build``.
"""
from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "libtns.so")
BUILD = os.path.join(ROOT, "_build")
SOURCES = ["engine.cpp", "kernels.cu", "solver.cu", "tc.cu", "noalloc.cu", "eig.cu", "devmem.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc():
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.exists(c) or c == "nvcc"):
            return c
    return "nvcc"


def build(verbose: bool = False, ptxas_v: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    inc = ["-I", CSRC, "-I", os.path.join(ROOT, "include")]
    common = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC"] + inc
    jobs = []
    for src in SOURCES:
        path = os.path.join(CSRC, src)
        obj = os.path.join(BUILD, src + ".o")
        if src.endswith(".cu"):
            cmd = [nvcc()] + ARCH + common + ["-c", path, "-o", obj]
            if ptxas_v:
                cmd += ["-Xptxas", "-v"]
        else:
            cmd = [nvcc()] + common + ["-x", "c++", "-c", path, "-o", obj]
        jobs.append((cmd, obj))

    def run(job):
        cmd, obj = job
        r = subprocess.run(cmd, capture_output=True, text=True)
        return cmd, r

    with ThreadPoolExecutor(max_workers=len(jobs)) as ex:
        results = list(ex.map(run, jobs))
    for cmd, r in results:
        if verbose or r.returncode != 0 or ptxas_v:
            sys.stderr.write(" ".join(cmd) + "\n" + r.stdout + r.stderr)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed: " + " ".join(cmd))
    link = [nvcc()] + ARCH + ["-shared", "-o", OUT] + [o for _, o in jobs] + ["-lcudart"]
    r = subprocess.run(link, capture_output=True, text=True)
    if r.returncode != 0:
        sys.stderr.write(r.stdout + r.stderr)
        raise RuntimeError("link failed")
    return OUT


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv, ptxas_v="--ptxas" in sys.argv))
