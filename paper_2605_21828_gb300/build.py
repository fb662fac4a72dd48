"""Compiles libmht.so in-tree: host C++ (FP64 build, packing, C ABI) + sm_103a CUDA kernels.

Usage: ``python -m paper_2605_21828_gb300.build`` or ``build_library()``.  Translation units
compile in parallel into ``_build/``; the shared library lands next to this file.  nvcc
cross-compiles for sm_103a without a GPU, so this runs on any host with the CUDA toolkit.
"""
from __future__ import annotations

import concurrent.futures as cf
import hashlib
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libmht.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found (CUDA toolkit required to build libmht)")


def _sources():
    host = sorted(os.path.join(CSRC, "host", f) for f in os.listdir(os.path.join(CSRC, "host"))
                  if f.endswith(".cpp"))
    cuda = sorted(os.path.join(CSRC, "cuda", f) for f in os.listdir(os.path.join(CSRC, "cuda"))
                  if f.endswith(".cu"))
    return host, cuda


def _digest(paths) -> str:
    h = hashlib.sha256()
    for p in sorted(paths):
        with open(p, "rb") as fh:
            h.update(p.encode() + b"\0" + fh.read())
    return h.hexdigest()


def build_library(force: bool = False, verbose: bool = False) -> str:
    """Builds (if sources changed) and returns the path of libmht.so."""
    host, cuda = _sources()
    headers = []
    for d in (os.path.join(CSRC, "host"), os.path.join(CSRC, "cuda"), CSRC, os.path.join(ROOT, "include")):
        headers += [os.path.join(d, f) for f in os.listdir(d) if f.endswith((".h", ".cuh"))]
    digest = _digest(host + cuda + headers + [os.path.abspath(__file__)])
    stamp = os.path.join(BUILD, "stamp")
    if not force and os.path.exists(LIB) and os.path.exists(stamp):
        with open(stamp) as fh:
            if fh.read().strip() == digest:
                return LIB
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    inc = ["-I", os.path.join(ROOT, "include"), "-I", CSRC]
    common = ["-O3", "-std=c++17"]
    jobs = []
    for src in host:
        obj = os.path.join(BUILD, os.path.basename(src) + ".o")
        jobs.append((["g++", *common, "-fPIC", "-fopenmp", "-Wall", "-Wno-unused-function",
                      "-I", os.path.join(ROOT, "include"), "-I", "/usr/local/cuda/include",
                      "-c", src, "-o", obj], obj))
    for src in cuda:
        obj = os.path.join(BUILD, os.path.basename(src) + ".o")
        jobs.append(([nvcc, *common, *ARCH, "-lineinfo", "-Xcompiler", "-fPIC", "-Xptxas", "-v",
                      *inc, "-c", src, "-o", obj], obj))

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("compile failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
        return r.stdout + r.stderr

    logs = []
    with cf.ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
        for out in ex.map(run, [j[0] for j in jobs]):
            logs.append(out)
    with open(os.path.join(BUILD, "ptxas.log"), "w") as fh:
        fh.write("\n".join(logs))
    tmp = LIB + ".tmp"
    run([nvcc, "-shared", *ARCH, "-Xcompiler", "-fopenmp", "-o", tmp, *[j[1] for j in jobs], "-lgomp"])
    os.replace(tmp, LIB)
    with open(stamp, "w") as fh:
        fh.write(digest)
    if verbose:
        print("built", LIB)
    return LIB


if __name__ == "__main__":
    build_library(force="--force" in sys.argv, verbose=True)
