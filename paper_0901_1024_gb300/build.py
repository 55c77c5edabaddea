"""Builds libdg.so (the C-ABI library of include/dg.h) in-tree with nvcc for sm_103a.

Every translation unit under csrc/ is compiled in parallel with
    nvcc -gencode arch=compute_103a,code=sm_103a -lineinfo -O3
into _build/, then linked into paper_0901_1024_gb300/libdg.so.  Objects are
rebuilt when their source, any header, or this script changed.
"""
from __future__ import annotations

import concurrent.futures as cf
import hashlib
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libdg.so")
INCLUDE = os.path.join(ROOT, "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I" + INCLUDE, "-I" + CSRC]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found (CUDA toolkit required to build libdg.so)")


def _headers_digest() -> str:
    h = hashlib.sha256()
    for d in (CSRC, INCLUDE):
        for name in sorted(os.listdir(d)):
            if name.endswith((".h", ".cuh")):
                with open(os.path.join(d, name), "rb") as f:
                    h.update(name.encode() + f.read())
    with open(__file__, "rb") as f:
        h.update(f.read())
    return h.hexdigest()


def _compile(nvcc, src, obj, stamp, ptxas_verbose):
    key = stamp + hashlib.sha256(open(src, "rb").read()).hexdigest()
    keyfile = obj + ".key"
    if os.path.exists(obj) and os.path.exists(keyfile) and open(keyfile).read() == key:
        return None
    cmd = [nvcc, *ARCH, *FLAGS, "-c", src, "-o", obj]
    if ptxas_verbose and src.endswith(".cu"):
        cmd += ["-Xptxas", "-v"]
    p = subprocess.run(cmd, capture_output=True, text=True)
    if p.returncode != 0:
        raise RuntimeError(f"compile failed: {' '.join(cmd)}\n{p.stdout}\n{p.stderr}")
    with open(keyfile, "w") as f:
        f.write(key)
    return p.stderr if ptxas_verbose else None


def build(verbose: bool = False, ptxas_verbose: bool = False, jobs: int | None = None) -> str:
    """Compile and link libdg.so; returns its path."""
    nvcc = _nvcc()
    os.makedirs(BUILD, exist_ok=True)
    srcs = sorted(os.path.join(CSRC, n) for n in os.listdir(CSRC) if n.endswith((".cu", ".cpp")))
    stamp = _headers_digest()
    objs = [os.path.join(BUILD, os.path.basename(s) + ".o") for s in srcs]
    jobs = jobs or min(len(srcs), os.cpu_count() or 4)
    with cf.ThreadPoolExecutor(jobs) as ex:
        futs = {ex.submit(_compile, nvcc, s, o, stamp, ptxas_verbose): s for s, o in zip(srcs, objs)}
        for fu in cf.as_completed(futs):
            out = fu.result()
            if out and verbose:
                sys.stderr.write(f"--- {os.path.basename(futs[fu])}\n{out}")
    newest = max(os.path.getmtime(o) for o in objs)
    if not os.path.exists(LIB) or os.path.getmtime(LIB) < newest:
        tmp = LIB + ".tmp"
        cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart_static", "-ldl", "-lrt", "-lpthread"]
        p = subprocess.run(cmd, capture_output=True, text=True)
        if p.returncode != 0:
            raise RuntimeError(f"link failed: {' '.join(cmd)}\n{p.stdout}\n{p.stderr}")
        os.replace(tmp, LIB)
    if verbose:
        sys.stderr.write(f"built {LIB}\n")
    return LIB


if __name__ == "__main__":
    build(verbose=True, ptxas_verbose="-v" in sys.argv)
