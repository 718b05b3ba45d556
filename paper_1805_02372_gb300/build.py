"""Build step of the CUDA library: nvcc for sm_103a, one object per source, in parallel.

Produces ``paper_1805_02372_gb300/_lib/libpa.so`` (in-tree, git-ignored). Run it
directly (``python -m paper_1805_02372_gb300.build``) or through
``__graft_entry__.build()``.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import hashlib
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
LIBDIR = os.path.join(PKG, "_lib")
LIB = os.path.join(LIBDIR, "libpa.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found: the CUDA library cannot be built")


def _flags(extra=()):
    return ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                   "-Xcompiler", "-O2", "-I", os.path.join(ROOT, "include"),
                   "--expt-relaxed-constexpr"] + list(extra)


# Per-source extra flags. The 64-bit-prime persistent kernel inlines 128-bit products
# into every radix-16 round; NVVM's -O3 pipeline takes minutes on it and ends with
# spills, -O2 takes about a minute and allocates it without spills.
PER_SOURCE = {"ntt_f64.cu": ["-Xcicc", "-O2"]}


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _stamp(srcs, extra) -> str:
    h = hashlib.sha256()
    for p in srcs + sorted(glob.glob(os.path.join(CSRC, "*.cuh")) +
                           glob.glob(os.path.join(CSRC, "*.h")) +
                           [os.path.join(ROOT, "include", "pa.h")]):
        with open(p, "rb") as f:
            h.update(p.encode() + f.read())
    h.update(" ".join(_flags(extra)).encode())
    h.update(repr(sorted(PER_SOURCE.items())).encode())
    return h.hexdigest()


def build(force: bool = False, verbose: bool = False, extra=()) -> str:
    """Compile every ``csrc/*.cu`` for sm_103a and link ``_lib/libpa.so``."""
    srcs = _sources()
    os.makedirs(BUILD, exist_ok=True)
    os.makedirs(LIBDIR, exist_ok=True)
    stamp_file = os.path.join(BUILD, "stamp")
    stamp = _stamp(srcs, extra)
    if not force and os.path.exists(LIB) and os.path.exists(stamp_file):
        with open(stamp_file) as f:
            if f.read() == stamp:
                return LIB
    cc = nvcc()

    def compile_one(src):
        obj = os.path.join(BUILD, os.path.basename(src) + ".o")
        cmd = [cc] + _flags(extra) + PER_SOURCE.get(os.path.basename(src), []) + [
            "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {os.path.basename(src)}:\n{r.stderr}")
        if verbose and r.stderr:
            sys.stderr.write(r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=min(len(srcs), os.cpu_count() or 4)) as ex:
        objs = list(ex.map(compile_one, srcs))
    tmp = LIB + f".tmp{os.getpid()}"
    r = subprocess.run([cc] + ARCH + ["-shared", "-o", tmp] + objs, capture_output=True,
                       text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, LIB)
    with open(stamp_file, "w") as f:
        f.write(stamp)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True,
                extra=["-Xptxas", "-v"] if "--ptxas-v" in sys.argv else ()))
