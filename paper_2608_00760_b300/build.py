"""Build libdmg.so (the CUDA kernels + C ABI) in-tree for sm_103a.

    python -m paper_2608_00760_b300.build          # build if sources changed
    python -m paper_2608_00760_b300.build --force

nvcc cross-compiles without a GPU. The library goes to
paper_2608_00760_b300/_lib/libdmg.so, next to the binding that loads it.
"""
from __future__ import annotations

import os
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
OUT = os.path.join(PKG, "_lib", "libdmg.so")
SOURCES = [os.path.join(CSRC, "dmg.cu"), os.path.join(CSRC, "noalloc.cu")]
DEPS = SOURCES + [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))] + [
    os.path.join(ROOT, "include", "dmg.h")]

NVCC_FLAGS = [
    "-gencode", "arch=compute_103a,code=sm_103a",
    "-O3", "-lineinfo", "-std=c++17",
    "-Xcompiler", "-fPIC", "-shared",
    "-I", os.path.join(ROOT, "include"),
]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.isabs(cand) and os.path.exists(cand) or not os.path.isabs(cand)):
            return cand
    return "nvcc"


OUT_CHECK = os.path.join(PKG, "_lib", "libdmg_check.so")


def build(force: bool = False, verbose: bool = False, check: bool = False) -> str:
    """Compile the library; check=True builds the bounds-checked variant
    (-DDMG_BOUNDS_CHECK) as _lib/libdmg_check.so."""
    out = OUT_CHECK if check else OUT
    os.makedirs(os.path.dirname(out), exist_ok=True)
    if not force and os.path.exists(out):
        t = os.path.getmtime(out)
        if all(os.path.getmtime(d) <= t for d in DEPS):
            return out
    tmp = out + ".tmp.%d" % os.getpid()
    cmd = ([nvcc()] + NVCC_FLAGS + (["-DDMG_BOUNDS_CHECK"] if check else []) +
           (["-Xptxas", "-v"] if verbose else []) + ["-o", tmp] + SOURCES)
    subprocess.check_call(cmd)
    os.replace(tmp, out)
    return out


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv, check="--check" in sys.argv))
