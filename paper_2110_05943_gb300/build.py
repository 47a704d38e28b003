"""Build the CUDA library libclb.so in-tree for sm_103a (GB300).

Three translation units (csrc/clb_api.cu includes the LB kernel headers;
csrc/clb_static.cu is the allocation-free reduction; csrc/nop_kernels.cu the
warm-start network's kernels), one -gencode, no cmake: seconds on either
machine.
"""
from __future__ import annotations

import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
LIB_DIR = os.path.join(HERE, "_lib")
LIB_PATH = os.path.join(LIB_DIR, "libclb.so")
SOURCES = ["clb_api.cu", "clb_static.cu", "nop_kernels.cu"]
ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def _nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libclb")
    return cand


def _inputs():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cu", ".cuh"))]
    files += [os.path.join(ROOT, "include", h) for h in ("clb.h", "clb_nop.h")]
    return files


def up_to_date() -> bool:
    if not os.path.exists(LIB_PATH):
        return False
    t = os.path.getmtime(LIB_PATH)
    return all(os.path.getmtime(f) <= t for f in _inputs())


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile libclb.so if any source is newer; return its path.  The
    translation units compile in parallel, then link once."""
    if not force and up_to_date():
        return LIB_PATH
    os.makedirs(LIB_DIR, exist_ok=True)
    tag = f"{os.getpid()}"
    common = [_nvcc(), ARCH, "-lineinfo", "-O3", "-std=c++17", "-Xcompiler", "-fPIC",
              "-I", os.path.join(ROOT, "include")]
    if verbose:
        common.insert(1, "-Xptxas=-v")
    objs, procs = [], []
    for src in SOURCES:
        obj = os.path.join(LIB_DIR, f"{os.path.splitext(src)[0]}.{tag}.o")
        objs.append(obj)
        procs.append(subprocess.Popen(common + ["-c", os.path.join(CSRC, src), "-o", obj]))
    codes = [p.wait() for p in procs]
    try:
        if any(codes):
            raise RuntimeError(f"nvcc failed for {[s for s, c in zip(SOURCES, codes) if c]}")
        tmp = LIB_PATH + f".{tag}.tmp"
        subprocess.run([_nvcc(), ARCH, "-shared", "-o", tmp] + objs, check=True)
        os.replace(tmp, LIB_PATH)
    finally:
        for o in objs:
            if os.path.exists(o):
                os.remove(o)
    return LIB_PATH


if __name__ == "__main__":
    print(build(force=True, verbose=True))
