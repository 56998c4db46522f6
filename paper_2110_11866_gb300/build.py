"""Compile the CUDA library (csrc/*.cu) for sm_103a into _build/libmorlet_sft.so.

Each translation unit is compiled by its own nvcc process, all at once, then linked. No cmake.
`python -m paper_2110_11866_gb300.build` or `build()` from Python.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libmorlet_sft.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-std=c++17", "-O3", "-lineinfo", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr"]


def _nvcc():
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.isabs(c) and os.path.exists(c) or not os.path.isabs(c)):
            return c
    return "nvcc"


def _newest_input():
    files = glob.glob(os.path.join(SRC, "*")) + [os.path.join(HERE, "..", "include", "morlet_sft.h"), __file__]
    return max(os.path.getmtime(f) for f in files if os.path.exists(f))


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(OUT, exist_ok=True)
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= _newest_input():
        return LIB
    nvcc = _nvcc()
    units = sorted(glob.glob(os.path.join(SRC, "*.cu")))
    objs = [os.path.join(OUT, os.path.basename(u)[:-3] + ".o") for u in units]

    def compile_one(u, o):
        cmd = [nvcc, *FLAGS, *ARCH, "-I", SRC, "-c", u, "-o", o]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {os.path.basename(u)}:\n{r.stderr[-4000:]}")
        return r.stderr

    with cf.ThreadPoolExecutor(max_workers=max(1, min(len(units), os.cpu_count() or 4))) as ex:
        futs = [ex.submit(compile_one, u, o) for u, o in zip(units, objs)]
        for f in futs:
            msg = f.result()
            if verbose and msg:
                sys.stderr.write(msg)
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [nvcc, "-shared", *ARCH, "-o", tmp, *objs, "-lpthread", "-ldl", "-lrt"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr[-4000:]}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
