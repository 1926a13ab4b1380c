"""Build libddg.so in-tree with nvcc for sm_103a (B300).

``python paper_2402_08296_b300/build.py`` compiles every ``csrc/*.cu`` into
``paper_2402_08296_b300/libddg.so``.  Object files go to ``_build/`` and are
rebuilt only when a source or the internal header changed.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "libddg.so")
OBJ = os.path.join(ROOT, "_build", "ddg")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr"]


def sources():
    return sorted(f for f in os.listdir(CSRC) if f.endswith(".cu"))


def _mtime(path):
    return os.path.getmtime(path) if os.path.exists(path) else -1.0


def build(verbose: bool = False, ptxas_info: bool = False) -> str:
    os.makedirs(OBJ, exist_ok=True)
    headers = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cuh")]
    headers.append(os.path.join(ROOT, "include", "ddg.h"))
    newest_header = max(_mtime(h) for h in headers)
    objs = []
    for src in sources():
        s = os.path.join(CSRC, src)
        o = os.path.join(OBJ, src[:-3] + ".o")
        objs.append(o)
        if _mtime(o) >= max(_mtime(s), newest_header):
            continue
        cmd = [NVCC, *ARCH, *FLAGS, "-c", s, "-o", o]
        if ptxas_info:
            cmd.insert(1, "-Xptxas=-v")
        if verbose:
            print(" ".join(cmd), flush=True)
        subprocess.run(cmd, check=True)
    if _mtime(OUT) < max(_mtime(o) for o in objs):
        cmd = [NVCC, *ARCH, "-shared", "-o", OUT, *objs, "-cudart", "shared",
               "-Xlinker", "-rpath,/usr/local/cuda/lib64"]
        if verbose:
            print(" ".join(cmd), flush=True)
        subprocess.run(cmd, check=True)
    return OUT


if __name__ == "__main__":
    print(build(verbose=True, ptxas_info="-v" in sys.argv))
