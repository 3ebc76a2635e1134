"""Build the CUDA library in-tree: nvcc for sm_103a -> paper_2609_10165_b300/libebr.so.

Each translation unit compiles to an object file in parallel (they share no
device symbols), then nvcc links the shared library.  Objects go to _build/
at the repository root; a unit is recompiled when it or any header of csrc/
(or include/ebr.h) is newer than its object.
"""

import concurrent.futures as cf
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libebr.so")
OBJ = os.path.join(ROOT, "_build")
SOURCES = ["api.cu", "classify.cu", "levels.cu", "scan.cu", "fill.cu", "forces.cu", "adjoint.cu",
           "packed.cu", "tiled.cu", "stats.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", *ARCH, "-Xcompiler", "-fPIC"]


def nvcc():
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.isabs(cand) and os.path.exists(cand) or not os.path.isabs(cand)):
            return cand
    return "nvcc"


def _headers():
    hs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    hs.append(os.path.join(ROOT, "include", "ebr.h"))
    return hs


def _stale(src, obj, newest_header):
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return os.path.getmtime(src) > t or newest_header > t


def build(verbose=False, extra=(), jobs=None):
    os.makedirs(OBJ, exist_ok=True)
    srcs = list(SOURCES)
    newest_header = max(os.path.getmtime(h) for h in _headers() if os.path.exists(h))
    objs = [os.path.join(OBJ, s[:-3] + ".o") for s in srcs]
    ptxas = ["-Xptxas", "-v"] if verbose else []
    todo = [(s, o) for s, o in zip(srcs, objs) if extra or _stale(os.path.join(CSRC, s), o, newest_header)]

    def compile_one(so):
        s, o = so
        cmd = [nvcc(), *FLAGS, *ptxas, *extra, "-c", "-o", o, os.path.join(CSRC, s)]
        if verbose:
            print(" ".join(cmd))
        r = subprocess.run(cmd, capture_output=True, text=True)
        return s, r

    if todo:
        with cf.ThreadPoolExecutor(max_workers=jobs or min(len(todo), os.cpu_count() or 4)) as ex:
            for s, r in ex.map(compile_one, todo):
                if verbose or r.returncode:
                    sys.stdout.write(r.stdout)
                    sys.stderr.write(r.stderr)
                if r.returncode:
                    raise subprocess.CalledProcessError(r.returncode, "nvcc " + s)
    if todo or not os.path.exists(LIB):
        subprocess.run([nvcc(), *ARCH, "-shared", "-o", LIB, *objs], check=True)
    return LIB


if __name__ == "__main__":
    build(verbose="-v" in sys.argv)
