"""Build libhomelbm.so in-tree with nvcc for sm_103a.

Each CUDA translation unit compiles in parallel into ``_build/``; the shared
library lands next to this file as ``libhomelbm.so``.  Sources newer than the
library trigger a rebuild.
"""
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(ROOT, "_build")
LIB = os.path.join(HERE, "libhomelbm.so")
SOURCES = ["api.cu", "stream_collide.cu", "stream_collide_f2.cu", "io_reduce.cu", "hierarchy.cu", "multilevel.cu",
           "ml_host.cu", "adjoint.cu", "adjoint_ml.cu", "batch.cu", "coupling.cu", "boundary.cu",
           "deposit.cu"]
HEADERS = ["hlbm_internal.h", "lbm_math.cuh", "storage.cuh", "io_reduce.h", "lattice_state.h", "hierarchy.cuh",
           "multilevel.cuh", "v2.cuh", "adjoint_math.cuh", "f2_common.cuh", "fp64_bits.cuh"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-std=c++17", "-O3", "-lineinfo", "-Xcompiler", "-fPIC", "-I", os.path.join(ROOT, "include")]


def nvcc():
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _stale():
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, f) for f in SOURCES + HEADERS] + [os.path.join(ROOT, "include", "homelbm.h"), __file__]
    return any(os.path.getmtime(p) > t for p in deps if os.path.exists(p))


def _run(cmd):
    r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if r.returncode != 0:
        raise RuntimeError("command failed: %s\n%s" % (" ".join(cmd), r.stdout))
    return r.stdout


def build(force=False, verbose=False):
    """Compile every CUDA source for sm_103a and link libhomelbm.so; returns its path."""
    if not force and not _stale():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    cc = nvcc()

    def one(src):
        obj = os.path.join(BUILD, src.replace(".cu", ".o"))
        out = _run([cc] + ARCH + FLAGS + ["-c", os.path.join(CSRC, src), "-o", obj])
        if verbose and out:
            sys.stdout.write(out)
        return obj

    with ThreadPoolExecutor(max_workers=min(len(SOURCES), os.cpu_count() or 1)) as ex:
        objs = list(ex.map(one, SOURCES))
    tmp = LIB + ".tmp"
    _run([cc] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart"])
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
