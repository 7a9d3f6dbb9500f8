"""Build libzd.so in-tree: every .cu under csrc/ compiled for sm_103a in
parallel, then linked into one shared library (static CUDA runtime).

build(debug=True) makes libzd_debug.so instead: the same sources compiled
with -DZD_DEBUG, whose kernels check their index arithmetic and record
ZD_ERR_INTERNAL (skipping the access) instead of touching memory they do not
own.  The binding loads it when the environment sets ZD_DEBUG=1."""
from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OBJ = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "_lib", "libzd.so")
OBJ_DEBUG = os.path.join(HERE, "_build_debug")
LIB_DEBUG = os.path.join(HERE, "_lib", "libzd_debug.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")

SOURCES = ["sort.cu", "build.cu", "knn_i32.cu", "knn_f32.cu", "knn_f32_2d.cu", "knn_f32_group.cu",
           "knn_f32_group_3n.cu", "knn_f32_group_3w.cu", "knn_f32_group_2n.cu", "knn_f32_group_2w.cu",
           "knn_wide.cu", "update.cu", "local.cu", "backward.cu", "api.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-I", INCLUDE]


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.sep not in c or os.path.exists(c)):
            return c
    return "nvcc"


def _deps():
    return [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(INCLUDE, "zd.h")]


def _stale(target, deps):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def _compile(src, extra, objdir=None):
    obj = os.path.join(objdir or OBJ, os.path.splitext(src)[0] + ".o")
    headers = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cuh")]
    if not _stale(obj, [os.path.join(CSRC, src)] + headers + [os.path.join(INCLUDE, "zd.h")]):
        return obj
    cmd = [nvcc()] + ARCH + FLAGS + extra + ["-c", os.path.join(CSRC, src), "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, " ".join(cmd), r.stderr))
    return obj


def build(force: bool = False, extra=None, jobs: int = 0, debug: bool = False) -> str:
    """Compile (when sources changed) and return the path of libzd.so
    (libzd_debug.so with debug=True)."""
    extra = list(extra or []) + (["-DZD_DEBUG"] if debug else [])
    lib, objdir = (LIB_DEBUG, OBJ_DEBUG) if debug else (LIB, OBJ)
    if not force and not _stale(lib, _deps()):
        return lib
    os.makedirs(objdir, exist_ok=True)
    os.makedirs(os.path.dirname(lib), exist_ok=True)
    if force:
        for f in os.listdir(objdir):
            if f.endswith(".o"):
                os.remove(os.path.join(objdir, f))
    jobs = jobs or min(len(SOURCES), os.cpu_count() or 4)
    with ThreadPoolExecutor(jobs) as ex:
        objs = list(ex.map(lambda s: _compile(s, extra, objdir), SOURCES))
    tmp = lib + ".tmp%d" % os.getpid()
    cmd = [nvcc()] + ARCH + ["-shared", "-o", tmp] + objs
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s\n%s" % (" ".join(cmd), r.stderr))
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, debug="--debug" in sys.argv))
