"""Build libmatgraph.so in-tree with nvcc for sm_103a (GB300).

Each CUDA translation unit compiles in parallel to an object file, then nvcc links
the shared library (static CUDA runtime).  Rebuilds only when a source is newer than
the library.
"""
from __future__ import annotations

import os
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD_DIR = os.path.join(HERE, "_build")
LIB_DIR = os.path.join(HERE, "_lib")
LIB = os.path.join(LIB_DIR, "libmatgraph.so")

UNITS = ["kernels_graph", "kernels_pairs", "kernels_knn", "kernels_edgevec", "kernels_ext", "api"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I" + INCLUDE, "-I" + CSRC]

_lock = threading.Lock()


def nvcc() -> str:
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _sources():
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(INCLUDE, "matgraph.h")]
    return [p for p in deps if os.path.isfile(p)]


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(p) > t for p in _sources())


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile (if needed) and return the path of libmatgraph.so."""
    with _lock:
        if not force and not _stale():
            return LIB
        os.makedirs(BUILD_DIR, exist_ok=True)
        os.makedirs(LIB_DIR, exist_ok=True)
        cc = nvcc()

        def compile_unit(u):
            obj = os.path.join(BUILD_DIR, u + ".o")
            cmd = [cc, *ARCH, *NVCC_FLAGS, "-c", os.path.join(CSRC, u + ".cu"), "-o", obj]
            r = subprocess.run(cmd, capture_output=True, text=True)
            if r.returncode != 0:
                raise RuntimeError(f"nvcc failed for {u}:\n{r.stdout}\n{r.stderr}")
            if verbose and (r.stdout or r.stderr):
                print(r.stdout, r.stderr)
            return obj

        with ThreadPoolExecutor(len(UNITS)) as ex:
            objs = list(ex.map(compile_unit, UNITS))
        tmp = LIB + f".{os.getpid()}.tmp"
        cmd = [cc, *ARCH, "-shared", "-Xcompiler", "-fPIC", *objs, "-o", tmp]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc link failed:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, LIB)
        return LIB
