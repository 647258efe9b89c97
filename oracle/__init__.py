"""FP64 CPU oracle for periodic cutoff / KNN multigraphs and edge-vector gradients.

TEST INFRASTRUCTURE: only ``tests/``, ``__graft_entry__.smoke()`` and the benchmark's
CPU-baseline leg may import this package.  The library (``paper_2307_05380_gb300``)
never does, and shares no code with it.

What it computes (paper, Sec. 2.1):

* :func:`cutoff` -- Def. 3 with a constant cutoff per structure:
  ``{(i, j, t) : ||(x_j - x_i + t) L|| < r}``, ``(i, i, 0)`` excluded, by brute force
  over an oversized, per-pair-centred box of offsets (see ``oracle.c``).
* :func:`knn` -- the KNN special case (Sec. 2.1 after Def. 3; Algorithm 1's output):
  exactly k edges per atom, ties broken by (d2, j, t).
* :func:`edge_vectors`, :func:`edge_grad` -- ``vec = (x_j - x_i + t) L``, ``len = |vec|``
  and the analytic gradient of a loss through them, edge set held fixed (Sec. 1 and
  Sec. 4: graphs updated inside a generative model's forward pass).

Outputs are in canonical order: (src, dst, tx, ty, tz) ascending, src/dst global atom
rows.  Inputs are promoted from float32 to float64 exactly as given.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

_ERRORS = {-1: "out of memory", -2: "singular or non-finite structure",
           -3: "offset box self-check failed", -4: "bad arguments"}


def build(force: bool = False) -> str:
    """Compile the oracle with gcc, -O2 -ffp-contract=off (no fused multiply-add)."""
    with _lock:
        if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
            tmp = _LIB + f".{os.getpid()}.tmp"
            subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
                                   "-shared", "-o", tmp, _SRC, "-lm"])
            os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        lib.oracle_buf_new.restype = P
        lib.oracle_buf_free.argtypes = [P]
        lib.oracle_buf_size.restype = ctypes.c_int64
        lib.oracle_buf_size.argtypes = [P]
        lib.oracle_buf_copy.argtypes = [P, P, P, P, P]
        lib.oracle_cutoff.restype = ctypes.c_int
        lib.oracle_cutoff.argtypes = [ctypes.c_int, P, P, P, P, ctypes.c_int, P, ctypes.c_int64, P]
        lib.oracle_knn.restype = ctypes.c_int
        lib.oracle_knn.argtypes = [ctypes.c_int, P, P, P, ctypes.c_int, ctypes.c_int, P,
                                   ctypes.c_int64, P]
        lib.oracle_edge_vectors.restype = ctypes.c_int
        lib.oracle_edge_vectors.argtypes = [ctypes.c_int, P, P, P, ctypes.c_int64, P, P, P, P, P]
        lib.oracle_edge_grad.restype = ctypes.c_int
        lib.oracle_edge_grad.argtypes = [ctypes.c_int, P, P, P, ctypes.c_int64, P, P, P, P, P, P, P]
        _lib = lib
    return _lib


def _geom(lattice, frac, atom_ptr):
    lat = np.ascontiguousarray(np.asarray(lattice, dtype=np.float64).reshape(-1, 9))
    fr = np.ascontiguousarray(np.asarray(frac, dtype=np.float64).reshape(-1, 3))
    ptr = np.ascontiguousarray(np.asarray(atom_ptr, dtype=np.int32))
    if ptr[-1] != fr.shape[0] or lat.shape[0] != ptr.shape[0] - 1:
        raise ValueError("atom_ptr does not match lattice/frac")
    return lat, fr, ptr


def _collect(lib, buf):
    n = lib.oracle_buf_size(buf)
    src = np.zeros(n, np.int32)
    dst = np.zeros(n, np.int32)
    off = np.zeros((n, 3), np.int32)
    d2 = np.zeros(n, np.float64)
    lib.oracle_buf_copy(buf, src.ctypes.data, dst.ctypes.data, off.ctypes.data, d2.ctypes.data)
    return dict(src=src, dst=dst, offset=off, d2=d2)


def _sources(sources):
    if sources is None:
        return None, 0
    s = np.ascontiguousarray(np.asarray(sources, dtype=np.int32))
    if s.size > 1 and np.any(np.diff(s) <= 0):
        raise ValueError("sources must be strictly ascending")
    return s, int(s.size)


def cutoff(lattice, frac, atom_ptr, r, sources=None, extra: int = 0):
    """Cutoff multigraph (Def. 3, constant cutoff per structure).

    ``r`` is a scalar or one radius per structure.  ``sources`` restricts the build to
    the given ascending global atom rows.  Returns dict(src, dst, offset, d2)."""
    lib = _load()
    lat, fr, ptr = _geom(lattice, frac, atom_ptr)
    B = lat.shape[0]
    rr = np.ascontiguousarray(np.broadcast_to(np.asarray(r, np.float64), (B,)).copy())
    src, ns = _sources(sources)
    buf = lib.oracle_buf_new()
    try:
        rc = lib.oracle_cutoff(B, ptr.ctypes.data, lat.ctypes.data, fr.ctypes.data, rr.ctypes.data,
                               int(extra), None if src is None else src.ctypes.data, ns, buf)
        if rc:
            raise RuntimeError(f"oracle_cutoff: {_ERRORS.get(rc, rc)}")
        return _collect(lib, buf)
    finally:
        lib.oracle_buf_free(buf)


def knn(lattice, frac, atom_ptr, k: int, sources=None, extra: int = 0):
    """KNN multigraph: exactly k edges per source atom, ties by (d2, j, t).

    Returns dict(src, dst, offset, d2) in canonical order."""
    lib = _load()
    lat, fr, ptr = _geom(lattice, frac, atom_ptr)
    src, ns = _sources(sources)
    buf = lib.oracle_buf_new()
    try:
        rc = lib.oracle_knn(lat.shape[0], ptr.ctypes.data, lat.ctypes.data, fr.ctypes.data, int(k),
                            int(extra), None if src is None else src.ctypes.data, ns, buf)
        if rc:
            raise RuntimeError(f"oracle_knn: {_ERRORS.get(rc, rc)}")
        return _collect(lib, buf)
    finally:
        lib.oracle_buf_free(buf)


def edge_vectors(lattice, frac, atom_ptr, src, dst, offset):
    """vec = (x_dst - x_src + t) L and len = |vec| in FP64 for a fixed edge list."""
    lib = _load()
    lat, fr, ptr = _geom(lattice, frac, atom_ptr)
    src = np.ascontiguousarray(src, np.int32)
    dst = np.ascontiguousarray(dst, np.int32)
    off = np.ascontiguousarray(np.asarray(offset, np.int32).reshape(-1, 3))
    E = src.shape[0]
    vec = np.zeros((E, 3), np.float64)
    ln = np.zeros(E, np.float64)
    rc = lib.oracle_edge_vectors(lat.shape[0], ptr.ctypes.data, lat.ctypes.data, fr.ctypes.data, E,
                                 src.ctypes.data, dst.ctypes.data, off.ctypes.data,
                                 vec.ctypes.data, ln.ctypes.data)
    if rc:
        raise RuntimeError(f"oracle_edge_vectors: {_ERRORS.get(rc, rc)}")
    return vec, ln


def edge_grad(lattice, frac, atom_ptr, src, dst, offset, grad_vec=None, grad_len=None):
    """Analytic gradient (FP64) of a loss through vec/len w.r.t. frac and lattice."""
    lib = _load()
    lat, fr, ptr = _geom(lattice, frac, atom_ptr)
    src = np.ascontiguousarray(src, np.int32)
    dst = np.ascontiguousarray(dst, np.int32)
    off = np.ascontiguousarray(np.asarray(offset, np.int32).reshape(-1, 3))
    E = src.shape[0]
    gv = None if grad_vec is None else np.ascontiguousarray(np.asarray(grad_vec, np.float64).reshape(E, 3))
    gl = None if grad_len is None else np.ascontiguousarray(np.asarray(grad_len, np.float64).reshape(E))
    gf = np.zeros_like(fr)
    gL = np.zeros((lat.shape[0], 9), np.float64)
    rc = lib.oracle_edge_grad(lat.shape[0], ptr.ctypes.data, lat.ctypes.data, fr.ctypes.data, E,
                              src.ctypes.data, dst.ctypes.data, off.ctypes.data,
                              None if gv is None else gv.ctypes.data,
                              None if gl is None else gl.ctypes.data,
                              gf.ctypes.data, gL.ctypes.data)
    if rc:
        raise RuntimeError(f"oracle_edge_grad: {_ERRORS.get(rc, rc)}")
    return gf, gL.reshape(-1, 3, 3)


def gaussian_loss_grads(vec, ln, w, sigma):
    """Per-edge loss terms of w * exp(-len^2 / 2 sigma^2) (the differentiation workload)
    and their derivatives w.r.t. len: returns (loss, dloss/dlen)."""
    e = np.exp(-(np.asarray(ln, np.float64) ** 2) / (2.0 * sigma * sigma))
    w = np.asarray(w, np.float64)
    return float(np.sum(w * e)), -w * e * np.asarray(ln, np.float64) / (sigma * sigma)


def pointers(src, atom_ptr):
    """edge_ptr [B+1] and src_ptr [N+1] (int64) of a canonical edge list."""
    src = np.asarray(src, np.int64)
    atom_ptr = np.asarray(atom_ptr, np.int64)
    N = int(atom_ptr[-1])
    src_ptr = np.zeros(N + 1, np.int64)
    np.add.at(src_ptr, src + 1, 1)
    src_ptr = np.cumsum(src_ptr)
    return src_ptr[atom_ptr], src_ptr
