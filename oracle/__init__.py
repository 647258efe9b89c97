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
* :func:`cutoff_atoms` -- Def. 3 with one cutoff c_i per atom (the source's radius decides).
* :func:`knn` with ``keep_ties`` -- Alg. 2's filter: every image at distance <= the k-th.
* :func:`symmetrize` -- the symmetric closure of a graph (tool list after Alg. 2).
* :func:`triplets` -- Gamma_2 of Def. 3: pairs of edges sharing a source.
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
        lib.oracle_knn.argtypes = [ctypes.c_int, P, P, P, ctypes.c_int, ctypes.c_int, ctypes.c_int, P,
                                   ctypes.c_int64, P]
        lib.oracle_cutoff_atoms.restype = ctypes.c_int
        lib.oracle_cutoff_atoms.argtypes = [ctypes.c_int, P, P, P, P, ctypes.c_int, P, ctypes.c_int64, P]
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


def cutoff_atoms(lattice, frac, atom_ptr, radii, sources=None, extra: int = 0):
    """Cutoff multigraph with one cutoff per atom (Def. 3 in full): (i, j, t) is an edge
    when |(x_j - x_i + t) L| < c_i, the source's radius.  ``radii`` holds c_i for every
    global atom row.  Returns dict(src, dst, offset, d2) in canonical order."""
    lib = _load()
    lat, fr, ptr = _geom(lattice, frac, atom_ptr)
    c = np.ascontiguousarray(np.asarray(radii, np.float64).reshape(-1))
    if c.shape[0] != fr.shape[0]:
        raise ValueError("one radius per atom")
    src, ns = _sources(sources)
    buf = lib.oracle_buf_new()
    try:
        rc = lib.oracle_cutoff_atoms(lat.shape[0], ptr.ctypes.data, lat.ctypes.data, fr.ctypes.data,
                                     c.ctypes.data, int(extra), None if src is None else src.ctypes.data, ns,
                                     buf)
        if rc:
            raise RuntimeError(f"oracle_cutoff_atoms: {_ERRORS.get(rc, rc)}")
        return _collect(lib, buf)
    finally:
        lib.oracle_buf_free(buf)


def knn(lattice, frac, atom_ptr, k: int, sources=None, extra: int = 0, keep_ties: bool = False):
    """KNN multigraph: exactly k edges per source atom, ties by (d2, j, t); with
    ``keep_ties`` every image whose d2 is <= the k-th one (Alg. 2's final filter).

    Returns dict(src, dst, offset, d2) in canonical order."""
    lib = _load()
    lat, fr, ptr = _geom(lattice, frac, atom_ptr)
    src, ns = _sources(sources)
    buf = lib.oracle_buf_new()
    try:
        rc = lib.oracle_knn(lat.shape[0], ptr.ctypes.data, lat.ctypes.data, fr.ctypes.data, int(k),
                            int(bool(keep_ties)), int(extra), None if src is None else src.ctypes.data, ns, buf)
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


def symmetrize(src, dst, offset):
    """Symmetric closure of a multigraph (the paper's tool list after Alg. 2): the input
    edges together with every reversed edge (j, i, -t), each distinct edge once.
    Returns dict(src, dst, offset) in canonical order (src, dst, t0, t1, t2)."""
    s = np.asarray(src, np.int64).reshape(-1)
    d = np.asarray(dst, np.int64).reshape(-1)
    t = np.asarray(offset, np.int64).reshape(-1, 3)
    edges = set()
    for q in range(s.shape[0]):
        e = (int(s[q]), int(d[q]), int(t[q, 0]), int(t[q, 1]), int(t[q, 2]))
        edges.add(e)
        edges.add((e[1], e[0], -e[2], -e[3], -e[4]))
    out = np.array(sorted(edges), dtype=np.int64).reshape(-1, 5)
    return dict(src=out[:, 0].astype(np.int32), dst=out[:, 1].astype(np.int32),
                offset=out[:, 2:5].astype(np.int32))


def triplets(src, include_self: bool = True):
    """Gamma_2 of Def. 3 over an edge list in canonical order: every ordered pair of edge
    ids (e, e') whose edges share a source; (e, e) is a member of the definition as
    written and is dropped when ``include_self`` is false.  Returns dict(a, b) sorted by
    (a, b)."""
    s = np.asarray(src, np.int64).reshape(-1)
    by_source = {}
    for e in range(s.shape[0]):
        by_source.setdefault(int(s[e]), []).append(e)
    a, b = [], []
    for e in range(s.shape[0]):
        for f in by_source[int(s[e])]:
            if include_self or e != f:
                a.append(e)
                b.append(f)
    return dict(a=np.asarray(a, np.int64), b=np.asarray(b, np.int64))
