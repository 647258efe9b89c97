"""Seeded synthetic crystal batches shaped like the paper's workloads (Sec. 3).

Inputs only: this module holds none of the graph method's arithmetic.  Both the CUDA
path (through the tests and the benchmark) and the FP64 oracle read what it returns.
The paper's dataset (Materials Project, Sec. 3) is not available, so these seeded
recipes stand in for it:

* ``1`` -- 16 structures, 4..16 atoms, lengths U[3,8] A, angles U[60,120] deg,
  1.0 A minimum separation; cutoff 5.0 A, k = 12.
* ``2`` -- 256 structures, atoms log-uniform in [1,64], lengths U[2.5,12] A, angles
  U[50,130] deg, 0.9 A separation; cutoff 6.0 A, k = 16.
* ``3`` -- 8192 structures, atoms from the mixture 70% [1,32] / 25% [33,128] / 5%
  [129,400] (log-uniform each), 10% skewed cells (one angle U[25,40] deg, one length
  U[12,30] A); cutoffs 4/6/8 A, k = 8/16/32.
* ``4`` -- 1024 structures, 8..64 atoms, lattices as in 2; cutoff 5.0 A, loss weights
  N(0,1), sigma 1.5 A, 20 perturbation steps (0.02 fractional, 1% strain).
* ``5`` -- 32 supercells, an 8-atom base cell (lengths U[3,6] A, angles U[70,110] deg)
  tiled n x n x n with n in [6,14], plus N(0, 0.05 A) Cartesian noise; cutoff 8 A,
  k = 32.

Every cell with volume below 0.3*abc is redrawn; a cell with less than 5 A^3 per atom
is scaled up isotropically to 5 A^3 per atom so the separation rule can be met.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gen.c")
_LIB = os.path.join(_HERE, "libmgsynth.so")
_lock = threading.Lock()
_lib = None

BASE_SEED = 2307053800

# Workload parameters of each recipe (cutoffs in Angstrom).
CONFIGS = {
    1: dict(B=16, cutoffs=[5.0], ks=[12]),
    2: dict(B=256, cutoffs=[6.0], ks=[16]),
    3: dict(B=8192, cutoffs=[4.0, 6.0, 8.0], ks=[8, 16, 32]),
    4: dict(B=1024, cutoffs=[5.0], ks=[], sigma=1.5, steps=20, sigma_x=0.02, strain=0.01),
    5: dict(B=32, cutoffs=[8.0], ks=[32]),
}


def build(force: bool = False) -> str:
    """Compile the generator (gcc, -ffp-contract=off) next to this file."""
    with _lock:
        if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
            tmp = _LIB + f".{os.getpid()}.tmp"
            subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared",
                                   "-o", tmp, _SRC, "-lm"])
            os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        lib.synth_counts.restype = ctypes.c_int64
        lib.synth_counts.argtypes = [ctypes.c_int, ctypes.c_uint64, ctypes.c_int, ctypes.c_void_p]
        lib.synth_fill.restype = ctypes.c_int
        lib.synth_fill.argtypes = [ctypes.c_int, ctypes.c_uint64, ctypes.c_int, ctypes.c_int,
                                   ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
        lib.synth_normal.restype = None
        lib.synth_normal.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int64,
                                     ctypes.c_double, ctypes.c_void_p]
        lib.synth_perturb.restype = None
        lib.synth_perturb.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int,
                                      ctypes.c_void_p, ctypes.c_double, ctypes.c_double,
                                      ctypes.c_void_p, ctypes.c_void_p]
        _lib = lib
    return _lib


class Batch:
    """A batch of crystal structures: lattice [B,3,3] (row r = lattice vector r, A),
    frac [N,3] fractional coordinates, atom_ptr [B+1] atom row ranges."""

    def __init__(self, lattice, frac, atom_ptr, cfg=None, seed=None):
        self.lattice = np.ascontiguousarray(lattice, dtype=np.float32).reshape(-1, 3, 3)
        self.frac = np.ascontiguousarray(frac, dtype=np.float32).reshape(-1, 3)
        self.atom_ptr = np.ascontiguousarray(atom_ptr, dtype=np.int32)
        self.cfg = cfg
        self.seed = seed

    @property
    def num_structures(self):
        return int(self.lattice.shape[0])

    @property
    def total_atoms(self):
        return int(self.frac.shape[0])

    @property
    def max_atoms(self):
        return int(np.max(np.diff(self.atom_ptr))) if self.num_structures else 0

    def subset(self, structures):
        """A new batch holding the given structure indices, in that order."""
        structures = list(structures)
        counts = [int(self.atom_ptr[s + 1] - self.atom_ptr[s]) for s in structures]
        ptr = np.zeros(len(structures) + 1, np.int32)
        ptr[1:] = np.cumsum(counts)
        frac = np.concatenate([self.frac[self.atom_ptr[s]:self.atom_ptr[s + 1]] for s in structures]
                              ) if structures else np.zeros((0, 3), np.float32)
        return Batch(self.lattice[structures], frac, ptr, self.cfg, self.seed)


def make_batch(cfg: int, seed: int | None = None, B: int | None = None, threads: int | None = None) -> Batch:
    """Generate the seeded batch of recipe ``cfg`` (optionally only its first B structures)."""
    lib = _load()
    if cfg not in CONFIGS:
        raise ValueError(f"unknown recipe {cfg}")
    seed = BASE_SEED + cfg if seed is None else int(seed)
    B = CONFIGS[cfg]["B"] if B is None else int(B)
    counts = np.zeros(B, np.int32)
    tot = lib.synth_counts(cfg, seed, B, counts.ctypes.data)
    if tot < 0:
        raise RuntimeError("synth_counts failed")
    ptr = np.zeros(B + 1, np.int32)
    ptr[1:] = np.cumsum(counts)
    lattice = np.zeros((B, 3, 3), np.float32)
    frac = np.zeros((int(tot), 3), np.float32)
    nthreads = threads or min(16, os.cpu_count() or 1)
    chunks = max(1, min(B, nthreads * 4))
    bounds = [B * c // chunks for c in range(chunks + 1)]

    def work(c):
        return lib.synth_fill(cfg, seed, bounds[c], bounds[c + 1], ptr.ctypes.data,
                              lattice.ctypes.data, frac.ctypes.data)

    with ThreadPoolExecutor(nthreads) as ex:
        rcs = list(ex.map(work, range(chunks)))
    for rc in rcs:
        if rc != 0:
            raise RuntimeError(f"synth_fill failed for structure {-rc - 1}")
    return Batch(lattice, frac, ptr, cfg, seed)


def normal(seed: int, purpose: int, n: int, sigma: float = 1.0) -> np.ndarray:
    """n seeded N(0, sigma^2) draws (float32)."""
    out = np.zeros(int(n), np.float32)
    if n:
        _load().synth_normal(int(seed), int(purpose), int(n), float(sigma), out.ctypes.data)
    return out


def perturb(batch: Batch, seed: int, step: int, sigma_x: float = 0.02, strain: float = 0.01) -> Batch:
    """One generative-loop perturbation of ``batch`` (returns a new batch)."""
    lat = batch.lattice.copy()
    frac = batch.frac.copy()
    _load().synth_perturb(int(seed), int(step), batch.num_structures, batch.atom_ptr.ctypes.data,
                          float(sigma_x), float(strain), lat.ctypes.data, frac.ctypes.data)
    return Batch(lat, frac, batch.atom_ptr.copy(), batch.cfg, batch.seed)


def crystal(lattice, frac) -> Batch:
    """A one-structure batch from explicit lattice rows and fractional coordinates."""
    frac = np.asarray(frac, np.float32).reshape(-1, 3)
    return Batch(np.asarray(lattice, np.float32).reshape(1, 3, 3), frac,
                 np.array([0, frac.shape[0]], np.int32))


def concat(batches) -> Batch:
    """Concatenate batches structure-wise."""
    lat = np.concatenate([b.lattice for b in batches])
    frac = np.concatenate([b.frac for b in batches])
    counts = np.concatenate([np.diff(b.atom_ptr) for b in batches])
    ptr = np.zeros(len(counts) + 1, np.int32)
    ptr[1:] = np.cumsum(counts)
    return Batch(lat, frac, ptr)
