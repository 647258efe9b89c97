"""ctypes declarations of the matgraph C-ABI (include/matgraph.h).

Argument marshalling only.  Loading fails loudly when libmatgraph.so is missing: there
is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

from . import _build

c_int32, c_int64, c_float, c_void_p, c_size_t = (ctypes.c_int32, ctypes.c_int64, ctypes.c_float,
                                                  ctypes.c_void_p, ctypes.c_size_t)

MG_OK = 0
MG_KIND_CUTOFF = 1
MG_KIND_KNN = 2
KIND_CUTOFF_ATOMS = 3  # binding-side tag: a cutoff graph with per-atom radii
STATUS_NAMES = {0: "MG_OK", 1: "MG_ERR_INVALID_ARGUMENT", 2: "MG_ERR_NONFINITE_INPUT",
                3: "MG_ERR_SINGULAR_LATTICE", 4: "MG_ERR_CAPACITY", 5: "MG_ERR_OFFSET_RANGE",
                6: "MG_ERR_TIMEOUT", 7: "MG_ERR_CUDA", 8: "MG_ERR_WORKSPACE", 9: "MG_ERR_NOT_BUILT",
                10: "MG_ERR_INTERNAL"}


class MgBatch(ctypes.Structure):
    _fields_ = [("num_structures", c_int32), ("total_atoms", c_int32), ("max_atoms", c_int32),
                ("lattice", c_void_p), ("frac", c_void_p), ("atom_ptr", c_void_p)]


class MgGraph(ctypes.Structure):
    _fields_ = [("capacity", c_int64), ("src", c_void_p), ("dst", c_void_p), ("offset", c_void_p),
                ("vec", c_void_p), ("len", c_void_p), ("edge_ptr", c_void_p), ("src_ptr", c_void_p),
                ("perm_dst", c_void_p), ("dst_ptr", c_void_p), ("status", c_void_p)]


class MgTriplets(ctypes.Structure):
    _fields_ = [("capacity", c_int64), ("edge_a", c_void_p), ("edge_b", c_void_p), ("trip_ptr", c_void_p),
                ("status", c_void_p)]


class MgGraphHost(ctypes.Structure):
    _fields_ = [("status", c_void_p), ("src", c_void_p), ("dst", c_void_p), ("offset", c_void_p),
                ("vec", c_void_p), ("len", c_void_p), ("edge_ptr", c_void_p), ("src_ptr", c_void_p)]


MG_SIZE_CLASSES = 8


class MgStep(ctypes.Structure):
    _fields_ = [("batch", c_void_p), ("frac_host", c_void_p), ("lattice_host", c_void_p),
                ("atom_ptr_host", c_void_p), ("graph", c_void_p * 2), ("ws", c_void_p * 2), ("ws_bytes", c_size_t * 2),
                ("stream", c_void_p * 3), ("graph_host", c_void_p * 2), ("host_edges", c_int64 * 2),
                ("grad_vec", c_void_p), ("grad_len", c_void_p), ("vec", c_void_p), ("len", c_void_p),
                ("grad_frac", c_void_p), ("grad_lattice", c_void_p), ("vec_host", c_void_p), ("len_host", c_void_p),
                ("grad_frac_host", c_void_p), ("grad_lattice_host", c_void_p), ("capture", c_int32)]


class MgOpts(ctypes.Structure):
    _fields_ = [("band_rel", c_float), ("knn_keep_ties", c_int32), ("schedule", c_int32),
                ("collect_stats", c_int32), ("fault_tile", c_int32)]


# exported symbols: (name, restype, argtypes)
SIGNATURES = [
    ("mg_create", c_int32, [ctypes.POINTER(c_void_p), c_int32]),
    ("mg_destroy", c_int32, [c_void_p]),
    ("mg_status_string", ctypes.c_char_p, [c_int32]),
    ("mg_workspace_size", c_int32, [c_void_p, ctypes.POINTER(MgBatch), c_int64, ctypes.POINTER(c_size_t)]),
    ("mg_cutoff_graph", c_int32, [c_void_p, ctypes.POINTER(MgBatch), c_float, c_void_p, ctypes.POINTER(MgOpts),
                                  ctypes.POINTER(MgGraph), c_void_p, c_size_t, c_void_p]),
    ("mg_cutoff_graph_atoms", c_int32, [c_void_p, ctypes.POINTER(MgBatch), c_void_p, ctypes.POINTER(MgOpts),
                                        ctypes.POINTER(MgGraph), c_void_p, c_size_t, c_void_p]),
    ("mg_knn_graph", c_int32, [c_void_p, ctypes.POINTER(MgBatch), c_int32, ctypes.POINTER(MgOpts),
                               ctypes.POINTER(MgGraph), c_void_p, c_size_t, c_void_p]),
    ("mg_update_graph", c_int32, [c_void_p, ctypes.POINTER(MgBatch), ctypes.POINTER(MgGraph), c_void_p, c_size_t,
                                  c_void_p]),
    ("mg_build_per_structure", c_int32, [c_void_p, ctypes.POINTER(MgBatch), c_int32, c_float, c_int32, c_void_p,
                                         ctypes.POINTER(MgOpts), ctypes.POINTER(MgGraph), c_void_p, c_size_t,
                                         c_void_p]),
    ("mg_edge_vectors_fwd", c_int32, [c_void_p, ctypes.POINTER(MgBatch), ctypes.POINTER(MgGraph), c_void_p,
                                      c_void_p, c_void_p]),
    ("mg_edge_vectors_bwd", c_int32, [c_void_p, ctypes.POINTER(MgBatch), ctypes.POINTER(MgGraph), c_void_p,
                                      c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_size_t,
                                      c_void_p]),
    ("mg_autotune", c_int32, [c_void_p, ctypes.POINTER(MgBatch), c_int32, c_float, c_int32,
                              ctypes.POINTER(MgGraph), c_void_p, c_size_t, c_void_p]),
    ("mg_last_launch_count", c_int64, [c_void_p]),
    ("mg_cutoff_graph_noalloc", c_int32, [c_void_p, ctypes.POINTER(MgBatch), c_float, ctypes.POINTER(MgOpts),
                                          ctypes.POINTER(MgGraph), c_void_p]),
    ("mg_triplets", c_int32, [c_void_p, ctypes.POINTER(MgBatch), ctypes.POINTER(MgGraph), c_int32,
                              ctypes.POINTER(MgTriplets), c_void_p, c_size_t, c_void_p]),
    ("mg_symmetrize", c_int32, [c_void_p, ctypes.POINTER(MgBatch), ctypes.POINTER(MgGraph),
                                ctypes.POINTER(MgGraph), c_void_p, c_size_t, c_void_p]),
    ("mg_graph_to_host", c_int32, [c_void_p, ctypes.POINTER(MgBatch), ctypes.POINTER(MgGraph), c_int64,
                                   ctypes.POINTER(MgGraphHost), c_void_p]),
    ("mg_graph_step", c_int32, [c_void_p, ctypes.POINTER(MgStep)]),
    ("mg_tuned_table", c_int32, [c_void_p, ctypes.POINTER(c_int32 * (2 * MG_SIZE_CLASSES)), c_int32]),
    ("mg_measure_fp_peaks", c_int32, [c_void_p, c_void_p, ctypes.POINTER(ctypes.c_double),
                                      ctypes.POINTER(ctypes.c_double), c_void_p]),
    ("mg_profile_enable", c_int32, [c_void_p, c_int32]),
    ("mg_stage_times", c_int32, [c_void_p, c_int32, c_int32, ctypes.POINTER(ctypes.c_char_p),
                                 ctypes.POINTER(c_float)]),
]

MG_PROF_CUTOFF, MG_PROF_KNN, MG_PROF_FWD, MG_PROF_BWD = 0, 1, 2, 3

_lib = None


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libmatgraph.so (building it first if allowed and needed)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if build_if_missing:
        path = _build.build()
    if not os.path.exists(path):
        raise RuntimeError(f"matgraph CUDA library not found at {path}; build it with "
                           "paper_2307_05380_gb300._build.build() (nvcc, sm_103a)")
    lib = ctypes.CDLL(path)
    for name, res, args in SIGNATURES:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def status_name(code: int) -> str:
    return STATUS_NAMES.get(int(code), f"status {code}")


def check(code: int, what: str):
    if code != MG_OK:
        raise RuntimeError(f"{what}: {status_name(code)}")
