"""PyTorch-facing binding of the matgraph C-ABI.

Torch supplies device memory and the current CUDA stream; every step of the graph
build, the edge vectors and their backward pass runs in the library's CUDA kernels.
Functions here only marshal arguments, allocate caller-owned buffers, read the device
status word and resize on MG_ERR_CAPACITY.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass, field
from typing import Optional

import torch

from . import _capi
from ._capi import MgBatch, MgGraph, MgOpts, MgTriplets

_CTX: dict = {}


def _dev_index(device: torch.device) -> int:
    return device.index if device.index is not None else torch.cuda.current_device()


_CTX_BY_DEVICE: dict = {}  # torch.device with an index -> its context (the per-call fast path)


def context(device=None) -> ctypes.c_void_p:
    """The library context of a CUDA device (created on first use)."""
    h = _CTX_BY_DEVICE.get(device) if isinstance(device, torch.device) else None
    if h is not None:
        return h
    device = torch.device("cuda") if device is None else torch.device(device)
    idx = _dev_index(device)
    if idx not in _CTX:
        lib = _capi.load()
        h = ctypes.c_void_p()
        _capi.check(lib.mg_create(ctypes.byref(h), idx), "mg_create")
        _CTX[idx] = h
    if device.index is not None:  # an index-less device follows the current device: not cached
        _CTX_BY_DEVICE[device] = _CTX[idx]
    return _CTX[idx]


# the current stream's raw handle without building a Stream object (about 2 us less per
# library call on the host); the public call when it is missing or the device has no index
_RAW_STREAM = getattr(torch._C, "_cuda_getCurrentRawStream", None)


def _stream(device) -> ctypes.c_void_p:
    if _RAW_STREAM is not None and isinstance(device, torch.device) and device.index is not None:
        return ctypes.c_void_p(_RAW_STREAM(device.index))
    return ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)


def _ptr(t: Optional[torch.Tensor]):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def make_opts(band_rel: float = 1e-5, schedule: int = 0, collect_stats: bool = False,
              fault_tile: int = -1, keep_ties: bool = False) -> MgOpts:
    """Build options (see mg_opts_t); fault_tile is a testing hook for the bounded waits."""
    return MgOpts(float(band_rel), int(bool(keep_ties)), int(schedule), int(bool(collect_stats)), int(fault_tile))


class Batch:
    """A batch of crystal structures on one CUDA device.

    frac [N, 3] float32 fractional coordinates, lattice [B, 3, 3] float32 (row r is
    lattice vector r, Angstrom), atom_ptr [B+1] int32 atom row ranges."""

    def __init__(self, frac: torch.Tensor, lattice: torch.Tensor, atom_ptr: torch.Tensor,
                 max_atoms: Optional[int] = None):
        if not (frac.is_cuda and lattice.is_cuda and atom_ptr.is_cuda):
            raise ValueError("frac, lattice and atom_ptr must be CUDA tensors")
        if frac.dtype != torch.float32 or lattice.dtype != torch.float32 or atom_ptr.dtype != torch.int32:
            raise TypeError("frac/lattice must be float32 and atom_ptr int32")
        if frac.dim() != 2 or frac.shape[1] != 3 or lattice.shape[-2:] != (3, 3):
            raise ValueError("frac must be [N, 3] and lattice [B, 3, 3]")
        if atom_ptr.numel() != lattice.reshape(-1, 9).shape[0] + 1:
            raise ValueError("atom_ptr must have B + 1 entries")
        self.frac = frac.contiguous()
        self.lattice = lattice.reshape(-1, 3, 3).contiguous()
        self.atom_ptr = atom_ptr.contiguous()
        self.device = frac.device
        if max_atoms is None:
            max_atoms = int((self.atom_ptr[1:] - self.atom_ptr[:-1]).max().item()) if self.B else 0
        self.max_atoms = int(max_atoms)
        self._c = MgBatch(self.B, self.N, self.max_atoms, self.lattice.data_ptr(),
                          self.frac.data_ptr() if self.N else None, self.atom_ptr.data_ptr())

    @property
    def B(self) -> int:
        return int(self.lattice.shape[0])

    @property
    def N(self) -> int:
        return int(self.frac.shape[0])

    def with_geometry(self, frac: torch.Tensor, lattice: torch.Tensor) -> "Batch":
        return Batch(frac, lattice, self.atom_ptr, self.max_atoms)

    @property
    def c(self) -> MgBatch:
        return self._c


@dataclass
class Graph:
    """Graph buffers (caller-owned device memory) and the result of the last build.

    The first ``num_edges`` rows of src/dst/offset/vec/len are valid, in canonical
    order (src, dst, tx, ty, tz).  edge_ptr [B+1] splits them by structure and
    src_ptr [N+1] by source atom; perm_dst/dst_ptr list edge ids by (dst, src, t)."""
    kind: int
    batch: Batch
    cutoff: float
    k: int
    capacity: int
    src: torch.Tensor
    dst: torch.Tensor
    offset: torch.Tensor
    vec: Optional[torch.Tensor]
    len: Optional[torch.Tensor]
    edge_ptr: torch.Tensor
    src_ptr: torch.Tensor
    perm_dst: Optional[torch.Tensor]
    dst_ptr: Optional[torch.Tensor]
    status: torch.Tensor
    ws: torch.Tensor
    opts: MgOpts
    radii: Optional[torch.Tensor] = None  # per-atom cutoffs (KIND_CUTOFF_ATOMS)
    num_edges: int = -1
    last_status: dict = field(default_factory=dict)
    _c: Optional[MgGraph] = None

    @property
    def c(self) -> MgGraph:
        if self._c is None:
            self._c = MgGraph(self.capacity, self.src.data_ptr(), self.dst.data_ptr(), self.offset.data_ptr(),
                              _ptr(self.vec), _ptr(self.len), self.edge_ptr.data_ptr(), self.src_ptr.data_ptr(),
                              _ptr(self.perm_dst), _ptr(self.dst_ptr), self.status.data_ptr())
        return self._c

    def edges(self):
        """(src, dst, offset) views of the valid edges (after a synchronised build)."""
        E = self.num_edges
        return self.src[:E], self.dst[:E], self.offset[:E]

    def read_status(self) -> dict:
        """Synchronise the stream and decode the device status word."""
        raw = self.status.cpu()
        code = int(raw[0].item() & 0xFFFFFFFF)
        first_bad = int((raw[0].item() >> 32) & 0xFFFFFFFF)
        if first_bad >= 2 ** 31:
            first_bad -= 2 ** 32
        st = dict(code=code, first_bad_structure=None if first_bad == 2 ** 31 - 1 else first_bad,
                  num_edges=int(raw[1]), required_capacity=int(raw[2]), rechecked=int(raw[3]),
                  candidates=int(raw[4]))
        self.last_status = st
        if code == 0:
            self.num_edges = st["num_edges"]
        return st


def _alloc_graph(kind, batch: Batch, cutoff, k, capacity, with_vectors, with_perm, opts, ws_edges=None) -> Graph:
    dev = batch.device
    capacity = int(max(capacity, 1))
    lib = _capi.load()
    ctx = context(dev)
    nbytes = ctypes.c_size_t(0)
    _capi.check(lib.mg_workspace_size(ctx, ctypes.byref(batch.c), int(ws_edges or capacity), ctypes.byref(nbytes)),
                "mg_workspace_size")
    i32 = dict(dtype=torch.int32, device=dev)
    f32 = dict(dtype=torch.float32, device=dev)
    i64 = dict(dtype=torch.int64, device=dev)
    return Graph(kind=kind, batch=batch, cutoff=float(cutoff), k=int(k), capacity=capacity,
                 src=torch.empty(capacity, **i32), dst=torch.empty(capacity, **i32),
                 offset=torch.empty(capacity, 3, **i32),
                 vec=torch.empty(capacity, 3, **f32) if with_vectors else None,
                 len=torch.empty(capacity, **f32) if with_vectors else None,
                 edge_ptr=torch.empty(batch.B + 1, **i64), src_ptr=torch.empty(batch.N + 1, **i64),
                 perm_dst=torch.empty(capacity, **i32) if with_perm else None,
                 dst_ptr=torch.empty(batch.N + 1, **i64) if with_perm else None,
                 status=torch.zeros(5, **i64), ws=torch.empty(int(nbytes.value), dtype=torch.uint8, device=dev),
                 opts=opts)


def _launch_build(g: Graph, per_structure: bool = False, atom_ptr_host=None):
    lib = _capi.load()
    ctx = context(g.batch.device)
    st = _stream(g.batch.device)
    if per_structure:
        ap = (ctypes.c_int32 * len(atom_ptr_host))(*atom_ptr_host)
        g._ap_keepalive = ap
        rc = lib.mg_build_per_structure(ctx, ctypes.byref(g.batch.c), g.kind, float(g.cutoff), int(g.k), ap,
                                        ctypes.byref(g.opts), ctypes.byref(g.c), _ptr(g.ws), g.ws.numel(), st)
        _capi.check(rc, "mg_build_per_structure")
    elif g.kind == _capi.MG_KIND_CUTOFF:
        rc = lib.mg_cutoff_graph(ctx, ctypes.byref(g.batch.c), float(g.cutoff), None, ctypes.byref(g.opts),
                                 ctypes.byref(g.c), _ptr(g.ws), g.ws.numel(), st)
        _capi.check(rc, "mg_cutoff_graph")
    elif g.kind == _capi.KIND_CUTOFF_ATOMS:
        rc = lib.mg_cutoff_graph_atoms(ctx, ctypes.byref(g.batch.c), _ptr(g.radii), ctypes.byref(g.opts),
                                       ctypes.byref(g.c), _ptr(g.ws), g.ws.numel(), st)
        _capi.check(rc, "mg_cutoff_graph_atoms")
    else:
        rc = lib.mg_knn_graph(ctx, ctypes.byref(g.batch.c), int(g.k), ctypes.byref(g.opts), ctypes.byref(g.c),
                              _ptr(g.ws), g.ws.numel(), st)
        _capi.check(rc, "mg_knn_graph")


def _finish(g: Graph, sync: bool) -> Graph:
    if not sync:
        return g
    st = g.read_status()
    if st["code"] != 0:
        raise RuntimeError(f"matgraph build failed: {_capi.status_name(st['code'])} "
                           f"(structure {st['first_bad_structure']})")
    return g


def _build(kind, batch: Batch, cutoff, k, capacity, with_vectors, with_perm, opts, sync, per_structure=False,
           radii=None):
    if opts is None:
        opts = make_opts()
    atom_ptr_host = batch.atom_ptr.cpu().tolist() if per_structure else None
    exact_k = kind == _capi.MG_KIND_KNN and not opts.knn_keep_ties
    if exact_k:
        capacity = int(k) * batch.N
    elif capacity is None:
        capacity = (2 * int(k) * batch.N + 1024) if kind == _capi.MG_KIND_KNN else 64 * batch.N + 1024
    g = _alloc_graph(kind, batch, cutoff, k, capacity, with_vectors, with_perm, opts)
    g.radii = radii
    _launch_build(g, per_structure, atom_ptr_host)
    if not sync:
        return g
    st = g.read_status()
    if st["code"] == 4 and not exact_k:  # MG_ERR_CAPACITY: exact size known now
        g = _alloc_graph(kind, batch, cutoff, k, st["required_capacity"], with_vectors, with_perm, opts)
        g.radii = radii
        _launch_build(g, per_structure, atom_ptr_host)
    return _finish(g, True)


def cutoff_graph(batch: Batch, cutoff: float, *, capacity: Optional[int] = None, with_vectors: bool = True,
                 with_perm: bool = True, opts: Optional[MgOpts] = None, sync: bool = True) -> Graph:
    """Cutoff multigraph (Def. 3 with a constant cutoff): every (i, j, t) with
    |(x_j - x_i + t) L| < cutoff, (i, i, 0) excluded."""
    return _build(_capi.MG_KIND_CUTOFF, batch, cutoff, 0, capacity, with_vectors, with_perm, opts, sync)


def cutoff_graph_atoms(batch: Batch, radii: torch.Tensor, *, capacity: Optional[int] = None,
                       with_vectors: bool = True, with_perm: bool = True, opts: Optional[MgOpts] = None,
                       sync: bool = True) -> Graph:
    """Cutoff multigraph with one cutoff per atom (Def. 3 in full): every (i, j, t) with
    |(x_j - x_i + t) L| < radii[i], (i, i, 0) excluded.  radii: float32 [N] on the device."""
    if radii.dtype != torch.float32 or radii.device != batch.device or radii.numel() != batch.N:
        raise ValueError("radii must be float32 [N] on the batch's device")
    radii = radii.contiguous()
    return _build(_capi.KIND_CUTOFF_ATOMS, batch, 0.0, 0, capacity, with_vectors, with_perm, opts, sync,
                  radii=radii)


def knn_graph(batch: Batch, k: int, *, with_vectors: bool = True, with_perm: bool = True,
              opts: Optional[MgOpts] = None, sync: bool = True, keep_ties: bool = False) -> Graph:
    """KNN multigraph: exactly k edges per atom, ties by (distance, j, t); with keep_ties
    every image at most as far as the k-th (Alg. 2's filter, >= k edges per atom)."""
    if keep_ties:
        opts = opts or make_opts()
        opts = MgOpts(opts.band_rel, 1, opts.schedule, opts.collect_stats, opts.fault_tile)
    return _build(_capi.MG_KIND_KNN, batch, 0.0, k, None, with_vectors, with_perm, opts, sync)


def build_per_structure(batch: Batch, kind: str, cutoff: float = 0.0, k: int = 0, *, capacity=None,
                        with_vectors=True, with_perm=True, opts=None, sync=True) -> Graph:
    """The plain comparison build: the same kernels, one launch sequence per structure."""
    kd = _capi.MG_KIND_CUTOFF if kind == "cutoff" else _capi.MG_KIND_KNN
    return _build(kd, batch, cutoff, k, capacity, with_vectors, with_perm, opts, sync, per_structure=True)


def rebuild(g: Graph, sync: bool = True, per_structure: bool = False, atom_ptr_host=None) -> Graph:
    """Run the build again into the same buffers (same parameters); per_structure
    selects the one-launch-sequence-per-structure comparison build."""
    if per_structure and atom_ptr_host is None:
        atom_ptr_host = g.batch.atom_ptr.cpu().tolist()
    _launch_build(g, per_structure, atom_ptr_host)
    return _finish(g, sync)


def update_graph(g: Graph, frac: Optional[torch.Tensor] = None, lattice: Optional[torch.Tensor] = None,
                 sync: bool = True) -> Graph:
    """Rebuild ``g`` for new geometry (Sec. 1: the graph follows the geometry inside a
    generative model).  New coordinates/lattices are copied into the graph's batch
    buffers; the recorded build is replayed as a CUDA graph.  If the edge count
    outgrows the capacity, the graph is rebuilt into larger buffers."""
    if frac is not None:
        g.batch.frac.copy_(frac)
    if lattice is not None:
        g.batch.lattice.copy_(lattice.reshape(g.batch.lattice.shape))
    lib = _capi.load()
    rc = lib.mg_update_graph(context(g.batch.device), ctypes.byref(g.batch.c), ctypes.byref(g.c), _ptr(g.ws),
                             g.ws.numel(), _stream(g.batch.device))
    _capi.check(rc, "mg_update_graph")
    if not sync:
        return g
    st = g.read_status()
    if st["code"] == 4:
        return _build(g.kind, g.batch, g.cutoff, g.k, st["required_capacity"], g.vec is not None,
                      g.perm_dst is not None, g.opts, True)
    return _finish(g, True)


def profile_enable(on: bool = True, device=None) -> None:
    """Record CUDA events between kernel stages of later builds and edge-vector calls."""
    _capi.check(_capi.load().mg_profile_enable(context(device), int(bool(on))), "mg_profile_enable")


def stage_times(which: str, device=None) -> dict:
    """{stage: milliseconds} of the last profiled call of kind 'cutoff', 'knn', 'fwd'
    or 'bwd' (waits for its events)."""
    code = {"cutoff": 0, "knn": 1, "fwd": 2, "bwd": 3}[which]
    names = (ctypes.c_char_p * 16)()
    ms = (ctypes.c_float * 16)()
    n = _capi.load().mg_stage_times(context(device), code, 16, names, ms)
    return {} if n < 0 else {names[q].decode(): float(ms[q]) for q in range(n)}


def measure_fp_peaks(device=None) -> dict:
    """FP32 and FP64 fused multiply-add rates of the device in TFLOP/s, from the library's
    own kernel (independent FMA chains on a full-occupancy grid, CUDA events; no clock or
    power setting touched).  Synchronises."""
    dev = torch.device("cuda") if device is None else torch.device(device)
    sink = torch.zeros(2, dtype=torch.float64, device=dev)
    f32, f64 = ctypes.c_double(0.0), ctypes.c_double(0.0)
    _capi.check(_capi.load().mg_measure_fp_peaks(context(dev), sink.data_ptr(), ctypes.byref(f32), ctypes.byref(f64),
                                                 _stream(dev)), "mg_measure_fp_peaks")
    return {"fp32_tflops": f32.value, "fp64_tflops": f64.value}


def last_launch_count(device=None) -> int:
    return int(_capi.load().mg_last_launch_count(context(device)))


def autotune(batch: Batch, kind: str, cutoff: float = 0.0, k: int = 0, capacity=None) -> None:
    """Time the schedules on this batch and keep the fastest for its size class."""
    kd = _capi.MG_KIND_CUTOFF if kind == "cutoff" else _capi.MG_KIND_KNN
    g = _build(kd, batch, cutoff, k, capacity, True, False, None, True)
    rc = _capi.load().mg_autotune(context(batch.device), ctypes.byref(batch.c), kd, float(cutoff), int(k),
                                  ctypes.byref(g.c), _ptr(g.ws), g.ws.numel(), _stream(batch.device))
    _capi.check(rc, "mg_autotune")


def tuned_table(device=None) -> list:
    """The context's tuned schedules: [kind - 1][size class] (0 = not tuned)."""
    n = _capi.MG_SIZE_CLASSES
    t = (ctypes.c_int32 * (2 * n))()
    _capi.check(_capi.load().mg_tuned_table(context(device), ctypes.byref(t), 0), "mg_tuned_table")
    return [list(t[0:n]), list(t[n:2 * n])]


def set_tuned_table(table, device=None) -> None:
    t = (ctypes.c_int32 * (2 * _capi.MG_SIZE_CLASSES))(*[int(v) for row in table for v in row])
    _capi.check(_capi.load().mg_tuned_table(context(device), ctypes.byref(t), 1), "mg_tuned_table")


def size_class(max_atoms: int, total_atoms: int) -> int:
    """The size class of a batch (as the library's): its largest structure, plus 4 from
    8192 atoms in the batch."""
    m = int(max_atoms)
    c = 1 if m <= 0 else 0 if m <= 32 else 1 if m <= 128 else 2 if m <= 512 else 3
    return c + (4 if int(total_atoms) >= 8192 else 0)


def _tune_path(device) -> str:
    import hashlib
    import os
    from . import _build
    h = hashlib.sha256()
    for f in sorted(_build._sources()):
        h.update(open(f, "rb").read())
    idx = _dev_index(torch.device(device))
    props = torch.cuda.get_device_properties(idx)
    name = "".join(c if c.isalnum() else "_" for c in props.name)
    d = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_tune")
    return os.path.join(d, f"{name}_sm{props.multi_processor_count}_{h.hexdigest()[:12]}.json")


def autotune_cached(batch: Batch, kind: str, cutoff: float = 0.0, k: int = 0, path=None) -> dict:
    """The schedule of this batch's size class from a per-device cache file (keyed by the
    device, its SM count and the library's sources); when the entry is missing,
    mg_autotune measures it on this batch and the file is written again.  Returns
    {"schedule", "size_class", "tuned_now", "path"}."""
    import json
    import os
    path = path or _tune_path(batch.device)
    cache = {}
    if os.path.exists(path):
        try:
            cache = json.load(open(path))
        except (OSError, ValueError):
            cache = {}
    ki = 0 if kind == "cutoff" else 1
    sc = size_class(batch.max_atoms, batch.N)
    table = tuned_table(batch.device)
    for key, sched in cache.items():  # "kind:class" -> schedule
        kk, cc = key.split(":")
        table[0 if kk == "cutoff" else 1][int(cc)] = int(sched)
    set_tuned_table(table, batch.device)
    tuned_now = f"{kind}:{sc}" not in cache
    if tuned_now:
        autotune(batch, kind, cutoff=cutoff, k=k)
        cache[f"{kind}:{sc}"] = tuned_table(batch.device)[ki][sc]
        os.makedirs(os.path.dirname(path), exist_ok=True)
        tmp = f"{path}.{os.getpid()}.tmp"
        json.dump(cache, open(tmp, "w"), indent=1, sort_keys=True)
        os.replace(tmp, path)
    return {"schedule": int(cache[f"{kind}:{sc}"]), "size_class": sc, "tuned_now": tuned_now, "path": path}


# ---------------------------------------------------------------------------- graph operations

@dataclass
class Triplets:
    """Gamma_2 of a graph: triplet q pairs edge edge_a[q] with edge edge_b[q] (same source);
    the triplets whose first edge is e are trip_ptr[e] .. trip_ptr[e+1]-1."""
    count: int
    edge_a: Optional[torch.Tensor]
    edge_b: torch.Tensor
    trip_ptr: torch.Tensor


def triplets(g: Graph, include_self: bool = True, with_edge_a: bool = True,
             capacity: Optional[int] = None) -> Triplets:
    """Ordered pairs (e, e') of edges with a common source (Def. 3's Gamma_2), as edge ids
    in canonical order; include_self keeps (e, e).  Synchronises to size the output."""
    batch = g.batch
    dev = batch.device
    if g.num_edges < 0:
        raise RuntimeError("graph has no synchronised build")
    E = g.num_edges
    lib = _capi.load()
    ctx = context(dev)
    st = _stream(dev)
    status = torch.zeros(5, dtype=torch.int64, device=dev)
    trip_ptr = torch.empty(E + 1, dtype=torch.int64, device=dev)
    nbytes = ctypes.c_size_t(0)
    _capi.check(lib.mg_workspace_size(ctx, ctypes.byref(batch.c), 0, ctypes.byref(nbytes)), "mg_workspace_size")
    ws = torch.empty(int(nbytes.value), dtype=torch.uint8, device=dev)
    if capacity is None:  # sum of squared degrees >= E^2 / N
        capacity = int(1.25 * E * E / max(batch.N, 1)) + 1024
    for _ in range(2):
        a = torch.empty(capacity, dtype=torch.int32, device=dev) if with_edge_a else None
        b = torch.empty(capacity, dtype=torch.int32, device=dev)
        out = MgTriplets(int(capacity), _ptr(a), b.data_ptr(), trip_ptr.data_ptr(), status.data_ptr())
        _capi.check(lib.mg_triplets(ctx, ctypes.byref(batch.c), ctypes.byref(g.c), int(bool(include_self)),
                                    ctypes.byref(out), ws.data_ptr(), ws.numel(), st), "mg_triplets")
        raw = status.cpu()
        code = int(raw[0].item() & 0xFFFFFFFF)
        T = int(raw[1])
        if code == 4:  # MG_ERR_CAPACITY: the exact count is known now
            capacity = max(T, 1)
            continue
        if code:
            raise RuntimeError(f"mg_triplets failed: {_capi.status_name(code)}")
        return Triplets(T, a[:T] if a is not None else None, b[:T], trip_ptr)
    raise RuntimeError("mg_triplets: capacity retry failed")


def symmetrize(g: Graph, *, with_vectors: bool = True, with_perm: bool = True,
               capacity: Optional[int] = None) -> Graph:
    """Symmetric closure of a graph built with a destination order (tool list after
    Alg. 2): its edges plus every reversed edge (j, i, -t), each once, canonical order."""
    if g.perm_dst is None or g.num_edges < 0:
        raise ValueError("symmetrize needs a synchronised graph built with with_perm=True")
    batch = g.batch
    lib = _capi.load()
    ctx = context(batch.device)
    st = _stream(batch.device)
    cap = capacity or max(2 * g.num_edges, 1)
    for _ in range(2):
        out = _alloc_graph(g.kind, batch, g.cutoff, g.k, cap, with_vectors, with_perm, g.opts,
                           ws_edges=max(g.capacity, cap))
        _capi.check(lib.mg_symmetrize(ctx, ctypes.byref(batch.c), ctypes.byref(g.c), ctypes.byref(out.c),
                                      _ptr(out.ws), out.ws.numel(), st), "mg_symmetrize")
        s = out.read_status()
        if s["code"] == 4:
            cap = s["required_capacity"]
            continue
        return _finish(out, True)
    raise RuntimeError("mg_symmetrize: capacity retry failed")


# ---------------------------------------------------------------------------- host copies

HOST_FIELDS = ("status", "src", "dst", "offset", "vec", "len", "edge_ptr", "src_ptr")


def host_buffers(g: Graph, num_edges: int, fields=HOST_FIELDS) -> dict:
    """Pinned host tensors for graph_to_host: the first num_edges rows of each field."""
    E = int(num_edges)
    shapes = {"status": ((5,), torch.int64), "src": ((E,), torch.int32), "dst": ((E,), torch.int32),
              "offset": ((E, 3), torch.int32), "vec": ((E, 3), torch.float32), "len": ((E,), torch.float32),
              "edge_ptr": ((g.batch.B + 1,), torch.int64), "src_ptr": ((g.batch.N + 1,), torch.int64)}
    return {f: torch.empty(shapes[f][0], dtype=shapes[f][1], pin_memory=True) for f in fields}


def graph_to_host(g: Graph, out: dict, num_edges: Optional[int] = None) -> dict:
    """Copy the graph's first num_edges rows (default: its last read edge count), pointers
    and status word into the host tensors of `out` (from host_buffers; any subset of the
    fields), asynchronously on the current stream: one library call for all of them."""
    E = g.num_edges if num_edges is None else int(num_edges)
    h = _capi.MgGraphHost(*[_ptr(out.get(f)) for f in HOST_FIELDS])
    dev = g.batch.device
    rc = _capi.load().mg_graph_to_host(context(dev), ctypes.byref(g.batch.c), ctypes.byref(g.c), E,
                                       ctypes.byref(h), _stream(dev))
    _capi.check(rc, "mg_graph_to_host")
    return out


class Step:
    """One step of a generative loop through a single library call (mg_graph_step): new
    geometry copied in from pinned host tensors, graphs[0] (and graphs[1], on its own
    stream) rebuilt, each graph's rows copied to its host buffers, edge vectors and the
    backward of grad_vec / grad_len on graphs[0], results copied out.  The argument
    block is built once here; run() only enqueues (synchronise streams[0] to read).

    graphs: one or two built Graphs on the same batch; streams: torch streams (the first
    is the step's); host: per graph a dict from host_buffers (or None); inputs: dict of
    pinned host tensors 'frac', 'lattice', 'atom_ptr' (any subset); outputs: dict of
    pinned host tensors 'vec', 'len', 'grad_frac', 'grad_lattice' (any subset); capture:
    record the step as one CUDA graph at the first run and replay it (one launch)."""

    def __init__(self, graphs, streams, host=(None, None), inputs=None, grad_vec=None, grad_len=None, vec=None,
                 ln=None, grad_frac=None, grad_lattice=None, outputs=None, host_edges=None, capture=True):
        g0 = graphs[0]
        g1 = graphs[1] if len(graphs) > 1 else None
        batch = g0.batch
        inputs = inputs or {}
        outputs = outputs or {}
        self._keep = [graphs, streams, host, inputs, outputs, grad_vec, grad_len, vec, ln, grad_frac, grad_lattice]
        st = _capi.MgStep()
        st.batch = ctypes.addressof(batch.c)
        st.frac_host = _ptr(inputs.get("frac"))
        st.lattice_host = _ptr(inputs.get("lattice"))
        st.atom_ptr_host = _ptr(inputs.get("atom_ptr"))
        self._hosts = []
        for q, g in enumerate((g0, g1)):
            if g is None:
                continue
            st.graph[q] = ctypes.addressof(g.c)
            st.ws[q] = g.ws.data_ptr()
            st.ws_bytes[q] = g.ws.numel()
            h = host[q] if q < len(host) else None
            if h is not None:
                hh = _capi.MgGraphHost(*[_ptr(h.get(f)) for f in HOST_FIELDS])
                self._hosts.append(hh)
                st.graph_host[q] = ctypes.addressof(hh)
            edges = host_edges[q] if host_edges is not None else g.num_edges
            st.host_edges[q] = int(edges)
        for q, s_ in enumerate(streams[:3]):
            st.stream[q] = s_.cuda_stream if s_ is not None else None
        st.grad_vec, st.grad_len = _ptr(grad_vec), _ptr(grad_len)
        st.vec, st.len = _ptr(vec), _ptr(ln)
        st.grad_frac, st.grad_lattice = _ptr(grad_frac), _ptr(grad_lattice)
        st.vec_host, st.len_host = _ptr(outputs.get("vec")), _ptr(outputs.get("len"))
        st.grad_frac_host, st.grad_lattice_host = _ptr(outputs.get("grad_frac")), _ptr(outputs.get("grad_lattice"))
        st.capture = int(bool(capture))  # record the step once as a CUDA graph, replay it after
        self._st = st
        self._ref = ctypes.byref(st)
        self._lib = _capi.load()
        self._ctx = context(batch.device)

    def run(self) -> None:
        rc = self._lib.mg_graph_step(self._ctx, self._ref)
        if rc:
            _capi.check(rc, "mg_graph_step")


# ---------------------------------------------------------------------------- edge vectors

def edge_vectors_fwd(g: Graph, batch: Optional[Batch] = None, out_vec=None, out_len=None):
    """vec = (x_j - x_i + t) L and len = |vec| for the graph's fixed edge set, from the
    batch's current coordinates (default: the graph's own batch)."""
    batch = g.batch if batch is None else batch
    dev = batch.device
    if out_vec is None:
        out_vec = torch.empty(g.capacity, 3, dtype=torch.float32, device=dev)
    if out_len is None:
        out_len = torch.empty(g.capacity, dtype=torch.float32, device=dev)
    rc = _capi.load().mg_edge_vectors_fwd(context(dev), ctypes.byref(batch.c), ctypes.byref(g.c), _ptr(out_vec),
                                          _ptr(out_len), _stream(dev))
    _capi.check(rc, "mg_edge_vectors_fwd")
    return out_vec, out_len


def edge_vectors_bwd(g: Graph, batch: Batch, grad_vec, grad_len, vec, ln, grad_frac=None, grad_lattice=None):
    """Gradients of a loss through vec/len w.r.t. frac [N,3] and lattice [B,3,3]."""
    dev = batch.device
    if grad_frac is None:
        grad_frac = torch.empty(batch.N, 3, dtype=torch.float32, device=dev)
    if grad_lattice is None:
        grad_lattice = torch.empty(batch.B, 3, 3, dtype=torch.float32, device=dev)
    rc = _capi.load().mg_edge_vectors_bwd(context(dev), ctypes.byref(batch.c), ctypes.byref(g.c), _ptr(grad_vec),
                                          _ptr(grad_len), _ptr(vec), _ptr(ln), _ptr(grad_frac),
                                          _ptr(grad_lattice), _ptr(g.ws), g.ws.numel(), _stream(dev))
    _capi.check(rc, "mg_edge_vectors_bwd")
    return grad_frac, grad_lattice


class EdgeVectors(torch.autograd.Function):
    """Differentiable edge vectors and lengths for a fixed edge set.

    forward(frac, lattice, graph) -> (vec [E,3], len [E]); backward gives gradients
    w.r.t. frac and lattice through the library's deterministic segmented kernels."""

    @staticmethod
    def forward(ctx, frac, lattice, graph: Graph):
        gb = graph.batch
        if (frac.data_ptr() == gb.frac.data_ptr() and lattice.data_ptr() == gb.lattice.data_ptr()
                and frac.shape == gb.frac.shape and lattice.shape == gb.lattice.shape
                and frac.is_contiguous() and lattice.is_contiguous()):
            batch = gb  # the graph's own coordinate buffers
        else:
            batch = gb.with_geometry(frac.detach().contiguous(), lattice.detach().contiguous())
        vec, ln = edge_vectors_fwd(graph, batch)
        E = graph.num_edges
        ctx.graph = graph
        ctx.batch = batch
        ctx.save_for_backward(vec, ln)
        ctx.set_materialize_grads(False)  # an unused output passes NULL, not a zero array
        return vec[:E], ln[:E]

    @staticmethod
    def backward(ctx, gvec, glen):
        vec, ln = ctx.saved_tensors
        g = ctx.graph
        gv = None if gvec is None else gvec.contiguous()
        gl = None if glen is None else glen.contiguous()
        # cutoff graphs need no destination order; other graphs need with_perm=True
        # (the library answers MG_ERR_INVALID_ARGUMENT otherwise)
        gf, gL = edge_vectors_bwd(g, ctx.batch, gv, gl, vec, ln)
        return gf, gL, None


def edge_vectors(frac: torch.Tensor, lattice: torch.Tensor, graph: Graph):
    """Differentiable (vec, len) of the graph's edges for coordinates frac and lattice."""
    return EdgeVectors.apply(frac, lattice, graph)
