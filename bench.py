#!/usr/bin/env python
"""Benchmark of the batched periodic-graph hot path on GB300.

One step = the whole path over one batch: the cutoff multigraph build (prep,
interplanar-box FP32 scan with FP64 re-test in the band; at this size the pair-lane
build over a cost-sorted work list, keys staged and written by a thread per edge), the
KNN build (a lane per target, candidates sorted in shared memory, adaptive radius,
FP64 ranking of the band; on a second stream) and the edge-vector forward and backward
passes on the cutoff graph.  Both builds replay their captured CUDA-graph plans
(mg_update_graph).  Units are edges built per step (cutoff + KNN).

Default workload: 8192 synthetic structures with a 70/25/5% mixture of 1-32, 33-128
and 129-400 atoms, 10% highly skewed cells; cutoff 6 A, k = 16 (--config 2: 256
structures with 1..64 atoms, log-uniform, lengths U[2.5,12] A, angles U[50,130] deg).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl mine|reference]
Prints one JSON line (rank 0).  With --sweep: the batch-size sweep of the KNN k = 32
build (Table 2's shape), one JSON line per batch size.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "edges/s batched vs per-structure build (+bwd), bit-exact edges; % roofline"
UNIT = "edges/s"
L2_FLUSH_BYTES = 256 << 20
FP32_LANES_PER_SM = 128
SMS = 152
WORKLOADS = {
    1: dict(cutoff=5.0, k=12, name="16 structures x 4-16 atoms, lengths U[3,8] A, cutoff 5 A, k=12"),
    2: dict(cutoff=6.0, k=16, name="256 structures x 1-64 atoms (log-uniform), lengths U[2.5,12] A, "
                                    "angles U[50,130] deg, cutoff 6 A, k=16"),
    3: dict(cutoff=6.0, k=16, name="8192 structures, 70/25/5% mixture up to 400 atoms, 10% skewed cells, "
                                    "cutoff 6 A, k=16"),
    4: dict(cutoff=5.0, k=16, name="1024 structures x 8-64 atoms, cutoff 5 A, k=16"),
    5: dict(cutoff=8.0, k=32, name="32 supercells of 1728-21952 atoms, cutoff 8 A, k=32"),
}
# Algorithmic work per unit of each stage (bytes or FP32 flops per edge, per atom).
# Edge record: src 4 + dst 4 + offset 12 + vec 12 + len 4 = 36 B.
STAGE_MODEL = {
    ("cutoff", "build"): ("hbm", 36.0, "cut"),
    ("knn", "knn"): ("hbm", 36.0, "knn"),
    ("fwd", "fwd"): ("hbm", 36.0, "cut"),
    ("bwd", "bwd_sym"): ("hbm", 36.0, "cut"),
    ("bwd", "bwd_src"): ("hbm", 36.0, "cut"),
    ("bwd", "bwd_dst"): ("hbm", 24.0, "cut"),
    ("bwd", "bwd_lat"): ("hbm", 0.0, "cut"),
}
# The other roofline term of a build: FP32 distance flops over the candidates in the cube
# around each atom's sphere (11 flops per candidate: 6 add/sub for v, 1 mul + 2 FMA for
# d^2), with (2r)^3 / (4/3 pi r^3) = 6/pi candidates per edge.
FLOPS_PER_CANDIDATE = 11.0
CANDIDATES_PER_EDGE = 6.0 / math.pi

# Stages that are one kernel launch; the roofline reports the slowest of these (the
# others bundle several launches: prep, the cell-list binning, the destination sort's
# histogram / scan / scatter / segment sort).
SINGLE_KERNEL_STAGES = {("cutoff", "build"), ("knn", "knn"), ("fwd", "fwd"),
                        ("bwd", "bwd_sym"), ("bwd", "bwd_src"), ("bwd", "bwd_dst"), ("bwd", "bwd_lat")}


def parse_args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=200)
    p.add_argument("--warmup", type=int, default=10)
    p.add_argument("--impl", default="mine", choices=["mine", "reference"])
    p.add_argument("--config", type=int, default=3, choices=sorted(WORKLOADS))
    p.add_argument("--no-baselines", action="store_true", help="skip the CPU oracle and per-structure legs")
    p.add_argument("--kernels-only", action="store_true",
                   help="setup, warm-up and the timed steps only (for profiler launch lists): no e2e, "
                        "per-structure, stage-time, float-error or CPU legs; the line says so")
    p.add_argument("--sweep", action="store_true", help="batch-size sweep of the KNN k=32 build")
    p.add_argument("--rows", action="store_true",
                   help="per-atom cutoff, keep-ties KNN, symmetric closure and triplets on --config")
    p.add_argument("--runs", action="store_true",
                   help="cutoff r = 4, 6, 8 and KNN k = 8, 16, 32 on --config, batched vs per structure")
    p.add_argument("--md", action="store_true",
                   help="the 20-step perturbation loop of the 1024-structure workload")
    p.add_argument("--link", action="store_true",
                   help="pinned host<->device copy bandwidth (the bound of the e2e numbers)")
    return p.parse_args()


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def replica_seed(config: int, rank: int) -> int:
    """Seed of rank `rank`'s batch: structures are independent units, so every rank builds
    its own full-size batch (weak scaling, no collective on the data path)."""
    import synth
    return synth.BASE_SEED + config + 1000 * rank


def reduce_over_ranks(units: float, ms: float, device) -> tuple:
    """Whole-job aggregate over the process group: edges summed over ranks, time the
    slowest rank's (the only cross-rank communication of the benchmark)."""
    import torch
    import torch.distributed as dist
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    m = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    dist.all_reduce(m, op=dist.ReduceOp.MAX)
    return float(u.item()), float(m.item())


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2307_05380_gb300", "csrc")
    for f in sorted(os.listdir(csrc)):
        h.update(f.encode())
        h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:16]


def fp32_term(edges, seconds, peak_tflops, peak_source):
    """The distance-flop side of a build's roofline, beside its edge-byte side."""
    per_edge = FLOPS_PER_CANDIDATE * CANDIDATES_PER_EDGE
    achieved = per_edge * edges / seconds / 1e12
    return {"achieved": achieved, "peak": peak_tflops, "unit": "TFLOP/s", "frac": achieved / peak_tflops,
            "work_per_launch": f"{per_edge:.1f} flop/edge (11 per candidate, 6/pi candidates per edge) x {edges} edges",
            "peak_source": peak_source}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return d.get("hbm_gbs", 6800.0), d.get("sm_max_mhz", 2070.0), "measured"
    return 6800.0, 2070.0, "fallback"


def recorded_traffic(config, stage_key):
    """DRAM bytes per launch from a committed ncu summary, if taken on this kernel source."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    d = json.load(open(path))
    ent = d.get(f"config{config}", {}).get(f"{stage_key[0]}.{stage_key[1]}")
    if not ent or ent.get("source_hash") != kernel_source_hash():
        return None
    return ent.get("bytes_per_launch")


class ClockSampler:
    """nvidia-smi clocks and throttle reasons while the timed region runs."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join("/tmp", f"mg_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = [r.split(",") for r in open(self.path).read().strip().splitlines() if r.strip()]
        os.unlink(self.path)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except (ValueError, IndexError):
                continue
            for name, val in zip(names, r[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------- reference arm

def run_reference(args, rank):
    """The FP64 oracle on the host cores, same workload, metric and unit."""
    if rank != 0:
        return 0
    import numpy as np

    import oracle
    import synth
    wl = WORKLOADS[args.config]
    b = synth.make_batch(args.config)
    sub, what = oracle_sample(args.config, b, first=64)

    def step():
        g = oracle.cutoff(sub.lattice, sub.frac, sub.atom_ptr, wl["cutoff"])
        h = oracle.knn(sub.lattice, sub.frac, sub.atom_ptr, wl["k"])
        vec, ln = oracle.edge_vectors(sub.lattice, sub.frac, sub.atom_ptr, g["src"], g["dst"], g["offset"])
        oracle.edge_grad(sub.lattice, sub.frac, sub.atom_ptr, g["src"], g["dst"], g["offset"], None, ln)
        return len(g["src"]) + len(h["src"])

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    edges = sum(step() for _ in range(args.steps))
    dt = time.perf_counter() - t0
    v = edges / dt
    sample = f"{what} per step"
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": wl["name"], "impl_note": "FP64 brute-force oracle, 1 thread"},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------- our arm

def oracle_sample(config, b, first=32, max_pairs=1.2e7):
    """The structures the host-side oracle legs time: the whole batch for the small
    workloads, the first `first` structures of the 8192-structure mixture, and for the
    supercells the smallest ones whose atom pairs (the brute force's cost, about 0.6 us
    each) stay within max_pairs, so that one pass takes seconds, not an hour."""
    import numpy as np
    if config in (1, 2, 4):
        return b, f"all {b.num_structures} structures"
    if config != 5:
        n = min(first, b.num_structures)
        return b.subset(range(n)), f"first {n} of {b.num_structures} structures"
    counts = np.diff(b.atom_ptr).astype(np.float64)
    take, tot = [], 0.0
    for s in np.argsort(counts, kind="stable"):
        if take and tot + counts[s] ** 2 > max_pairs:
            break
        take.append(int(s))
        tot += counts[s] ** 2
    take.sort()
    return b.subset(take), f"the {len(take)} smallest of {b.num_structures} supercells ({int(counts[take].sum())} atoms)"


def cpu_baseline_leg(args, b, wl, budget_s=12.0):
    import oracle
    sub, what = oracle_sample(args.config, b)
    edges, passes = 0, 0
    t0 = time.perf_counter()
    while True:
        g = oracle.cutoff(sub.lattice, sub.frac, sub.atom_ptr, wl["cutoff"])
        h = oracle.knn(sub.lattice, sub.frac, sub.atom_ptr, wl["k"])
        vec, ln = oracle.edge_vectors(sub.lattice, sub.frac, sub.atom_ptr, g["src"], g["dst"], g["offset"])
        oracle.edge_grad(sub.lattice, sub.frac, sub.atom_ptr, g["src"], g["dst"], g["offset"], None, ln)
        edges += len(g["src"]) + len(h["src"])
        passes += 1
        if time.perf_counter() - t0 >= budget_s:
            break
    dt = time.perf_counter() - t0
    return {"value": edges / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{passes} passes of cutoff+KNN+edge vectors+gradient over {what} "
                      f"({dt:.1f} s, single thread)"}


def cpu_info():
    """nproc and the CPU model of this host."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.startswith("Model name:"):
                model = ln.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    return os.cpu_count(), model


def _oracle_worker(payload):
    """One spawned process: passes of the oracle's step (cutoff + KNN + edge vectors +
    gradient) over its share of the structures for about budget_s seconds."""
    lat, frac, ptr, cutoff, k, budget_s = payload
    import oracle
    edges = passes = 0
    t0 = time.perf_counter()
    while True:
        g = oracle.cutoff(lat, frac, ptr, cutoff)
        h = oracle.knn(lat, frac, ptr, k)
        vec, ln = oracle.edge_vectors(lat, frac, ptr, g["src"], g["dst"], g["offset"])
        oracle.edge_grad(lat, frac, ptr, g["src"], g["dst"], g["offset"], None, ln)
        edges += len(g["src"]) + len(h["src"])
        passes += 1
        if time.perf_counter() - t0 >= budget_s:
            break
    return edges, passes, time.perf_counter() - t0


def cpu_baseline_threaded(sub, wl, budget_s=12.0):
    """The same oracle step threaded across structures: one spawned process per core, each
    on a contiguous range of structures of about equal cost (atoms squared); the rate is
    the sum of the processes' rates over their concurrent windows."""
    import multiprocessing as mp

    import numpy as np
    ncores = os.cpu_count() or 1
    counts = np.diff(sub.atom_ptr).astype(np.int64)
    cost = np.cumsum(counts * counts)
    cuts = [0] + [int(np.searchsorted(cost, cost[-1] * q / ncores, side="right")) for q in range(1, ncores)] \
        + [sub.num_structures]
    payloads = []
    for lo, hi in zip(cuts[:-1], cuts[1:]):
        if hi <= lo:
            continue
        a0, a1 = int(sub.atom_ptr[lo]), int(sub.atom_ptr[hi])
        payloads.append((sub.lattice[lo:hi].copy(), sub.frac[a0:a1].copy(),
                         (sub.atom_ptr[lo:hi + 1] - a0).astype(np.int32), wl["cutoff"], wl["k"], budget_s))
    with mp.get_context("spawn").Pool(len(payloads)) as pool:
        res = pool.map(_oracle_worker, payloads)
    return sum(e / dt for e, _, dt in res), len(payloads)


def float_errors(b, g_cut, g_knn, grad_len, grad_frac, grad_lat, seed=7, edge_sample=1 << 20, struct_sample=64):
    """Error of every float output against the FP64 oracle, outside every timed region:
    vec and len of both graphs on a uniform sample of edges (relative to the exact
    length), and grad_frac / grad_lattice of the step's backward on a sample of whole
    structures (the gradient of a structure depends on its edges only).  Gradient errors
    are given relative to the oracle's norm (per atom and per structure) and in units of
    the condition-aware scale sum_e |contribution| per component."""
    import numpy as np
    import torch

    import oracle
    rng = np.random.default_rng(seed)
    out = {}
    for name, g in (("cutoff", g_cut), ("knn", g_knn)):
        E = g.num_edges
        idx = np.sort(rng.choice(E, min(E, edge_sample), replace=False)) if E else np.zeros(0, np.int64)
        ti = torch.from_numpy(idx).to(g.src.device)
        src, dst, off = g.src[ti].cpu().numpy(), g.dst[ti].cpu().numpy(), g.offset[ti].cpu().numpy()
        vec, ln = g.vec[ti].cpu().numpy().astype(np.float64), g.len[ti].cpu().numpy().astype(np.float64)
        ov, ol = oracle.edge_vectors(b.lattice, b.frac, b.atom_ptr, src, dst, off)
        out[f"{name}_len_rel_max"] = float(np.max(np.abs(ln - ol) / ol, initial=0))
        out[f"{name}_vec_rel_max"] = float(np.max(np.linalg.norm(vec - ov, axis=1) / ol, initial=0))
        out[f"{name}_edges_sampled"] = int(len(idx))
    B = b.num_structures
    structs = np.sort(rng.choice(B, min(B, struct_sample), replace=False))
    edge_ptr = g_cut.edge_ptr.cpu().numpy()
    gl_all = grad_len.cpu().numpy().astype(np.float64)
    gf_gpu = grad_frac.cpu().numpy().astype(np.float64)
    gL_gpu = grad_lat.cpu().numpy().astype(np.float64).reshape(-1, 3, 3)
    f_rel = L_rel = f_cond = L_cond = 0.0
    for s in structs:
        e0, e1 = int(edge_ptr[s]), int(edge_ptr[s + 1])
        a0, a1 = int(b.atom_ptr[s]), int(b.atom_ptr[s + 1])
        if e1 == e0:
            continue
        sub = b.subset([int(s)])
        src = g_cut.src[e0:e1].cpu().numpy() - a0
        dst = g_cut.dst[e0:e1].cpu().numpy() - a0
        off = g_cut.offset[e0:e1].cpu().numpy()
        gl = gl_all[e0:e1]
        gf, gL = oracle.edge_grad(sub.lattice, sub.frac, sub.atom_ptr, src, dst, off, None, gl)
        df_err = np.abs(gf_gpu[a0:a1] - gf)
        dL_err = np.abs(gL_gpu[s] - gL[0])
        nf = np.linalg.norm(gf, axis=1)
        ok = nf > 0
        if ok.any():
            f_rel = max(f_rel, float(np.max(np.linalg.norm(gf_gpu[a0:a1] - gf, axis=1)[ok] / nf[ok])))
        if np.linalg.norm(gL[0]) > 0:
            L_rel = max(L_rel, float(np.linalg.norm(gL_gpu[s] - gL[0]) / np.linalg.norm(gL[0])))
        # condition-aware scale: |g_e,c| <= |grad_len_e|, edge e adds +-g_e L^T and df^T g_e
        Lt = np.abs(sub.lattice[0].astype(np.float64))
        h = np.abs(gl)[:, None] * Lt.sum(axis=1)[None, :]
        scale_f = np.zeros((a1 - a0, 3))
        np.add.at(scale_f, src, h)
        np.add.at(scale_f, dst, h)
        dfr = np.abs(sub.frac[dst].astype(np.float64) - sub.frac[src] + off)
        scale_L = (dfr[:, :, None] * np.abs(gl)[:, None, None] * np.ones((1, 1, 3))).sum(axis=0)
        f_cond = max(f_cond, float(np.max(df_err / (scale_f + 1e-30))))
        L_cond = max(L_cond, float(np.max(dL_err / (scale_L + 1e-30))))
    out.update({"grad_frac_rel_max": f_rel, "grad_lattice_rel_max": L_rel,
                "grad_frac_cond_max": f_cond, "grad_lattice_cond_max": L_cond,
                "structures_sampled": int(len(structs)),
                "how": "vec/len: |x - x64| / len64 over sampled edges of both graphs; gradients of the step's "
                       "backward (loss sum w*len) on sampled structures: per-atom / per-structure norm-wise "
                       "relative error, and max |err| / sum_e |contribution| per component (cond)"})
    return out


def run_mine(args, rank, world, local_rank):
    import numpy as np
    import torch

    import paper_2307_05380_gb300 as mg
    import synth

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    # explicit streams: the legacy default stream cannot be captured into the plans that
    # mg_update_graph replays; the KNN build runs on a second stream, concurrently
    main_stream = torch.cuda.Stream(dev)
    knn_stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(main_stream)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    wl = WORKLOADS[args.config]
    # weak scaling: every rank builds its own seeded batch of the full workload size
    b = synth.make_batch(args.config, seed=replica_seed(args.config, rank))
    batch = mg.Batch(torch.from_numpy(b.frac).to(dev), torch.from_numpy(b.lattice).to(dev),
                     torch.from_numpy(b.atom_ptr).to(dev), max_atoms=b.max_atoms)
    # schedules per size class from the per-device autotune cache (measured here, outside
    # every timed region, when the device or the library's sources are new to it)
    tune = {"cutoff": mg.autotune_cached(batch, "cutoff", cutoff=wl["cutoff"]),
            "knn": mg.autotune_cached(batch, "knn", k=wl["k"])}
    # the cutoff graph is symmetric: its backward needs no destination order, so the
    # optional perm_dst output is not requested; the step differentiates through the
    # cutoff graph only, so the KNN graph's destination order is not requested either
    g_cut = mg.cutoff_graph(batch, wl["cutoff"], with_perm=False)
    g_knn = mg.knn_graph(batch, wl["k"], with_perm=False)
    E_cut, E_knn = g_cut.num_edges, g_knn.num_edges
    units = E_cut + E_knn
    # share of the FP32 candidates re-tested in FP64 (a counting build, outside every timed region)
    st_stats = mg.cutoff_graph(batch, wl["cutoff"], with_perm=False, capacity=g_cut.capacity,
                               opts=mg.make_opts(collect_stats=True)).read_status()
    fp64_recheck = {"graph": "cutoff", "candidates": st_stats["candidates"], "rechecked": st_stats["rechecked"],
                    "fraction": st_stats["rechecked"] / max(1, st_stats["candidates"])}
    grad_len = torch.from_numpy(synth.normal(17, 0, g_cut.capacity)).to(dev)
    out_vec = torch.empty(g_cut.capacity, 3, device=dev)
    out_len = torch.empty(g_cut.capacity, device=dev)
    grad_frac = torch.empty(batch.N, 3, device=dev)
    grad_lat = torch.empty(batch.B, 3, 3, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    launches = {"n": 0}

    ev_fork = torch.cuda.Event()
    ev_join = torch.cuda.Event()

    def step():
        n = 0
        ev_fork.record(main_stream)
        knn_stream.wait_event(ev_fork)
        torch.cuda.set_stream(knn_stream)
        mg.update_graph(g_knn, sync=False)
        n += mg.last_launch_count(dev)
        torch.cuda.set_stream(main_stream)
        ev_join.record(knn_stream)
        mg.update_graph(g_cut, sync=False)
        n += mg.last_launch_count(dev)
        mg.edge_vectors_fwd(g_cut, out_vec=out_vec, out_len=out_len)
        n += mg.last_launch_count(dev)
        mg.edge_vectors_bwd(g_cut, batch, None, grad_len, out_vec, out_len, grad_frac, grad_lat)
        n += mg.last_launch_count(dev)
        main_stream.wait_event(ev_join)  # the step ends when both builds are done
        launches["n"] += n

    for _ in range(max(3, args.warmup)):
        flush.zero_()
        step()
    torch.cuda.synchronize(dev)
    st = g_cut.read_status()
    sk = g_knn.read_status()
    assert st["code"] == 0 and sk["code"] == 0 and g_cut.num_edges == E_cut, (st, sk)

    # the library's stage events stay off in the warm-up, the timed steps and e2e (an event
    # between two kernels would also keep a kernel from launching behind the one before
    # it); the serialized per-stage pass below turns them on, and the plans are recorded
    # again with their events
    sampler = ClockSampler(local_rank)
    sampler.start()
    time.sleep(0.3)
    stage_tot: dict = {}
    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    launches["n"] = 0
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize(dev)
    t_wall = time.perf_counter()
    torch.cuda.nvtx.range_push("timed_steps")  # lets a profiler select the timed region
    for s in range(args.steps):
        flush.zero_()  # L2 flush between timed steps (outside the events)
        ev0[s].record(stream)
        step()
        ev1[s].record(stream)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize(dev)
    t_wall = time.perf_counter() - t_wall
    if world > 1:
        torch.distributed.barrier()
    step_ms = [ev0[s].elapsed_time(ev1[s]) for s in range(args.steps)]
    total_ms = sum(step_ms)
    gpu_launches = launches["n"]

    # whole-job aggregate: all ranks' edges over the slowest rank's time
    tot_units, max_ms = units * args.steps, total_ms
    if world > 1:
        tot_units, max_ms = reduce_over_ranks(tot_units, max_ms, dev)
    value = tot_units / (max_ms / 1e3)
    if args.kernels_only:
        sampler.stop()
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                              "warmup": args.warmup, "ms_per_step": max_ms / args.steps, "higher_is_better": True,
                              "kernels_only": True, "gpu_launches": gpu_launches,
                              "config": {"workload": wl["name"], "edges_per_step": {"cutoff": E_cut, "knn": E_knn}}}),
                  flush=True)
        if world > 1:
            torch.distributed.destroy_process_group()
        return 0

    # e2e: the step (both graph updates, forward, backward with the loss gradient) from
    # pinned host inputs to pinned host outputs.  Every step copies the inputs in and every
    # output back: both graphs' edges, status words, vectors and gradients.  Each graph's
    # copy is issued right behind its build, on another stream, so the copies overlap the
    # rest of the step; the step's outputs follow the backward.  The host waits once, at
    # the end, then checks both status words.
    frac_h = torch.from_numpy(b.frac).pin_memory()
    lat_h = torch.from_numpy(b.lattice).pin_memory()
    ptr_h = torch.from_numpy(b.atom_ptr).pin_memory()
    w_dev = grad_len  # dLoss/dlen of the loss sum(w * len)
    e2e_steps = max(5, min(args.steps, 50))
    copy_stream = torch.cuda.Stream(dev)
    host_knn = mg.host_buffers(g_knn, E_knn, ("status", "src", "dst", "offset", "vec", "len"))
    host_cut = mg.host_buffers(g_cut, E_cut, ("status", "src", "dst", "offset"))
    step_out = (out_vec[:E_cut], out_len[:E_cut], grad_frac, grad_lat)
    host_step = [torch.empty(t.shape, dtype=t.dtype, pin_memory=True) for t in step_out]
    d2h = sum(t.numel() * t.element_size() for t in list(host_knn.values()) + list(host_cut.values()) + host_step)

    # the whole step through one library call (mg_graph_step): inputs in, both graphs
    # rebuilt (KNN on its own stream) and copied out (the cutoff graph's copy on the copy
    # stream), edge vectors and backward, results out; one synchronisation per step
    out_host = {"vec": host_step[0], "len": host_step[1], "grad_frac": host_step[2], "grad_lattice": host_step[3]}
    step_call = mg.Step([g_cut, g_knn], [main_stream, knn_stream, copy_stream], host=(host_cut, host_knn),
                        inputs={"frac": frac_h, "lattice": lat_h, "atom_ptr": ptr_h}, grad_len=w_dev, vec=out_vec,
                        ln=out_len, grad_frac=grad_frac, grad_lattice=grad_lat, outputs=out_host,
                        host_edges=(E_cut, E_knn))

    def e2e_step():
        step_call.run()
        main_stream.synchronize()
        for st_h, E in ((host_cut["status"], E_cut), (host_knn["status"], E_knn)):  # code 0, same edge count
            assert int(st_h[0]) & 0xFFFFFFFF == 0 and int(st_h[1]) == E, st_h
        return E_cut + E_knn, d2h

    e2e_step()
    e2e_t, e2e_units = 0.0, 0
    for _ in range(e2e_steps):
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        u_, _ = e2e_step()
        e2e_t += time.perf_counter() - t0
        e2e_units += u_
    mg.profile_enable(True, dev)
    h2d = (frac_h.numel() * 4 + lat_h.numel() * 4 + ptr_h.numel() * 4)
    e2e_val = e2e_units / e2e_t
    if world > 1:  # e2e throughput of the replicas adds up
        e2e_val, _ = reduce_over_ranks(e2e_val, 0.0, dev)

    # plain comparison: the same kernels, one launch sequence per structure
    per_structure = None
    if not args.no_baselines:
        ap_host = b.atom_ptr.tolist()
        ps_cut = mg.cutoff_graph(batch, wl["cutoff"], capacity=E_cut)
        ps_knn = mg.knn_graph(batch, wl["k"], with_perm=False)
        ps_ms = []
        for rep in range(4):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            mg.rebuild(ps_cut, sync=False, per_structure=True, atom_ptr_host=ap_host)
            mg.rebuild(ps_knn, sync=False, per_structure=True, atom_ptr_host=ap_host)
            mg.edge_vectors_fwd(ps_cut, out_vec=out_vec, out_len=out_len)
            mg.edge_vectors_bwd(ps_cut, batch, None, grad_len, out_vec, out_len, grad_frac, grad_lat)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            if rep:
                ps_ms.append(e0.elapsed_time(e1))
        assert ps_cut.read_status()["num_edges"] == E_cut
        ps_step = statistics.mean(ps_ms)
        per_structure = {"value": units / (ps_step / 1e3), "unit": UNIT, "ms_per_step": ps_step,
                         "speedup_batched": ps_step / (total_ms / args.steps)}

    # Per-kernel timing for the roofline: the same steps with both builds serialized on
    # one stream (concurrent streams would make stage events overlap other kernels),
    # CUDA events recorded by the library between its kernels, L2 flushed between steps.
    n_roof = max(5, min(args.steps, 50))
    for _ in range(n_roof):
        flush.zero_()
        mg.update_graph(g_knn, sync=False)
        mg.update_graph(g_cut, sync=False)
        mg.edge_vectors_fwd(g_cut, out_vec=out_vec, out_len=out_len)
        mg.edge_vectors_bwd(g_cut, batch, None, grad_len, out_vec, out_len, grad_frac, grad_lat)
        for which in ("cutoff", "knn", "fwd", "bwd"):
            for name, ms in mg.stage_times(which, dev).items():
                stage_tot[(which, name)] = stage_tot.get((which, name), 0.0) + ms

    clocks = sampler.stop()
    ferr = None
    if rank == 0 and not args.no_baselines:
        torch.cuda.synchronize(dev)
        ferr = float_errors(b, g_cut, g_knn, grad_len[:E_cut], grad_frac, grad_lat)

    # roofline of the dominant stage
    hbm_peak, sm_max, peak_src = measured_peaks()
    # the FP32 peak measured by the library's own FMA kernel (CUDA events, no clock
    # setting touched), the nominal lanes x clock beside it
    fp_peaks = mg.measure_fp_peaks(dev)
    fp32_nominal = SMS * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12  # TFLOP/s
    fp32_peak = fp_peaks["fp32_tflops"]
    fp32_src = (f"measured: library FFMA kernel, 16 chains per thread, full occupancy "
                f"({fp32_peak:.1f} TFLOP/s; nominal 152 SM x 128 lanes x 2 x {sm_max:.0f} MHz = {fp32_nominal:.1f})")
    stages = {f"{k[0]}.{k[1]}": v / n_roof for k, v in stage_tot.items()}
    # the staged cutoff build (large batches) is three stages: scan and stage the keys,
    # scan the counts, write the edges; its edge emission is the unit of the roofline
    staged = ("cutoff", "stage") in stage_tot
    pair_lane = ("cutoff", "plan") in stage_tot
    if staged:
        stage_tot[("cutoff", "build")] = sum(stage_tot.get(("cutoff", k), 0.0)
                                             for k in ("plan", "stage", "count_scan", "emit"))
    singles = {k: v for k, v in stage_tot.items() if k in SINGLE_KERNEL_STAGES and k in STAGE_MODEL}
    dom = max(singles, key=singles.get)
    bound, per_unit, which_units = STAGE_MODEL.get(dom, ("hbm", 36.0, "cut"))
    n_units = E_cut if which_units == "cut" else E_knn
    t_launch = stage_tot[dom] / n_roof / 1e3
    if bound == "hbm":
        achieved = per_unit * n_units / t_launch / 1e9
        roof = {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                "frac": achieved / hbm_peak}
    else:
        achieved = per_unit * n_units / t_launch / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
                "frac": achieved / fp32_peak}
    roof["kernel"] = f"{dom[0]}.{dom[1]}"
    if pair_lane and dom == ("cutoff", "build"):
        roof["kernel"] += " (pair-lane: cost-sorted plan, stage, count scan, emit; 9 launches)"
    elif staged and dom == ("cutoff", "build"):
        roof["kernel"] += " (staged: scan-and-stage, count scan, emit; 7 launches)"
    roof["peak_source"] = f"{peak_src} ({'MEASURED_PEAKS.json hbm_gbs' if bound == 'hbm' else fp32_src})"
    roof["traffic"] = recorded_traffic(args.config, dom)
    roof["work_per_launch"] = f"{per_unit:g} {'B' if bound == 'hbm' else 'flop'}/edge x {n_units} edges"
    if dom in (("cutoff", "build"), ("knn", "knn")):
        roof["fp32_term"] = fp32_term(n_units, t_launch, fp32_peak, fp32_src)

    if rank == 0:
        cpu = None
        if world == 1 and not args.no_baselines:
            cpu = cpu_baseline_leg(args, b, wl)
            nproc, model = cpu_info()
            sub, _ = oracle_sample(args.config, b)
            rate, procs = cpu_baseline_threaded(sub, wl)
            cpu.update({"nproc": nproc, "cpu_model": model,
                        "threaded": {"value": rate, "unit": UNIT, "cores": procs,
                                     "note": "the same oracle step, one spawned process per core on "
                                             "cost-balanced structure ranges"}})
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "fp64_recheck": fp64_recheck,
                "warmup": args.warmup, "ms_per_step": max_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": wl["name"], "structures": b.num_structures, "atoms": b.total_atoms,
                           "cutoff_A": wl["cutoff"], "k": wl["k"], "edges_per_step": {"cutoff": E_cut, "knn": E_knn},
                           "l2": "flushed between timed steps (256 MiB write, outside the step events)",
                           "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                           "step": "cutoff build + KNN build (CUDA-graph plans) + edge-vector fwd + bwd on the "
                                   "cutoff graph; destination orders not requested (unused by the step)"},
                "roofline": roof, "cpu_baseline": cpu, "float_error": ferr, "fp_peaks_measured": fp_peaks,
                "autotune": {kd: {"schedule": v["schedule"], "size_class": v["size_class"], "tuned_now": v["tuned_now"]}
                             for kd, v in tune.items()},
                "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
                "gpu_launches": gpu_launches, "clocks": clocks, "per_structure": per_structure,
                "stage_ms_per_step": stages, "wall_s_timed_region": t_wall}
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


SWEEP_BATCHES = (32, 64, 128, 256, 512)
SWEEP_K = 32
DATASET_STRUCTURES = 119701  # structures of the paper's filtered dataset (Sec. 3)


def run_sweep(args, local_rank):
    """Time of one KNN k=32 build per batch size (plan replay, L2 flushed between
    batches) and the device memory it holds (workspace + graph buffers), on batches of
    the default workload's recipe; the dataset column scales the batch time to the
    paper's structure count (Table 2's columns, synthetic stand-in)."""
    import torch

    import paper_2307_05380_gb300 as mg
    import synth

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    steps = max(5, min(args.steps, 200))
    for B in SWEEP_BATCHES:
        b = synth.make_batch(2, B=B)
        batch = mg.Batch(torch.from_numpy(b.frac).to(dev), torch.from_numpy(b.lattice).to(dev),
                         torch.from_numpy(b.atom_ptr).to(dev), max_atoms=b.max_atoms)
        g = mg.knn_graph(batch, SWEEP_K, with_perm=False)
        held = g.ws.numel() + sum(t.numel() * t.element_size() for t in
                                  (g.src, g.dst, g.offset, g.vec, g.len, g.edge_ptr, g.src_ptr, g.status))
        for _ in range(max(3, args.warmup)):
            mg.update_graph(g, sync=False)
        ms = []
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        for _ in range(steps):
            flush.zero_()
            e0.record(stream)
            mg.update_graph(g, sync=False)
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        st = g.read_status()
        assert st["code"] == 0, st
        t = statistics.median(ms)
        print(json.dumps({"sweep": f"knn k={SWEEP_K} batch size", "batch": B, "atoms": b.total_atoms,
                          "edges": g.num_edges, "ms_per_batch": t, "structures_per_s": B / t * 1e3,
                          "edges_per_s": g.num_edges / t * 1e3, "device_bytes": int(held),
                          "dataset_s": DATASET_STRUCTURES / B * t / 1e3, "steps": steps,
                          "timing": "CUDA events around each plan replay, median; L2 flushed between batches"}),
              flush=True)
    return 0


def run_rows(args, local_rank):
    """Throughput and HBM roofline of the operations after the hot path, one JSON line
    each, on the --config workload: per-atom cutoff build (radii U[0.75 c, c]), keep-ties
    KNN build, symmetric closure of the KNN graph, triplets of the cutoff graph.  Builds
    replay their plans; closure and triplets call the C-ABI on preallocated buffers.  L2
    is flushed between iterations; CUDA events around each call, median."""
    import ctypes

    import numpy as np
    import torch

    import paper_2307_05380_gb300 as mg
    import synth
    from paper_2307_05380_gb300 import _capi
    from paper_2307_05380_gb300.graph import MgTriplets, _stream, context

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    hbm_peak, _, peak_src = measured_peaks()
    wl = WORKLOADS[args.config]
    b = synth.make_batch(args.config)
    batch = mg.Batch(torch.from_numpy(b.frac).to(dev), torch.from_numpy(b.lattice).to(dev),
                     torch.from_numpy(b.atom_ptr).to(dev), max_atoms=b.max_atoms)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    steps = max(5, min(args.steps, 100))
    lib = _capi.load()
    ctx = context(dev)

    def timed(fn):
        for _ in range(max(3, args.warmup)):
            fn()
        ms = []
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        for _ in range(steps):
            flush.zero_()
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        return statistics.median(ms)

    def line(op, units, unit_name, ms, bytes_per_unit, note):
        gbs = units * bytes_per_unit / ms / 1e6
        print(json.dumps({"row": op, "workload": wl["name"], "units": int(units), "unit": unit_name,
                          "ms": ms, "units_per_s": units / ms * 1e3,
                          "roofline": {"bound": "hbm", "achieved": gbs, "peak": hbm_peak, "unit": "GB/s",
                                       "frac": gbs / hbm_peak, "peak_source": peak_src,
                                       "work_per_unit": note}, "steps": steps}), flush=True)

    radii = np.random.default_rng(args.config).uniform(0.75 * wl["cutoff"], wl["cutoff"], b.total_atoms)
    g_atoms = mg.cutoff_graph_atoms(batch, torch.from_numpy(radii.astype(np.float32)).to(dev), with_perm=False)
    ms = timed(lambda: mg.update_graph(g_atoms, sync=False))
    assert g_atoms.read_status()["code"] == 0
    line("cutoff graph, per-atom radii", g_atoms.num_edges, "edges", ms, 36.0, "36 B written per edge")

    g_ties = mg.knn_graph(batch, wl["k"], keep_ties=True, with_perm=False)
    ms = timed(lambda: mg.update_graph(g_ties, sync=False))
    assert g_ties.read_status()["code"] == 0
    line(f"knn graph k={wl['k']}, keep ties", g_ties.num_edges, "edges", ms, 36.0, "36 B written per edge")

    g_knn = mg.knn_graph(batch, wl["k"])
    sym = mg.symmetrize(g_knn)
    E_in = g_knn.num_edges
    ms = timed(lambda: _capi.check(lib.mg_symmetrize(ctx, ctypes.byref(batch.c), ctypes.byref(g_knn.c),
                                                     ctypes.byref(sym.c), sym.ws.data_ptr(), sym.ws.numel(),
                                                     _stream(dev)), "mg_symmetrize"))
    assert sym.read_status()["code"] == 0
    line(f"symmetric closure of the knn graph k={wl['k']}", sym.num_edges, "edges", ms,
         40.0 + 24.0 * E_in / sym.num_edges,
         "40 B written per output edge (36 + perm_dst 4) + 24 B read per input edge (dst, offset, perm, src)")

    g_cut = mg.cutoff_graph(batch, wl["cutoff"], with_perm=False)
    tr = mg.triplets(g_cut)
    T = tr.count
    status = torch.zeros(5, dtype=torch.int64, device=dev)
    nbytes = ctypes.c_size_t(0)
    lib.mg_workspace_size(ctx, ctypes.byref(batch.c), 0, ctypes.byref(nbytes))
    ws = torch.empty(int(nbytes.value), dtype=torch.uint8, device=dev)
    out = MgTriplets(T, tr.edge_a.data_ptr(), tr.edge_b.data_ptr(), tr.trip_ptr.data_ptr(), status.data_ptr())
    ms = timed(lambda: _capi.check(lib.mg_triplets(ctx, ctypes.byref(batch.c), ctypes.byref(g_cut.c), 1,
                                                   ctypes.byref(out), ws.data_ptr(), ws.numel(), _stream(dev)),
                                   "mg_triplets"))
    assert int(status.cpu()[1]) == T
    line("triplets of the cutoff graph", T, "triplets", ms, 8.0 + 8.0 * g_cut.num_edges / T,
         "8 B written per triplet (two edge ids) + 8 B per edge (trip_ptr)")
    return 0


def run_runs(args, local_rank):
    """The radius and k runs of the --config workload (cutoff r = 4, 6, 8 A; KNN k = 8, 16,
    32), one JSON line each: the batched build (plan replay, CUDA events, median; L2
    flushed between builds) against the same kernels launched once per structure (mean of
    three), with the HBM roofline of 36 B per edge written."""
    import torch

    import paper_2307_05380_gb300 as mg
    import synth

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    hbm_peak, _, peak_src = measured_peaks()
    wl = WORKLOADS[args.config]
    b = synth.make_batch(args.config)
    batch = mg.Batch(torch.from_numpy(b.frac).to(dev), torch.from_numpy(b.lattice).to(dev),
                     torch.from_numpy(b.atom_ptr).to(dev), max_atoms=b.max_atoms)
    ap_host = b.atom_ptr.tolist()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    steps = max(5, min(args.steps, 50))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn, n):
        ms = []
        for _ in range(n):
            flush.zero_()
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        return ms

    runs = [("cutoff", r, 0) for r in (4.0, 6.0, 8.0)] + [("knn", 0.0, k) for k in (8, 16, 32)]
    for kind, r, k in runs:
        g = mg.cutoff_graph(batch, r, with_perm=False) if kind == "cutoff" else mg.knn_graph(batch, k, with_perm=False)
        for _ in range(max(3, args.warmup)):
            mg.update_graph(g, sync=False)
        t = statistics.median(timed(lambda: mg.update_graph(g, sync=False), steps))
        assert g.read_status()["code"] == 0
        E = g.num_edges
        ps = mg.cutoff_graph(batch, r, with_perm=False, capacity=E) if kind == "cutoff" \
            else mg.knn_graph(batch, k, with_perm=False)
        tp = statistics.mean(timed(lambda: mg.rebuild(ps, sync=False, per_structure=True, atom_ptr_host=ap_host),
                                   3))
        assert ps.read_status()["num_edges"] == E
        gbs = 36.0 * E / t / 1e6
        print(json.dumps({"run": f"{kind} {'r = %g A' % r if kind == 'cutoff' else 'k = %d' % k}",
                          "workload": wl["name"], "edges": E, "ms": t, "edges_per_s": E / t * 1e3,
                          "per_structure_ms": tp, "speedup_batched": tp / t,
                          "roofline": {"bound": "hbm", "achieved": gbs, "peak": hbm_peak, "unit": "GB/s",
                                       "frac": gbs / hbm_peak, "peak_source": peak_src,
                                       "work_per_unit": "36 B written per edge"}, "steps": steps}), flush=True)
        del g, ps
    return 0


def run_md(args, local_rank):
    """The perturbation loop of the 1024-structure workload: 20 steps of (seeded
    perturbation x += N(0, 0.02), 1% strain) -> graph update (plan replay) -> edge vectors
    -> backward of the Gaussian edge loss sum_e w_e exp(-len_e^2 / 2 sigma^2), sigma = 1.5.
    Every step's coordinates are generated on the host beforehand and held on the device;
    each step copies its own into the batch buffers.  The edge count of every step is
    kept on the device and read once, after the timed loop; CUDA events around the 20
    steps (a loop: no L2 flush inside)."""
    import torch

    import paper_2307_05380_gb300 as mg
    import synth

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    cfg, nsteps, sigma = 4, 20, 1.5
    wl = WORKLOADS[cfg]
    traj = [synth.make_batch(cfg)]
    for t in range(1, nsteps + 1):
        traj.append(synth.perturb(traj[-1], seed=41, step=t))
    fr_d = torch.stack([torch.from_numpy(x.frac) for x in traj[1:]]).to(dev)
    la_d = torch.stack([torch.from_numpy(x.lattice) for x in traj[1:]]).to(dev)
    b0 = traj[0]
    batch = mg.Batch(torch.from_numpy(b0.frac).to(dev), torch.from_numpy(b0.lattice).to(dev),
                     torch.from_numpy(b0.atom_ptr).to(dev), max_atoms=b0.max_atoms)
    E0 = mg.cutoff_graph(batch, wl["cutoff"], with_perm=False).num_edges
    g = mg.cutoff_graph(batch, wl["cutoff"], with_perm=False, capacity=int(1.3 * E0))
    w = torch.from_numpy(synth.normal(43, 0, g.capacity)).to(dev)
    out_vec = torch.empty(g.capacity, 3, device=dev)
    out_len = torch.empty(g.capacity, device=dev)
    grad_frac = torch.empty(batch.N, 3, device=dev)
    grad_lat = torch.empty(batch.B, 3, 3, device=dev)
    counts = torch.zeros(nsteps, 2, dtype=torch.int64, device=dev)

    def loop():
        for t in range(nsteps):
            batch.frac.copy_(fr_d[t])
            batch.lattice.copy_(la_d[t])
            mg.update_graph(g, sync=False)
            mg.edge_vectors_fwd(g, out_vec=out_vec, out_len=out_len)
            gl = -w * out_len / (sigma * sigma) * torch.exp(-out_len * out_len / (2 * sigma * sigma))
            mg.edge_vectors_bwd(g, batch, None, gl, out_vec, out_len, grad_frac, grad_lat)
            counts[t].copy_(g.status[:2])

    # the plain comparison: the same loop with every graph built by the same kernels
    # launched once per structure (a per-structure graph is not recorded as symmetric, so
    # its backward goes through the destination order it also builds)
    ap_host = b0.atom_ptr.tolist()
    ps = mg.cutoff_graph(batch, wl["cutoff"], with_perm=True, capacity=int(1.3 * E0))
    ps_counts = torch.zeros(nsteps, 2, dtype=torch.int64, device=dev)

    def loop_per_structure():
        for t in range(nsteps):
            batch.frac.copy_(fr_d[t])
            batch.lattice.copy_(la_d[t])
            mg.rebuild(ps, sync=False, per_structure=True, atom_ptr_host=ap_host)
            mg.edge_vectors_fwd(ps, out_vec=out_vec, out_len=out_len)
            gl = -w * out_len / (sigma * sigma) * torch.exp(-out_len * out_len / (2 * sigma * sigma))
            mg.edge_vectors_bwd(ps, batch, None, gl, out_vec, out_len, grad_frac, grad_lat)
            ps_counts[t].copy_(ps.status[:2])

    def timed(fn):
        for _ in range(max(1, args.warmup // 3)):
            fn()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1)

    ms = timed(loop)
    ms_ps = timed(loop_per_structure)
    c = counts.cpu()
    cp = ps_counts.cpu()
    assert all(int(x) & 0xFFFFFFFF == 0 for x in c[:, 0]), c
    assert torch.equal(c[:, 1], cp[:, 1]), (c, cp)  # the same edge count every step
    edges = int(c[:, 1].sum())
    print(json.dumps({"md": "perturbation loop: update -> edge vectors -> Gaussian-loss backward",
                      "workload": wl["name"], "steps": nsteps, "edges_per_step_mean": edges / nsteps,
                      "edges_min_max": [int(c[:, 1].min()), int(c[:, 1].max())], "ms_per_step": ms / nsteps,
                      "edges_per_s": edges / ms * 1e3,
                      "per_structure": {"ms_per_step": ms_ps / nsteps, "edges_per_s": edges / ms_ps * 1e3,
                                        "speedup_batched": ms_ps / ms,
                                        "how": "the same loop, every graph built by mg_build_per_structure "
                                               "(one launch sequence per structure) with its destination order"},
                      "timing": "CUDA events around the 20 steps"}), flush=True)
    return 0


def run_link(args, local_rank):
    """Pinned host memory <-> device copy bandwidth by the copy engines (what the e2e
    step's copies run at): one line per size and direction, the best of the
    repetitions, CUDA events around each copy; also several copies on separate streams
    at once."""
    import torch
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    reps = max(5, min(args.steps, 50))
    for mb in (2, 16, 256, 1024):
        n = (mb << 20) // 4
        d = torch.empty(n, dtype=torch.float32, device=dev).fill_(1.0)
        h = torch.empty(n, dtype=torch.float32, pin_memory=True)
        for name, dst, src in (("D2H", h, d), ("H2D", d, h)):
            best = 1e30
            for _ in range(reps):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record()
                dst.copy_(src, non_blocking=True)
                e1.record()
                torch.cuda.synchronize(dev)
                best = min(best, e0.elapsed_time(e1))
            print(json.dumps({"link": name, "MB": mb, "ms": best, "GB_per_s": (mb << 20) / best / 1e6,
                              "how": "one pinned copy, best of %d, CUDA events" % reps}), flush=True)
    # four D2H copies of 256 MB on four streams at once
    streams = [torch.cuda.Stream(dev) for _ in range(4)]
    n = (256 << 20) // 4
    ds = [torch.empty(n, dtype=torch.float32, device=dev).fill_(1.0) for _ in streams]
    hs = [torch.empty(n, dtype=torch.float32, pin_memory=True) for _ in streams]
    best = 1e30
    for _ in range(reps):
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for st, d_, h_ in zip(streams, ds, hs):
            with torch.cuda.stream(st):
                h_.copy_(d_, non_blocking=True)
        torch.cuda.synchronize(dev)
        best = min(best, time.perf_counter() - t0)
    print(json.dumps({"link": "D2H x4 streams", "MB": 4 * 256, "ms": best * 1e3,
                      "GB_per_s": 4 * (256 << 20) / best / 1e9,
                      "how": "four pinned copies on four streams, host clock around all four"}), flush=True)
    return 0


def main():
    args = parse_args()
    rank, world, local_rank = dist_env()
    if args.impl == "reference":
        return run_reference(args, rank)
    if args.sweep:
        return run_sweep(args, local_rank) if rank == 0 else 0
    if args.rows:
        return run_rows(args, local_rank) if rank == 0 else 0
    if args.runs:
        return run_runs(args, local_rank) if rank == 0 else 0
    if args.md:
        return run_md(args, local_rank) if rank == 0 else 0
    if args.link:
        return run_link(args, local_rank) if rank == 0 else 0
    return run_mine(args, rank, world, local_rank)


if __name__ == "__main__":
    sys.exit(main())
