"""The N > 1 path of the benchmark on CPU: two gloo ranks.

Structures are independent, so ranks run replicas (each its own seeded batch) and the
only communication is the aggregate: edges summed, time taken from the slowest rank.
Each rank computes its replica's edge count with the FP64 oracle here (no GPU)."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench
import oracle
import synth


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out_path):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    b = synth.make_batch(1, seed=bench.replica_seed(1, rank))
    edges = len(oracle.cutoff(b.lattice, b.frac, b.atom_ptr, 5.0)["src"])
    ms = 10.0 + 5.0 * rank  # stand-in step times: rank 1 is the slowest
    units, max_ms = bench.reduce_over_ranks(edges, ms, torch.device("cpu"))
    np.save(f"{out_path}.{rank}.npy", np.array([edges, units, max_ms, float(b.frac.sum())]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_replicas_aggregate(tmp_path):
    world = 2
    out = str(tmp_path / "agg")
    mp.start_processes(_rank_main, args=(world, _free_port(), out), nprocs=world, start_method="spawn", join=True)
    r = [np.load(f"{out}.{q}.npy") for q in range(world)]
    assert r[0][3] != r[1][3]  # the replicas hold different seeded batches
    total = r[0][0] + r[1][0]
    for q in range(world):
        assert r[q][1] == total  # edges summed over ranks
        assert r[q][2] == 15.0  # the slowest rank's time


def test_replica_seeds_distinct():
    seeds = {bench.replica_seed(2, q) for q in range(8)}
    assert len(seeds) == 8
