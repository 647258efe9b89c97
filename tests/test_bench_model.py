"""The benchmark's algorithmic work model, checked on CPU.

The FP32 side of a build's roofline counts 11 flops per candidate and 6/pi candidates per
edge: the candidates are the images in the cube of half-width r around each atom, the
edges those inside the sphere of radius r, and (2r)^3 / (4/3 pi r^3) = 6/pi.  Here both
are counted by brute force on the 16-structure workload; the sphere count is the
oracle's edge count."""
import math

import numpy as np

import bench
import oracle
import synth


def test_candidates_per_edge_model_against_a_brute_force_count():
    b = synth.make_batch(1)
    r = 5.0
    cube = sphere = 0
    for s in range(b.num_structures):
        lo, hi = b.atom_ptr[s], b.atom_ptr[s + 1]
        L = b.lattice[s].astype(np.float64)
        x = b.frac[lo:hi].astype(np.float64)
        # every image with |v|_inf < r has |df_k| <= sqrt(3) r ||L^-1||_F
        B = int(np.ceil(math.sqrt(3.0) * r * np.linalg.norm(np.linalg.inv(L)))) + 1
        T = np.stack(np.meshgrid(*[np.arange(-B, B + 1)] * 3, indexing="ij"), -1).reshape(-1, 3)
        for i in range(hi - lo):
            df = x - x[i]
            c = -np.round(df)
            v = ((df + c)[:, None, :] + T[None, :, :]) @ L
            self_img = np.zeros(v.shape[:2], bool)
            self_img[i] = np.all(T + c[i] == 0, axis=1)
            cube += int(((np.abs(v).max(-1) < r) & ~self_img).sum())
            sphere += int((((v * v).sum(-1) < r * r) & ~self_img).sum())
    edges = oracle.cutoff(b.lattice, b.frac, b.atom_ptr, r)["src"].shape[0]
    assert sphere == edges
    assert abs(cube / sphere - bench.CANDIDATES_PER_EDGE) < 0.03 * bench.CANDIDATES_PER_EDGE


def test_fp32_term_arithmetic():
    t = bench.fp32_term(1_000_000, 1e-3, 80.0, "measured")
    per_edge = 11.0 * 6.0 / math.pi
    assert math.isclose(t["achieved"], per_edge * 1e6 / 1e-3 / 1e12)
    assert math.isclose(t["frac"], t["achieved"] / 80.0)
    assert t["unit"] == "TFLOP/s" and t["peak_source"] == "measured"


def test_recorded_traffic_only_for_the_sources_it_was_captured_on(monkeypatch):
    """DRAM traffic from a committed ncu capture is reported only while the kernel
    sources hash to the value stored with it; any other source gives null."""
    entry = bench.recorded_traffic(3, ("cutoff", "build"))
    current = bench.kernel_source_hash()
    import json
    import os
    d = json.load(open(os.path.join(os.path.dirname(bench.__file__), "profiles", "traffic.json")))
    stored = d["config3"]["cutoff.build"]
    if stored["source_hash"] == current:
        assert entry == stored["bytes_per_launch"]
    else:
        assert entry is None
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "0" * 16)
    assert bench.recorded_traffic(3, ("cutoff", "build")) is None
    assert bench.recorded_traffic(9, ("cutoff", "build")) is None


def test_oracle_sample_is_bounded():
    """The host-side oracle legs time a bounded sample: the whole batch for the small
    workloads, the first 32 structures of the 8192-structure mixture, and for the
    supercells the smallest ones within 1.2e7 atom pairs (one pass of the brute force
    in seconds, not the hour the whole batch takes)."""
    import numpy as np

    import synth
    b2 = synth.make_batch(2)
    sub, _ = bench.oracle_sample(2, b2)
    assert sub.num_structures == b2.num_structures
    sub, what = bench.oracle_sample(3, synth.make_batch(3, B=64))
    assert sub.num_structures == 32 and "first 32" in what
    b5 = synth.make_batch(5)
    sub, what = bench.oracle_sample(5, b5)
    n = np.diff(sub.atom_ptr).astype(np.float64)
    assert 1 <= sub.num_structures < b5.num_structures
    assert (n ** 2).sum() <= 1.2e7 or sub.num_structures == 1
    assert n.max() <= np.diff(b5.atom_ptr).min() * 2  # the smallest supercells
