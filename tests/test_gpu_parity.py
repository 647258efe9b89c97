"""GPU parity: the CUDA path against the FP64 oracle, element by element.

Edge sets bit-exact after canonical order; vec/len within 1e-6 relative; gradients
within a condition-aware bound.  Every call goes through the C-ABI library.
"""
import numpy as np
import pytest

import oracle
import synth
from helpers import (assert_perm_dst, assert_same_edges, assert_vectors, grad_check, graph_arrays,
                     oracle_all_sources, oracle_sources, pointers_ok, rows_of_sources, to_device)

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2307_05380_gb300 as mg  # noqa: E402


def cutoff_parity(b, r, **kw):
    g = mg.cutoff_graph(to_device(b), r, **kw)
    got = graph_arrays(g)
    want = oracle.cutoff(b.lattice, b.frac, b.atom_ptr, r)
    assert_same_edges(got, want, f"cutoff r={r}")
    pointers_ok(got, b)
    if g.vec is not None:
        assert_vectors(b, got)
    if g.perm_dst is not None:
        assert_perm_dst(got, b.total_atoms)
    return got


def knn_parity(b, k, **kw):
    g = mg.knn_graph(to_device(b), k, **kw)
    got = graph_arrays(g)
    want = oracle.knn(b.lattice, b.frac, b.atom_ptr, k)
    assert_same_edges(got, want, f"knn k={k}")
    pointers_ok(got, b)
    if g.vec is not None:
        assert_vectors(b, got)
    if g.perm_dst is not None:
        assert_perm_dst(got, b.total_atoms)
    return got


# ------------------------------------------------------------------ workloads

def test_config1_cutoff_and_knn():
    b = synth.make_batch(1)
    cutoff_parity(b, 5.0)
    knn_parity(b, 12)


def test_config2_full_batch_cutoff_and_knn():
    b = synth.make_batch(2)
    cutoff_parity(b, 6.0)
    knn_parity(b, 16)


@pytest.mark.parametrize("r", [4.0, 6.0, 8.0])
def test_config3_sampled_structures_cutoff(r):
    """Full 8192-structure batch on the GPU; every structure of a seeded sample (skewed
    cells included) compared with the oracle."""
    b = synth.make_batch(3)
    g = mg.cutoff_graph(to_device(b), r, with_perm=False)
    got = graph_arrays(g)
    rng = np.random.default_rng(int(r))
    sample = sorted(set(rng.choice(b.num_structures, 48, replace=False).tolist()) |
                    {int(np.argmax(np.diff(b.atom_ptr)))})
    for s in sample:
        lo, hi = got["edge_ptr"][s], got["edge_ptr"][s + 1]
        sub = b.subset([s])
        want = oracle.cutoff(sub.lattice, sub.frac, sub.atom_ptr, r)
        part = {key: got[key][lo:hi] for key in ("src", "dst", "offset", "vec", "len")}
        part["src"] = part["src"] - b.atom_ptr[s]
        part["dst"] = part["dst"] - b.atom_ptr[s]
        assert_same_edges(part, want, f"structure {s}")
        assert_vectors(sub, part)


@pytest.mark.parametrize("k", [8, 16, 32])
def test_config3_sampled_structures_knn(k):
    b = synth.make_batch(3)
    g = mg.knn_graph(to_device(b), k, with_perm=False)
    got = graph_arrays(g)
    rng = np.random.default_rng(k)
    sample = sorted(rng.choice(b.num_structures, 64, replace=False).tolist())
    for s in sample:
        lo, hi = got["edge_ptr"][s], got["edge_ptr"][s + 1]
        sub = b.subset([s])
        want = oracle.knn(sub.lattice, sub.frac, sub.atom_ptr, k)
        part = {key: got[key][lo:hi] for key in ("src", "dst", "offset", "vec", "len")}
        part["src"] = part["src"] - b.atom_ptr[s]
        part["dst"] = part["dst"] - b.atom_ptr[s]
        assert_same_edges(part, want, f"structure {s}")
        assert_vectors(sub, part)


@pytest.mark.parametrize("cfg,r,k", [(3, 6.0, 16), (4, 5.0, 16)])
def test_every_edge_against_the_oracle(cfg, r, k):
    """A workload at full size (8192 structures with 295,952 atoms; 1024 structures with
    37k atoms): every edge of the cutoff graph (the staged build the bench times) and of
    the KNN graph bit-exact against the oracle over all sources (spawned processes on
    source ranges); every vector and length within 1e-6.  On the 1024-structure
    workload also the gradient of its Gaussian edge loss over the whole batch."""
    b = synth.make_batch(cfg)
    batch = to_device(b)
    g = mg.cutoff_graph(batch, r, with_perm=False)
    got = graph_arrays(g)
    assert_same_edges(got, oracle_all_sources("cutoff", b, r), f"cutoff r={r}, all sources")
    pointers_ok(got, b)
    assert_vectors(b, got)
    if cfg == 4:
        grad_check(b, g, synth.normal(4, 2, g.num_edges))
    del got
    got = graph_arrays(mg.knn_graph(batch, k, with_perm=False))
    assert_same_edges(got, oracle_all_sources("knn", b, k), f"knn k={k}, all sources")
    assert_vectors(b, got)


def test_supercells_up_to_4096_atoms_every_edge():
    """The supercell workload's parameters (cutoff 8 A, k = 32; cell list, staged build) on
    its eleven smallest supercells (1,728-4,096 atoms, 34,912 atoms in all): every edge of
    both graphs bit-exact against the oracle over all sources, vectors within 1e-6."""
    b5 = synth.make_batch(5)
    n = np.diff(b5.atom_ptr)
    b = b5.subset(sorted(np.argsort(n, kind="stable")[:11].tolist()))
    assert int(np.diff(b.atom_ptr).max()) <= 4096 and b.total_atoms >= 8192  # the staged build
    batch = to_device(b)
    got = graph_arrays(mg.cutoff_graph(batch, 8.0, with_perm=False))
    assert_same_edges(got, oracle_all_sources("cutoff", b, 8.0), "cutoff r=8, all sources")
    pointers_ok(got, b)
    assert_vectors(b, got)
    got = graph_arrays(mg.knn_graph(batch, 32, with_perm=False))
    assert_same_edges(got, oracle_all_sources("knn", b, 32), "knn k=32, all sources")
    assert_vectors(b, got)


def supercell_sources(b, per, seed):
    """`per` seeded source rows of every structure of b (all of a smaller one), ascending."""
    rng = np.random.default_rng(seed)
    out = []
    for s in range(b.num_structures):
        lo, hi = int(b.atom_ptr[s]), int(b.atom_ptr[s + 1])
        out.append(np.sort(rng.choice(np.arange(lo, hi), min(per, hi - lo), replace=False)))
    return np.concatenate(out).astype(np.int32)


def test_config5_supercells_sampled_sources():
    """Every supercell (1,728-21,952 atoms, cell list, staged build), 256 seeded sources
    each, all their edges at cutoff 8 A bit-exact against the oracle; vectors of those
    edges within 1e-6; in-degree equal to out-degree over the whole batch (a constant
    cutoff gives a symmetric graph)."""
    b = synth.make_batch(5)
    g = mg.cutoff_graph(to_device(b), 8.0, with_perm=False)
    src_ptr = g.src_ptr.cpu().numpy()
    srcs = supercell_sources(b, 256, 5)
    want = oracle_sources("cutoff", b, 8.0, srcs)
    rows = torch.from_numpy(rows_of_sources(src_ptr, srcs)).to(g.src.device)
    got = dict(src=g.src[rows].cpu().numpy(), dst=g.dst[rows].cpu().numpy(), offset=g.offset[rows].cpu().numpy(),
               vec=g.vec[rows].cpu().numpy(), len=g.len[rows].cpu().numpy())
    assert_same_edges(got, want, "supercells, 256 sources each")
    assert_vectors(b, got)
    E = g.num_edges
    deg_out = np.diff(src_ptr)
    deg_in = np.bincount(g.dst[:E].cpu().numpy(), minlength=b.total_atoms)
    np.testing.assert_array_equal(deg_out, deg_in)


def test_config5_knn_sampled_sources():
    """Every supercell, 256 seeded sources each: their k = 32 nearest images bit-exact
    against the oracle, vectors within 1e-6."""
    b = synth.make_batch(5)
    k = 32
    g = mg.knn_graph(to_device(b), k, with_perm=False)
    srcs = supercell_sources(b, 256, 55)
    want = oracle_sources("knn", b, k, srcs)
    rows = torch.from_numpy((srcs[:, None].astype(np.int64) * k + np.arange(k)).reshape(-1)).to(g.src.device)
    got = dict(src=g.src[rows].cpu().numpy(), dst=g.dst[rows].cpu().numpy(), offset=g.offset[rows].cpu().numpy(),
               vec=g.vec[rows].cpu().numpy(), len=g.len[rows].cpu().numpy())
    assert_same_edges(got, want, "supercells knn k=32, 256 sources each")
    assert_vectors(b, got)


def test_config5_three_largest_supercells_every_edge():
    """The three largest supercells (21,952, 21,952 and 17,576 atoms) at cutoff 8 A, built
    inside the whole 32-structure batch: every edge of the three bit-exact against the
    oracle over all their sources (about 1.3e9 atom pairs, spawned processes on source
    ranges), so the edge count of each is exact too."""
    b = synth.make_batch(5)
    g = mg.cutoff_graph(to_device(b), 8.0, with_perm=False)
    edge_ptr = g.edge_ptr.cpu().numpy()
    big = sorted(np.argsort(np.diff(b.atom_ptr), kind="stable")[-3:].tolist())
    srcs = np.concatenate([np.arange(b.atom_ptr[s], b.atom_ptr[s + 1]) for s in big]).astype(np.int32)
    want = oracle_sources("cutoff", b, 8.0, srcs)
    rows = torch.from_numpy(np.concatenate([np.arange(edge_ptr[s], edge_ptr[s + 1]) for s in big])).to(g.src.device)
    got = dict(src=g.src[rows].cpu().numpy(), dst=g.dst[rows].cpu().numpy(), offset=g.offset[rows].cpu().numpy())
    assert_same_edges(got, want, "three largest supercells, every edge")


# ------------------------------------------------------------------ closed forms and edge cases

def test_closed_forms_on_gpu():
    sc = synth.crystal(np.eye(3), [[0, 0, 0]])
    for r, deg in [(1.0, 0), (1.01, 6), (1.42, 18), (1.74, 26)]:
        g = mg.cutoff_graph(to_device(sc), r)
        assert g.num_edges == deg
    a = 3.6
    fcc = synth.crystal(np.array([[0, .5, .5], [.5, 0, .5], [.5, .5, 0]]) * a, [[0, 0, 0]])
    g = mg.knn_graph(to_device(fcc), 12)
    np.testing.assert_allclose(g.len[:12].cpu().numpy(), a / np.sqrt(2), rtol=1e-6)
    tie = synth.crystal(np.eye(3), [[0.25, 0.5, 0.75]])
    g = mg.knn_graph(to_device(tie), 8)
    assert g.offset[:8].cpu().numpy().tolist() == [[-1, -1, 0], [-1, 0, -1], [-1, 0, 0], [0, -1, 0],
                                                    [0, 0, -1], [0, 0, 1], [0, 1, 0], [1, 0, 0]]


def edge_case_batch():
    parts = [
        synth.crystal(np.eye(3) * 2.0, [[0.1, 0.2, 0.3]]),                      # one atom
        synth.crystal([[4, 0, 0], [3.6, 1.7, 0], [0.2, 0.3, 5]], [[0, 0, 0], [0.3, 0.6, 0.2]]),  # ~25 deg skew
        synth.crystal(np.eye(3) * 3.0, [[1.3, -2.2, 0.7], [-0.4, 0.5, 3.9]]),    # unwrapped coordinates
        synth.crystal([[2.5, 0, 0], [0, 14, 0], [0, 0, 30]], [[0.5, 0.5, 0.5], [0.9, 0.1, 0.2]]),  # long cell
        synth.make_batch(2, B=8),
    ]
    b = synth.concat(parts)
    # insert an empty structure in the middle
    counts = np.diff(b.atom_ptr).tolist()
    counts.insert(3, 0)
    lat = np.concatenate([b.lattice[:3], np.eye(3, dtype=np.float32)[None] * 5, b.lattice[3:]])
    ptr = np.concatenate([[0], np.cumsum(counts)]).astype(np.int32)
    return synth.Batch(lat, b.frac, ptr)


def test_edge_cases_cutoff():
    b = edge_case_batch()
    for r in (3.0, 5.5):
        cutoff_parity(b, r)


def test_edge_cases_knn():
    b = edge_case_batch()
    for k in (1, 5, 27, 33, 64, 100, 128):
        knn_parity(b, k)


def test_pair_lane_knn_small_batches_and_edge_cases():
    """The pair-lane KNN forced (schedule 5; batches below 8192 atoms take the warp
    enumeration by default) on the 16- and 256-structure workloads, the edge cases (one
    atom, a 25 degree skew, unwrapped coordinates, a long cell, an empty structure; k up
    to 64, and k = 100 handed to the warp enumeration), the needle cells and the
    cell-list structures, against the oracle."""
    opts = mg.make_opts(schedule=5)
    knn_parity(synth.make_batch(1), 12, opts=opts)
    knn_parity(synth.make_batch(2), 16, opts=opts)
    knn_parity(synth.make_batch(2), 32, opts=opts)
    b = edge_case_batch()
    for k in (1, 5, 27, 33, 64, 100):
        knn_parity(b, k, opts=opts)
    knn_parity(cell_list_batch(), 16, opts=opts)
    c, s_ = np.cos(0.7), np.sin(0.7)  # the needle cells: the radius grows along L_0
    R = np.array([[c, -s_, 0.0], [s_, c, 0.0], [0.0, 0.0, 1.0]]) @ np.array([[1.0, 0.0, 0.0], [0.0, c, -s_], [0.0, s_, c]])
    lat = np.stack([np.diag([1.0, 10.0, 10.0]), np.diag([1.0, 10.0, 10.0]) @ R.T,
                    np.array([[1.0, 0.0, 0.0], [5.0, 10.0, 0.0], [3.0, 4.0, 10.0]])])
    needles = synth.Batch(lat, np.array([[0.3, 0.6, 0.2]] * 3), np.array([0, 1, 2, 3], np.int32))
    for k in (5, 18):
        knn_parity(needles, k, opts=opts)


def cell_list_batch():
    """Structures large enough for the cell list: a skewed 2-atom cell tiled 6x6x6 with
    some atoms moved by whole cells (unwrapped coordinates), and a noisy 5x5x5 tiling of
    a random 8-atom cell."""
    rng = np.random.default_rng(42)
    base_L = np.array([[3.1, 0.0, 0.0], [2.2, 2.4, 0.0], [0.4, 0.6, 3.3]])
    base_x = np.array([[0.1, 0.2, 0.3], [0.6, 0.55, 0.8]])
    n = 6
    xs = np.concatenate([(base_x + np.array(c)) / n for c in np.ndindex(n, n, n)])
    xs[::7] += rng.integers(-2, 3, size=xs[::7].shape)
    a = synth.Batch((n * base_L)[None], xs, np.array([0, len(xs)], np.int32))
    b = synth.make_batch(5, B=1)
    lo = b.atom_ptr[0]
    m = 5
    c8 = synth.make_batch(1, B=1)
    xb = c8.frac[:min(8, len(c8.frac))].astype(np.float64)
    xt = np.concatenate([(xb + np.array(c)) / m for c in np.ndindex(m, m, m)])
    xt += rng.normal(0, 0.002, xt.shape)
    c = synth.Batch((m * c8.lattice[0].astype(np.float64))[None], xt, np.array([0, len(xt)], np.int32))
    del lo
    return synth.concat([a, synth.crystal(np.eye(3) * 3.0, [[0.5, 0.5, 0.5]]), c])


def test_cell_list_cutoff_and_knn_full_parity():
    b = cell_list_batch()
    for r in (2.5, 4.0):
        cutoff_parity(b, r)
    for k in (8, 40):
        knn_parity(b, k)


def test_cell_list_per_structure_build_identical():
    b = cell_list_batch()
    batch = to_device(b)
    ref = graph_arrays(mg.cutoff_graph(batch, 4.0))
    ps = graph_arrays(mg.build_per_structure(batch, "cutoff", cutoff=4.0))
    for key in ref:
        np.testing.assert_array_equal(ref[key], ps[key], err_msg=key)
    kref = graph_arrays(mg.knn_graph(batch, 12))
    kps = graph_arrays(mg.build_per_structure(batch, "knn", k=12))
    for key in kref:
        np.testing.assert_array_equal(kref[key], kps[key], err_msg=key)


def test_ragged_sizes_many_tiles():
    """Batches whose atom counts straddle warp and scan-tile boundaries."""
    b = synth.concat([synth.make_batch(3, B=40), synth.make_batch(1, B=5)])
    cutoff_parity(b, 5.0)
    knn_parity(b, 9)


def test_one_pass_build_across_waves():
    """The one-pass build keeps 6 blocks of 4 source warps per SM resident; larger batches
    run their last tiles in later waves, whose look-back reads tiles that have already
    retired.  A batch just past one wave is compared with the oracle; the 1024-structure
    workload (about ten waves) forced through the one-pass build gives the same arrays,
    bit for bit, as the staged build."""
    b = synth.make_batch(2, seed=0)  # 3,674 atoms: 919 tiles
    assert b.total_atoms > 152 * 6 * 4
    cutoff_parity(b, 6.0, opts=mg.make_opts(schedule=3))
    b4 = synth.make_batch(4)
    batch = to_device(b4)
    onepass = graph_arrays(mg.cutoff_graph(batch, 5.0, opts=mg.make_opts(schedule=3)))
    staged = graph_arrays(mg.cutoff_graph(batch, 5.0, opts=mg.make_opts(schedule=4)))
    assert onepass.keys() == staged.keys()
    for key in staged:
        np.testing.assert_array_equal(onepass[key], staged[key], err_msg=key)


def test_needle_cells_knn_radius_growth():
    """One atom in 1 x 10 x 10 A cells (straight, rotated and skewed): the k nearest
    images lie along L_0 up to 9 A away, so the KNN search grows its radius several times
    along one axis; exact-k, keep-ties and a 9.5 A cutoff graph against the oracle."""
    c, s_ = np.cos(0.7), np.sin(0.7)
    R = np.array([[c, -s_, 0.0], [s_, c, 0.0], [0.0, 0.0, 1.0]]) @ np.array([[1.0, 0.0, 0.0], [0.0, c, -s_], [0.0, s_, c]])
    lat = np.stack([np.diag([1.0, 10.0, 10.0]), np.diag([1.0, 10.0, 10.0]) @ R.T,
                    np.array([[1.0, 0.0, 0.0], [5.0, 10.0, 0.0], [3.0, 4.0, 10.0]])])
    b = synth.Batch(lat, np.array([[0.3, 0.6, 0.2]] * 3), np.array([0, 1, 2, 3], np.int32))
    for k in (5, 18):
        knn_parity(b, k)
        got = graph_arrays(mg.knn_graph(to_device(b), k, keep_ties=True))
        assert_same_edges(got, oracle.knn(b.lattice, b.frac, b.atom_ptr, k, keep_ties=True), f"ties k={k}")
    cutoff_parity(b, 9.5)


def test_capacity_error_then_exact_rebuild():
    b = synth.make_batch(1)
    batch = to_device(b)
    g = mg.cutoff_graph(batch, 5.0, capacity=10, sync=False)
    st = g.read_status()
    want = oracle.cutoff(b.lattice, b.frac, b.atom_ptr, 5.0)
    assert st["code"] == 4 and st["required_capacity"] == len(want["src"])
    g2 = mg.cutoff_graph(batch, 5.0, capacity=st["required_capacity"])
    assert g2.num_edges == len(want["src"])


def test_bad_inputs_reported_on_device():
    b = synth.make_batch(1, B=3)
    lat = b.lattice.copy()
    lat[1] = 0.0  # singular
    frac = b.frac.copy()
    frac[b.atom_ptr[2]] = np.nan
    g = mg.cutoff_graph(to_device(synth.Batch(lat, frac, b.atom_ptr)), 5.0, sync=False)
    st = g.read_status()
    assert st["code"] in (2, 3) and st["first_bad_structure"] == 1
    # the good structure is still built
    want = oracle.cutoff(b.lattice[:1], b.frac[:b.atom_ptr[1]], b.atom_ptr[:2], 5.0)
    E0 = int(g.edge_ptr[1].item())
    assert E0 == len(want["src"])


# ------------------------------------------------------------------ pair-lane build

def pair_opts(**kw):
    return mg.make_opts(schedule=5, **kw)


def test_pair_lane_build_small_batches_against_the_oracle():
    """The pair-lane build (work list, count pass, scan, write pass) forced on the
    16- and 256-structure workloads and on the edge cases (one-atom cells, a 25 degree
    skew, unwrapped coordinates, a long cell, an empty structure): edges, pointers,
    vectors and destination order against the oracle."""
    for b, r in ((synth.make_batch(1), 5.0), (synth.make_batch(2), 6.0), (edge_case_batch(), 3.0),
                 (edge_case_batch(), 5.5)):
        cutoff_parity(b, r, opts=pair_opts())


def test_pair_lane_build_with_warp_enumerated_structures():
    """Structures outside the pair-lane scan (cell lists, boxes of more than 64 cells,
    a source with more than 1024 edges) are scanned by the warp enumeration inside the
    pair-lane passes, next to pair-lane structures."""
    b = synth.concat([cell_list_batch(), synth.crystal(np.eye(3), [[0.1, 0.2, 0.3]]), synth.make_batch(2, B=16)])
    for r in (2.5, 4.0):
        cutoff_parity(b, r, opts=pair_opts())
    cutoff_parity(b, 7.3, opts=pair_opts())  # the unit cube's source: ~1600 edges, re-enumerated


@pytest.mark.parametrize("r", [4.0, 6.0, 8.0])
def test_pair_lane_build_identical_to_staged_build_8192_structures(r):
    """The 8192-structure mixture (skewed cells included) at every radius of the
    workload: the pair-lane build (the default there) and the staged build give the same
    arrays bit for bit, destination order included; the staged build is checked against
    the oracle edge by edge elsewhere, and here sampled structures are too."""
    b = synth.make_batch(3)
    batch = to_device(b)
    pair = graph_arrays(mg.cutoff_graph(batch, r, opts=pair_opts()))
    staged = graph_arrays(mg.cutoff_graph(batch, r, opts=mg.make_opts(schedule=4)))
    assert pair.keys() == staged.keys()
    for key in staged:
        np.testing.assert_array_equal(pair[key], staged[key], err_msg=key)
    rng = np.random.default_rng(100 + int(r))
    for s in sorted(rng.choice(b.num_structures, 16, replace=False).tolist()):
        lo, hi = pair["edge_ptr"][s], pair["edge_ptr"][s + 1]
        sub = b.subset([s])
        part = {key: pair[key][lo:hi] for key in ("src", "dst", "offset")}
        part["src"] = part["src"] - b.atom_ptr[s]
        part["dst"] = part["dst"] - b.atom_ptr[s]
        assert_same_edges(part, oracle.cutoff(sub.lattice, sub.frac, sub.atom_ptr, r), f"structure {s}")


def test_pair_lane_build_capacity_bad_inputs_and_gradient():
    """Too small a capacity: MG_ERR_CAPACITY with the exact requirement, nothing written;
    a singular and a non-finite structure reported while the others are built; the
    gradient through the pair table the write pass records, against the oracle."""
    b = synth.make_batch(4, B=256)
    batch = to_device(b)
    want = oracle.cutoff(b.lattice, b.frac, b.atom_ptr, 5.0)
    g = mg.cutoff_graph(batch, 5.0, capacity=1000, opts=pair_opts(), sync=False)
    st = g.read_status()
    assert st["code"] == 4 and st["required_capacity"] == len(want["src"]), st
    g = mg.cutoff_graph(batch, 5.0, opts=pair_opts(), with_perm=False)
    got = graph_arrays(g)
    assert_same_edges(got, want, "pair-lane, 256 structures")
    pointers_ok(got, b)
    grad_check(b, g, synth.normal(8, 1, g.num_edges), c=synth.normal(8, 2, 3 * g.num_edges).reshape(-1, 3))
    lat = b.lattice.copy()
    lat[3] = 0.0
    frac = b.frac.copy()
    frac[b.atom_ptr[7] + 1] = np.inf
    gb = mg.cutoff_graph(to_device(synth.Batch(lat, frac, b.atom_ptr)), 5.0, opts=pair_opts(), sync=False)
    st = gb.read_status()
    assert st["code"] in (2, 3) and st["first_bad_structure"] == 3, st
    ep = gb.edge_ptr.cpu().numpy()
    assert ep[4] - ep[3] == 0 and ep[8] - ep[7] == 0
    for s in (0, 5, 9):
        assert ep[s + 1] - ep[s] == int(np.sum((want["src"] >= b.atom_ptr[s]) & (want["src"] < b.atom_ptr[s + 1])))


def onepass_opts(**kw):
    return mg.make_opts(schedule=6, **kw)


def test_pair_lane_one_pass_build_against_the_oracle():
    """The one-pass pair-lane build (schedule 6: items in canonical order, masks, a
    decoupled look-back, edges written from the masks) on the 16- and 256-structure
    workloads, the edge cases, warp-enumerated structures (cell lists, large boxes, a
    source re-enumerated past the shared staging) beside pair-lane ones, and across many
    tiles: edges, pointers, vectors and destination order against the oracle."""
    for b, r in ((synth.make_batch(1), 5.0), (synth.make_batch(2), 6.0), (edge_case_batch(), 3.0),
                 (edge_case_batch(), 5.5)):
        cutoff_parity(b, r, opts=onepass_opts())
    b = synth.concat([cell_list_batch(), synth.crystal(np.eye(3), [[0.1, 0.2, 0.3]]), synth.make_batch(2, B=16)])
    for r in (2.5, 4.0, 7.3):
        cutoff_parity(b, r, opts=onepass_opts())


def test_pair_lane_one_pass_build_identical_to_one_pass_build():
    """Schedule 6 against the one-pass build of the warp enumeration (schedule 3), bit for
    bit with destination order, on the 256- and 1024-structure workloads and on 160
    structures of the 8192-structure mixture (up to 400 atoms, skewed cells); capacity
    error with the exact requirement; the backward through its pair table."""
    for b, r in ((synth.make_batch(2), 6.0), (synth.make_batch(4), 5.0), (synth.make_batch(3, B=160), 6.0)):
        batch = to_device(b)
        one = graph_arrays(mg.cutoff_graph(batch, r, opts=onepass_opts()))
        ref = graph_arrays(mg.cutoff_graph(batch, r, opts=mg.make_opts(schedule=3)))
        assert one.keys() == ref.keys()
        for key in ref:
            np.testing.assert_array_equal(one[key], ref[key], err_msg=key)
    b = synth.make_batch(2)
    batch = to_device(b)
    want = oracle.cutoff(b.lattice, b.frac, b.atom_ptr, 6.0)
    g = mg.cutoff_graph(batch, 6.0, capacity=1000, opts=onepass_opts(), sync=False)
    st = g.read_status()
    assert st["code"] == 4 and st["required_capacity"] == len(want["src"]), st
    g = mg.cutoff_graph(batch, 6.0, opts=onepass_opts(), with_perm=False)
    grad_check(b, g, synth.normal(9, 1, g.num_edges), c=synth.normal(9, 2, 3 * g.num_edges).reshape(-1, 3))
    g3 = mg.cutoff_graph(batch, 6.0, opts=mg.make_opts(schedule=3), with_perm=False)
    gl = torch.from_numpy(synth.normal(9, 3, g.num_edges)).cuda()
    v, ln = mg.edge_vectors_fwd(g)
    f1, L1 = mg.edge_vectors_bwd(g, batch, None, gl, v, ln)
    v3, ln3 = mg.edge_vectors_fwd(g3)
    f3, L3 = mg.edge_vectors_bwd(g3, batch, None, gl, v3, ln3)
    assert torch.equal(f1, f3) and torch.equal(L1, L3)


def test_pair_lane_one_pass_build_without_staging_space():
    """A large batch whose workspace does not cover the capacity cannot stage keys: the
    automatic choice is then the one-pass pair-lane build (stage events name one 'build'
    stage), with the same arrays as the pair-lane build of a full workspace."""
    import ctypes
    from paper_2307_05380_gb300 import _capi
    from paper_2307_05380_gb300 import graph as G
    b = synth.make_batch(3, B=1024)
    batch = to_device(b)
    ref = graph_arrays(mg.cutoff_graph(batch, 6.0, with_perm=False))
    g = mg.cutoff_graph(batch, 6.0, with_perm=False)
    nbytes = ctypes.c_size_t(0)
    _capi.check(_capi.load().mg_workspace_size(G.context(batch.device), ctypes.byref(batch.c), 0,
                                               ctypes.byref(nbytes)), "mg_workspace_size")
    g.ws = g.ws[:int(nbytes.value)]  # the per-atom regions only: no room to stage edges
    mg.profile_enable(True, batch.device)
    try:
        mg.rebuild(g)
        n_auto = mg.last_launch_count(batch.device)
        stages = mg.stage_times("cutoff", batch.device)
    finally:
        mg.profile_enable(False, batch.device)
    assert "build" in stages and "stage" not in stages, stages
    mg.cutoff_graph(batch, 6.0, with_perm=False, opts=mg.make_opts(schedule=3))
    assert n_auto == mg.last_launch_count(batch.device) + 1  # the item scan, then the one pass
    got = graph_arrays(g)
    for key in ref:
        np.testing.assert_array_equal(got[key], ref[key], err_msg=key)


def test_pair_lane_build_stats():
    b = synth.make_batch(3, B=512)
    g = mg.cutoff_graph(to_device(b), 6.0, opts=pair_opts(collect_stats=True))
    st = g.last_status
    assert st["candidates"] >= g.num_edges > 0
    assert 0 <= st["rechecked"] < st["candidates"] * 1e-2


@pytest.mark.parametrize("cfg,k", [(3, 8), (3, 16), (3, 32), (5, 32)])
def test_pair_lane_knn_identical_to_warp_knn(cfg, k):
    """The pair-lane KNN (the default: a lane per target, candidates sorted in shared
    memory, sources with large boxes handed to the warp-enumeration KNN) against the
    warp-enumeration KNN for every source (schedule 1): the same arrays bit for bit on
    the 8192-structure mixture and on the supercells, plus sampled structures against
    the oracle."""
    b = synth.make_batch(cfg)
    batch = to_device(b)
    pl = graph_arrays(mg.knn_graph(batch, k, with_perm=False))
    wk = graph_arrays(mg.knn_graph(batch, k, with_perm=False, opts=mg.make_opts(schedule=1)))
    for key in wk:
        np.testing.assert_array_equal(pl[key], wk[key], err_msg=key)
    rng = np.random.default_rng(200 + k)
    srcs = np.sort(rng.choice(b.total_atoms, 512, replace=False)).astype(np.int32)
    rows = (srcs[:, None].astype(np.int64) * k + np.arange(k)).reshape(-1)
    got = {key: pl[key][rows] for key in ("src", "dst", "offset")}
    assert_same_edges(got, oracle_sources("knn", b, k, srcs), f"knn k={k}, 512 sources")


def test_autotuned_schedules_identical_on_8192_structures(tmp_path):
    """mg_autotune on the 8192-structure mixture (cutoff 6 A, k = 16) through the per-device
    cache file: the tuned builds give the same arrays, bit for bit, as every fixed
    schedule, and sampled structures match the oracle; a second call reads the cache
    instead of tuning again."""
    b = synth.make_batch(3)
    batch = to_device(b)
    path = str(tmp_path / "tune.json")
    saved = mg.tuned_table(batch.device)
    try:
        t1 = mg.autotune_cached(batch, "cutoff", cutoff=6.0, path=path)
        t2 = mg.autotune_cached(batch, "knn", k=16, path=path)
        assert t1["tuned_now"] and t2["tuned_now"]
        assert not mg.autotune_cached(batch, "cutoff", cutoff=6.0, path=path)["tuned_now"]
        tuned = graph_arrays(mg.cutoff_graph(batch, 6.0, with_perm=False))
        for sched in (3, 4, 5):
            other = graph_arrays(mg.cutoff_graph(batch, 6.0, with_perm=False, opts=mg.make_opts(schedule=sched)))
            for key in tuned:
                np.testing.assert_array_equal(tuned[key], other[key], err_msg=f"cutoff schedule {sched} {key}")
        ktuned = graph_arrays(mg.knn_graph(batch, 16, with_perm=False))
        for sched in (1, 2, 5):
            other = graph_arrays(mg.knn_graph(batch, 16, with_perm=False, opts=mg.make_opts(schedule=sched)))
            for key in ktuned:
                np.testing.assert_array_equal(ktuned[key], other[key], err_msg=f"knn schedule {sched} {key}")
        rng = np.random.default_rng(31)
        for s in sorted(rng.choice(b.num_structures, 12, replace=False).tolist()):
            lo, hi = tuned["edge_ptr"][s], tuned["edge_ptr"][s + 1]
            sub = b.subset([s])
            part = {key: tuned[key][lo:hi] - (b.atom_ptr[s] if key in ("src", "dst") else 0)
                    for key in ("src", "dst", "offset")}
            assert_same_edges(part, oracle.cutoff(sub.lattice, sub.frac, sub.atom_ptr, 6.0), f"structure {s}")
    finally:
        mg.set_tuned_table(saved, batch.device)


# ------------------------------------------------------------------ schedules, per-structure, update

def test_schedules_and_per_structure_identical():
    b = synth.make_batch(2)
    batch = to_device(b)
    ref = graph_arrays(mg.cutoff_graph(batch, 6.0, opts=mg.make_opts(schedule=1)))
    per = graph_arrays(mg.cutoff_graph(batch, 6.0, opts=mg.make_opts(schedule=2)))
    onepass = graph_arrays(mg.cutoff_graph(batch, 6.0, opts=mg.make_opts(schedule=3)))
    staged = graph_arrays(mg.cutoff_graph(batch, 6.0, opts=mg.make_opts(schedule=4)))
    ps = graph_arrays(mg.build_per_structure(batch, "cutoff", cutoff=6.0))
    mg.autotune(batch, "cutoff", cutoff=6.0)
    tuned = graph_arrays(mg.cutoff_graph(batch, 6.0))
    for other in (per, onepass, staged, ps, tuned):
        for key in ref:
            np.testing.assert_array_equal(ref[key], other[key], err_msg=key)
    kref = graph_arrays(mg.knn_graph(batch, 16, opts=mg.make_opts(schedule=1)))
    kper = graph_arrays(mg.knn_graph(batch, 16, opts=mg.make_opts(schedule=2)))
    kps = graph_arrays(mg.build_per_structure(batch, "knn", k=16))
    for other in (kper, kps):
        for key in kref:
            np.testing.assert_array_equal(kref[key], other[key], err_msg=key)


def test_update_graph_replay_tracks_geometry():
    b = synth.make_batch(4, B=64)
    batch = to_device(b)
    g = mg.cutoff_graph(batch, 5.0, capacity=400000)
    cur = b
    for step in range(3):
        cur = synth.perturb(cur, seed=11, step=step)
        g = mg.update_graph(g, torch.from_numpy(cur.frac).cuda(), torch.from_numpy(cur.lattice).cuda())
        got = graph_arrays(g)
        want = oracle.cutoff(cur.lattice, cur.frac, cur.atom_ptr, 5.0)
        assert_same_edges(got, want, f"step {step}")
        assert_vectors(cur, got)


def test_bounded_wait_reports_timeout_and_context_survives():
    """A tile of the one-pass build that never publishes its offset (testing hook): the
    look-back waits of the tiles after it give up, the status reports MG_ERR_TIMEOUT, and
    the next build on the same context is correct."""
    b = synth.make_batch(1)
    batch = to_device(b)
    g = mg.cutoff_graph(batch, 5.0, opts=mg.make_opts(fault_tile=1), sync=False)
    st = g.read_status()
    assert st["code"] == 6, st  # MG_ERR_TIMEOUT
    good = graph_arrays(mg.cutoff_graph(batch, 5.0))
    assert_same_edges(good, oracle.cutoff(b.lattice, b.frac, b.atom_ptr, 5.0), "after timeout")


def test_stats_counters():
    b = synth.make_batch(2, B=32)
    g = mg.cutoff_graph(to_device(b), 6.0, opts=mg.make_opts(collect_stats=True))
    st = g.last_status
    assert st["candidates"] >= g.num_edges > 0
    assert 0 <= st["rechecked"] < st["candidates"]


# ------------------------------------------------------------------ edge vectors and gradients

def test_edge_vectors_fwd_matches_build():
    b = synth.make_batch(2)
    g = mg.cutoff_graph(to_device(b), 6.0)
    vec, ln = mg.edge_vectors_fwd(g)
    E = g.num_edges
    assert torch.equal(vec[:E], g.vec[:E]) and torch.equal(ln[:E], g.len[:E])


def test_gradients_match_oracle_and_are_deterministic():
    b = synth.make_batch(4, B=128)
    g = mg.cutoff_graph(to_device(b), 5.0)
    w = synth.normal(4, 0, g.num_edges)
    g1 = grad_check(b, g, w)
    g2 = grad_check(b, g, w)
    assert torch.equal(g1[0], g2[0]) and torch.equal(g1[1], g2[1])


def test_symmetric_and_destination_order_backward_agree():
    """A cutoff graph's backward through reverse edges (no perm_dst) against the
    destination-order path (a per-structure build is not recorded as symmetric)."""
    b = synth.make_batch(4, B=64)
    batch = to_device(b)
    g_sym = mg.cutoff_graph(batch, 5.0, with_perm=False)
    g_gen = mg.build_per_structure(batch, "cutoff", cutoff=5.0)
    assert g_sym.num_edges == g_gen.num_edges
    gl = torch.from_numpy(synth.normal(3, 0, g_sym.num_edges)).cuda()
    v1, l1 = mg.edge_vectors_fwd(g_sym)
    v2, l2 = mg.edge_vectors_fwd(g_gen)
    f1, L1 = mg.edge_vectors_bwd(g_sym, batch, None, gl, v1, l1)
    f2, L2 = mg.edge_vectors_bwd(g_gen, batch, None, gl, v2, l2)
    torch.testing.assert_close(f1, f2, rtol=1e-5, atol=1e-5 * float(f2.abs().max()))
    torch.testing.assert_close(L1, L2, rtol=1e-5, atol=1e-5 * float(L2.abs().max()))


def test_gradients_knn_graph_grad_vec_path():
    b = synth.make_batch(2, B=64)
    g = mg.knn_graph(to_device(b), 16)
    E = g.num_edges
    # grad_vec alone (zero loss weights on the lengths), then both paths together
    grad_check(b, g, np.zeros(E, np.float32), c=synth.normal(5, 1, 3 * E).reshape(-1, 3))
    grad_check(b, g, synth.normal(5, 2, E), c=synth.normal(5, 1, 3 * E).reshape(-1, 3))
