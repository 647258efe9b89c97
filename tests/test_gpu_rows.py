"""GPU parity for the rows after the hot path: per-atom cutoffs and keep-ties KNN graphs
(Def. 3 in full; Alg. 2's filter), against the FP64 oracle through the C-ABI library.

Edge sets bit-exact in canonical order; vec/len within 1e-6 relative; destination order
and gradients as for the constant-cutoff graph.
"""
import dataclasses
import json
import os

import numpy as np
import pytest

import oracle
import synth
from helpers import (assert_grad_bound, assert_perm_dst, assert_same_edges, assert_vectors, grad_check, graph_arrays,
                     pointers_ok, to_device)

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2307_05380_gb300 as mg  # noqa: E402

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "next_rows.json")))


def radii_for(b, seed, lo, hi):
    """Seeded per-atom radii, uniform in [lo, hi)."""
    return np.random.default_rng(seed).uniform(lo, hi, b.total_atoms).astype(np.float32)


def atoms_parity(b, radii, **kw):
    batch = to_device(b)
    g = mg.cutoff_graph_atoms(batch, torch.from_numpy(radii).cuda(), **kw)
    got = graph_arrays(g)
    want = oracle.cutoff_atoms(b.lattice, b.frac, b.atom_ptr, radii.astype(np.float64))
    assert_same_edges(got, want, "per-atom cutoff")
    pointers_ok(got, b)
    if g.vec is not None:
        assert_vectors(b, got)
    if g.perm_dst is not None:
        assert_perm_dst(got, b.total_atoms)
    return g, got


def ties_parity(b, k, **kw):
    g = mg.knn_graph(to_device(b), k, keep_ties=True, **kw)
    got = graph_arrays(g)
    want = oracle.knn(b.lattice, b.frac, b.atom_ptr, k, keep_ties=True)
    assert_same_edges(got, want, f"keep-ties knn k={k}")
    pointers_ok(got, b)
    if g.vec is not None:
        assert_vectors(b, got)
    if g.perm_dst is not None:
        assert_perm_dst(got, b.total_atoms)
    return g, got


# ------------------------------------------------------------------ per-atom cutoffs

def test_per_atom_cutoff_closed_forms_on_gpu():
    d = GOLD["per_atom_cutoff_sc_pair"]
    b = synth.crystal(d["lattice"], d["frac"])
    for radii, degs in d["cases"]:  # radius 1.0 sits exactly on a shell: strict inequality
        g = mg.cutoff_graph_atoms(to_device(b), torch.tensor(radii, dtype=torch.float32, device="cuda"))
        got = graph_arrays(g)
        assert np.bincount(got["src"], minlength=2).tolist() == degs


@pytest.mark.parametrize("cfg,lo,hi", [(1, 2.0, 6.0), (2, 3.0, 7.0), (4, 2.5, 6.0)])
def test_per_atom_cutoff_full_batches(cfg, lo, hi):
    b = synth.make_batch(cfg, B=None if cfg == 1 else 96)
    atoms_parity(b, radii_for(b, cfg, lo, hi))


def test_per_atom_cutoff_cell_list_sources():
    """Two supercells (cell-list path, thousands of atoms) against the oracle on a sample
    of sources: every edge of each sampled source, in canonical order."""
    b = synth.make_batch(5).subset([0, 1])
    radii = radii_for(b, 5, 5.0, 8.0)
    g = mg.cutoff_graph_atoms(to_device(b), torch.from_numpy(radii).cuda(), with_perm=False)
    got = graph_arrays(g)
    rng = np.random.default_rng(5)
    srcs = np.sort(rng.choice(b.total_atoms, 64, replace=False)).astype(np.int32)
    want = oracle.cutoff_atoms(b.lattice, b.frac, b.atom_ptr, radii.astype(np.float64), sources=srcs)
    sel = np.concatenate([np.arange(got["src_ptr"][s], got["src_ptr"][s + 1]) for s in srcs])
    part = {k: got[k][sel] for k in ("src", "dst", "offset", "vec", "len")}
    assert_same_edges(part, want, "cell-list sources")
    assert_vectors(b, part)
    assert got["src_ptr"][-1] == g.num_edges


def test_per_atom_cutoff_equal_radii_is_the_constant_cutoff_graph():
    b = synth.make_batch(2, B=64)
    batch = to_device(b)
    ga = mg.cutoff_graph_atoms(batch, torch.full((b.total_atoms,), 6.0, device="cuda"))
    gc = mg.cutoff_graph(batch, 6.0)
    a, c = graph_arrays(ga), graph_arrays(gc)
    for key in ("src", "dst", "offset", "vec", "len", "edge_ptr", "src_ptr", "perm_dst", "dst_ptr"):
        np.testing.assert_array_equal(a[key], c[key], err_msg=key)


def test_per_atom_cutoff_gradients_through_destination_order():
    b = synth.make_batch(4, B=48)
    g, _ = atoms_parity(b, radii_for(b, 44, 3.0, 6.0))
    w = synth.normal(4, 2, g.num_edges)
    g1 = grad_check(b, g, w)
    g2 = grad_check(b, g, w)
    assert torch.equal(g1[0], g2[0]) and torch.equal(g1[1], g2[1])


def test_per_atom_cutoff_bad_radius_reported():
    b = synth.make_batch(1)
    radii = np.full(b.total_atoms, 4.0, np.float32)
    radii[int(b.atom_ptr[3]) + 1] = -1.0
    batch = to_device(b)
    with pytest.raises(RuntimeError, match="INVALID_ARGUMENT"):
        mg.cutoff_graph_atoms(batch, torch.from_numpy(radii).cuda())
    radii[int(b.atom_ptr[3]) + 1] = float("nan")
    with pytest.raises(RuntimeError, match="structure 3"):
        mg.cutoff_graph_atoms(batch, torch.from_numpy(radii).cuda())


def test_per_atom_cutoff_update_replay():
    b = synth.make_batch(4, B=32)
    batch = to_device(b)
    radii = torch.from_numpy(radii_for(b, 9, 3.0, 5.0)).cuda()
    g = mg.cutoff_graph_atoms(batch, radii, capacity=200 * b.total_atoms)
    moved = synth.perturb(b, 9, 1)
    batch.frac.copy_(torch.from_numpy(moved.frac).cuda())
    batch.lattice.copy_(torch.from_numpy(moved.lattice).cuda())
    for _ in range(2):
        mg.update_graph(g)
        got = graph_arrays(g)
        want = oracle.cutoff_atoms(moved.lattice, moved.frac, moved.atom_ptr,
                                   radii.cpu().numpy().astype(np.float64))
        assert_same_edges(got, want, "per-atom replay")


# ------------------------------------------------------------------ keep-ties KNN

@pytest.mark.parametrize("name", ["knn_keep_ties_sc", "knn_keep_ties_fcc", "knn_keep_ties_bcc"])
def test_keep_ties_closed_forms_on_gpu(name):
    d = GOLD[name]
    L = np.asarray(d.get("lattice_over_a", np.eye(3)), float) * 3.0
    b = synth.crystal(L, [[0, 0, 0]])
    for k, m in d["cases"]:
        g, got = ties_parity(b, k)
        assert g.num_edges == m, (name, k)


def test_keep_ties_perfect_supercell_many_ties():
    L = np.eye(3) * 2.0
    x = [[a, b_, c] for a in (0, .5) for b_ in (0, .5) for c in (0, .5)]
    b = synth.concat([synth.crystal(L, x), synth.crystal(np.diag([3.0, 3.0, 4.0]), [[0, 0, 0], [.5, .5, .5]])])
    for k in (1, 6, 7, 19, 33, 100):
        ties_parity(b, k)


@pytest.mark.parametrize("cfg,k", [(1, 12), (2, 16), (3, 8)])
def test_keep_ties_batches(cfg, k):
    b = synth.make_batch(cfg, B=None if cfg == 1 else 96)
    g, got = ties_parity(b, k)
    # with generic coordinates the only ties are an atom's own images t and -t
    assert g.num_edges >= k * b.total_atoms


def test_keep_ties_gradients():
    b = synth.make_batch(2, B=32)
    g, _ = ties_parity(b, 16)
    grad_check(b, g, synth.normal(6, 1, g.num_edges))


# ------------------------------------------------------------------ triplets (Gamma_2)

def _oracle_triplets_check(got_g, tr, include_self):
    want = oracle.triplets(got_g["src"], include_self=include_self)
    assert tr.count == want["a"].shape[0]
    np.testing.assert_array_equal(tr.edge_b.cpu().numpy(), want["b"])
    if tr.edge_a is not None:
        np.testing.assert_array_equal(tr.edge_a.cpu().numpy(), want["a"])
    ptr = np.searchsorted(want["a"], np.arange(got_g["src"].shape[0] + 1))
    np.testing.assert_array_equal(tr.trip_ptr.cpu().numpy(), ptr)


def test_triplets_closed_form_on_gpu():
    d = GOLD["triplets_sc"]
    b = synth.crystal(np.eye(3), [[0, 0, 0]])
    g = mg.cutoff_graph(to_device(b), d["cutoff"])
    assert mg.triplets(g).count == d["with_self"]
    assert mg.triplets(g, include_self=False).count == d["without_self"]


@pytest.mark.parametrize("include_self", [True, False])
def test_triplets_config1_cutoff_and_config2_knn(include_self):
    b1 = synth.make_batch(1)
    g1 = mg.cutoff_graph(to_device(b1), 5.0)
    _oracle_triplets_check(graph_arrays(g1), mg.triplets(g1, include_self=include_self), include_self)
    b2 = synth.make_batch(2, B=64)
    g2 = mg.knn_graph(to_device(b2), 16)
    tr = mg.triplets(g2, include_self=include_self, with_edge_a=include_self)
    _oracle_triplets_check(graph_arrays(g2), tr, include_self)


def test_triplets_full_size_sampled():
    """The bench workload's cutoff graph (tens of millions of triplets): the count is
    the sum of squared degrees and sampled triplets follow from the definition."""
    b = synth.make_batch(2)
    g = mg.cutoff_graph(to_device(b), 6.0, with_perm=False)
    got = graph_arrays(g)
    tr = mg.triplets(g, capacity=1024)  # forces the capacity retry
    deg = np.diff(got["src_ptr"]).astype(np.int64)
    assert tr.count == int(np.sum(deg * deg))
    rng = np.random.default_rng(7)
    q = np.sort(rng.choice(tr.count, 4096, replace=False))
    a = tr.edge_a.cpu().numpy()[q]
    bb = tr.edge_b.cpu().numpy()[q]
    np.testing.assert_array_equal(got["src"][a], got["src"][bb])  # same source
    tp = tr.trip_ptr.cpu().numpy()
    e = np.searchsorted(tp, q, side="right") - 1
    np.testing.assert_array_equal(a, e)
    lo = got["src_ptr"][got["src"][e]]
    np.testing.assert_array_equal(bb, lo + (q - tp[e]))


# ------------------------------------------------------------------ symmetric closure

def sym_parity(b, g):
    s = mg.symmetrize(g)
    got_in = graph_arrays(g)
    got = graph_arrays(s)
    want = oracle.symmetrize(got_in["src"], got_in["dst"], got_in["offset"])
    assert_same_edges(got, want, "symmetric closure")
    pointers_ok(got, b)
    assert_vectors(b, got)
    assert_perm_dst(got, b.total_atoms)
    return s, got


def test_symmetrize_closed_form_on_gpu():
    b = synth.crystal(np.eye(3), [[0, 0, 0]])
    g = mg.knn_graph(to_device(b), 8)
    s, got = sym_parity(b, g)
    assert got["offset"].tolist() == GOLD["symmetrize_sc_k8"]["offsets"]


@pytest.mark.parametrize("cfg,k", [(1, 12), (2, 16), (3, 32)])
def test_symmetrize_knn_graphs(cfg, k):
    b = synth.make_batch(cfg, B=None if cfg == 1 else 128)
    sym_parity(b, mg.knn_graph(to_device(b), k))


def test_symmetrize_cutoff_graph_is_identity_and_per_atom_closure():
    b = synth.make_batch(2, B=64)
    batch = to_device(b)
    g = mg.cutoff_graph(batch, 6.0)
    s, got = sym_parity(b, g)
    ref = graph_arrays(g)
    for key in ("src", "dst", "offset", "edge_ptr", "src_ptr"):
        np.testing.assert_array_equal(got[key], ref[key], err_msg=key)
    ga = mg.cutoff_graph_atoms(batch, torch.from_numpy(radii_for(b, 3, 3.0, 7.0)).cuda())
    sym_parity(b, ga)


def test_symmetrize_keep_ties_graph():
    L = np.eye(3) * 2.0
    x = [[a, b_, c] for a in (0, .5) for b_ in (0, .5) for c in (0, .5)]
    b = synth.concat([synth.crystal(L, x), synth.make_batch(1, B=4)])
    sym_parity(b, mg.knn_graph(to_device(b), 7, keep_ties=True))


def test_symmetrized_graph_backward_uses_reverse_edges():
    """The closure is recorded as symmetric: its backward (reverse-edge path) against the
    oracle gradient, and equal to the destination-order path on the same edges."""
    b = synth.make_batch(2, B=48)
    batch = to_device(b)
    s, _ = sym_parity(b, mg.knn_graph(batch, 16))
    w = synth.normal(8, 0, s.num_edges)
    grad_check(b, s, w)
    gl = torch.from_numpy(w).cuda()
    v, ln = mg.edge_vectors_fwd(s)
    f1, L1 = mg.edge_vectors_bwd(s, batch, None, gl, v, ln)
    assert mg.last_launch_count() == 2  # symmetric path: bwd_sym + bwd_lat
    # the same edges in other buffers are not recorded as symmetric: destination order
    c = dataclasses.replace(s, src=s.src.clone(), dst=s.dst.clone(), offset=s.offset.clone(),
                            edge_ptr=s.edge_ptr.clone(), src_ptr=s.src_ptr.clone(), perm_dst=s.perm_dst.clone(),
                            dst_ptr=s.dst_ptr.clone(), _c=None)
    f2, L2 = mg.edge_vectors_bwd(c, batch, None, gl, v, ln)
    assert mg.last_launch_count() == 3  # bwd_src + bwd_dst + bwd_lat
    torch.testing.assert_close(f1, f2, rtol=1e-5, atol=1e-5 * float(f2.abs().max()))
    torch.testing.assert_close(L1, L2, rtol=1e-5, atol=1e-5 * float(L2.abs().max()))


# ------------------------------------------------------------------ symmetric backward paths

def test_symmetric_backward_pair_table_and_search_paths_identical():
    """The reverse-edge backward finds reverse edges through the build's pair table
    (structures of <= 512 atoms) or by binary search; both give bit-identical sums.
    A per-structure rebuild records no pair table, so the same graph then takes the
    search path."""
    b = synth.make_batch(3, B=160)  # structures of 1 to about 400 atoms
    assert int(np.diff(b.atom_ptr).max()) > 128
    batch = to_device(b)
    g = mg.cutoff_graph(batch, 5.0, with_perm=False)
    gl = torch.from_numpy(synth.normal(12, 0, g.num_edges)).cuda()
    v, ln = mg.edge_vectors_fwd(g)
    f1, L1 = mg.edge_vectors_bwd(g, batch, None, gl, v, ln)
    mg.rebuild(g, per_structure=True)
    v2, ln2 = mg.edge_vectors_fwd(g)
    assert torch.equal(v, v2) and torch.equal(ln, ln2)
    f2, L2 = mg.edge_vectors_bwd(g, batch, None, gl, v2, ln2)
    assert torch.equal(f1, f2) and torch.equal(L1, L2)
    grad_check(b, g, synth.normal(12, 0, g.num_edges))


def test_knn_band_past_the_kept_images_takes_the_second_scan():
    """FCC shells hold 12, 6 and 24 images: at k = 20 the k-th distance lies in a shell
    that runs past the 32 images pass 1 keeps, so the selection scans again; exact-k
    ties broken by (d2, j, t) and keep-ties (all 42) both match the oracle."""
    a = 3.0
    b = synth.crystal(np.asarray(GOLD["knn_keep_ties_fcc"]["lattice_over_a"]) * a, [[0, 0, 0]])
    g = mg.knn_graph(to_device(b), 20)
    got = graph_arrays(g)
    assert_same_edges(got, oracle.knn(b.lattice, b.frac, b.atom_ptr, 20), "fcc k=20")
    gt, _ = ties_parity(b, 20)
    assert gt.num_edges == 42


# ------------------------------------------------------------------ the two cutoff builds

@pytest.mark.parametrize("schedule", [3, 4])
def test_one_pass_and_staged_builds_match_the_oracle(schedule):
    """schedule 3 forces the one-pass build (look-back), 4 the staged build (scan and
    stage, scan the counts, write); both are exact on every kind of source: all-pairs,
    cell-list, per-atom radii and keep-ties KNN."""
    opts = mg.make_opts(schedule=schedule)
    b = synth.make_batch(2, B=96)
    cutoff_got = graph_arrays(mg.cutoff_graph(to_device(b), 6.0, opts=opts))
    assert_same_edges(cutoff_got, oracle.cutoff(b.lattice, b.frac, b.atom_ptr, 6.0), "cutoff")
    assert_perm_dst(cutoff_got, b.total_atoms)
    b5 = synth.make_batch(5).subset([0])
    g5 = mg.cutoff_graph(to_device(b5), 8.0, with_perm=False, opts=opts)
    got5 = graph_arrays(g5)
    srcs = np.arange(0, b5.total_atoms, 97, dtype=np.int32)
    want5 = oracle.cutoff(b5.lattice, b5.frac, b5.atom_ptr, 8.0, sources=srcs)
    sel = np.concatenate([np.arange(got5["src_ptr"][s], got5["src_ptr"][s + 1]) for s in srcs])
    assert_same_edges({k: got5[k][sel] for k in ("src", "dst", "offset")}, want5, "cell-list")
    radii = radii_for(b, 17, 3.0, 6.0)
    ga = mg.cutoff_graph_atoms(to_device(b), torch.from_numpy(radii).cuda(), opts=opts)
    assert_same_edges(graph_arrays(ga), oracle.cutoff_atoms(b.lattice, b.frac, b.atom_ptr,
                                                            radii.astype(np.float64)), "per-atom")
    gk = mg.knn_graph(to_device(b), 16, keep_ties=True, opts=opts)
    assert_same_edges(graph_arrays(gk), oracle.knn(b.lattice, b.frac, b.atom_ptr, 16, keep_ties=True), "ties")
    # the symmetric backward reads the pair table either build records
    batch = to_device(b)
    g = mg.cutoff_graph(batch, 6.0, with_perm=False, opts=opts)
    grad_check(b, g, synth.normal(21, schedule, g.num_edges))


@pytest.mark.parametrize("schedule", [3, 4])
def test_elongated_cells_in_every_axis_order(schedule):
    """Cells whose shortest direction is lattice axis 0, 1 or 2, and a skewed one: the
    staged build (schedule 4) scans the first two with that axis innermost and restores
    canonical order per target; the one-pass build (schedule 3) scans in lattice order.
    Both give the oracle's edges, in canonical order, and the same gradients."""
    kinds = np.array([
        [[3.1, 0.0, 0.0], [1.0, 10.5, 0.0], [2.0, -1.5, 12.0]],    # shortest along L_0
        [[10.5, 0.0, 0.0], [1.2, 3.2, 0.0], [2.1, 1.3, 11.8]],     # shortest along L_1
        [[11.0, 0.0, 0.0], [1.0, 10.8, 0.0], [0.5, 0.7, 3.3]],     # shortest along L_2
        [[4.29, 0.0, 0.0], [0.69, 5.02, 0.0], [6.39, -3.69, 11.62]],  # skewed, long L_2
    ])
    b0 = synth.make_batch(2, B=64)
    lat = np.stack([kinds[s % len(kinds)] for s in range(b0.num_structures)])
    b = synth.Batch(lat, b0.frac, b0.atom_ptr)
    opts = mg.make_opts(schedule=schedule)
    got = graph_arrays(mg.cutoff_graph(to_device(b), 6.0, opts=opts))
    assert_same_edges(got, oracle.cutoff(b.lattice, b.frac, b.atom_ptr, 6.0), "elongated")
    assert_vectors(b, got)
    assert_perm_dst(got, b.total_atoms)
    g = mg.cutoff_graph(to_device(b), 6.0, with_perm=False, opts=opts)
    grad_check(b, g, synth.normal(23, schedule, g.num_edges))


def test_fused_lattice_reduction_with_empty_structures():
    """The symmetric backward reduces each structure's lattice gradient in the last warp
    to finish it; empty structures (first, middle, last) still get a zero gradient, and
    the result equals the separate reduction kernel bit for bit."""
    parts = [synth.make_batch(2, B=6)]
    b0 = synth.concat(parts)
    counts = [0] + np.diff(b0.atom_ptr).tolist()[:3] + [0, 0] + np.diff(b0.atom_ptr).tolist()[3:] + [0]
    lat = np.concatenate([np.eye(3, dtype=np.float32)[None] * 4, b0.lattice[:3],
                          np.eye(3, dtype=np.float32)[None].repeat(2, 0) * 5, b0.lattice[3:],
                          np.eye(3, dtype=np.float32)[None] * 6])
    ptr = np.concatenate([[0], np.cumsum(counts)]).astype(np.int32)
    b = synth.Batch(lat, b0.frac, ptr)
    batch = to_device(b)
    g = mg.cutoff_graph(batch, 5.0, with_perm=False)
    gl = torch.from_numpy(synth.normal(31, 0, g.num_edges)).cuda()
    v, ln = mg.edge_vectors_fwd(g)
    gf_fused = torch.full((b.total_atoms, 3), float("nan"), device="cuda")
    gL_fused = torch.full((b.num_structures, 3, 3), float("nan"), device="cuda")
    mg.edge_vectors_bwd(g, batch, None, gl, v, ln, gf_fused, gL_fused)
    assert mg.last_launch_count() == 1  # the reduction joined the backward kernel
    for s in np.flatnonzero(np.diff(ptr) == 0):
        assert torch.all(gL_fused[s] == 0)
    mg.rebuild(g, per_structure=True)  # no pair table, no counters: the separate kernel
    v2, ln2 = mg.edge_vectors_fwd(g)
    gf2, gL2 = mg.edge_vectors_bwd(g, batch, None, gl, v2, ln2)
    assert mg.last_launch_count() == 2
    assert torch.equal(gf_fused, gf2) and torch.equal(gL_fused, gL2)
    grad_check(b, g, synth.normal(31, 1, g.num_edges))


def test_symmetric_backward_large_structures_and_grad_vec():
    """Structures above 1024 atoms: the symmetric backward followed by the block-per-
    structure lattice reduction.  Both incoming gradients (grad_vec and grad_len)
    against the oracle; deterministic."""
    b = synth.make_batch(5, B=4)
    assert int(np.diff(b.atom_ptr).max()) > 1024
    batch = to_device(b)
    g = mg.cutoff_graph(batch, 5.0, with_perm=False)
    E = g.num_edges
    v, ln = mg.edge_vectors_fwd(g)
    gv = torch.from_numpy(synth.normal(41, 0, 3 * E).reshape(-1, 3)).cuda()
    gl = torch.from_numpy(synth.normal(41, 1, E)).cuda()
    f1, L1 = mg.edge_vectors_bwd(g, batch, gv, gl, v, ln)
    assert mg.last_launch_count() == 2  # bwd_sym + the block-per-structure reduction
    f2, L2 = mg.edge_vectors_bwd(g, batch, gv, gl, v, ln)
    assert torch.equal(f1, f2) and torch.equal(L1, L2)
    got = graph_arrays(g)
    assert_grad_bound(b, got, gv.cpu().numpy(), gl.cpu().numpy(), f1.cpu().numpy(), L1.cpu().numpy())
    grad_check(b, g, synth.normal(41, 2, E), c=synth.normal(41, 3, 3 * E).reshape(-1, 3))


@pytest.mark.parametrize("schedule", [3, 4])
def test_sources_beyond_the_shared_staging_are_enumerated_again(schedule):
    """A source with more than 1024 edges does not fit the shared-memory staging: both
    builds count it, then enumerate it again in canonical order (here one atom in a
    unit cube at cutoff 7.3: every image within 7.3 of it, ~1600 edges, next to normal
    sources)."""
    opts = mg.make_opts(schedule=schedule)
    b = synth.concat([synth.crystal(np.eye(3), [[0.1, 0.2, 0.3]]), synth.make_batch(1, B=3)])
    g = mg.cutoff_graph(to_device(b), 7.3, opts=opts)
    got = graph_arrays(g)
    want = oracle.cutoff(b.lattice, b.frac, b.atom_ptr, 7.3)
    assert np.diff(got["src_ptr"]).max() > 1024
    assert_same_edges(got, want, "spilled source")
    assert_vectors(b, got)
    assert_perm_dst(got, b.total_atoms)
    grad_check(b, g, synth.normal(41, schedule, g.num_edges))


def test_staged_build_replay_and_device_errors():
    """The staged build captured in a plan and replayed for moving geometry, and a
    structure with bad input reported while the others are still built."""
    opts = mg.make_opts(schedule=4)
    b = synth.make_batch(4, B=64)
    batch = to_device(b)
    g = mg.cutoff_graph(batch, 5.0, capacity=400000, opts=opts)
    cur = b
    for step in range(3):
        cur = synth.perturb(cur, seed=13, step=step)
        g = mg.update_graph(g, torch.from_numpy(cur.frac).cuda(), torch.from_numpy(cur.lattice).cuda())
        got = graph_arrays(g)
        assert_same_edges(got, oracle.cutoff(cur.lattice, cur.frac, cur.atom_ptr, 5.0), f"step {step}")
        assert_vectors(cur, got)
    grad_check(cur, g, synth.normal(51, 0, g.num_edges))
    bad = synth.make_batch(1, B=3)
    lat = bad.lattice.copy()
    lat[1] = 0.0  # singular
    gb = mg.cutoff_graph(to_device(synth.Batch(lat, bad.frac, bad.atom_ptr)), 5.0, sync=False, opts=opts)
    st = gb.read_status()
    assert st["code"] == 3 and st["first_bad_structure"] == 1
    want = oracle.cutoff(bad.lattice[:1], bad.frac[:bad.atom_ptr[1]], bad.atom_ptr[:2], 5.0)
    assert int(gb.edge_ptr[1].item()) == len(want["src"])


# ------------------------------------------------------------------ host copies

def test_graph_to_host_matches_device_arrays():
    """mg_graph_to_host copies the first num_edges rows, the pointers and the status word
    of each requested field (pinned buffers, asynchronous on the current stream)."""
    b = synth.make_batch(2, B=48)
    batch = to_device(b)
    for g in (mg.cutoff_graph(batch, 6.0, with_perm=False), mg.knn_graph(batch, 12, with_perm=False)):
        E = g.num_edges
        out = mg.host_buffers(g, E)
        mg.graph_to_host(g, out, E)
        torch.cuda.current_stream().synchronize()
        assert torch.equal(out["status"], g.status.cpu())
        for f in ("src", "dst", "offset", "vec", "len"):
            assert torch.equal(out[f], getattr(g, f)[:E].cpu()), f
        assert torch.equal(out["edge_ptr"], g.edge_ptr.cpu()) and torch.equal(out["src_ptr"], g.src_ptr.cpu())
        part = mg.host_buffers(g, 10, ("src", "len"))  # a subset, fewer rows
        mg.graph_to_host(g, part, 10)
        torch.cuda.current_stream().synchronize()
        assert torch.equal(part["src"], g.src[:10].cpu()) and torch.equal(part["len"], g.len[:10].cpu())
    with pytest.raises(RuntimeError, match="INVALID_ARGUMENT"):
        mg.graph_to_host(g, part, g.capacity + 1)


def test_plans_recorded_again_when_profiling_changes():
    """A plan recorded without stage events is recorded again with them once profiling is
    on (and the stage times appear), and again without them when it is off; the edges
    stay identical."""
    b = synth.make_batch(2, B=32)
    batch = to_device(b)
    mg.profile_enable(False)
    g = mg.cutoff_graph(batch, 6.0, with_perm=False)
    mg.update_graph(g)
    want = graph_arrays(g)
    mg.profile_enable(True)
    mg.update_graph(g)
    stages = mg.stage_times("cutoff")
    assert "build" in stages and all(v >= 0 for v in stages.values()), stages
    assert_same_edges(graph_arrays(g), want, "profiled replay")
    mg.profile_enable(False)
    mg.update_graph(g)
    assert_same_edges(graph_arrays(g), want, "replay without events")


def test_measured_fp_peaks_are_plausible():
    """The library's FMA issue-rate kernel: FP32 within a factor of two of the nominal
    152 SM x 128 lanes x 2 flops x clock (80.5 TFLOP/s at 2070 MHz), FP64 at a small
    fraction of it (this GPU's FP64 pipe is narrow), both positive and finite."""
    p = mg.measure_fp_peaks(torch.device("cuda:0"))
    assert 40.0 < p["fp32_tflops"] < 160.0, p
    assert 0.0 < p["fp64_tflops"] < 0.25 * p["fp32_tflops"], p


def test_graph_step_one_call_matches_the_oracle_and_separate_calls():
    """mg_graph_step: new coordinates copied in from pinned host memory, the cutoff graph
    and the KNN graph (on a second stream) rebuilt and copied out, edge vectors and the
    backward of a length gradient, results copied out, all from one call.  The host
    copies of both graphs equal the oracle's graphs of the new geometry; the gradients
    equal those of separate library calls, bit for bit."""
    b = synth.make_batch(2)
    batch = to_device(b)
    s0, s1, s2 = torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.Stream()
    with torch.cuda.stream(s0):
        g_cut = mg.cutoff_graph(batch, 6.0, with_perm=False)
        g_knn = mg.knn_graph(batch, 16, with_perm=False)
    cur = synth.perturb(b, seed=3, step=1)
    inputs = {"frac": torch.from_numpy(cur.frac).pin_memory(), "lattice": torch.from_numpy(cur.lattice).pin_memory()}
    cap = g_cut.capacity
    host_cut = mg.host_buffers(g_cut, cap, ("status", "src", "dst", "offset", "src_ptr"))
    host_knn = mg.host_buffers(g_knn, g_knn.capacity, ("status", "src", "dst", "offset", "vec", "len"))
    gl = torch.from_numpy(synth.normal(6, 1, cap)).cuda()
    vec = torch.empty(cap, 3, device="cuda")
    ln = torch.empty(cap, device="cuda")
    gf = torch.empty(b.total_atoms, 3, device="cuda")
    gL = torch.empty(b.num_structures, 3, 3, device="cuda")
    out = {"grad_frac": torch.empty(b.total_atoms, 3).pin_memory(),
           "grad_lattice": torch.empty(b.num_structures, 3, 3).pin_memory(),
           "len": torch.empty(cap).pin_memory()}
    step = mg.Step([g_cut, g_knn], [s0, s1, s2], host=(host_cut, host_knn), inputs=inputs, grad_len=gl, vec=vec, ln=ln,
                   grad_frac=gf, grad_lattice=gL, outputs=out, host_edges=(cap, g_knn.capacity))
    for _ in range(2):  # twice: the argument block is reused
        step.run()
        s0.synchronize()
    st = host_cut["status"]
    assert int(st[0]) & 0xFFFFFFFF == 0
    E = int(st[1])
    want = oracle.cutoff(cur.lattice, cur.frac, cur.atom_ptr, 6.0)
    got = {"src": host_cut["src"][:E].numpy(), "dst": host_cut["dst"][:E].numpy(), "offset": host_cut["offset"][:E].numpy()}
    assert_same_edges(got, want, "step: cutoff graph of the new geometry")
    kst = host_knn["status"]
    Ek = int(kst[1])
    kgot = {"src": host_knn["src"][:Ek].numpy(), "dst": host_knn["dst"][:Ek].numpy(),
            "offset": host_knn["offset"][:Ek].numpy(), "vec": host_knn["vec"][:Ek].numpy(),
            "len": host_knn["len"][:Ek].numpy()}
    assert_same_edges(kgot, oracle.knn(cur.lattice, cur.frac, cur.atom_ptr, 16), "step: knn graph")
    assert_vectors(cur, kgot)
    with torch.cuda.stream(s0):
        g_cut.num_edges = E
        f2, L2 = mg.edge_vectors_bwd(g_cut, batch, None, gl, vec, ln)
    s0.synchronize()
    assert torch.equal(out["grad_frac"], f2.cpu()) and torch.equal(out["grad_lattice"], L2.cpu())
    assert torch.equal(out["len"][:E], ln[:E].cpu())
    # the same step enqueued call by call (not recorded): the same results
    out2 = {key: torch.empty_like(v).pin_memory() for key, v in out.items()}
    step2 = mg.Step([g_cut, g_knn], [s0, s1, s2], host=(host_cut, host_knn), inputs=inputs, grad_len=gl, vec=vec,
                    ln=ln, grad_frac=gf, grad_lattice=gL, outputs=out2, host_edges=(cap, g_knn.capacity),
                    capture=False)
    step2.run()
    s0.synchronize()
    for key in out:
        assert torch.equal(out[key], out2[key]), key
