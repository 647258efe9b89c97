"""Pins for the oracle's per-atom cutoff, keep-ties KNN, symmetric closure and triplet
functions (no GPU).

Closed forms (tests/golden/next_rows.json), a separate brute force on tiny inputs written
with Cartesian matrix products instead of the oracle's canonical formula, and the
invariants the definitions imply.
"""
import itertools
import json
import os

import numpy as np
import pytest

import oracle
import synth

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "next_rows.json")))


def edge_set(g):
    return {(int(s), int(d), tuple(int(v) for v in t)) for s, d, t in zip(g["src"], g["dst"], g["offset"])}


def canonical(g):
    keys = list(zip(g["src"].tolist(), g["dst"].tolist(), [tuple(t) for t in g["offset"].tolist()]))
    return keys == sorted(keys)


def small_batch(seed, B=3):
    return synth.make_batch(1, seed=seed, B=B).subset(list(range(B)))


def brute_images(L, x, i, box=5):
    """Every image (j, t) != (i, 0) of atom i within |t_k| <= box, with its Cartesian
    squared distance from a matrix product (a different evaluation order from the
    oracle's canonical one)."""
    n = x.shape[0]
    out = []
    for j in range(n):
        for t in itertools.product(range(-box, box + 1), repeat=3):
            if j == i and t == (0, 0, 0):
                continue
            v = (x[j] - x[i] + np.asarray(t, float)) @ L
            out.append((float(v @ v), j, t))
    return out


# ------------------------------------------------------------------ per-atom cutoffs

def test_per_atom_cutoff_closed_forms():
    d = GOLD["per_atom_cutoff_sc_pair"]
    L = np.asarray(d["lattice"], float)[None]
    x = np.asarray(d["frac"], float)
    ptr = np.array([0, 2], np.int32)
    for radii, degs in d["cases"]:
        g = oracle.cutoff_atoms(L, x, ptr, radii)
        assert np.bincount(g["src"], minlength=2).tolist() == degs, radii
        assert canonical(g)


@pytest.mark.parametrize("seed", [11, 12, 13])
def test_per_atom_cutoff_brute_force(seed):
    b = small_batch(seed)
    rng = np.random.default_rng(seed)
    radii = rng.uniform(2.0, 5.0, size=b.frac.shape[0])
    g = oracle.cutoff_atoms(b.lattice, b.frac, b.atom_ptr, radii)
    want = set()
    for s in range(b.num_structures):
        lo, hi = int(b.atom_ptr[s]), int(b.atom_ptr[s + 1])
        L = b.lattice[s].astype(float)
        x = b.frac[lo:hi].astype(float)
        for i in range(hi - lo):
            c = radii[lo + i]
            for d2, j, t in brute_images(L, x, i):
                assert abs(np.sqrt(d2) - c) > 1e-9  # no edge sits on the sphere
                if d2 < c * c:
                    want.add((lo + i, lo + j, t))
    assert edge_set(g) == want
    assert canonical(g)


def test_per_atom_cutoff_is_the_sources_constant_cutoff_graph_and_asymmetric():
    b = small_batch(21)
    rng = np.random.default_rng(21)
    radii = rng.uniform(2.5, 5.0, size=b.frac.shape[0])
    g = edge_set(oracle.cutoff_atoms(b.lattice, b.frac, b.atom_ptr, radii))
    for a in range(b.frac.shape[0]):
        r = float(radii[a])
        ref = oracle.cutoff(b.lattice, b.frac, b.atom_ptr, r, sources=[a])
        assert {e for e in g if e[0] == a} == edge_set(ref)
    # an edge and its reverse are both present exactly when d < min(c_i, c_j)
    full = oracle.cutoff_atoms(b.lattice, b.frac, b.atom_ptr, radii)
    for s, d, t, d2 in zip(full["src"], full["dst"], full["offset"], full["d2"]):
        rev = (int(d), int(s), tuple(-int(v) for v in t))
        assert (rev in g) == (d2 < min(radii[s], radii[d]) ** 2)


def test_per_atom_cutoff_rejects_bad_radius():
    b = small_batch(3)
    radii = np.full(b.frac.shape[0], 3.0)
    radii[1] = 0.0
    with pytest.raises(RuntimeError):
        oracle.cutoff_atoms(b.lattice, b.frac, b.atom_ptr, radii)


# ------------------------------------------------------------------ keep-ties KNN

@pytest.mark.parametrize("name", ["knn_keep_ties_sc", "knn_keep_ties_fcc", "knn_keep_ties_bcc"])
def test_keep_ties_closed_forms(name):
    d = GOLD[name]
    L = np.asarray(d.get("lattice_over_a", np.eye(3)), float) * 3.0
    b = synth.crystal(L, [[0, 0, 0]])
    for k, m in d["cases"]:
        g = oracle.knn(b.lattice, b.frac, b.atom_ptr, k, keep_ties=True)
        assert len(g["src"]) == m, (name, k)
        assert canonical(g)


@pytest.mark.parametrize("seed", [31, 32])
def test_keep_ties_brute_force(seed):
    b = small_batch(seed)
    for k in (3, 7):
        g = oracle.knn(b.lattice, b.frac, b.atom_ptr, k, keep_ties=True)
        want = set()
        for s in range(b.num_structures):
            lo, hi = int(b.atom_ptr[s]), int(b.atom_ptr[s + 1])
            L = b.lattice[s].astype(float)
            x = b.frac[lo:hi].astype(float)
            for i in range(hi - lo):
                imgs = sorted(brute_images(L, x, i, box=3))
                D = imgs[k - 1][0]
                for d2, j, t in imgs:
                    if d2 <= D * (1 + 1e-12):
                        want.add((lo + i, lo + j, t))
        assert edge_set(g) == want


def test_keep_ties_extends_exact_k_by_the_kth_shell_only():
    # a perfect 2x2x2 supercell has many exact ties; generic coordinates only those of
    # an atom's own images
    L = np.eye(3) * 2.0
    x = np.array([[a, b, c] for a in (0, .5) for b in (0, .5) for c in (0, .5)], float)
    crystal = synth.crystal(L, x)
    generic = small_batch(41)
    for b in (crystal, generic):
        for k in (5, 9, 20):
            ex = oracle.knn(b.lattice, b.frac, b.atom_ptr, k)
            kt = oracle.knn(b.lattice, b.frac, b.atom_ptr, k, keep_ties=True)
            es, ts = edge_set(ex), edge_set(kt)
            assert es <= ts
            N = b.frac.shape[0]
            Dk = np.zeros(N)
            for s, d2 in zip(ex["src"], ex["d2"]):
                Dk[s] = max(Dk[s], d2)
            for s, d, t, d2 in zip(kt["src"], kt["dst"], kt["offset"], kt["d2"]):
                assert d2 <= Dk[s]
                if (int(s), int(d), tuple(int(v) for v in t)) not in es:
                    assert d2 == Dk[s]
            if b is generic:
                # the only exact ties left are an atom's own images t and -t (bit-equal d2)
                for (i, j, t) in ts - es:
                    assert i == j and (i, j, tuple(-v for v in t)) in es


# ------------------------------------------------------------------ symmetric closure

def test_symmetrize_closed_form():
    b = synth.crystal(np.eye(3), [[0, 0, 0]])
    g = oracle.knn(b.lattice, b.frac, b.atom_ptr, 8)
    s = oracle.symmetrize(g["src"], g["dst"], g["offset"])
    assert s["offset"].tolist() == GOLD["symmetrize_sc_k8"]["offsets"]


@pytest.mark.parametrize("seed", [51, 52])
def test_symmetrize_fixes_cutoff_graphs_and_closes_knn_graphs(seed):
    b = small_batch(seed, B=4)
    c = oracle.cutoff(b.lattice, b.frac, b.atom_ptr, 4.0)
    sc = oracle.symmetrize(c["src"], c["dst"], c["offset"])
    assert edge_set(sc) == edge_set(c)  # a constant-cutoff graph is already symmetric
    for k in (4, 9):
        g = oracle.knn(b.lattice, b.frac, b.atom_ptr, k)
        s = oracle.symmetrize(g["src"], g["dst"], g["offset"])
        es, gs = edge_set(s), edge_set(g)
        assert len(es) == len(s["src"])  # each edge once
        assert canonical(s)
        assert gs <= es
        for (i, j, t) in es:
            rev = (j, i, tuple(-v for v in t))
            assert rev in es
            assert (i, j, t) in gs or rev in gs  # nothing beyond the closure


# ------------------------------------------------------------------ triplets

def test_triplets_closed_form():
    d = GOLD["triplets_sc"]
    b = synth.crystal(np.eye(3), [[0, 0, 0]])
    g = oracle.cutoff(b.lattice, b.frac, b.atom_ptr, d["cutoff"])
    assert len(oracle.triplets(g["src"])["a"]) == d["with_self"]
    assert len(oracle.triplets(g["src"], include_self=False)["a"]) == d["without_self"]


@pytest.mark.parametrize("include_self", [True, False])
def test_triplets_brute_force_and_count(include_self):
    b = small_batch(61, B=2)
    g = oracle.cutoff(b.lattice, b.frac, b.atom_ptr, 3.0)
    tr = oracle.triplets(g["src"], include_self=include_self)
    src = g["src"]
    E = src.shape[0]
    want = [(e, f) for e in range(E) for f in range(E) if src[e] == src[f] and (include_self or e != f)]
    got = list(zip(tr["a"].tolist(), tr["b"].tolist()))
    assert got == want
    deg = np.bincount(src, minlength=b.frac.shape[0]).astype(np.int64)
    assert len(got) == int(np.sum(deg * (deg if include_self else deg - 1)))
