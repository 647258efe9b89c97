"""Pins for the FP64 oracle, independent of the oracle's own code (no GPU).

Closed forms (tests/golden/closed_forms.json), invariants the definition implies, a
separate brute force on tiny inputs, and central finite differences for the gradient.
"""
import itertools
import json
import math
import os

import numpy as np
import pytest

import oracle
import synth

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "closed_forms.json")))


def edge_set(g):
    return {(int(s), int(d), tuple(int(v) for v in t)) for s, d, t in zip(g["src"], g["dst"], g["offset"])}


def cut(b, r, **kw):
    return oracle.cutoff(b.lattice, b.frac, b.atom_ptr, r, **kw)


def knn(b, k, **kw):
    return oracle.knn(b.lattice, b.frac, b.atom_ptr, k, **kw)


def degrees(g, n):
    return np.bincount(g["src"], minlength=n)


# ------------------------------------------------------------------ closed forms

def test_sc_degrees_and_strict_cutoff():
    d = GOLD["sc_cutoff_degree"]
    b = synth.crystal(d["lattice"], d["frac"])
    for r, deg in d["cases"]:
        assert len(cut(b, r)["src"]) == deg, r


def test_sc_shell_counts_match_sums_of_three_squares():
    d = GOLD["sc_shell_counts"]
    b = synth.crystal(np.eye(3), [[0, 0, 0]])
    g = cut(b, 3.01)
    # squared lengths of integer vectors are exact in FP64
    for m, r3 in zip(d["m"], d["r3"]):
        assert int(np.sum(g["d2"] == m)) == r3, m
        # independent direct count of integer vectors
        direct = sum(1 for t in itertools.product(range(-3, 4), repeat=3) if t[0] ** 2 + t[1] ** 2 + t[2] ** 2 == m)
        assert direct == r3


@pytest.mark.parametrize("name", ["fcc_primitive", "bcc_primitive"])
def test_cubic_primitive_shells(name):
    d = GOLD[name]
    a = d["a"]
    b = synth.crystal(np.asarray(d["lattice_over_a"]) * a, [[0, 0, 0]])
    g = knn(b, d["k"])
    assert len(g["src"]) == d["k"]
    np.testing.assert_allclose(np.sqrt(g["d2"]), d["first_shell_over_a"] * a, rtol=1e-6)
    mid = 0.5 * (d["first_shell_over_a"] + d["second_shell_over_a"]) * a
    assert len(cut(b, mid)["src"]) == d["first_shell_count"]
    # second shell adds 6
    assert len(cut(b, 1.05 * a)["src"]) == d["first_shell_count"] + 6


@pytest.mark.parametrize("name", ["fcc_conventional", "bcc_conventional"])
def test_conventional_cells(name):
    d = GOLD[name]
    a = d["a"]
    b = synth.crystal(np.eye(3) * a, d["frac"])
    g = cut(b, d["cutoff_over_a"] * a)
    assert np.all(degrees(g, len(d["frac"])) == d["degree"])


def test_hexagonal_non_symmetric_lattice():
    d = GOLD["hexagonal"]
    a, c = d["a"], d["c"]
    L = [[a, 0, 0], [-a / 2, a * np.sqrt(3) / 2, 0], [0, 0, c]]
    b = synth.crystal(L, [[0.1, 0.2, 0.3]])
    for r, deg in d["cases"]:
        assert len(cut(b, r)["src"]) == deg, r


def test_knn_tiebreak_sc():
    d = GOLD["sc_knn_tiebreak"]
    b = synth.crystal(np.eye(3), [[0.25, 0.5, 0.75]])
    g = knn(b, d["k"])
    assert g["offset"].tolist() == d["offsets"]


@pytest.mark.parametrize("shape", ["needle", "rotated", "skewed"])
def test_knn_needle_cell_closed_form(shape):
    """One atom in a 1 x 10 x 10 A cell: every image off the L_0 line is at least 10 A away
    (for the skewed cell too: its L_1 and L_2 move y by 10 t_1 + 4 t_2 and z by 10 t_2), so
    for k <= 18 the k nearest are (+-m, 0, 0) at m A, m <= 9, the tie at each m broken
    by t ((-m, 0, 0) first).  The search must grow far along L_0 alone (Alg. 1), and
    Alg. 2's filter keeps both images of the k-th shell."""
    L = {"needle": np.diag([1.0, 10.0, 10.0]),
         "skewed": np.array([[1.0, 0.0, 0.0], [5.0, 10.0, 0.0], [3.0, 4.0, 10.0]])}.get(shape)
    if shape == "rotated":
        c, s_ = math.cos(0.7), math.sin(0.7)
        R = np.array([[c, -s_, 0.0], [s_, c, 0.0], [0.0, 0.0, 1.0]]) @ np.array([[1.0, 0.0, 0.0], [0.0, c, -s_], [0.0, s_, c]])
        L = np.diag([1.0, 10.0, 10.0]) @ R.T
    b = synth.crystal(L, [[0.3, 0.6, 0.2]])
    order = [(sgn * m, 0, 0) for m in range(1, 10) for sgn in (-1, 1)]
    for k in (1, 5, 6, 17, 18):
        g = knn(b, k)
        assert g["offset"].tolist() == sorted(list(t) for t in order[:k])
        l0 = np.linalg.norm(b.lattice[0][0].astype(np.float64))  # |L_0| of the stored FP32 lattice
        np.testing.assert_allclose(np.sort(np.sqrt(g["d2"])), l0 * np.array(sorted(abs(t[0]) for t in order[:k])),
                                   rtol=1e-12)
        ties = oracle.knn(b.lattice, b.frac, b.atom_ptr, k, keep_ties=True)
        shell = abs(order[k - 1][0])
        assert ties["offset"].tolist() == sorted([s * m, 0, 0] for m in range(1, shell + 1) for s in (-1, 1))


def test_triclinic_vectors_hand_computed():
    d = GOLD["triclinic_vectors"]
    b = synth.crystal(d["lattice"], d["frac"])
    src = [e[0] for e in d["edges"]]
    dst = [e[1] for e in d["edges"]]
    off = [e[2] for e in d["edges"]]
    vec, ln = oracle.edge_vectors(b.lattice, b.frac, b.atom_ptr, src, dst, off)
    want = np.array([e[3] for e in d["edges"]])
    np.testing.assert_allclose(vec, want, atol=1e-12)
    np.testing.assert_allclose(ln, np.linalg.norm(want, axis=1), rtol=1e-14)
    # and the cutoff graph finds exactly these vectors' lengths among its edges
    g = cut(b, 5.0)
    s = edge_set(g)
    for e in d["edges"]:
        if np.linalg.norm(e[3]) < 5.0:
            assert (e[0], e[1], tuple(e[2])) in s


# ------------------------------------------------------------------ brute force

def brute_force(b, r=None, k=None, box=5):
    """Independent brute force over a large fixed box |t| <= box (tiny inputs only)."""
    out = []
    for s in range(b.num_structures):
        L = b.lattice[s].astype(np.float64)
        lo, hi = b.atom_ptr[s], b.atom_ptr[s + 1]
        x = b.frac[lo:hi].astype(np.float64)
        ts = np.array(list(itertools.product(range(-box, box + 1), repeat=3)), np.float64)
        for i in range(hi - lo):
            cands = []
            for j in range(hi - lo):
                df = (x[j] - x[i])[None, :] + ts
                v0 = ((df[:, 0] * L[0, 0]) + (df[:, 1] * L[1, 0])) + (df[:, 2] * L[2, 0])
                v1 = ((df[:, 0] * L[0, 1]) + (df[:, 1] * L[1, 1])) + (df[:, 2] * L[2, 1])
                v2 = ((df[:, 0] * L[0, 2]) + (df[:, 1] * L[1, 2])) + (df[:, 2] * L[2, 2])
                d2 = ((v0 * v0) + (v1 * v1)) + (v2 * v2)
                for q in range(len(ts)):
                    t = tuple(int(v) for v in ts[q])
                    if j == i and t == (0, 0, 0):
                        continue
                    cands.append((d2[q], j, t))
            if r is not None:
                sel = [c for c in cands if c[0] < r * r]
            else:
                cands.sort()
                sel = cands[:k]
                # the box must hold every image up to the k-th distance
                assert np.sqrt(sel[-1][0]) * np.linalg.norm(np.linalg.inv(L)) + 1 < box
            for d2, j, t in sorted(sel, key=lambda c: (c[1], c[2])):
                out.append((lo + i, lo + j, t))
    return out


def tiny_batch():
    return synth.concat([synth.make_batch(1, B=3), synth.crystal(np.eye(3) * 2.0, [[0.1, 0.2, 0.3]]),
                         synth.crystal([[3, 0, 0], [2.5, 1.2, 0], [0.3, 0.2, 2.8]], [[0.0, 0.0, 0.0], [0.4, 0.6, 0.5]])])


def test_cutoff_matches_independent_brute_force():
    b = tiny_batch()
    g = cut(b, 3.3)
    got = list(zip(g["src"].tolist(), g["dst"].tolist(), [tuple(t) for t in g["offset"].tolist()]))
    assert got == brute_force(b, r=3.3)  # same set, same canonical order


def test_knn_matches_independent_brute_force():
    b = tiny_batch()
    g = knn(b, 7)
    got = list(zip(g["src"].tolist(), g["dst"].tolist(), [tuple(t) for t in g["offset"].tolist()]))
    assert got == brute_force(b, k=7)


def test_larger_box_same_result():
    b = synth.make_batch(1)
    assert edge_set(cut(b, 5.0)) == edge_set(cut(b, 5.0, extra=2))
    assert edge_set(knn(b, 12)) == edge_set(knn(b, 12, extra=2))


# ------------------------------------------------------------------ invariants

@pytest.fixture(scope="module")
def cfg1():
    return synth.make_batch(1)


def test_edge_symmetry(cfg1):
    s = edge_set(cut(cfg1, 5.0))
    assert s == {(j, i, tuple(-v for v in t)) for i, j, t in s}


def test_canonical_order_and_pointers(cfg1):
    g = cut(cfg1, 5.0)
    keys = np.column_stack([g["src"], g["dst"], g["offset"]])
    order = np.lexsort(keys.T[::-1])
    assert np.all(order == np.arange(len(order)))
    edge_ptr, src_ptr = oracle.pointers(g["src"], cfg1.atom_ptr)
    assert edge_ptr[-1] == len(g["src"])


def test_pointers_against_hand_counted_csr():
    """oracle.pointers against CSR arrays counted by hand (tests/golden/pointers.json):
    empty structures at either end and in the middle, atoms without edges, no edges at
    all.  An off-by-one in the source index (counting at src instead of src + 1) shifts
    every src_ptr entry and fails here."""
    cases = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "pointers.json")))["cases"]
    for c in cases:
        edge_ptr, src_ptr = oracle.pointers(np.asarray(c["src"], np.int32), np.asarray(c["atom_ptr"], np.int32))
        np.testing.assert_array_equal(src_ptr, c["src_ptr"], err_msg=c["what"])
        np.testing.assert_array_equal(edge_ptr, c["edge_ptr"], err_msg=c["what"])


def test_permutation_invariance(cfg1):
    rng = np.random.default_rng(0)
    g = cut(cfg1, 5.0)
    h = knn(cfg1, 12)
    perm = np.arange(cfg1.total_atoms)
    for s in range(cfg1.num_structures):
        lo, hi = cfg1.atom_ptr[s], cfg1.atom_ptr[s + 1]
        perm[lo:hi] = lo + rng.permutation(hi - lo)
    # new row q holds old atom perm[q]
    pb = synth.Batch(cfg1.lattice, cfg1.frac[perm], cfg1.atom_ptr)
    inv = np.empty_like(perm)
    inv[perm] = np.arange(len(perm))
    remap = lambda st: {(int(inv[i]), int(inv[j]), t) for i, j, t in st}
    assert edge_set(cut(pb, 5.0)) == remap(edge_set(g))
    # KNN: ties across atoms may legitimately change with relabelling; compare distances
    hp = knn(pb, 12)
    for q in range(cfg1.total_atoms):
        a = np.sort(h["d2"][h["src"] == perm[q]])
        b = np.sort(hp["d2"][hp["src"] == q])
        np.testing.assert_allclose(a, b, rtol=1e-12)


UNIMODULAR = [np.array([[1, 1, 0], [0, 1, 0], [0, 0, 1]]),
              np.array([[1, 0, 0], [2, 1, 1], [-1, 0, 1]]),
              np.array([[0, 1, 0], [0, 0, 1], [1, 0, 0]])]


@pytest.mark.parametrize("U", UNIMODULAR)
def test_unimodular_basis_change(cfg1, U):
    assert round(abs(np.linalg.det(U))) == 1
    Ui = np.linalg.inv(U)
    lat = np.einsum("ab,sbc->sac", U, cfg1.lattice.astype(np.float64))
    frac = cfg1.frac.astype(np.float64) @ Ui
    g = cut(cfg1, 5.0)
    g2 = oracle.cutoff(lat, frac, cfg1.atom_ptr, 5.0)
    mapped = {(i, j, tuple(int(v) for v in np.rint(np.array(t) @ Ui))) for i, j, t in edge_set(g)}
    assert edge_set(g2) == mapped
    # and the vectors agree
    v1, _ = oracle.edge_vectors(cfg1.lattice, cfg1.frac, cfg1.atom_ptr, g["src"], g["dst"], g["offset"])
    off2 = np.rint(g["offset"] @ Ui).astype(np.int32)
    v2, _ = oracle.edge_vectors(lat, frac, cfg1.atom_ptr, g["src"], g["dst"], off2)
    np.testing.assert_allclose(v1, v2, atol=1e-10)


def test_integer_translation(cfg1):
    rng = np.random.default_rng(1)
    n = rng.integers(-3, 4, size=(cfg1.total_atoms, 3))
    tb = synth.Batch(cfg1.lattice, cfg1.frac.astype(np.float64) + n, cfg1.atom_ptr)
    g = cut(cfg1, 5.0)
    g2 = oracle.cutoff(cfg1.lattice, cfg1.frac.astype(np.float64) + n, cfg1.atom_ptr, 5.0)
    want = {(i, j, tuple(int(v) for v in np.array(t) + n[i] - n[j])) for i, j, t in edge_set(g)}
    assert edge_set(g2) == want
    del tb


def test_supercell_consistency():
    base = synth.make_batch(1, B=2)
    for s in range(2):
        lo, hi = base.atom_ptr[s], base.atom_ptr[s + 1]
        x = base.frac[lo:hi].astype(np.float64)
        L = base.lattice[s].astype(np.float64)
        xs = np.concatenate([(x + np.array(c)) / 2.0 for c in itertools.product(range(2), repeat=3)])
        # float64 throughout: the tiled coordinates are not float32 values
        ptr1, ptr8 = np.array([0, len(x)], np.int32), np.array([0, len(xs)], np.int32)
        g1 = oracle.cutoff(L[None], x, ptr1, 5.0)
        g2 = oracle.cutoff((2 * L)[None], xs, ptr8, 5.0)
        assert len(g2["src"]) == 8 * len(g1["src"])
        d1 = degrees(g1, len(x))
        d2 = degrees(g2, len(xs))
        assert np.all(d2 == np.tile(d1, 8))
        k1, k2 = oracle.knn(L[None], x, ptr1, 12), oracle.knn((2 * L)[None], xs, ptr8, 12)
        for a in range(len(x)):
            np.testing.assert_allclose(np.sort(k1["d2"][k1["src"] == a]),
                                       np.sort(k2["d2"][k2["src"] == a]), rtol=1e-9)


def test_monotone_in_r_and_knn_inside_cutoff(cfg1):
    s4, s5 = edge_set(cut(cfg1, 4.0)), edge_set(cut(cfg1, 5.0))
    assert s4 <= s5
    h = knn(cfg1, 12)
    kth = np.sqrt(h["d2"].max())
    big = cut(cfg1, kth * (1 + 1e-9) + 1e-9)
    assert edge_set(h) <= edge_set(big)
    # KNN is the first k of the cutoff list ordered by (d2, j, t)
    for a in range(cfg1.total_atoms):
        m = big["src"] == a
        order = np.lexsort((big["offset"][m, 2], big["offset"][m, 1], big["offset"][m, 0],
                            big["dst"][m], big["d2"][m]))
        first = {(a, int(big["dst"][m][q]), tuple(int(v) for v in big["offset"][m][q])) for q in order[:12]}
        assert first == {e for e in edge_set(h) if e[0] == a}


def test_unwrapped_coordinates_allowed(cfg1):
    x = cfg1.frac.astype(np.float64).copy()
    x[0] += np.array([1.0, -2.0, 3.0])
    g = oracle.cutoff(cfg1.lattice, x, cfg1.atom_ptr, 5.0)
    v, ln = oracle.edge_vectors(cfg1.lattice, x, cfg1.atom_ptr, g["src"], g["dst"], g["offset"])
    assert np.all(ln < 5.0)
    assert len(g["src"]) == len(cut(cfg1, 5.0)["src"])


# ------------------------------------------------------------------ gradients

def loss_fn(lat, frac, ptr, g, w, sigma):
    vec, ln = oracle.edge_vectors(lat, frac, ptr, g["src"], g["dst"], g["offset"])
    return oracle.gaussian_loss_grads(vec, ln, w, sigma)[0]


def test_gradient_central_differences():
    b = synth.make_batch(4, B=3)
    g = cut(b, 5.0)
    w = synth.normal(7, 0, len(g["src"]))
    lat = b.lattice.astype(np.float64)
    fr = b.frac.astype(np.float64)
    vec, ln = oracle.edge_vectors(lat, fr, b.atom_ptr, g["src"], g["dst"], g["offset"])
    _, dlen = oracle.gaussian_loss_grads(vec, ln, w, 1.5)
    gf, gL = oracle.edge_grad(lat, fr, b.atom_ptr, g["src"], g["dst"], g["offset"], None, dlen)
    h = 1e-6
    rng = np.random.default_rng(3)
    for q in rng.choice(fr.size, 40, replace=False):
        p, m = fr.copy(), fr.copy()
        p.flat[q] += h
        m.flat[q] -= h
        fd = (loss_fn(lat, p, b.atom_ptr, g, w, 1.5) - loss_fn(lat, m, b.atom_ptr, g, w, 1.5)) / (2 * h)
        assert abs(fd - gf.flat[q]) <= 1e-6 * max(1.0, np.abs(gf).max())
    for q in range(lat.size):
        p, m = lat.copy(), lat.copy()
        p.flat[q] += h
        m.flat[q] -= h
        fd = (loss_fn(p, fr, b.atom_ptr, g, w, 1.5) - loss_fn(m, fr, b.atom_ptr, g, w, 1.5)) / (2 * h)
        assert abs(fd - gL.flat[q]) <= 1e-6 * max(1.0, np.abs(gL).max())


def test_gradient_vec_term_central_differences():
    """A loss that is linear in vec pins the grad_vec path (sum_e c_e . vec_e)."""
    b = synth.make_batch(1, B=2)
    g = cut(b, 4.0)
    c = synth.normal(9, 1, 3 * len(g["src"])).reshape(-1, 3).astype(np.float64)
    lat = b.lattice.astype(np.float64)
    fr = b.frac.astype(np.float64)
    gf, gL = oracle.edge_grad(lat, fr, b.atom_ptr, g["src"], g["dst"], g["offset"], c, None)

    def f(l, x):
        v, _ = oracle.edge_vectors(l, x, b.atom_ptr, g["src"], g["dst"], g["offset"])
        return float(np.sum(v * c))
    h = 1e-6
    for q in range(0, fr.size, 5):
        p, m = fr.copy(), fr.copy()
        p.flat[q] += h
        m.flat[q] -= h
        assert abs((f(lat, p) - f(lat, m)) / (2 * h) - gf.flat[q]) <= 1e-6 * max(1.0, np.abs(gf).max())
    for q in range(lat.size):
        p, m = lat.copy(), lat.copy()
        p.flat[q] += h
        m.flat[q] -= h
        assert abs((f(p, fr) - f(m, fr)) / (2 * h) - gL.flat[q]) <= 1e-6 * max(1.0, np.abs(gL).max())


def test_gradient_invariants():
    b = synth.make_batch(4, B=4)
    g = cut(b, 5.0)
    w = synth.normal(7, 0, len(g["src"]))
    vec, ln = oracle.edge_vectors(b.lattice, b.frac, b.atom_ptr, g["src"], g["dst"], g["offset"])
    _, dlen = oracle.gaussian_loss_grads(vec, ln, w, 1.5)
    gf, gL = oracle.edge_grad(b.lattice, b.frac, b.atom_ptr, g["src"], g["dst"], g["offset"], None, dlen)
    for s in range(b.num_structures):
        lo, hi = b.atom_ptr[s], b.atom_ptr[s + 1]
        # the loss depends on coordinate differences only
        np.testing.assert_allclose(gf[lo:hi].sum(0), 0.0, atol=1e-9 * np.abs(gf[lo:hi]).max())
        # rotation invariance of a radial loss: L^T dLoss/dL is symmetric
        M = b.lattice[s].astype(np.float64).T @ gL[s]
        np.testing.assert_allclose(M, M.T, atol=1e-9 * np.abs(M).max())
        # uniform strain L -> (1 + e) L with x fixed scales every length by (1 + e), so
        # d Loss / d e = trace(L^T dLoss/dL) = sum_e (dLoss/dl_e) l_e over the structure
        sel = (g["src"] >= lo) & (g["src"] < hi)
        virial = float(np.sum(dlen[sel] * ln[sel]))
        np.testing.assert_allclose(np.trace(M), virial, rtol=1e-9, atol=1e-12 * np.abs(dlen[sel] * ln[sel]).sum())
