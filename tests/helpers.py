"""Shared test helpers: moving synthetic batches to the GPU and comparing graphs."""
import numpy as np

import oracle


def to_device(b, dev="cuda:0"):
    import torch

    import paper_2307_05380_gb300 as mg
    return mg.Batch(torch.from_numpy(b.frac).to(dev), torch.from_numpy(b.lattice).to(dev),
                    torch.from_numpy(b.atom_ptr).to(dev), max_atoms=b.max_atoms)


_POOL_BATCH = None


def _pool_init(lattice, frac, atom_ptr):
    global _POOL_BATCH
    _POOL_BATCH = (lattice, frac, atom_ptr)


def _oracle_range(task):
    kind, param, lo, hi = task
    lattice, frac, atom_ptr = _POOL_BATCH
    src = np.arange(lo, hi, dtype=np.int32) if not isinstance(lo, np.ndarray) else lo
    g = oracle.cutoff(lattice, frac, atom_ptr, param, sources=src) if kind == "cutoff" \
        else oracle.knn(lattice, frac, atom_ptr, param, sources=src)
    return g["src"], g["dst"], g["offset"]


def oracle_all_sources(kind, b, param, workers=None):
    """The oracle's graph over every source atom of batch b ('cutoff' with radius param,
    'knn' with k = param), computed by spawned processes on contiguous source ranges of
    about equal cost (a source costs the atoms of its structure) and joined in source
    order: the same edges as one call, in a fraction of the time."""
    import multiprocessing as mp
    import os
    workers = workers or os.cpu_count() or 1
    n = np.diff(b.atom_ptr).astype(np.float64)
    cum = np.cumsum(np.repeat(n, np.diff(b.atom_ptr)))
    pieces = 4 * workers
    cuts = sorted({0, b.total_atoms} | {int(np.searchsorted(cum, cum[-1] * q / pieces)) for q in range(1, pieces)})
    tasks = [(kind, param, lo, hi) for lo, hi in zip(cuts[:-1], cuts[1:]) if hi > lo]
    with mp.get_context("spawn").Pool(workers, initializer=_pool_init,
                                      initargs=(b.lattice, b.frac, b.atom_ptr)) as pool:
        parts = pool.map(_oracle_range, tasks)
    return dict(src=np.concatenate([p[0] for p in parts]), dst=np.concatenate([p[1] for p in parts]),
                offset=np.concatenate([p[2] for p in parts]).reshape(-1, 3))


def oracle_sources(kind, b, param, sources, workers=None):
    """The oracle's graph restricted to the given ascending source rows of batch b,
    computed by spawned processes on pieces of the source list of about equal cost (a
    source costs the atoms of its structure) and joined in source order."""
    import multiprocessing as mp
    import os
    workers = workers or os.cpu_count() or 1
    sources = np.asarray(sources, np.int32)
    n = np.diff(b.atom_ptr).astype(np.float64)
    atom_s = np.repeat(np.arange(b.num_structures), np.diff(b.atom_ptr))
    cum = np.cumsum(n[atom_s[sources]])
    pieces = 4 * workers
    cuts = sorted({0, len(sources)} | {int(np.searchsorted(cum, cum[-1] * q / pieces)) for q in range(1, pieces)})
    tasks = [(kind, param, sources[lo:hi], None) for lo, hi in zip(cuts[:-1], cuts[1:]) if hi > lo]
    with mp.get_context("spawn").Pool(workers, initializer=_pool_init,
                                      initargs=(b.lattice, b.frac, b.atom_ptr)) as pool:
        parts = pool.map(_oracle_range, tasks)
    return dict(src=np.concatenate([p[0] for p in parts]), dst=np.concatenate([p[1] for p in parts]),
                offset=np.concatenate([p[2] for p in parts]).reshape(-1, 3))


def rows_of_sources(src_ptr, sources):
    """Edge rows of the given sources, concatenated in source order (CSR src_ptr)."""
    lo = np.asarray(src_ptr)[sources]
    hi = np.asarray(src_ptr)[np.asarray(sources) + 1]
    return np.concatenate([np.arange(a, c, dtype=np.int64) for a, c in zip(lo, hi)]) if len(lo) else \
        np.zeros(0, np.int64)


def graph_arrays(g):
    E = g.num_edges
    out = dict(src=g.src[:E].cpu().numpy(), dst=g.dst[:E].cpu().numpy(), offset=g.offset[:E].cpu().numpy(),
               edge_ptr=g.edge_ptr.cpu().numpy(), src_ptr=g.src_ptr.cpu().numpy())
    if g.vec is not None:
        out["vec"] = g.vec[:E].cpu().numpy()
        out["len"] = g.len[:E].cpu().numpy()
    if g.perm_dst is not None:
        out["perm_dst"] = g.perm_dst[:E].cpu().numpy()
        out["dst_ptr"] = g.dst_ptr.cpu().numpy()
    return out


def assert_same_edges(got, want, what=""):
    """Bit-exact comparison of canonical edge lists."""
    assert got["src"].shape == want["src"].shape, f"{what}: {got['src'].shape[0]} vs {want['src'].shape[0]} edges"
    np.testing.assert_array_equal(got["src"], want["src"], err_msg=what)
    np.testing.assert_array_equal(got["dst"], want["dst"], err_msg=what)
    np.testing.assert_array_equal(got["offset"], want["offset"], err_msg=what)


def assert_vectors(b, got, rtol=1e-6):
    """vec/len within rtol of the FP64 oracle (vec error relative to the length)."""
    vec, ln = oracle.edge_vectors(b.lattice, b.frac, b.atom_ptr, got["src"], got["dst"], got["offset"])
    lerr = np.abs(got["len"].astype(np.float64) - ln) / ln
    verr = np.linalg.norm(got["vec"].astype(np.float64) - vec, axis=1) / ln
    assert lerr.max(initial=0) <= rtol, f"len rel err {lerr.max()}"
    assert verr.max(initial=0) <= rtol, f"vec rel err {verr.max()}"
    return lerr.max(initial=0), verr.max(initial=0)


def assert_perm_dst(got, N):
    """perm_dst lists edge ids by (dst, src, t); dst_ptr is its CSR."""
    E = got["src"].shape[0]
    order = np.lexsort((got["offset"][:, 2], got["offset"][:, 1], got["offset"][:, 0], got["src"], got["dst"]))
    np.testing.assert_array_equal(got["perm_dst"], order)
    counts = np.bincount(got["dst"], minlength=N)
    np.testing.assert_array_equal(got["dst_ptr"], np.concatenate([[0], np.cumsum(counts)]))
    assert got["dst_ptr"][-1] == E


def pointers_ok(got, b):
    edge_ptr, src_ptr = oracle.pointers(got["src"], b.atom_ptr)
    np.testing.assert_array_equal(got["edge_ptr"], edge_ptr)
    np.testing.assert_array_equal(got["src_ptr"], src_ptr)


def assert_grad_bound(b, got, grad_vec, grad_len, gf_gpu, gL_gpu, rel=1e-5):
    """GPU gradients w.r.t. frac and lattice against the oracle's FP64 analytic gradient
    of the same incoming edge gradients, per component within rel times the summed
    magnitudes of the contributions (a condition-aware bound).  Edge e contributes
    g_e L^T to its destination and -g_e L^T to its source, and (x_j - x_i + t)^T g_e to
    the lattice gradient, with g_e = grad_vec_e + grad_len_e vec_e / len_e; since
    |vec_c / len| <= 1, |g_e,c| <= |grad_vec_e,c| + |grad_len_e| componentwise.  Either
    incoming gradient may be None.  Returns the largest error in units of the bound."""
    E = got["src"].shape[0]
    gv = None if grad_vec is None else np.asarray(grad_vec, np.float64).reshape(E, 3)
    gl = None if grad_len is None else np.asarray(grad_len, np.float64).reshape(E)
    gf, gL = oracle.edge_grad(b.lattice, b.frac, b.atom_ptr, got["src"], got["dst"], got["offset"], gv, gl)
    gabs = np.zeros((E, 3))
    if gv is not None:
        gabs += np.abs(gv)
    if gl is not None:
        gabs += np.abs(gl)[:, None]
    Lt = np.abs(b.lattice.astype(np.float64))
    atom_s = np.repeat(np.arange(b.num_structures), np.diff(b.atom_ptr))
    s_e = atom_s[got["src"]]
    # |g_e| |L|^T per edge and component k: sum_c |g_e,c| |L_kc|
    h = np.einsum("ec,ekc->ek", gabs, Lt[s_e])
    scale_f = np.zeros((b.total_atoms, 3))
    np.add.at(scale_f, got["src"], h)
    np.add.at(scale_f, got["dst"], h)
    err_f = np.abs(np.asarray(gf_gpu, np.float64) - gf)
    df = b.frac[got["dst"]].astype(np.float64) - b.frac[got["src"]] + got["offset"]
    scale_L = np.zeros((b.num_structures, 3, 3))
    np.add.at(scale_L, s_e, np.abs(df)[:, :, None] * gabs[:, None, :])
    err_L = np.abs(np.asarray(gL_gpu, np.float64).reshape(-1, 3, 3) - gL)
    bf = rel * scale_f + 1e-12
    bL = rel * scale_L + 1e-12
    assert np.all(err_f <= bf), f"grad_frac: max err {err_f.max()}, worst ratio {(err_f / bf).max()}"
    assert np.all(err_L <= bL), f"grad_lattice: max err {err_L.max()}, worst ratio {(err_L / bL).max()}"
    return max(float((err_f / bf).max(initial=0)), float((err_L / bL).max(initial=0)))


def grad_check(b, g, w, sigma=1.5, c=None):
    """Autograd through the library's edge vectors for the loss
    sum_e w_e exp(-len_e^2 / 2 sigma^2) (+ sum_e c_e . vec_e when c [E, 3] is given, the
    grad_vec path), against the oracle's analytic gradient within the condition-aware
    bound of assert_grad_bound.  Returns the two gradients."""
    import torch

    import paper_2307_05380_gb300 as mg
    batch = g.batch
    frac = batch.frac.clone().requires_grad_(True)
    lat = batch.lattice.clone().requires_grad_(True)
    vec, ln = mg.edge_vectors(frac, lat, g)
    wt = torch.from_numpy(w).to(batch.device)
    loss = (wt * torch.exp(-ln ** 2 / (2 * sigma ** 2))).sum()
    if c is not None:
        loss = loss + (vec * torch.from_numpy(np.asarray(c, np.float32)).to(batch.device)).sum()
    loss.backward()
    got = graph_arrays(g)
    ov, ol = oracle.edge_vectors(b.lattice, b.frac, b.atom_ptr, got["src"], got["dst"], got["offset"])
    _, dlen = oracle.gaussian_loss_grads(ov, ol, w, sigma)
    assert_grad_bound(b, got, c, dlen, frac.grad.cpu().numpy(), lat.grad.cpu().numpy())
    return frac.grad.clone(), lat.grad.clone()
