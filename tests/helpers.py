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
    src = np.arange(lo, hi, dtype=np.int32)
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


def grad_check(b, g, w, sigma=1.5):
    """Autograd through the library's edge vectors for a Gaussian edge loss, against the
    oracle's analytic gradient within a condition-aware bound (1e-5 of the summed
    magnitudes of the contributions).  Returns the two gradients."""
    import torch

    import paper_2307_05380_gb300 as mg
    batch = g.batch
    frac = batch.frac.clone().requires_grad_(True)
    lat = batch.lattice.clone().requires_grad_(True)
    vec, ln = mg.edge_vectors(frac, lat, g)
    wt = torch.from_numpy(w).to(batch.device)
    loss = (wt * torch.exp(-ln ** 2 / (2 * sigma ** 2))).sum()
    loss.backward()
    got = graph_arrays(g)
    ov, ol = oracle.edge_vectors(b.lattice, b.frac, b.atom_ptr, got["src"], got["dst"], got["offset"])
    _, dlen = oracle.gaussian_loss_grads(ov, ol, w, sigma)
    gf, gL = oracle.edge_grad(b.lattice, b.frac, b.atom_ptr, got["src"], got["dst"], got["offset"], None, dlen)
    # condition-aware bound: 1e-5 of the summed magnitudes of the contributions
    gabs = np.abs(dlen)[:, None] * np.ones((1, 3))
    scale_f = np.zeros_like(gf)
    Lt = np.abs(b.lattice.astype(np.float64))
    atom_s = np.repeat(np.arange(b.num_structures), np.diff(b.atom_ptr))
    # |g_e| L^T magnitudes per edge and component (|dLoss/dlen| bounds |g_e| componentwise)
    h = np.einsum("ec,ekc->ek", gabs, Lt[atom_s[got["src"]]])
    np.add.at(scale_f, got["src"], h)
    np.add.at(scale_f, got["dst"], h)
    err_f = np.abs(frac.grad.cpu().numpy() - gf)
    assert np.all(err_f <= 1e-5 * scale_f + 1e-12), err_f.max()
    df = (b.frac[got["dst"]].astype(np.float64) - b.frac[got["src"]] + got["offset"])
    scale_L = np.zeros((b.num_structures, 3, 3))
    np.add.at(scale_L, atom_s[got["src"]], np.abs(df)[:, :, None] * gabs[:, None, :])
    err_L = np.abs(lat.grad.cpu().numpy() - gL)
    assert np.all(err_L <= 1e-5 * scale_L + 1e-12), err_L.max()
    return frac.grad.clone(), lat.grad.clone()
