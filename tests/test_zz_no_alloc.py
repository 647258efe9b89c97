"""mg_cutoff_graph_noalloc: the cutoff build for callers that cannot provide a
workspace (their device memory belongs to another framework's pool, or they may not
call cudaMalloc at that point).  Its scratch is a fixed device array inside the
library.  Two calls in a row, on different batches, must each reproduce the output of
the workspace entry point mg_cutoff_graph exactly, so nothing left in the shared array
by the first call leaks into the second.  This file sorts last so that a run which
stops at the first failure has run every other test before it."""
import ctypes

import numpy as np
import pytest

import oracle
import synth
from helpers import assert_same_edges, grad_check, graph_arrays, to_device

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2307_05380_gb300 as mg  # noqa: E402
from paper_2307_05380_gb300 import _capi  # noqa: E402


def noalloc_into(g, cutoff):
    """Call the C-ABI entry point on graph buffers the caller already owns."""
    batch = g.batch
    rc = _capi.load().mg_cutoff_graph_noalloc(mg.context(batch.device), ctypes.byref(batch.c),
                                              ctypes.c_float(cutoff), ctypes.byref(g.opts), ctypes.byref(g.c),
                                              ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0, _capi.status_name(rc)
    st = g.read_status()
    assert st["code"] == 0, _capi.status_name(st["code"])
    return g


def noalloc_build(batch, cutoff, capacity):
    """Allocate the outputs here (the caller's job), then call the C-ABI entry point."""
    g = mg.graph._alloc_graph(_capi.MG_KIND_CUTOFF, batch, cutoff, 0, capacity, True, True, mg.make_opts())
    return noalloc_into(g, cutoff)


def test_noalloc_matches_workspace_entry_point_twice():
    cases = [(synth.make_batch(2), 6.0), (synth.make_batch(1), 5.0)]
    for b, r in cases:  # two calls in a row on the shared scratch array
        batch = to_device(b)
        want = graph_arrays(mg.cutoff_graph(batch, r))
        got = graph_arrays(noalloc_build(batch, r, want["src"].shape[0]))
        for key in ("src", "dst", "offset", "edge_ptr", "src_ptr", "perm_dst", "dst_ptr"):
            np.testing.assert_array_equal(got[key], want[key], err_msg=key)
        np.testing.assert_allclose(got["len"], want["len"], rtol=1e-6, atol=0)
        np.testing.assert_allclose(got["vec"], want["vec"], rtol=0, atol=1e-6 * float(want["len"].max()))


def test_noalloc_rejects_batches_beyond_the_scratch_limit():
    b = synth.make_batch(5)  # ~3e5 atoms plus an edge capacity of 1e7 needs more than 32 MiB
    batch = to_device(b)
    g = mg.graph._alloc_graph(_capi.MG_KIND_CUTOFF, batch, 8.0, 0, 10_000_000, True, True, mg.make_opts(),
                              ws_edges=1)
    rc = _capi.load().mg_cutoff_graph_noalloc(mg.context(batch.device), ctypes.byref(batch.c), ctypes.c_float(8.0),
                                              ctypes.byref(g.opts), ctypes.byref(g.c),
                                              ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 8  # MG_ERR_WORKSPACE, before any launch


def test_noalloc_graph_backward_matches_the_oracle():
    """The backward of a graph built without a workspace: it is a constant-cutoff graph,
    so its in-edges are its reversed out-edges, found by search (no pair table was
    recorded in a caller workspace).  Gradient of a Gaussian edge loss against the
    oracle's analytic gradient."""
    b = synth.make_batch(4, B=64)
    batch = to_device(b)
    E = len(oracle.cutoff(b.lattice, b.frac, b.atom_ptr, 5.0)["src"])
    g = noalloc_build(batch, 5.0, E)
    grad_check(b, g, synth.normal(4, 1, g.num_edges))


def test_noalloc_rebuild_drops_the_records_of_an_earlier_workspace_build():
    """A workspace build at 6 A into some buffers, then a build without a workspace at
    5 A into the same buffers: the backward must not use the pair table the first build
    left in the workspace (it indexes the 6 A edge set), and mg_update_graph must not
    replay the 6 A plan."""
    b = synth.make_batch(2)
    batch = to_device(b)
    g = mg.cutoff_graph(batch, 6.0, with_perm=False)
    noalloc_into(g, 5.0)
    got = graph_arrays(g)
    assert_same_edges(got, oracle.cutoff(b.lattice, b.frac, b.atom_ptr, 5.0), "noalloc rebuild at 5 A")
    grad_check(b, g, synth.normal(2, 7, g.num_edges))
    rc = _capi.load().mg_update_graph(mg.context(batch.device), ctypes.byref(batch.c), ctypes.byref(g.c),
                                      ctypes.c_void_p(g.ws.data_ptr()), ctypes.c_size_t(g.ws.numel()),
                                      ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 9  # MG_ERR_NOT_BUILT
