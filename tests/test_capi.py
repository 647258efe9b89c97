"""The C-ABI library without a GPU: it loads, exports every symbol include/matgraph.h
declares, its structs have the layout the binding assumes, and host-side argument
checks answer before anything is launched."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "matgraph.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2307_05380_gb300 import _capi
    return _capi.load(build_if_missing=True)


def declared_functions():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:mg_status_t|const char \*|int64_t|int32_t)\s*(mg_\w+)\s*\(", text, re.M)))


def test_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert len(names) >= 12
    for n in names:
        assert hasattr(lib, n), n
    from paper_2307_05380_gb300 import _capi
    assert {s[0] for s in _capi.SIGNATURES} == set(names)


def test_struct_layout_matches_header(tmp_path):
    from paper_2307_05380_gb300._capi import MgBatch, MgGraph, MgOpts
    prog = tmp_path / "layout.c"
    prog.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "matgraph.h"\n'
                    'int main(void){printf("%zu %zu %zu %zu %zu %zu %zu\\n", sizeof(mg_batch_t), '
                    'sizeof(mg_graph_t), sizeof(mg_opts_t), sizeof(mg_device_status_t), '
                    'offsetof(mg_batch_t, lattice), offsetof(mg_graph_t, status), '
                    'offsetof(mg_device_status_t, candidates));return 0;}\n')
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I" + os.path.dirname(HEADER), str(prog), "-o", str(exe)])
    vals = [int(v) for v in subprocess.check_output([str(exe)]).split()]
    assert vals[0] == ctypes.sizeof(MgBatch)
    assert vals[1] == ctypes.sizeof(MgGraph)
    assert vals[2] == ctypes.sizeof(MgOpts)
    assert vals[3] == 40  # five 64-bit words, read back as int64[5]
    assert vals[4] == MgBatch.lattice.offset
    assert vals[5] == MgGraph.status.offset
    assert vals[6] == 32


def test_output_struct_layouts_match_header(tmp_path):
    """The triplet buffers and the host-copy buffers as the binding builds them."""
    from paper_2307_05380_gb300._capi import MgGraphHost, MgTriplets
    prog = tmp_path / "layout2.c"
    prog.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "matgraph.h"\n'
                    'int main(void){printf("%zu %zu %zu %zu %zu %zu\\n", sizeof(mg_triplets_t), '
                    'offsetof(mg_triplets_t, trip_ptr), offsetof(mg_triplets_t, status), sizeof(mg_graph_host_t), '
                    'offsetof(mg_graph_host_t, vec), offsetof(mg_graph_host_t, src_ptr));return 0;}\n')
    exe = tmp_path / "layout2"
    subprocess.check_call(["gcc", "-I" + os.path.dirname(HEADER), str(prog), "-o", str(exe)])
    vals = [int(v) for v in subprocess.check_output([str(exe)]).split()]
    assert vals == [ctypes.sizeof(MgTriplets), MgTriplets.trip_ptr.offset, MgTriplets.status.offset,
                    ctypes.sizeof(MgGraphHost), MgGraphHost.vec.offset, MgGraphHost.src_ptr.offset], vals


def test_step_struct_layout_matches_header(tmp_path):
    """mg_step_t, field by field, as the C compiler lays it out."""
    import ctypes
    import subprocess
    from paper_2307_05380_gb300._capi import MgStep
    names = [f[0] for f in MgStep._fields_]
    src = tmp_path / "step.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "matgraph.h"\n'
                   'int main(void){printf("%zu", sizeof(mg_step_t));' +
                   "".join(f'printf(" %zu", offsetof(mg_step_t, {n}));' for n in names) + 'return 0;}\n')
    exe = tmp_path / "step"
    subprocess.check_call(["gcc", "-I" + os.path.dirname(HEADER), str(src), "-o", str(exe)])
    vals = [int(v) for v in subprocess.check_output([str(exe)]).split()]
    assert vals == [ctypes.sizeof(MgStep)] + [getattr(MgStep, n).offset for n in names], vals


def test_status_strings(lib):
    for code in range(11):
        s = lib.mg_status_string(code).decode()
        assert s.startswith("MG_")


def test_host_argument_checks_without_device(lib):
    from paper_2307_05380_gb300._capi import MgBatch, MgGraph, MgOpts
    # no context: rejected on the host
    assert lib.mg_cutoff_graph(None, None, ctypes.c_float(5.0), None, None, None, None, 0, None) == 1
    assert lib.mg_knn_graph(None, None, 4, None, None, None, 0, None) == 1
    assert lib.mg_update_graph(None, None, None, None, 0, None) == 1
    assert lib.mg_edge_vectors_fwd(None, None, None, None, None, None) == 1
    assert lib.mg_last_launch_count(None) == -1
    sz = ctypes.c_size_t(0)
    assert lib.mg_workspace_size(None, ctypes.byref(MgBatch()), 0, ctypes.byref(sz)) == 1
    del MgGraph, MgOpts


def test_create_without_gpu_fails_cleanly(lib):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    assert lib.mg_create(ctypes.byref(h), 0) == 7  # MG_ERR_CUDA
    assert not h.value
