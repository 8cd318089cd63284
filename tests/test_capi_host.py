"""Host-side checks of the C ABI: the library builds, loads and exports every
declared symbol, struct layouts agree with the header, argument errors that
are caught before any device work return the documented status, and the
host-only relabelling is a correct graph isomorphism."""
import ctypes
import os
import re
import subprocess
import tempfile

import numpy as np
import pytest

import paper_2608_01907_gb300 as snap
from synth import edges_to_csr, rmat_graph, sbm_graph, tiny_graph

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "snap_layout.h")


@pytest.fixture(scope="module")
def lib():
    snap.build()
    return snap.load_library()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"\b(snap_[a-z_]+)\s*\(", text)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert "snap_layout_create" in names and "snap_layout_epochs" in names and "snap_layout_objective" in names
    for nm in names:
        assert hasattr(lib, nm), nm
    out = subprocess.run(["nm", "-D", "--defined-only", snap.library_path()], capture_output=True, text=True).stdout
    for nm in names:
        assert re.search(rf"\bT {nm}\b", out), nm


def _declared_parameters():
    """Parameter declarations of every function in the header (comments removed)."""
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    out = {}
    for m in re.finditer(r"\b(snap_[a-z_]+)\s*\(([^;{]*?)\)\s*;", text, flags=re.S):
        params = m.group(2).strip()
        out[m.group(1)] = [] if params in ("", "void") else [re.sub(r"\s+", " ", p.strip())
                                                               for p in params.split(",")]
    return out


def _ctypes_of(decl):
    """The ctypes type a C parameter declaration is passed as."""
    if "*" in decl or decl.startswith(("snap_layout_t ", "snap_multi_t ")):
        return ctypes.c_void_p
    base = decl.rsplit(" ", 1)[0].replace("const ", "")
    return {"int32_t": ctypes.c_int32, "int64_t": ctypes.c_int64, "uint64_t": ctypes.c_uint64,
            "double": ctypes.c_double, "float": ctypes.c_float}[base]


def test_binding_arguments_match_header(lib):
    decls = _declared_parameters()
    assert len(decls["snap_layout_autotune"]) == 14 and len(decls["snap_layout_epochs"]) == 8
    for name, params in decls.items():
        argtypes = getattr(lib, name).argtypes
        assert argtypes is not None, f"{name} has no argtypes in the binding"
        assert len(argtypes) == len(params), f"{name}: header {len(params)} parameters, binding {len(argtypes)}"
        for decl, t in zip(params, argtypes):
            assert t == _ctypes_of(decl), f"{name}: '{decl}' passed as {t.__name__}"
    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    returns = {"void": None, "snap_status": ctypes.c_int, "int64_t": ctypes.c_int64, "const char *": ctypes.c_char_p}
    decl_re = r"(?:^|\n)\s*((?:const\s+)?[a-z_0-9]+\s*\**)\s*(snap_[a-z_]+)\s*\([^;{]*?\)\s*;"
    seen = 0
    for m in re.finditer(decl_re, text, flags=re.S):
        ret = re.sub(r"\s+", " ", m.group(1).strip()).replace(" *", " *")
        assert getattr(lib, m.group(2)).restype == returns[ret], m.group(2)
        seen += 1
    assert seen == len(decls)


def test_struct_layouts_match_header(lib):
    src = r'''
#include <stdio.h>
#include <stddef.h>
#include "snap_layout.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu %d\n", sizeof(snap_schedule), offsetof(snap_schedule, eta0),
         offsetof(snap_schedule, eta_min), sizeof(snap_options), offsetof(snap_options, node_weights),
         offsetof(snap_options, sync_substeps), offsetof(snap_options, sync_cap),
         offsetof(snap_options, block_threads), offsetof(snap_options, flags), SNAP_FLAG_CUDA_GRAPH);
  printf("%zu\n", offsetof(snap_options, max_inflight));
  return 0;
}
'''
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        exe = os.path.join(d, "t")
        open(c, "w").write(src)
        subprocess.check_call(["gcc", "-I", os.path.dirname(HEADER), c, "-o", exe])
        vals = [int(v) for v in subprocess.check_output([exe]).split()]
    S, O = snap.SnapSchedule, snap.SnapOptions
    assert vals == [ctypes.sizeof(S), S.eta0.offset, S.eta_min.offset, ctypes.sizeof(O), O.node_weights.offset,
                    O.sync_substeps.offset, O.sync_cap.offset, O.block_threads.offset, O.flags.offset,
                    snap.FLAG_CUDA_GRAPH, O.max_inflight.offset]


def test_options_default(lib):
    o = snap.snap_options_default()
    assert (o.mode, o.sampler, o.sync_substeps, o.sync_cap, o.segment_edges, o.block_threads, o.flags) == \
        (snap.MODE_HOGWILD_RED, snap.SAMPLER_UNIFORM, 1, 0.0, 0, 0, 0)


def _status(fn, *a, **kw):
    if fn is snap.snap_layout_create:
        kw.setdefault("stream", 0)      # no torch stream without a GPU
    with pytest.raises(snap.SnapError) as ei:
        fn(*a, **kw)
    return ei.value.status, str(ei.value)


def test_host_side_argument_errors(lib):
    g = tiny_graph(20, 30, seed=1)
    rp = g.row_ptr.copy()
    rp[0] = 1
    assert _status(snap.snap_layout_create, rp, g.col_idx)[0] == 1
    rp = g.row_ptr.copy()
    rp[-1] = -2                      # a decreasing row_ptr inside is caught on the device (GPU tests)
    assert _status(snap.snap_layout_create, rp, g.col_idx)[0] == 1
    deg = g.degrees.copy()
    deg[3] += 1
    st, msg = _status(snap.snap_layout_create, g.row_ptr, g.col_idx, deg)
    assert st == 1 and "degrees[3]" in msg
    assert _status(snap.snap_layout_create, g.row_ptr, g.col_idx, None, 0)[0] == 1
    o = snap.make_options(sampler=snap.SAMPLER_WEIGHTS)          # no node_weights
    assert _status(snap.snap_layout_create, g.row_ptr, g.col_idx, opts=o)[0] == 1
    o = snap.make_options(sampler=3)
    assert _status(snap.snap_layout_create, g.row_ptr, g.col_idx, opts=o)[0] == 1
    for bad in (dict(mode=7), dict(sync_substeps=0), dict(segment_edges=6), dict(block_threads=48),
                dict(sync_cap=-1.0), dict(block_threads=512), dict(max_inflight=1.5)):
        assert _status(snap.snap_layout_create, g.row_ptr, g.col_idx, opts=snap.make_options(**bad))[0] == 1, bad
    o = snap.make_options()
    o.flags = 8
    st, msg = _status(snap.snap_layout_create, g.row_ptr, g.col_idx, opts=o)
    assert st == 1 and "flags" in msg


def test_null_handle_errors(lib):
    P = ctypes.c_void_p
    assert lib.snap_layout_check(None, None) == 1
    assert lib.snap_layout_device_bytes(None) == 0
    out = ctypes.c_uint64(7)
    assert lib.snap_memory_cached(0, None) == 1 and lib.snap_memory_cached(-1, ctypes.byref(out)) == 1
    assert lib.snap_memory_cached(0, ctypes.byref(out)) == 0 and out.value == 0   # nothing allocated here
    assert lib.snap_memory_trim(-1, 0) == 1 and lib.snap_memory_trim(0, 0) == 0
    lib.snap_layout_destroy(None)
    sched = snap.linear_schedule()
    assert lib.snap_layout_epochs(None, P(8), 0, 1, 3, ctypes.byref(sched), 1, None) == 1
    assert b"NULL" in lib.snap_last_error()
    assert lib.snap_layout_autotune(None, P(8), P(8), 3, ctypes.byref(sched), 1, 0.02, None, None, None, None,
                                    None, None, None) == 1
    assert b"NULL" in lib.snap_last_error()


def _edge_set(rp, ci):
    rows = np.repeat(np.arange(rp.size - 1), np.diff(rp))
    return set(zip(rows.tolist(), ci.tolist()))


@pytest.mark.parametrize("gen", ["tiny", "sbm", "rmat"])
def test_reorder_is_isomorphism_with_sorted_rows(lib, gen):
    g = {"tiny": lambda: tiny_graph(300, 700, seed=2),
         "sbm": lambda: sbm_graph(n=500, blocks=5, p_in=0.05, p_out=0.002, seed=3),
         "rmat": lambda: rmat_graph(scale=12, num_edges=20000, seed=4)}[gen]()
    perm, rp, ci = snap.snap_graph_reorder(g.row_ptr, g.col_idx)
    n = g.n
    assert sorted(perm.tolist()) == list(range(n))
    assert rp[0] == 0 and rp[-1] == g.nnz
    for v in range(n):
        row = ci[rp[v]:rp[v + 1]]
        assert np.all(np.diff(row) > 0)
    old = _edge_set(g.row_ptr, g.col_idx)
    new = _edge_set(rp, ci)
    mapped = {(int(perm[a]), int(perm[b])) for a, b in old}
    assert mapped == new
    # degrees carried over
    assert np.array_equal(np.diff(rp)[perm], np.diff(g.row_ptr))
    # label 0 goes to a highest-degree vertex
    assert np.diff(g.row_ptr)[np.argmin(perm)] == np.diff(g.row_ptr).max()


def test_reorder_bfs_locality_on_a_path(lib):
    n = 50
    rng = np.random.default_rng(1)
    labels = rng.permutation(n)
    rp, ci = edges_to_csr(n, labels[:-1], labels[1:])
    perm, rp2, ci2 = snap.snap_graph_reorder(rp, ci)
    rows = np.repeat(np.arange(n), np.diff(rp2))
    # a BFS from a path vertex keeps every edge within a small label distance
    assert np.abs(rows - ci2).max() <= 2


def test_reorder_rejects_bad_input(lib):
    rp = np.array([0, 1, 2], np.int64)
    assert _status(snap.snap_graph_reorder, rp, np.array([1, 5], np.int32))[0] == 1
    assert _status(snap.snap_graph_reorder, rp, np.array([1, 1], np.int32))[0] == 1


def test_batch_union_is_a_disjoint_union():
    from synth import tiny_graph
    graphs = [tiny_graph(n, m, seed=s) for s, (n, m) in enumerate([(30, 60), (1, 0), (50, 120), (7, 9)])]
    rp, ci, offs = snap.batch_union([(g.row_ptr, g.col_idx) for g in graphs])
    assert rp.dtype == np.int64 and ci.dtype == np.int32 and offs.dtype == np.int32
    assert offs.tolist() == [0, 30, 31, 81, 88] and rp.size == 89
    assert rp[-1] == sum(int(g.row_ptr[-1]) for g in graphs) == ci.size
    for q, g in enumerate(graphs):
        a, b = int(offs[q]), int(offs[q + 1])
        sub_rp = rp[a:b + 1] - rp[a]
        sub_ci = ci[rp[a]:rp[b]] - a
        assert np.array_equal(sub_rp, g.row_ptr) and np.array_equal(sub_ci, g.col_idx)
    # no edge leaves its graph
    rows = np.repeat(np.arange(rp.size - 1), np.diff(rp))
    graph_of = np.searchsorted(offs, np.arange(rp.size - 1), side="right") - 1
    assert np.array_equal(graph_of[rows], graph_of[ci])


@pytest.mark.parametrize("gen", ["tiny", "sbm", "rmat"])
def test_synth_relabel_gives_the_library_relabelling(lib, gen):
    """The input generators relabel graphs with their own code (so the
    oracle's inputs never pass through the library); both must give the same
    labels and the same CSR, so that both arms of the bench and the stored
    oracle values see the graph the library lays out."""
    from synth import bfs_relabel
    g = {"tiny": lambda: tiny_graph(300, 700, seed=2),
         "sbm": lambda: sbm_graph(n=500, blocks=5, p_in=0.05, p_out=0.002, seed=3),
         "rmat": lambda: rmat_graph(scale=14, num_edges=60000, seed=4)}[gen]()
    perm, rp, ci = snap.snap_graph_reorder(g.row_ptr, g.col_idx)
    r = bfs_relabel(g)
    assert np.array_equal(r.meta["perm"], perm)
    assert np.array_equal(r.row_ptr, rp) and np.array_equal(r.col_idx, ci)
