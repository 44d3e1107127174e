"""The C-ABI library builds, loads and exports every symbol include/tc.h declares
(no GPU: no compute calls).  Also the host-side argument checks that fail
before any device work."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2403_02997_gb300 import build
    build.build()
    import paper_2403_02997_gb300 as tc
    return tc.load_library()


def declared_functions():
    text = open(os.path.join(ROOT, "include", "tc.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(tc_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_the_abi():
    names = declared_functions()
    for want in ["tc_graph_create", "tc_graph_destroy", "tc_count", "tc_count_many",
                 "tc_count_split", "tc_count_forward", "tc_count_fe",
                 "tc_get_levels", "tc_get_cover_edges", "tc_status_string"]:
        assert want in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_status_strings(lib):
    for s in range(7):
        assert lib.tc_status_string(s).startswith(b"TC_")


def test_host_side_argument_checks(lib):
    import paper_2403_02997_gb300 as tc
    out = ctypes.c_void_p()
    # NULL out pointer, NULL arrays with edges, n >= 2^31: rejected before any CUDA call
    assert lib.tc_graph_create(None, None, 0, 4, 0, None, None) == 1
    assert lib.tc_graph_create(None, None, 5, 4, 0, None, ctypes.byref(out)) == 1
    assert lib.tc_graph_create(None, None, 0, 1 << 31, 0, None, ctypes.byref(out)) == 1
    assert lib.tc_count(None, 0, None, None) == 1
    assert lib.tc_count_split(None, 0, None, None) == 1
    assert lib.tc_count_forward(None, None, None) == 1
    assert lib.tc_count_fe(None, 0, 0.7, None, None, None) == 1
    assert lib.tc_graph_relabel_degree(None, None, None, None) == 1
    assert lib.tc_list_triangles(None, 0, None, None, 0, None, None, None) == 1
    assert lib.tc_count_many(None, None, 0, None, None) == 0
    assert lib.tc_graph_destroy(None) == 0
    p = tc.tc_params()
    assert lib.tc_params_default(ctypes.byref(p)) == 0
    assert p.hash_chunk % 32 == 0
    assert p.hash_block == 512 and p.edges_per_item <= p.hash_block


def test_binding_fails_loudly_without_library(tmp_path):
    import paper_2403_02997_gb300 as tc
    saved = tc._lib
    try:
        tc._lib = None
        with pytest.raises(ImportError):
            tc.load_library(str(tmp_path / "missing.so"))
    finally:
        tc._lib = saved
