"""GPU path vs the CPU oracle, element by element (needs a GB300).

Counts, c1 / c2, BFS levels, the cover-edge set and the CSR are integers and
must be bit-exact.  The cover set has no defined order on the device, so both
sides are compared sorted.  Parameter sets steer every cover edge through each
intersection kernel: the direct merge, the owner hash with one chunk, and the
owner hash with many chunks and many slices, with 512- and 1024-thread blocks.
"""
import json
import os
from math import comb

import numpy as np
import pytest

import oracle
import paper_2403_02997_gb300 as tc
from paper_2403_02997_gb300 import gen
from tests import graphs

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))

PARAMS = {
    "default": {},
    "all_hash": dict(small_max_degree=0),
    "all_merge": dict(small_max_degree=1 << 30),
    "tiny_chunks": dict(small_max_degree=0, hash_chunk=32, edges_per_item=3),
    "chunk64_slice1": dict(small_max_degree=2, hash_chunk=64, edges_per_item=1),
    "sorted_lookup": dict(small_max_degree=0, hash_chunk=128, edges_per_item=7, sorted_lookup=1),
    "medium_bin": dict(small_max_degree=4, medium_max_degree=1024),
    "medium_only": dict(small_max_degree=0, medium_max_degree=1024, hash_chunk=64),
    "block1024": dict(small_max_degree=0, hash_block=1024, hash_chunk=16384, edges_per_item=1024),
    "block1024_tiny": dict(small_max_degree=0, hash_block=1024, hash_chunk=32, edges_per_item=5),
    # items longer than the block (cursors held as 32-bit positions)
    "items1024": dict(small_max_degree=0, hash_chunk=128, edges_per_item=1024),
    "block1024_items4096": dict(small_max_degree=0, hash_block=1024, hash_chunk=256,
                                edges_per_item=4096),
}


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2403_02997_gb300 import build
    build.build_all()
    oracle.build()


def gpu_run(n, src, dst, root, params=None, device_edges=False):
    import torch
    if device_edges:
        s = torch.from_numpy(np.asarray(src, np.uint32).astype(np.int32)).cuda()
        d = torch.from_numpy(np.asarray(dst, np.uint32).astype(np.int32)).cuda()
    else:
        s, d = src, dst
    g = tc.Graph(s, d, n)
    if params:
        g.set_params(**params)
    T = g.count(root)
    return g, T


def check_against_oracle(n, src, dst, root, params=None, device_edges=False, check_csr=True):
    ref = oracle.count(n, src, dst, root, want_cover=True)
    g, T = gpu_run(n, src, dst, root, params, device_edges)
    try:
        st = g.stats()
        assert T == ref["T"]
        assert (st["c1"], st["c2"]) == (ref["c1"], ref["c2"])
        assert st["num_cover"] == ref["num_cover"]
        assert g.m == ref["m"]
        if n:
            assert np.array_equal(g.levels(), ref["level"])
            u, v = g.cover_edges()
            o = np.lexsort((v, u))
            assert np.array_equal(u[o], ref["cover_u"]) and np.array_equal(v[o], ref["cover_v"])
            if check_csr:
                rp, col = g.csr()
                assert np.array_equal(rp.astype(np.int64), ref["row_ptr"])
                assert np.array_equal(col, ref["col"])
        return T, st
    finally:
        g.close()


@pytest.mark.parametrize("pname", list(PARAMS))
@pytest.mark.parametrize("seed", [1, 2, 3])
def test_random_graphs(pname, seed):
    rng = np.random.default_rng(seed)
    for trial in range(4):
        n = int(rng.integers(2, 3000))
        E = int(rng.integers(0, 20 * n))
        src = rng.integers(0, n, E).astype(np.uint32)
        dst = rng.integers(0, n, E).astype(np.uint32)
        root = int(rng.integers(0, n))
        check_against_oracle(n, src, dst, root, PARAMS[pname])


@pytest.mark.parametrize("pname", list(PARAMS))
@pytest.mark.parametrize("scale,ef,seed", [(8, 16, 1), (12, 16, 2), (14, 8, 3)])
def test_rmat(pname, scale, ef, seed):
    src, dst = gen.rmat_edges(scale, ef, seed)
    n = 1 << scale
    rp, _ = oracle.build_csr(n, src, dst)
    root = oracle.max_degree_root(rp)
    check_against_oracle(n, src, dst, root, PARAMS[pname])


@pytest.mark.parametrize("pname", ["default", "all_hash", "tiny_chunks"])
def test_rmat16_multiroot(pname):
    src, dst = gen.rmat_edges(16, 16, 2)
    n = 1 << 16
    ref_T = json.load(open(os.path.join(HERE, "golden", "rmat16.json")))["T"]
    g, T = gpu_run(n, src, dst, 0, PARAMS[pname])
    try:
        assert T == ref_T
        for root in [g.max_degree_vertex(), 1, 12345, n - 1]:
            assert g.count(root) == ref_T
            st = g.stats()
            assert st["c2"] % 3 == 0 and st["c1"] + st["c2"] // 3 == ref_T
    finally:
        g.close()


def test_closed_forms():
    for n in [3, 4, 7, 33, 100]:
        assert check_against_oracle(*graphs.complete(n), 0)[0] == comb(n, 3)
    for n in [5, 9, 64]:
        assert check_against_oracle(*graphs.wheel(n), 0)[0] == n - 1
        assert check_against_oracle(*graphs.wheel(n), n - 1)[0] == n - 1
    assert check_against_oracle(*graphs.complete_bipartite(7, 40), 3)[0] == 0
    assert check_against_oracle(*graphs.diag_grid(9, 17), 0)[0] == 2 * 8 * 16
    assert check_against_oracle(*graphs.cycle(7), 2)[0] == 0
    assert check_against_oracle(*graphs.path(100), 0)[0] == 0


def test_disconnected_and_isolated():
    parts = [graphs.complete(6), graphs.wheel(7), graphs.cycle(3), graphs.path(4),
             graphs.diag_grid(3, 4), graphs.complete(1), graphs.star(9)]
    g = graphs.relabel(graphs.disjoint_union(*parts), 9)
    n, s, d = g
    for root in range(0, n, 7):
        check_against_oracle(n, s, d, root)
    # isolated vertices only
    check_against_oracle(10, np.array([3], np.uint32), np.array([3], np.uint32), 4)


def test_mesh_small_closed_form():
    rows, cols = 64, 48
    s, d = gen.mesh_edges(rows, cols, 0.5, 7)
    T, st = check_against_oracle(rows * cols, s, d, 0)
    assert T == 2 * int(gen.mesh_diagonals(rows, cols, 0.5, 7).sum())
    assert st["num_levels"] == rows + cols - 1


def test_device_and_host_edges_agree():
    src, dst = gen.er_edges(5000, 60000, 4)
    a = check_against_oracle(5000, src, dst, 17, device_edges=True)[0]
    b = check_against_oracle(5000, src, dst, 17, device_edges=False)[0]
    assert a == b


def test_empty_and_tiny():
    e = np.zeros(0, np.uint32)
    g = tc.Graph(e, e, 0)
    assert g.count(0) == 0
    g.close()
    check_against_oracle(1, e, e, 0)
    check_against_oracle(5, e, e, 3)
    check_against_oracle(2, np.array([0, 1, 1], np.uint32), np.array([1, 0, 1], np.uint32), 1)


def test_errors():
    with pytest.raises(tc.TCError) as ei:
        tc.Graph(np.array([0, 5], np.uint32), np.array([1, 2], np.uint32), 5)
    assert ei.value.status == 2
    g = tc.Graph(np.array([0], np.uint32), np.array([1], np.uint32), 3)
    with pytest.raises(tc.TCError) as ei:
        g.count(3)
    assert ei.value.status == 1
    assert g.count(2) == 0  # the handle stays usable
    with pytest.raises(tc.TCError):
        g.set_params(hash_chunk=100)
    with pytest.raises(tc.TCError):
        g.set_params(hash_block=768)
    with pytest.raises(tc.TCError):  # items of up to 2x a 512-thread block
        g.set_params(edges_per_item=1025)
    with pytest.raises(tc.TCError):  # and 4x a 1024-thread one
        g.set_params(hash_block=1024, edges_per_item=4097)
    g.set_params(hash_block=1024, edges_per_item=4096)
    assert g.count(2) == 0
    g.close()


def test_count_many_matches_single():
    specs = [gen.er_spec(300 + 50 * i, 3000 + 700 * i, 10 + i) for i in range(6)]
    specs += [gen.rmat_spec(9 + i % 3, 8 + i, 20 + i) for i in range(6)]
    gs, roots, want = [], [], []
    for sp in specs:
        s, d = sp.edges()
        rp, col = oracle.build_csr(sp.n, s, d)
        root = oracle.max_degree_root(rp) if sp.root == "maxdeg" else 0
        gs.append(tc.Graph(s, d, sp.n))
        roots.append(root)
        want.append(oracle.cetc(rp, col, oracle.bfs_levels(rp, col, root))["T"])
    try:
        assert tc.count_many(gs, roots) == want
        assert [g.count(r) for g, r in zip(gs, roots)] == want
    finally:
        for g in gs:
            g.close()
