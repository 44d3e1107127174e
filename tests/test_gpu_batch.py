"""Batched counting (one union of many graphs) against the oracle (GPU).

Each graph's count from tc_count_many / tc_batch_count must equal the oracle's
count for that graph and root, and the batch's per-graph levels must equal the
oracle's levels, for graphs of uneven size (empty ones included) and with the
tunables that send every cover edge through the owner-hash path with many
chunks and slices (so every kernel's per-graph attribution is exercised).
"""
import numpy as np
import pytest

import oracle
import paper_2403_02997_gb300 as tc
from paper_2403_02997_gb300 import gen
from tests import graphs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2403_02997_gb300 import build
    build.build_all()
    oracle.build()


def mixed_graphs():
    out = []
    for sp in gen.batched_specs(40, master_seed=4, log2_min=4, log2_max=12):
        s, d = sp.edges()
        out.append((sp.n, s, d, "maxdeg" if sp.root == "maxdeg" else 0))
    out.append((0, np.zeros(0, np.uint32), np.zeros(0, np.uint32), 0))        # empty
    out.append((7, np.zeros(0, np.uint32), np.zeros(0, np.uint32), 3))        # edgeless
    n, s, d = graphs.relabel(graphs.disjoint_union(graphs.complete(8), graphs.wheel(9),
                                                   graphs.path(5)), 1)
    out.append((n, s, d, 4))
    n, s, d = graphs.complete(40)
    out.append((n, s, d, 0))
    return out


def oracle_truth(items):
    want, roots, levels = [], [], []
    for n, s, d, root in items:
        rp, col = oracle.build_csr(n, s, d)
        r = oracle.max_degree_root(rp) if root == "maxdeg" else root
        roots.append(r)
        if n == 0:
            want.append(0)
            levels.append(np.zeros(0, np.int32))
            continue
        lv = oracle.bfs_levels(rp, col, r)
        want.append(oracle.cetc(rp, col, lv)["T"])
        levels.append(lv)
    return want, roots, levels


@pytest.mark.parametrize("params", [{}, dict(small_max_degree=0, hash_chunk=32, edges_per_item=2),
                                    dict(small_max_degree=1 << 30),
                                    dict(small_max_degree=8, medium_max_degree=256),
                                    dict(small_max_degree=0, hash_block=1024, hash_chunk=64,
                                         edges_per_item=700),
                                    dict(small_max_degree=0, hash_block=1024, hash_chunk=96,
                                         edges_per_item=3000)])
def test_batch_counts_and_levels(params):
    items = mixed_graphs()
    want, roots, levels = oracle_truth(items)
    gs = [tc.Graph(s, d, n) for n, s, d, _ in items]
    try:
        b = tc.Batch(gs)
        if params:
            b.set_params(**params)
        assert b.count(roots) == want
        for i, lv in enumerate(levels):
            assert np.array_equal(b.levels(i), lv), i
        st = b.stats()
        assert st["triangles"] == sum(want)
        assert st["c2"] % 3 == 0
        # the handles may go away; the batch holds its own copy
        for g in gs:
            g.close()
        assert b.count(roots) == want
        b.close()
    finally:
        for g in gs:
            g.close()


def test_count_many_matches_per_graph_counts():
    items = mixed_graphs()
    want, roots, _ = oracle_truth(items)
    gs = [tc.Graph(s, d, n) for n, s, d, _ in items]
    try:
        assert tc.count_many(gs, roots) == want
        assert [g.count(r) if g.n else 0 for g, r in zip(gs, roots)] == want
        with pytest.raises(tc.TCError):
            tc.count_many([gs[0], gs[0]], [roots[0], roots[0]])
    finally:
        for g in gs:
            g.close()


def test_batch_of_one_equals_single():
    s, d = gen.rmat_edges(14, 16, 3)
    g = tc.Graph(s, d, 1 << 14)
    try:
        r = g.max_degree_vertex()
        single = g.count(r)
        b = tc.Batch([g])
        assert b.count([r]) == [single]
        assert np.array_equal(b.levels(0), g.levels())
        b.close()
    finally:
        g.close()


def test_batch_from_edge_lists():
    items = mixed_graphs()
    want, roots, levels = oracle_truth(items)
    b = tc.Batch.from_edges([(s, d, n) for n, s, d, _ in items])
    try:
        md = b.max_degree_vertices()
        for i, (n, s, d, root) in enumerate(items):
            if root == "maxdeg":
                assert md[i] == roots[i], i
        assert b.count(roots) == want
        for i, lv in enumerate(levels):
            assert np.array_equal(b.levels(i), lv), i
        b.set_params(small_max_degree=0, hash_chunk=64, edges_per_item=5)
        assert b.count(roots) == want
    finally:
        b.close()
    # an id beyond its own graph's size is an error even inside the union's range
    n1, s1, d1 = graphs.complete(5)
    with pytest.raises(tc.TCError) as ei:
        tc.Batch.from_edges([(s1, d1, 5), (np.array([0, 7], np.uint32),
                                             np.array([1, 2], np.uint32), 6)])
    assert ei.value.status == 2


@pytest.mark.parametrize("params", [{}, dict(small_max_degree=0), dict(small_max_degree=1 << 30),
                                    dict(small_max_degree=8)])
def test_persistent_batch_counts_and_levels(params):
    """One persistent launch, one graph per block: every graph's count and levels equal the
    oracle's, with every cover edge merged by a lane (small_max_degree huge), searched by a warp
    (0), or split between the two; a second call (graph order cached) and the union path agree."""
    items = mixed_graphs()
    s, d = gen.rmat_edges(14, 16, 3)          # frontiers of thousands of vertices, hub pairs
    items.append((1 << 14, s, d, "maxdeg"))
    want, roots, levels = oracle_truth(items)
    gs = [tc.Graph(s_, d_, n) for n, s_, d_, _ in items]
    try:
        b = tc.Batch(gs)
        if params:
            b.set_params(**params)
        assert b.count_persistent(roots) == want
        for i, lv in enumerate(levels):
            assert np.array_equal(b.levels(i), lv), i
        st = b.stats()
        assert st["triangles"] == sum(want) and st["c2"] % 3 == 0
        assert b.count(roots) == want
        assert b.count_persistent(roots) == want
        b.close()
    finally:
        for g in gs:
            g.close()


def test_persistent_batch_from_edge_lists():
    items = mixed_graphs()
    want, roots, levels = oracle_truth(items)
    b = tc.Batch.from_edges([(s, d, n) for n, s, d, _ in items])
    try:
        assert b.count_persistent(roots) == want
        for i, lv in enumerate(levels):
            assert np.array_equal(b.levels(i), lv), i
    finally:
        b.close()
