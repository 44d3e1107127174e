"""BFS levels on long, thin graphs: the persistent cooperative kernel (GPU).

Levels are compared exactly with the oracle, with the persistent kernel on and
off.  The bounded grid-barrier wait is exercised by a testing knob that makes
one block leave without arriving: the count must fail with TC_ERR_TIMEOUT
within the configured budget and the handle must stay usable.
"""
import time

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


def levels_and_count(n, src, dst, root, **params):
    g = tc.Graph(src, dst, n)
    try:
        if params:
            g.set_params(**params)
        T = g.count(root)
        return g.levels(), T, g.stats()
    finally:
        g.close()


def check(n, src, dst, root):
    ref = oracle.count(n, src, dst, root)
    for persistent in (1, 0):
        lv, T, st = levels_and_count(n, src, dst, root, persistent_bfs=persistent)
        assert np.array_equal(lv, ref["level"]), persistent
        assert T == ref["T"]
    return st


def test_long_path_levels():
    n = 200_000
    n_, s, d = graphs.path(n)
    st = check(n, s, d, 0)
    assert st["num_levels"] == n
    check(n, s, d, n // 2 + 7)


def lollipop(k, tail):
    """K_k with a path of `tail` vertices hanging off vertex 0."""
    n1, s1, d1 = graphs.complete(k)
    ps = np.arange(tail, dtype=np.uint32) + k
    pd = np.concatenate([[0], ps[:-1]]).astype(np.uint32)
    return k + tail, np.concatenate([s1, ps]), np.concatenate([d1, pd])


def test_lollipop_and_cycle():
    n, s, d = lollipop(300, 20_000)
    check(n, s, d, 5)
    check(n, s, d, n - 1)
    n, s, d = graphs.cycle(100_001)
    check(n, s, d, 3)


def test_path_into_power_law_core():
    """The frontier stays tiny for 3000 levels, then explodes inside an R-MAT
    core: the persistent run must hand over to the host-driven loop."""
    scale = 17
    s1, d1 = gen.rmat_edges(scale, 16, 9)
    core = 1 << scale
    rp, _ = oracle.build_csr(core, s1, d1)
    hub = oracle.max_degree_root(rp)
    tail = 3000
    ps = np.arange(tail, dtype=np.uint32) + core
    pd = np.concatenate([[hub], ps[:-1]]).astype(np.uint32)
    n = core + tail
    s = np.concatenate([s1, ps])
    d = np.concatenate([d1, pd])
    st = check(n, s, d, n - 1)
    assert st["num_levels"] > tail


def test_barrier_timeout_is_reported_and_handle_survives():
    rows, cols = 300, 200
    s, d = gen.mesh_edges(rows, cols, 0.5, 3)
    n = rows * cols
    g = tc.Graph(s, d, n)
    try:
        good = g.count(0)
        # the persistent kernel (not the cluster search) takes the mesh's frontiers
        g.set_params(test_barrier_skip=1, barrier_timeout_ms=50, cluster_bfs=0)
        t0 = time.time()
        with pytest.raises(tc.TCError) as ei:
            g.count(0)
        assert ei.value.status == 5  # TC_ERR_TIMEOUT
        assert time.time() - t0 < 30
        g.set_params()  # defaults again
        assert g.count(0) == good
    finally:
        g.close()
